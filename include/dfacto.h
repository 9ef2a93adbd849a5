/*
 * dfacto.h -- C ABI of libdfacto, a GB300 (sm_103a) implementation of DFacTo
 * (Choi & Vishwanathan, "DFacTo: Distributed Factorization of Tensors",
 * NIPS 2014): CP decomposition of sparse 3-way tensors by ALS and GD, with the
 * matricized-tensor times Khatri-Rao product (MTTKRP) computed as the paper's two
 * sparse matrix-vector products over flattened CSR copies of the tensor, batched
 * across all R columns.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Indices are 0-based.  A tensor X is I x J x K = dims[0] x dims[1] x dims[2].
 *  - "Mode" n is 0, 1 or 2 and names the factor being solved for: mode 0 is
 *    N = X^1 (C kr B) (updates A), mode 1 is X^2 (A kr C) (updates B), mode 2 is
 *    X^3 (B kr A) (updates C), with the flattenings of Eq. x1 and the operand
 *    order of Algorithm 4.  For mode n the CSR copy pairs rows (o, f) with
 *    entries `in`, where o = n, in = (n+1) mod 3, f = (n+2) mod 3.
 *  - Factor matrices are row-major: row t of F_m holds F_m[t, 0..R-1].
 *  - Pointers may be host or device memory unless a function says otherwise;
 *    the library finds out with cudaPointerGetAttributes.  Device pointers must
 *    be 16-byte aligned.  The caller keeps ownership of every buffer it passes;
 *    the library never keeps a caller pointer after the call returns.
 *  - Work is queued on the handle's stream.  Functions that return a host value
 *    (fit, loss, lambda, CSR sizes) synchronize that stream; the others do not.
 *  - Every function returns a status and never aborts the process.  After
 *    DFACTO_ECUDA the handle must be destroyed.  dfacto_last_error() gives a
 *    one-line description of the last failure on a handle.
 *  - Calls on one handle are not thread-safe; distinct handles are independent.
 */
#ifndef DFACTO_H_
#define DFACTO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dfacto_status {
  DFACTO_OK = 0,
  DFACTO_EINVAL = 1,    /* bad argument (null pointer, mode, rank, sizes)         */
  DFACTO_ERANGE = 2,    /* a coordinate lies outside dims                         */
  DFACTO_EDUP = 3,      /* two nonzeros share a coordinate                        */
  DFACTO_ENOMEM = 4,    /* device (or pinned host) allocation failed              */
  DFACTO_ECUDA = 5,     /* a CUDA call failed; the handle is unusable             */
  DFACTO_ESINGULAR = 6, /* informational: a Gram-Hadamard matrix was not positive
                           definite and its pseudo-inverse was used              */
  DFACTO_ELSFAIL = 7,   /* GD line search found no acceptable step; the factors
                           are unchanged                                          */
  DFACTO_ETIMEOUT = 8,  /* reserved: no kernel of this version waits on another  */
  DFACTO_EINTERNAL = 9  /* an internal consistency check failed                   */
} dfacto_status;

typedef enum dfacto_dtype {
  DFACTO_F32 = 0,  /* float                                  */
  DFACTO_BF16 = 1, /* bfloat16 (round-to-nearest-even stores) */
  DFACTO_F64 = 2   /* double (set/get of factors only)        */
} dfacto_dtype;

/*
 * Build and solver options.  Initialise with dfacto_options_init().
 *   rank          R, 1..128 (R > 32 must be a multiple of 4).
 *   factor_dtype  storage of A, B, C on the device: DFACTO_F32 or DFACTO_BF16.
 *                 Products are always accumulated in FP32; Grams, the R x R
 *                 solves, line-search and fit scalars in FP64.
 *   lambda_reg    ridge term added to every Gram-Hadamard matrix (ALS) and to
 *                 the objective (GD): the regularized forms of Appendix B
 *                 (Eq. tensorapprx-ref-sol) and Appendix C (Eq. gd-obj-fn-reg).
 *                 Must be >= 0; 0 (the default) is the plain method.
 *   seg_nnz       nonzeros walked by one lane group in the MTTKRP kernel, at
 *                 most 4096; 0 lets the library choose.  Rounded to a multiple
 *                 of 32.
 *   vec           factor columns per lane in the MTTKRP kernel (1, 2, 4 or 8;
 *                 must divide R); 0 lets the library choose.  With 0, at a rank
 *                 R > 2 that is not a multiple of 4, the MTTKRP and the GD line
 *                 search gather from zero-padded FP32 copies of the factors at
 *                 R rounded up to a multiple of 4 (16-byte gathers; the result
 *                 is the same sums up to their order), which the handle
 *                 allocates on first use.
 *   walk          MTTKRP kernel: 1 detects fiber ends from the fiber pointers
 *                 as it walks, 2 from a per-nonzero end bitmask and closes the
 *                 fibers of a few steps together; 0 lets the library choose.
 *                 Other values are refused (DFACTO_EINVAL).  Both compute the
 *                 same sums in the same order.
 *   line_search   GD step size (dfacto_gd_iter): 0 (default) backtracking from
 *                 min(2 alpha_prev, 1), halving until the Armijo condition holds
 *                 (the rule read into Algorithm 5's "line search"); 1 the exact
 *                 minimiser of f(theta - alpha grad) over alpha > 0.  Along the
 *                 ray f is a polynomial of degree 6 in alpha (its cubic data term
 *                 from one pass over the nonzeros, its model term from R x R
 *                 Grams); the roots of its derivative are isolated in FP64 on
 *                 the device and the local minimum with the smallest f is taken
 *                 when it lowers f (otherwise the step falls back to
 *                 backtracking).  The paper states no rule; this option is an
 *                 addition.  Other values are refused (DFACTO_EINVAL).
 */
typedef struct dfacto_options {
  int32_t rank;
  int32_t factor_dtype;
  double lambda_reg;
  int32_t seg_nnz;
  int32_t vec;
  int32_t walk;
  int32_t line_search;
  int32_t reserved[4];
} dfacto_options;

/* Sizes of a built tensor. */
typedef struct dfacto_info {
  int32_t dims[3];
  int32_t rank;
  int64_t nnz;
  int64_t nfib[3];       /* fibers (= nnzc of the paired flattening) per mode */
  int64_t device_bytes;  /* device memory held by the handle                  */
  double norm_x2;        /* ||X||^2 in FP64                                    */
  int32_t factor_dtype;
  int32_t seg_nnz[3];    /* MTTKRP segment length in use per mode              */
  int32_t vec[3];        /* MTTKRP columns per lane in use per mode (of the
                            padded FP32 copies at a padded rank, see vec)       */
} dfacto_info;

/*
 * Device pointers to the flattened CSR copy of one mode (Sec. 3, Lemma 3 and
 * Lemma 4).  For mode n:
 *   fiber_ptr[dim_o + 1]  row(M^r): the fibers of output row o are
 *                         fiber_ptr[o] .. fiber_ptr[o+1]-1 (empty rows kept)
 *   fiber_idx[nfib]       col(M^r): the index f of each fiber
 *   nz_ptr[nfib + 1]      row pointer of (Xhat^{n+1})^T: fiber q holds the
 *                         nonzeros nz_ptr[q] .. nz_ptr[q+1]-1
 *   nz_idx[nnz], nz_val[nnz]  column (index `in`) and value of each nonzero
 * Fibers are the distinct (o, f) pairs in lexicographic order, entries ascend
 * in `in` within a fiber.  The arrays belong to the handle and stay valid until
 * dfacto_destroy().
 */
typedef struct dfacto_csr_view {
  int64_t dim_o;
  int64_t nfib;
  int64_t nnz;
  const int64_t* fiber_ptr;
  const int32_t* fiber_idx;
  const int64_t* nz_ptr;
  const int32_t* nz_idx;
  const float* nz_val;
} dfacto_csr_view;

typedef struct dfacto_handle dfacto_t;

/* Fill *opt with the defaults for rank R (FP32 factors, lambda_reg 0, tuned). */
void dfacto_options_init(dfacto_options* opt, int32_t rank);

/* Static string for a status code. */
const char* dfacto_status_str(dfacto_status s);

/*
 * dfacto_build -- validate a COO tensor and build its three flattened CSR
 * copies on the device (the (Xhat^2)^T, (Xhat^3)^T, (Xhat^1)^T of Sec. 3 with
 * the fixed sparsity pattern of M^r, Lemma 4), by a radix sort per mode.
 *   idx     int32[3][nnz], structure of arrays: idx[m*nnz + t] is coordinate m
 *           of nonzero t.  Host or device.
 *   val     float[nnz], host or device.  Explicit zeros are kept as observed
 *           entries (the observed set of Sec. 2).
 *   nnz     0 <= nnz <= 2^31 - 2^16 (2,147,418,112).
 *   dims    host int32[3], each >= 1.
 *   opt     build options (rank, factor storage, ...); NULL means rank 1.
 *   stream  cudaStream_t the handle will use for all its work (NULL: the
 *           legacy default stream).
 *   out     receives the new handle.  The handle owns all device memory it
 *           allocates.  Factors start at zero: set them before solving.
 * Errors: EINVAL (null pointers, dims < 1, bad rank/options), ERANGE (a
 * coordinate outside dims), EDUP (repeated coordinate), ENOMEM, ECUDA.  On error
 * *out is NULL.
 */
dfacto_status dfacto_build(const int32_t* idx, const float* val, int64_t nnz,
                           const int32_t dims[3], const dfacto_options* opt, void* stream,
                           dfacto_t** out);

/* Release every resource of the handle (NULL is allowed). */
void dfacto_destroy(dfacto_t* h);

/* One-line description of the last failure on the handle ("" if none). */
const char* dfacto_last_error(const dfacto_t* h);

/*
 * Number of CUDA kernels this library has launched in this process so far
 * (all handles).  The difference around a call is that call's launch count.
 */
int64_t dfacto_launch_count(void);

/* Sizes of the built tensor (host struct). */
dfacto_status dfacto_get_info(dfacto_t* h, dfacto_info* info);

/* Change the stream used by later calls on this handle. */
dfacto_status dfacto_set_stream(dfacto_t* h, void* stream);

/* Wait for all work queued on the handle's stream. */
dfacto_status dfacto_sync(dfacto_t* h);

/*
 * dfacto_set_factors / dfacto_get_factors -- copy factor matrix `mode`
 * (dims[mode] x R, row-major) in or out, converting between `dtype` and the
 * handle's storage type (BF16 storage rounds to nearest even).  The
 * initialization is the caller's (the paper leaves it open, Algorithm 2).
 * Setting a factor invalidates its cached Gram.  Host or device buffers.
 */
dfacto_status dfacto_set_factors(dfacto_t* h, int mode, const void* F, dfacto_dtype dtype);
dfacto_status dfacto_get_factors(dfacto_t* h, int mode, void* F, dfacto_dtype dtype);

/*
 * CP weights lambda_r of Eq. parafac (host double[R]).  ALS writes them (the
 * column norms of the last updated factor); they are 1 after dfacto_build and
 * the GD model ignores them.
 */
dfacto_status dfacto_get_lambda(dfacto_t* h, double* lambda);
dfacto_status dfacto_set_lambda(dfacto_t* h, const double* lambda);

/*
 * dfacto_mttkrp -- N = X^n (F_f kr F_in) for the current factors (Algorithm 1,
 * Lemma 2): for every column r, value(M^r) <- (Xhat^{n+1})^T F_in[:, r] and
 * N[:, r] <- M^r F_f[:, r], all R columns in one pass, the intermediate M^r
 * held in registers only.
 *   out  device float[dims[mode] x R], row-major, caller-owned; every entry is
 *        written (rows with no nonzeros get 0).
 * Asynchronous.  Errors: EINVAL, ECUDA.
 */
dfacto_status dfacto_mttkrp(dfacto_t* h, int mode, float* out);

/*
 * dfacto_als_iter -- one DFacTo-ALS sweep (Algorithm 4 with Algorithm 2):
 * for modes 0, 1, 2 in turn, N = MTTKRP(mode), Gamma = Gram(F_f) * Gram(F_in)
 * (+ lambda_reg I) (Eq. kr-product), F_mode = N Gamma^{-1} by Cholesky (the
 * pseudo-inverse of Eq. kr-pseudo when Gamma is not positive definite), then
 * column normalisation with lambda = the column 2-norms.  Afterwards the fit
 * 1 - ||X - [[lambda; A,B,C]]|| / ||X|| is computed in FP64.
 *   fit_out  host double, nullable.  When NULL nothing is read back and the
 *            call does not synchronize.
 * Returns DFACTO_ESINGULAR (after completing the sweep) if a pseudo-inverse was
 * needed; that status is only seen when fit_out is non-NULL.
 */
dfacto_status dfacto_als_iter(dfacto_t* h, double* fit_out);

/*
 * dfacto_gd_iter -- one DFacTo-GD step (Algorithm 5, with the gradient sign of
 * Eq. gd-A): the three gradients dF_n = -N_n + F_n Gamma_n (+ lambda_reg F_n) at
 * the current point, then a backtracking line search -- alpha0 = min(2
 * alpha_prev, 1) (1 on the first step), accept the first alpha with
 * f(theta - alpha grad) <= f(theta) - 1e-4 alpha ||grad||^2, halving at most 100
 * times -- or, with the line_search option 1, the exact minimiser of
 * f(theta - alpha grad) over alpha > 0, and the update theta <- theta - alpha
 * grad.  f is the objective of
 * Eq. gd-obj-fn (regularized: Eq. gd-obj-fn-reg), evaluated in FP64.
 *   loss_out, alpha_out  host doubles, nullable; when both are NULL the call
 *                        does not synchronize.  loss_out gets f at the returned
 *                        point, alpha_out the accepted step.
 * Returns DFACTO_ELSFAIL (factors unchanged) when no trial is accepted; that
 * status is only seen when an output pointer is non-NULL.
 */
dfacto_status dfacto_gd_iter(dfacto_t* h, double* loss_out, double* alpha_out);

/*
 * dfacto_fit -- fit of the current model [[lambda; A,B,C]]:
 * 1 - sqrt(max(0, ||X||^2 - 2<X, Xhat> + ||Xhat||^2)) / ||X||, all in FP64, with
 * <X, Xhat> by one pass over the nonzeros and ||Xhat||^2 = lambda^T (A^T A *
 * B^T B * C^T C) lambda.  Synchronizes.
 */
dfacto_status dfacto_fit(dfacto_t* h, double* fit_out);

/* Device pointers to the CSR copy of one mode (see dfacto_csr_view). */
dfacto_status dfacto_get_csr(dfacto_t* h, int mode, dfacto_csr_view* view);

/*
 * dfacto_mttkrp_noalloc -- the same MTTKRP as dfacto_mttkrp for one mode, for
 * callers that are not allowed to allocate device memory: code whose device
 * memory is owned and accounted by another allocator (a framework's caching
 * allocator, a memory-capped service), code running in a section where an
 * allocation could block or fail at the wrong moment, or code that only borrows
 * device pointers from their owner.  dfacto_mttkrp may allocate its work
 * buffers on first use; this entry point never calls cudaMalloc, cudaFree or
 * any allocating routine.  The paper has no counterpart.
 *
 * Its scratch (segment starts and the partial sums of rows shared between
 * blocks) lives in one fixed 16 MiB device array inside the library.  Every
 * GPU that loads the library holds that array until the process exits.  The
 * problem must fit in it: about 260 million nonzeros at R = 32 (4 bytes per
 * 128 nonzeros plus 8 * R + 8 bytes per 8,192 nonzeros when R is a multiple of
 * 8) and about 310 million at R = 10 (the same per 4,096 nonzeros).
 *   csr     host struct of device pointers to the flattened CSR copy of mode n,
 *           in the layout dfacto_get_csr describes (from a handle, or built by
 *           the caller the same way); nnz <= 2^31 - 2^16.
 *   F_in    device float[dims[(n+1) mod 3] x R], row-major: the factor indexed
 *           by nz_idx.
 *   F_f     device float[dims[(n+2) mod 3] x R], row-major: the factor indexed
 *           by fiber_idx.
 *   R       1..128 (R > 32 a multiple of 4).
 *   out     device float[dim_o x R], row-major; every entry is written.
 *   stream  cudaStream_t for the work (NULL: the legacy default stream).
 * Returns DFACTO_ENOMEM when the problem needs more scratch than the 16 MiB
 * array holds, DFACTO_EINVAL for bad arguments, DFACTO_ECUDA if a launch
 * failed.  Asynchronous otherwise.
 *
 * The first call on a device, with that device current, looks up the device
 * address of the array (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Under CUDA's lazy module loading (the default) that first
 * call, and the first call for each walk shape (R), may also load the
 * library's device code and the array itself, which takes device memory: make
 * one call per device and R before the section that must not allocate (its
 * results can be discarded), or run with CUDA_MODULE_LOADING=EAGER.  All calls
 * share the one array and a call leaves its contents behind: calls whose work
 * may overlap on the GPU (different streams or threads without ordering) race
 * on it and must be serialised by the caller.  Nothing in the array needs to
 * start at zero: each call writes every scratch value it later reads.
 */
dfacto_status dfacto_mttkrp_noalloc(const dfacto_csr_view* csr, const float* F_in, const float* F_f,
                                    int32_t R, float* out, void* stream);

/* ------------------------------------------------------------------------
 * Joint matrix completion and tensor factorization (Appendix F).
 *
 * A ratings matrix Y (users x items, dims[0] x dims[1], observed entries
 * Omega^Y) and the handle's user x item x word tensor X share the user factor
 * A and the item factor B (Eq. joint-obj-fn):
 *   f = 1/2 sum_{(i,j) in Omega^Y} (y_ij - a_i . b_j)^2
 *       + mu 1/2 ||X - [[A, B, C]]||^2 + lambda 1/2 (||A||^2 + ||B||^2 + ||C||^2)
 * with lambda the handle's lambda_reg.  The model has no CP weights (they
 * are kept at 1) and needs R <= 32.
 * ------------------------------------------------------------------------ */

/*
 * dfacto_joint_set_ratings -- attach the ratings to a built handle (replacing
 * earlier ones) and build their two CSR copies on the device (by user and by
 * item, columns ascending within a row).
 *   yidx  int32[2][nnzY], structure of arrays: yidx[t] is the user (row of A,
 *         < dims[0]) and yidx[nnzY + t] the item (row of B, < dims[1]) of
 *         rating t.  Host or device; the caller keeps ownership.
 *   yval  float[nnzY], host or device.
 *   nnzY  0 <= nnzY <= 2^31 - 2^16.
 *   mu    weight of the tensor term, >= 0.
 * Errors: EINVAL (bad arguments, R > 32, handle in a batch), ERANGE (a rating
 * outside dims[0] x dims[1]), EDUP (two ratings of one (user, item)), ENOMEM,
 * ECUDA.  Synchronizes.
 */
dfacto_status dfacto_joint_set_ratings(dfacto_t* h, const int32_t* yidx, const float* yval,
                                       int64_t nnzY, double mu);

/* Device pointers to one CSR copy of the ratings: side 0 rows are users
 * (col = item), side 1 rows are items (col = user); ptr[rows + 1]. */
typedef struct dfacto_ratings_view {
  int64_t rows;
  int64_t nnz;
  const int64_t* ptr;
  const int32_t* col;
  const float* val;
} dfacto_ratings_view;
dfacto_status dfacto_get_ratings_csr(dfacto_t* h, int side, dfacto_ratings_view* view);

/*
 * dfacto_joint_als_iter -- one ALS sweep of the joint model: every row of A by
 * the closed form of Appendix F,
 *   a_i = [sum_{j in Omega_i} y_ij b_j + mu N_A[i]]
 *         [sum_{j in Omega_i} b_j^T b_j + mu C^T C * B^T B + lambda I]^-1
 * (N_A = X^1 (C kr B), the MTTKRP of Algorithm 1; the sum in the bracket runs
 * over the user's own ratings), then B the same way with the new A, then C
 * (tensor term only).  One R x R Cholesky solve per row in FP64; needs
 * lambda_reg > 0 (EINVAL otherwise), which makes every system positive
 * definite.
 *   obj_out  host double, nullable: f after the sweep (synchronizes).
 */
dfacto_status dfacto_joint_als_iter(dfacto_t* h, double* obj_out);

/*
 * dfacto_joint_gd_iter -- one GD step of the joint model: the gradients of
 * Eq. grad-joint-A for A, B and C at the current point, then the step size by
 * the handle's line_search option (backtracking as dfacto_gd_iter, or the
 * exact minimiser: along the ray f is a polynomial of degree 6, its ratings
 * term a quartic from one pass over the ratings), then the update.
 *   obj_out, alpha_out  host doubles, nullable (both NULL: no synchronization).
 * Returns DFACTO_ELSFAIL (factors unchanged) when no step is accepted.
 */
dfacto_status dfacto_joint_gd_iter(dfacto_t* h, double* obj_out, double* alpha_out);

/* f of the joint model at the current factors (synchronizes). */
dfacto_status dfacto_joint_objective(dfacto_t* h, double* obj_out);

/* ------------------------------------------------------------------------
 * Batches: many independent decompositions advanced together.
 *
 * The paper factorizes one tensor at a time; a batch runs the ALS sweep of
 * Algorithm 4 (with the MTTKRP of Algorithm 1) for n independent jobs at
 * once.  Jobs that share (R, factor type) form a rank class: their flattened
 * CSR copies are concatenated into one block-diagonal tensor (indices offset
 * per job) and their factors are pooled, so the MTTKRP of a mode for every
 * job of every class is one persistent kernel launch.  The per-job steps
 * (Gamma^{-1}, N Gamma^{-1}, normalisation, Grams, fit) run as one batched
 * launch per step and rank class, and from the second sweep on the whole
 * sweep is replayed as one CUDA graph.
 * ------------------------------------------------------------------------ */
typedef struct dfacto_batch dfacto_batch_t;

typedef struct {
  int32_t use_graph;    /* nonzero: capture the sweep into a CUDA graph and
                           replay it from the second sweep on */
  int32_t autotune;     /* nonzero: time walk shapes per rank class at creation */
  int32_t reserved[6];  /* zero */
} dfacto_batch_options;

/* Defaults: graph on, autotune on. */
void dfacto_batch_options_init(dfacto_batch_options* opt);

/*
 * dfacto_batch_create -- group n built handles (dfacto_build, factors set)
 * into a batch.
 *   jobs    host array of n distinct handles on the current device, none in
 *           another batch.  The batch borrows them: their factors move into
 *           the batch's pools (the handles keep working, with their factor
 *           pointers inside the pools) until dfacto_batch_destroy moves them
 *           back.  Destroy the batch before its jobs; a job destroyed first
 *           leaves the batch unusable (its calls return DFACTO_EINVAL).
 *   n       1..65536.
 *   opt     options, or NULL for the defaults.
 *   stream  cudaStream_t the batch's calls are ordered after, and that waits
 *           for each call's work (NULL: the legacy default stream).  The batch
 *           runs on two non-blocking streams of its own.
 * The batch owns a second copy of every job's CSR arrays (concatenated per
 * rank class) and one MTTKRP output buffer per class and mode.  Returns
 * DFACTO_EINVAL for bad arguments, DFACTO_ENOMEM, DFACTO_ECUDA.  Synchronous.
 */
dfacto_status dfacto_batch_create(dfacto_t* const* jobs, int32_t n, const dfacto_batch_options* opt,
                                  void* stream, dfacto_batch_t** out);

/* Free the batch's memory, streams and graph and hand the factors back to
 * the jobs (copied into allocations of their own).  NULL is ignored. */
void dfacto_batch_destroy(dfacto_batch_t* b);

/*
 * dfacto_batch_mttkrp -- the MTTKRP of mode `mode` (Algorithm 1) for every
 * job, from the jobs' current factors.
 *   out     host array of n device pointers; out[j] is float[dims_j[mode] x
 *           R_j], row-major, written completely.
 * Asynchronous on the batch stream.
 */
dfacto_status dfacto_batch_mttkrp(dfacto_batch_t* b, int mode, float* const* out);

/*
 * dfacto_batch_als_iter -- one ALS sweep (Algorithm 4: modes 1, 2, 3) for
 * every job, then every job's fit.  The first sweep (and any sweep after a
 * job's factors were changed outside the batch) is issued launch by launch;
 * later sweeps replay the captured graph.
 *   fits    host double[n] or NULL: fit of each job after the sweep (the
 *           call then waits for the sweep).
 * Returns DFACTO_ESINGULAR (informational) if any job's Gamma needed the
 * pseudo-inverse, DFACTO_EINTERNAL if a consistency check failed.
 */
dfacto_status dfacto_batch_als_iter(dfacto_batch_t* b, double* fits);

/* Wait for all work of the batch. */
dfacto_status dfacto_batch_sync(dfacto_batch_t* b);

/* One rank class of a batch: its jobs share rank and factor type. */
typedef struct {
  int32_t rank;
  int32_t factor_dtype;
  int32_t n_jobs;
  int32_t vec;       /* columns per lane of the walk */
  int32_t lanes;     /* lanes per segment (G); a warp walks 32 / lanes segments */
  int32_t seg_nnz;   /* nonzeros per segment */
  int64_t nnz;       /* nonzeros of the class (all its jobs) */
  double tuned_ms;   /* MTTKRP time of the three modes at the chosen shape
                        (0 when not tuned) */
} dfacto_batch_class;

/* Number of rank classes, and class k's description (0 <= k < classes). */
int32_t dfacto_batch_num_classes(const dfacto_batch_t* b);
dfacto_status dfacto_batch_get_class(const dfacto_batch_t* b, int32_t k, dfacto_batch_class* out);

/* Message of the last failure on b (empty if none). */
const char* dfacto_batch_last_error(const dfacto_batch_t* b);

#ifdef __cplusplus
}
#endif

#endif /* DFACTO_H_ */
