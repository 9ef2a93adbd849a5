// internal.h -- private state of a libdfacto handle and the host-side entry
// points of each kernel family.  Not part of the public ABI (include/dfacto.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/dfacto.h"

namespace dfacto {

struct JointState;  // joint.cu

// Lane-group configuration of the MTTKRP walk: each group of G lanes owns one
// segment of the nonzero stream and each lane owns VEC consecutive columns.
struct WalkCfg {
  int vec = 0;    // columns per lane (1, 2, 4, 8)
  int G = 0;      // lanes per group (power of two, G * vec >= R)
  int seg = 0;    // nonzeros per segment (multiple of 32)
  int kernel = 1; // 1: mttkrp_walk, 2: mttkrp_walk2 (fiber ends from a bitmask)
};

constexpr int kWalkWarps = 8;  // warps per MTTKRP CTA

// Largest nonzero count of a tensor (and of a batch's rank class) and largest
// MTTKRP segment: the walks keep nonzero positions in 32-bit integers, and a
// segment end (position + segment length + one lane group) must stay below
// 2^31.
constexpr int64_t kMaxNnz = (int64_t(1) << 31) - (int64_t(1) << 16);
constexpr int kMaxSeg = 4096;

// Flattened CSR copy of one mode (Sec. 3): the nonzero rows of
// (X^{n+1})^T ("fibers") and the fixed pattern of M^r.
struct ModeCSR {
  int o = 0, in = 0, f = 0;    // axes
  int64_t dim_o = 0;
  int64_t nfib = 0;
  int64_t* fiber_ptr = nullptr;  // [dim_o + 1]  row(M^r)
  int32_t* fiber_idx = nullptr;  // [nfib]       col(M^r) = f
  int32_t* fiber_row = nullptr;  // [nfib]       o of each fiber (COO form of row(M^r))
  int64_t* nz_ptr = nullptr;     // [nfib + 1]
  int32_t* nz_idx = nullptr;     // [nnz]        index `in`
  float* nz_val = nullptr;       // [nnz]
  uint32_t* end_bits = nullptr;  // [(nnz + 31) / 32] bit p set iff nonzero p ends its fiber
  WalkCfg cfg;
  int64_t nseg = 0;              // segments of cfg.seg nonzeros
  int32_t* seg_fib = nullptr;    // [nseg] fiber holding the first nonzero of each segment
  int32_t seg_fib_for = 0;       // segment length seg_fib was computed for
};

// Scalar slots in device memory (double).
enum Scalar : int {
  kNormX2 = 0,   // ||X||^2
  kFit,          // last fit
  kInner,        // <X, Xhat>
  kLoss,         // GD objective at the current point
  kAlpha,        // last accepted GD step (alpha_prev)
  kG2,           // ||grad||^2
  kModelNorm2,   // ||Xhat||^2
  kT000, kT100, kT010, kT001, kT110, kT101, kT011, kT111,  // GD trilinear terms
  kStep,         // step applied by the last GD update (0 after a failed search)
  kNumScalars
};

// Integer status flags in device memory.
enum Flag : int {
  kFlagRange = 0,     // coordinate out of range
  kFlagDup,           // duplicate coordinate
  kFlagSingular,      // a pseudo-inverse was used
  kFlagLsFail,        // line search failed
  kFlagInternal,      // internal check failed
  kNumFlags
};

}  // namespace dfacto

struct dfacto_handle {
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;        // Gamma^{-1} beside the MTTKRP (created at build)
  cudaEvent_t aux_fork = nullptr;
  cudaEvent_t aux_join = nullptr;
  int device = 0;
  int32_t dims[3] = {0, 0, 0};
  int64_t nnz = 0;
  int R = 1;
  int dtype = DFACTO_F32;  // factor storage
  double lambda_reg = 0.0;
  dfacto_options opt{};
  dfacto::ModeCSR m[3];
  void* F[3] = {nullptr, nullptr, nullptr};   // factors, storage dtype
  float* N = nullptr;                         // [max dim x R] MTTKRP output scratch
  float* Fh = nullptr;                        // [max dim x R] N Gamma^{-1} before normalisation
  float* grad[3] = {nullptr, nullptr, nullptr};  // GD gradients (lazy)
  double* lambda = nullptr;                   // [R]
  float* inv_lambda = nullptr;                // [R] 1/lambda (1 where lambda = 0)
  double* ipart = nullptr;                    // [blocks x R] partials of <X, Xhat>
  int ipart_blocks = 0;
  double* gram[3] = {nullptr, nullptr, nullptr};  // [R x R] Grams of the stored factors
  bool gram_valid[3] = {false, false, false};
  double* gd_mats = nullptr;                  // [3 x 3 x R x R] P0/P1/P2 per factor
  uint32_t* gd_scratch = nullptr;             // [8] gradient max bits and scales (dual pass)
  double* ls_vals = nullptr;                  // [1 + trials] f(0) and the backtracking trials (lazy)
  double* W = nullptr;                        // [R x R] Gamma^{-1} (FP64)
  double* rr_work = nullptr;                  // [2 R^2 + R] workspace of the R x R solve
  float* W32 = nullptr;                       // [R x R] Gamma^{-1} (FP32)
  double* scal = nullptr;                     // [kNumScalars]
  int32_t* flags = nullptr;                   // [kNumFlags]
  double* partials = nullptr;                 // reduction partials
  int64_t partials_cap = 0;                   // doubles
  float* carry = nullptr;                     // MTTKRP CTA carries [ncta x 2 x walk rank]
  int32_t* carry_row = nullptr;               // [ncta x 4] head row, tail row, slot info
  int64_t carry_cap = 0;                      // CTAs
  int carry_rank = 0;                         // columns of a carry row the buffer holds
  // MTTKRP at a rank that is not a multiple of four: the two gathered factors
  // and the output as zero-padded FP32 rows of a multiple of four columns
  // [max dim x padded rank] each (lazy)
  float* pad_in = nullptr;
  float* pad_f = nullptr;
  float* pad_out = nullptr;
  // the line search's trilinear pass at such a rank: A, B, C and their
  // gradients as padded FP32 rows [(dims[0] + dims[1] + dims[2]) x padded rank x 2] (lazy)
  float* pad_dual = nullptr;
  double* host_scal = nullptr;                // host mirror of scal
  int32_t* host_flags = nullptr;              // host mirror of flags
  int64_t bytes = 0;
  std::string err;
  // Set while the handle is in a batch: F[m] then point into the batch's
  // factor pools and are not the handle's to free.
  dfacto_batch* batch = nullptr;
  // Ratings of the joint model (Appendix F), set by dfacto_joint_set_ratings.
  dfacto::JointState* joint = nullptr;
};

namespace dfacto {

// Kernels launched by this library in this process (dfacto_launch_count).
extern std::atomic<long long> g_launches;
#define DF_COUNT() ::dfacto::g_launches.fetch_add(1, std::memory_order_relaxed)

// ---- errors ---------------------------------------------------------------
dfacto_status fail(dfacto_t* h, dfacto_status s, const std::string& what);
dfacto_status cuda_fail(dfacto_t* h, cudaError_t e, const char* what);
#define DF_CUDA(h, call)                                              \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return ::dfacto::cuda_fail((h), e_, #call); \
  } while (0)

// ---- kernels with more than 48 KB of dynamic shared memory ---------------
// Raise `kernel`'s dynamic shared memory limit to `bytes` on the current
// device, once per (kernel, device, size) and thread-safe (the attribute is a
// per-device setting).  No-op at or below the default 48 KB.
cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes);

// ---- memory ---------------------------------------------------------------
dfacto_status dalloc(dfacto_t* h, void** p, size_t bytes);
void dfree(dfacto_t* h, void* p, size_t bytes);
bool is_device_ptr(const void* p);
dfacto_status grow_partials(dfacto_t* h, int64_t doubles);

// ---- scan (scan.cu) -------------------------------------------------------
// Exclusive prefix sum of n int32 values (n < 2^31), out may alias in.
// Temporary storage is taken with cudaMallocAsync on `s`.
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);

// ---- build (build.cu) -----------------------------------------------------
dfacto_status build_modes(dfacto_t* h, const int32_t* d_idx, const float* d_val);
// Stable LSD radix sort of (key, payload) pairs by key bits [lo_bit, hi_bit);
// the result is in (k0, v0), or in (k1, v1) when *in_alt is set.
cudaError_t sort_pairs64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                         int lo_bit, int hi_bit, cudaStream_t s, bool* in_alt);
dfacto_status ensure_segments(dfacto_t* h, int mode);

// ---- MTTKRP (mttkrp*.cu) --------------------------------------------------
WalkCfg choose_walk(int R, int dtype, int64_t nnz, int64_t nfib, int seg_opt, int vec_opt);
// Rank the MTTKRP walk runs at: R, or R rounded up to a multiple of four (the
// factors then gathered from zero-padded FP32 copies) when R > 2 is not one
// and no lane width was asked for.
int walk_rank(int R, int vec_opt);
// dst[r, c] = src[r, c] for c < R, 0 for R <= c < RP (FP32 rows of RP columns).
cudaError_t pad_factor_rows(const void* src, int src_dtype, int64_t rows, int R, int RP, float* dst,
                            cudaStream_t s);
dfacto_status mttkrp_launch(dfacto_t* h, int mode, float* out);

// ---- batches (batch.cu, dense.cu) -----------------------------------------
// One job of a batch for one mode, as the batched R x R and row kernels see
// it: the pointers the per-job kernels would take from the job's handle.
struct DenseJob {
  const double* Gf;        // Gram of factor f
  const double* Gi;        // Gram of factor in
  double lambda_reg;
  double* W;               // Gamma^{-1} (FP64), [R x R]
  float* W32;              // Gamma^{-1} (FP32)
  int32_t* singular;       // the job's singular flag
  double* rr_work;         // R x R solve workspace
  const float* N;          // MTTKRP output rows of the job, [rows x R]
  int64_t rows;            // dims[mode]
  int nb;                  // row blocks of the row passes
  float* Fh;               // N Gamma^{-1} (R > 32 only)
  double* partials;        // per-block partials
  double* lambda;          // [R]
  float* inv_lambda;       // [R]
  void* F;                 // the factor of this mode (storage type)
  double* gram_out;        // Gram of the new factor
  double* ipart;           // partials of <X, Xhat> (mode 3)
  const double* GA;        // Grams of the three factors (fit)
  const double* GB;
  const double* GC;
  double* scal;            // the job's scalars
};
int dense_row_blocks(int64_t rows, int R);  // blocks of the row passes of one mode
// Batched steps of one rank class (all jobs share R and the factor type):
// Gamma^{-1} of every job; N Gamma^{-1}, normalisation, store and Gram (and on
// the last mode the fit's inner product); the fit.  begin[j] is the first row
// block of job j (prefix sums of nb, begin[n] = total).
cudaError_t batch_gamma_inverse(const DenseJob* jobs, int n, int R, cudaStream_t s);
cudaError_t batch_als_post(const DenseJob* jobs, const int32_t* begin, int n, int total_blocks, int R,
                           int dtype, bool last, cudaStream_t s);
cudaError_t batch_fit(const DenseJob* jobs, int n, int R, cudaStream_t s);

// Called by dfacto_destroy for a handle still in a batch: the batch drops it.
void batch_forget(dfacto_batch* b, dfacto_t* h);

// Frees the joint model's ratings and buffers (joint.cu); called by dfacto_destroy.
void joint_free(dfacto_t* h);

// ---- dense R x R and row-wise kernels (dense.cu) --------------------------
dfacto_status gram_of_factor(dfacto_t* h, int m);
dfacto_status als_mode(dfacto_t* h, int mode);
dfacto_status als_pre(dfacto_t* h, int mode);
dfacto_status als_post(dfacto_t* h, int mode, float* N);
dfacto_status als_fit(dfacto_t* h);
dfacto_status fit_direct(dfacto_t* h);
dfacto_status gd_step(dfacto_t* h);
dfacto_status convert_factor_in(dfacto_t* h, int m, const void* src, int src_dtype);
dfacto_status convert_factor_out(dfacto_t* h, int m, void* dst, int dst_dtype);
dfacto_status norm_x2(dfacto_t* h);
// GD pieces shared with the joint model (joint.cu): the R x R matrices of the
// search ray (P0, P1, P2 per factor from h->F and h->grad), the line search
// on the ray (tensor term weighted by mu, plus the ratings quartic ycoef[0..4]
// when non-null; step into scal[kStep]), and theta <- theta - step grad.
dfacto_status ray_matrices(dfacto_t* h);
dfacto_status line_search(dfacto_t* h, double mu, const double* ycoef);
dfacto_status apply_step(dfacto_t* h);
dfacto_status dual_pass(dfacto_t* h);  // T110, T101, T011, T111 of the ray (dual.cu)

}  // namespace dfacto
