// batch.cu -- many independent decompositions advanced together.
//
// Jobs that share (R, factor type) form a rank class.  A class is one
// block-diagonal tensor: the flattened CSR copies of its jobs (Sec. 3) are
// concatenated with every index offset by the job's position in the class
// (rows of mode o, columns `in` and `f` by the running sums of the earlier
// jobs' dimensions), and the factors of each mode sit in one pool in the same
// order.  The MTTKRP of Algorithm 1 over the class is then exactly the
// MTTKRPs of its jobs stacked: a nonzero of job j only ever reads rows of job
// j's factors and writes rows of job j's output.  The walk of every class of
// one factor type runs in one persistent launch (mttkrp_walk2_multi).
//
// The R x R and row steps of Algorithm 2 run once per rank class as batched
// launches (each block finds its job and runs that job's step); from the
// second sweep on the whole sweep is one CUDA graph.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mttkrp.cuh"

struct dfacto_batch;

namespace dfacto {
namespace {

constexpr int kTuneSegs[] = {64, 128, 256};

__global__ void copy_add_i32(const int32_t* __restrict__ src, int64_t n, int32_t add,
                             int32_t* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = src[i] + add;
}

__global__ void copy_add_i64(const int64_t* __restrict__ src, int64_t n, int64_t add,
                             int64_t* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = src[i] + add;
}

__global__ void set_i64(int64_t* p, int64_t v) { *p = v; }

// Zero the status flags of every job (the start of a sweep).
__global__ void zero_job_flags(int32_t* const* __restrict__ flags, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kNumFlags; i += gridDim.x * blockDim.x)
    flags[i / kNumFlags][i % kNumFlags] = 0;
}

// Collect every job's fit and flags into one array each (one read-back).
__global__ void gather_results(double* const* __restrict__ scal, int32_t* const* __restrict__ flags,
                               int n, const int32_t* __restrict__ bad, double* __restrict__ fits,
                               int32_t* __restrict__ status) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    fits[j] = scal[j][kFit];
    status[j] = (flags[j][kFlagSingular] ? 1 : 0) | (flags[j][kFlagInternal] || *bad ? 2 : 0);
  }
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

size_t elem_bytes(int dtype) { return dtype == DFACTO_BF16 ? 2 : 4; }


int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct ClassMode {
  int64_t dim_o = 0, nfib = 0;
  int64_t* fiber_ptr = nullptr;  // [dim_o + 1]
  int32_t* fiber_idx = nullptr;  // [nfib]
  int32_t* fiber_row = nullptr;  // [nfib]
  int64_t* nz_ptr = nullptr;     // [nfib + 1]
  int32_t* nz_idx = nullptr;     // [nnz]
  float* nz_val = nullptr;       // [nnz]
  uint32_t* end_bits = nullptr;  // [(nnz + 31) / 32]
  int32_t* seg_fib = nullptr;    // [nseg_cap]
  float* N = nullptr;            // [dim_o x R] MTTKRP output of every job of the class
};

struct BatchClass {
  int R = 0, dtype = DFACTO_F32;
  std::vector<int> jobs;           // batch job indices, in class order
  std::vector<int64_t> off[3];     // per job: first row in the pools of mode m
  int64_t rows[3] = {0, 0, 0};     // pool rows per mode
  int64_t nnz = 0;
  std::vector<int64_t> nnz_off, fib_off[3];
  void* F[3] = {nullptr, nullptr, nullptr};  // factor pools [rows[m] x R]
  ClassMode m[3];
  WalkCfg cfg;
  int shape = -1;                  // multi shape id (-1: own launch)
  int64_t nseg_cap = 0;            // seg_fib capacity (segments)
  float* carry = nullptr;          // [carry_cap x 2 x R]
  int32_t* carry_row = nullptr;    // [carry_cap x 2]
  int64_t carry_cap = 0;           // CTAs
  double tuned_ms = 0.0;
  DenseJob* dense[3] = {nullptr, nullptr, nullptr};  // device [jobs] per mode
  int32_t* begin[3] = {nullptr, nullptr, nullptr};   // device [jobs + 1] first row block
  int total_blocks[3] = {0, 0, 0};
  std::vector<int> nb[3];                            // row blocks per job and mode

  int segs() const { return kWalkWarps * (32 / cfg.G); }
  int64_t ncta() const {
    const int64_t P = (int64_t)segs() * cfg.seg;
    return (nnz + P - 1) / P;
  }
};

}  // namespace
}  // namespace dfacto

struct dfacto_batch {
  int device = 0;
  int sms = 152;
  std::vector<dfacto_t*> jobs;
  std::vector<dfacto::BatchClass> cls;
  cudaStream_t user = nullptr;   // the caller's stream
  cudaStream_t main = nullptr;
  cudaStream_t side = nullptr;   // Gamma^{-1} of the next mode, beside the MTTKRP
  cudaEvent_t side_ev = nullptr;
  cudaEvent_t fork_ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ready = false;
  int64_t graph_kernels = 0;     // kernels launched by one replay of the graph
  bool broken = false;
  int64_t sweeps = 0;
  dfacto_batch_options opt{};
  double** d_scal = nullptr;     // [n] per-job scalar arrays
  int32_t** d_flags = nullptr;   // [n] per-job flag arrays
  double* d_fits = nullptr;      // [n]
  int32_t* d_status = nullptr;   // [n]
  int32_t* d_bad = nullptr;      // fix-up consistency flag
  double* h_fits = nullptr;      // host [n]
  int32_t* h_status = nullptr;   // host [n]
  std::vector<void*> owned;      // device allocations of the batch
  std::string err;
};

namespace dfacto {
namespace {

dfacto_status bfail(dfacto_batch* b, dfacto_status s, const std::string& what) {
  b->err = what;
  return s;
}

dfacto_status bcuda(dfacto_batch* b, cudaError_t e, const char* what) {
  b->err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? DFACTO_ENOMEM : DFACTO_ECUDA;
}

#define DB_CUDA(b, call)                                 \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bcuda((b), e_, #call); \
  } while (0)

// Batch memory comes from the device's stream-ordered pool, on the batch's
// main stream (freed there when the batch is destroyed).
template <typename P>
dfacto_status balloc(dfacto_batch* b, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(bytes, 16), b->main);
  if (e != cudaSuccess) {
    *p = nullptr;
    return bcuda(b, e, "cudaMalloc (batch)");
  }
  b->owned.push_back(q);
  *p = static_cast<P*>(q);
  return DFACTO_OK;
}

// ---- construction ----------------------------------------------------------

// Concatenate the CSR copies of mode `mode` of the class's jobs.
dfacto_status build_class_mode(dfacto_batch* b, BatchClass& C, int mode) {
  cudaStream_t s = b->main;
  const int o = mode, in = (mode + 1) % 3, f = (mode + 2) % 3;
  ClassMode& M = C.m[mode];
  M.dim_o = C.rows[o];
  M.nfib = 0;
  C.fib_off[mode].assign(C.jobs.size(), 0);
  for (size_t t = 0; t < C.jobs.size(); ++t) {
    C.fib_off[mode][t] = M.nfib;
    M.nfib += b->jobs[C.jobs[t]]->m[mode].nfib;
  }
  if (M.nfib >= (int64_t(1) << 31)) return bfail(b, DFACTO_EINVAL, "rank class has 2^31 fibers or more");
  dfacto_status st;
  if ((st = balloc(b, &M.fiber_ptr, sizeof(int64_t) * (size_t)(M.dim_o + 1))) != DFACTO_OK) return st;
  if ((st = balloc(b, &M.fiber_idx, sizeof(int32_t) * (size_t)M.nfib)) != DFACTO_OK) return st;
  if ((st = balloc(b, &M.fiber_row, sizeof(int32_t) * (size_t)M.nfib)) != DFACTO_OK) return st;
  if ((st = balloc(b, &M.nz_ptr, sizeof(int64_t) * (size_t)(M.nfib + 1))) != DFACTO_OK) return st;
  if ((st = balloc(b, &M.nz_idx, sizeof(int32_t) * (size_t)C.nnz)) != DFACTO_OK) return st;
  if ((st = balloc(b, &M.nz_val, sizeof(float) * (size_t)C.nnz)) != DFACTO_OK) return st;
  if ((st = balloc(b, &M.end_bits, sizeof(uint32_t) * (size_t)((C.nnz + 31) / 32))) != DFACTO_OK) return st;
  if ((st = balloc(b, &M.N, sizeof(float) * (size_t)M.dim_o * C.R)) != DFACTO_OK) return st;
  for (size_t t = 0; t < C.jobs.size(); ++t) {
    const dfacto_t* h = b->jobs[C.jobs[t]];
    const ModeCSR& J = h->m[mode];
    const int64_t ro = C.off[o][t], rf = C.off[f][t], ri = C.off[in][t];
    const int64_t q0 = C.fib_off[mode][t], p0 = C.nnz_off[t];
    // fiber_ptr rows of this job (its last entry is the next job's first)
    copy_add_i64<<<grid_of(J.dim_o), 256, 0, s>>>(J.fiber_ptr, J.dim_o, q0, M.fiber_ptr + ro);
    DF_COUNT();
    if (J.nfib > 0) {
      copy_add_i32<<<grid_of(J.nfib), 256, 0, s>>>(J.fiber_idx, J.nfib, (int32_t)rf, M.fiber_idx + q0);
      DF_COUNT();
      copy_add_i32<<<grid_of(J.nfib), 256, 0, s>>>(J.fiber_row, J.nfib, (int32_t)ro, M.fiber_row + q0);
      DF_COUNT();
      copy_add_i64<<<grid_of(J.nfib), 256, 0, s>>>(J.nz_ptr, J.nfib, p0, M.nz_ptr + q0);
      DF_COUNT();
    }
    if (h->nnz > 0) {
      copy_add_i32<<<grid_of(h->nnz), 256, 0, s>>>(J.nz_idx, h->nnz, (int32_t)ri, M.nz_idx + p0);
      DF_COUNT();
      DB_CUDA(b, cudaMemcpyAsync(M.nz_val + p0, J.nz_val, sizeof(float) * (size_t)h->nnz,
                                 cudaMemcpyDeviceToDevice, s));
    }
    DB_CUDA(b, cudaGetLastError());
  }
  set_i64<<<1, 1, 0, s>>>(M.fiber_ptr + M.dim_o, M.nfib);
  DF_COUNT();
  set_i64<<<1, 1, 0, s>>>(M.nz_ptr + M.nfib, C.nnz);
  DF_COUNT();
  DB_CUDA(b, cudaGetLastError());
  DB_CUDA(b, launch_fiber_end_bits(M.nz_ptr, M.nfib, C.nnz, M.end_bits, s));
  return DFACTO_OK;
}

// Segment starts and carry room for the class's current walk configuration.
dfacto_status prepare_walk(dfacto_batch* b, BatchClass& C) {
  const int64_t nseg = (C.nnz + C.cfg.seg - 1) / C.cfg.seg;
  if (nseg > C.nseg_cap) return bfail(b, DFACTO_EINTERNAL, "segment table too small");
  if (C.ncta() > C.carry_cap) return bfail(b, DFACTO_EINTERNAL, "carry table too small");
  for (int mode = 0; mode < 3; ++mode)
    DB_CUDA(b, launch_segment_starts(C.m[mode].nz_ptr, C.m[mode].nfib, nseg, C.cfg.seg,
                                     C.m[mode].seg_fib, b->main));
  return DFACTO_OK;
}

MttkrpParams class_params(const BatchClass& C, int mode, int32_t* bad) {
  (void)bad;
  const ClassMode& M = C.m[mode];
  MttkrpParams a;
  a.fiber_ptr = M.fiber_ptr;
  a.fiber_idx = M.fiber_idx;
  a.fiber_row = M.fiber_row;
  a.nz_ptr = M.nz_ptr;
  a.nz_idx = M.nz_idx;
  a.nz_val = M.nz_val;
  a.seg_fib = M.seg_fib;
  a.end_bits = M.end_bits;
  a.Fin = C.F[(mode + 1) % 3];
  a.Ff = C.F[(mode + 2) % 3];
  a.out = M.N;
  a.carry = C.carry;
  a.carry_row = C.carry_row;
  a.nnz = C.nnz;
  a.nfib = M.nfib;
  a.dim_o = M.dim_o;
  a.R = C.R;
  a.seg = C.cfg.seg;
  return a;
}

// MTTKRP of `mode` for the classes in `which` (all classes if empty): the
// classes with a compiled multi shape share one persistent launch per factor
// type (kMaxClasses at a time), the others get their own walk; then one
// fix-up per class.
dfacto_status batch_mttkrp_issue(dfacto_batch* b, int mode, cudaStream_t s,
                                 const std::vector<int>& which) {
  std::vector<int> ks = which;
  if (ks.empty())
    for (int k = 0; k < (int)b->cls.size(); ++k) ks.push_back(k);
  for (int dtype : {DFACTO_F32, DFACTO_BF16}) {
    std::vector<int> multi;
    for (int k : ks) {
      const BatchClass& C = b->cls[k];
      if (C.dtype != dtype || C.nnz == 0) continue;
      if (C.shape >= 0) {
        multi.push_back(k);
      } else {
        const MttkrpParams a = class_params(C, mode, b->d_bad);
        cudaError_t e = dtype == DFACTO_BF16
                            ? launch_walk2<__nv_bfloat16>(C.cfg.vec, C.cfg.G, a, C.ncta(), s)
                            : launch_walk2<float>(C.cfg.vec, C.cfg.G, a, C.ncta(), s);
        if (e != cudaSuccess) return bcuda(b, e, "batched walk (own launch)");
      }
    }
    for (size_t i0 = 0; i0 < multi.size(); i0 += kMaxClasses) {
      MultiWalkParams mp;
      std::memset(&mp, 0, sizeof(mp));
      size_t smem = 0;
      int total = 0;
      mp.nclass = (int)std::min<size_t>(kMaxClasses, multi.size() - i0);
      for (int c = 0; c < mp.nclass; ++c) {
        const BatchClass& C = b->cls[multi[i0 + c]];
        mp.p[c] = class_params(C, mode, b->d_bad);
        mp.shape[c] = C.shape;
        mp.cta_begin[c] = total;
        total += (int)C.ncta();
        smem = std::max(smem, walk2_smem_bytes(C.cfg.vec, C.cfg.G, C.R));
      }
      mp.cta_begin[mp.nclass] = total;
      for (int c = mp.nclass + 1; c <= kMaxClasses; ++c) mp.cta_begin[c] = total;
      // Persistent grid: as many blocks as stay resident (3 per SM at 80
      // registers, fewer if shared memory limits them).
      const int per_sm = std::max<int>(1, std::min<int>(3, (int)((228 * 1024) / (smem + 2048 + 1024))));
      const int grid = std::min(total, b->sms * per_sm);
      cudaError_t e = dtype == DFACTO_BF16 ? launch_walk2_multi<__nv_bfloat16>(mp, smem, grid, s)
                                           : launch_walk2_multi<float>(mp, smem, grid, s);
      if (e != cudaSuccess) return bcuda(b, e, "batched walk");
    }
  }
  for (int k : ks) {
    const BatchClass& C = b->cls[k];
    const int64_t P = (int64_t)C.segs() * C.cfg.seg;
    DB_CUDA(b, launch_mttkrp_fixup(C.carry_row, C.carry, C.m[mode].fiber_ptr, C.m[mode].nz_ptr,
                                   C.m[mode].N, C.R, P, C.nnz > 0 ? C.ncta() : 0, C.m[mode].dim_o,
                                   b->d_bad, s));
  }
  return DFACTO_OK;
}

// Time the MTTKRP of the three modes of class k (mean of `reps` calls each).
dfacto_status time_class(dfacto_batch* b, int k, int reps, double* ms) {
  cudaEvent_t e0, e1;
  DB_CUDA(b, cudaEventCreate(&e0));
  DB_CUDA(b, cudaEventCreate(&e1));
  dfacto_status st = DFACTO_OK;
  double total = 0.0;
  for (int mode = 0; mode < 3 && st == DFACTO_OK; ++mode) {
    st = batch_mttkrp_issue(b, mode, b->main, {k});  // warm-up
    if (st != DFACTO_OK) break;
    cudaEventRecord(e0, b->main);
    for (int r = 0; r < reps && st == DFACTO_OK; ++r) st = batch_mttkrp_issue(b, mode, b->main, {k});
    cudaEventRecord(e1, b->main);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = bcuda(b, cudaGetLastError(), "autotune timing");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    total += t / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = total;
  return st;
}

// Candidate walk configurations of class C: columns per lane (the R tile of a
// lane) and nonzeros per segment; the lanes per segment follow from R.
std::vector<WalkCfg> candidates(const BatchClass& C) {
  std::vector<WalkCfg> out;
  for (int vec : {4, 8}) {
    if (C.R % vec != 0) continue;
    const int G = next_pow2((C.R + vec - 1) / vec);
    if (G > 32 || multi_shape_id(vec, G) < 0) continue;
    for (int seg : kTuneSegs) {
      WalkCfg c;
      c.vec = vec;
      c.G = G;
      c.seg = seg;
      c.kernel = 2;
      out.push_back(c);
    }
  }
  return out;
}

dfacto_status autotune_class(dfacto_batch* b, int k) {
  BatchClass& C = b->cls[k];
  const std::vector<WalkCfg> cands = candidates(C);
  if (cands.size() < 2 || C.nnz == 0) return DFACTO_OK;
  WalkCfg best = C.cfg;
  double best_ms = 1e300;
  for (const WalkCfg& c : cands) {
    C.cfg = c;
    C.shape = multi_shape_id(c.vec, c.G);
    dfacto_status st = prepare_walk(b, C);
    if (st != DFACTO_OK) return st;
    double ms = 0;
    if ((st = time_class(b, k, 3, &ms)) != DFACTO_OK) return st;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  C.cfg = best;
  C.shape = multi_shape_id(best.vec, best.G);
  C.tuned_ms = best_ms;
  return prepare_walk(b, C);
}

// ---- the sweep ---------------------------------------------------------------

// Per-job pointers of every class and mode for the batched dense kernels.
dfacto_status build_dense_tables(dfacto_batch* b) {
  for (BatchClass& C : b->cls) {
    const int n = (int)C.jobs.size();
    for (int mode = 0; mode < 3; ++mode) {
      const int in = (mode + 1) % 3, f = (mode + 2) % 3;
      std::vector<DenseJob> tab(n);
      std::vector<int32_t> begin(n + 1, 0);
      C.nb[mode].assign(n, 0);
      for (int t = 0; t < n; ++t) {
        dfacto_t* h = b->jobs[C.jobs[t]];
        DenseJob& J = tab[t];
        J.Gf = h->gram[f];
        J.Gi = h->gram[in];
        J.lambda_reg = h->lambda_reg;
        J.W = h->W;
        J.W32 = h->W32;
        J.singular = h->flags + kFlagSingular;
        J.rr_work = h->rr_work;
        J.N = C.m[mode].N + (size_t)C.off[mode][t] * C.R;
        J.rows = h->dims[mode];
        J.nb = dense_row_blocks(J.rows, C.R);
        J.Fh = h->Fh;
        J.partials = h->partials;
        J.lambda = h->lambda;
        J.inv_lambda = h->inv_lambda;
        J.F = h->F[mode];
        J.gram_out = h->gram[mode];
        J.ipart = h->ipart;
        J.GA = h->gram[0];
        J.GB = h->gram[1];
        J.GC = h->gram[2];
        J.scal = h->scal;
        C.nb[mode][t] = J.nb;
        begin[t + 1] = begin[t] + J.nb;
      }
      C.total_blocks[mode] = begin[n];
      dfacto_status st;
      if ((st = balloc(b, &C.dense[mode], sizeof(DenseJob) * (size_t)n)) != DFACTO_OK) return st;
      if ((st = balloc(b, &C.begin[mode], sizeof(int32_t) * (size_t)(n + 1))) != DFACTO_OK) return st;
      DB_CUDA(b, cudaMemcpy(C.dense[mode], tab.data(), sizeof(DenseJob) * (size_t)n, cudaMemcpyHostToDevice));
      DB_CUDA(b, cudaMemcpy(C.begin[mode], begin.data(), sizeof(int32_t) * (size_t)(n + 1),
                            cudaMemcpyHostToDevice));
    }
  }
  return DFACTO_OK;
}

// Issue one ALS sweep of every job plus its fit, ending on b->main.  Per mode:
// Gamma^{-1} of every job (side stream) beside the MTTKRP of every class
// (main), then N Gamma^{-1}, normalisation, store and Gram, one launch per step
// and rank class.
dfacto_status issue_sweep(dfacto_batch* b) {
  const int n = (int)b->jobs.size();
  zero_job_flags<<<grid_of((int64_t)n * kNumFlags), 256, 0, b->main>>>(b->d_flags, n);
  DF_COUNT();
  // Grams of factors set from outside the batch (only before the graph exists).
  for (int j = 0; j < n; ++j) {
    dfacto_t* h = b->jobs[j];
    bool missing = false;
    for (int m = 0; m < 3; ++m) missing = missing || !h->gram_valid[m];
    if (!missing) continue;
    cudaStream_t saved = h->stream;
    h->stream = b->main;
    dfacto_status st = DFACTO_OK;
    for (int m = 0; m < 3 && st == DFACTO_OK; ++m)
      if (!h->gram_valid[m]) st = gram_of_factor(h, m);
    h->stream = saved;
    if (st != DFACTO_OK) {
      b->err = "job " + std::to_string(j) + ": " + h->err;
      return st;
    }
  }
  for (int mode = 0; mode < 3; ++mode) {
    DB_CUDA(b, cudaEventRecord(b->fork_ev, b->main));
    DB_CUDA(b, cudaStreamWaitEvent(b->side, b->fork_ev, 0));
    for (const BatchClass& C : b->cls)
      DB_CUDA(b, batch_gamma_inverse(C.dense[mode], (int)C.jobs.size(), C.R, b->side));
    dfacto_status st = batch_mttkrp_issue(b, mode, b->main, {});
    if (st != DFACTO_OK) {
      cudaEventRecord(b->side_ev, b->side);  // rejoin before returning
      cudaStreamWaitEvent(b->main, b->side_ev, 0);
      return st;
    }
    DB_CUDA(b, cudaEventRecord(b->side_ev, b->side));
    DB_CUDA(b, cudaStreamWaitEvent(b->main, b->side_ev, 0));
    for (BatchClass& C : b->cls) {
      DB_CUDA(b, batch_als_post(C.dense[mode], C.begin[mode], (int)C.jobs.size(), C.total_blocks[mode],
                                C.R, C.dtype, mode == 2, b->main));
      for (size_t t = 0; t < C.jobs.size(); ++t) {
        dfacto_t* h = b->jobs[C.jobs[t]];
        h->gram_valid[mode] = true;
        if (mode == 2) h->ipart_blocks = C.nb[2][t];
      }
    }
  }
  for (const BatchClass& C : b->cls) DB_CUDA(b, batch_fit(C.dense[2], (int)C.jobs.size(), C.R, b->main));
  gather_results<<<grid_of(n), 256, 0, b->main>>>(b->d_scal, b->d_flags, n, b->d_bad, b->d_fits,
                                                  b->d_status);
  DF_COUNT();
  DB_CUDA(b, cudaGetLastError());
  return DFACTO_OK;
}

void drop_graph(dfacto_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_ready = false;
}

// Order the batch after the jobs' own streams and the caller's stream.
dfacto_status enter(dfacto_batch* b) {
  if (b->broken) return bfail(b, DFACTO_EINVAL, "a job of this batch was destroyed");
  for (dfacto_t* h : b->jobs) DB_CUDA(b, cudaStreamSynchronize(h->stream));
  DB_CUDA(b, cudaEventRecord(b->fork_ev, b->user));
  DB_CUDA(b, cudaStreamWaitEvent(b->main, b->fork_ev, 0));
  return DFACTO_OK;
}

void release(dfacto_batch* b) {
  for (void* p : b->owned) cudaFreeAsync(p, b->main);
  b->owned.clear();
  if (b->main) cudaStreamSynchronize(b->main);
  drop_graph(b);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->side_ev) cudaEventDestroy(b->side_ev);
  b->side = nullptr;
  b->side_ev = nullptr;
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->main) cudaStreamDestroy(b->main);
  delete[] b->h_fits;
  delete[] b->h_status;
  b->fork_ev = nullptr;
  b->main = nullptr;
  b->h_fits = nullptr;
  b->h_status = nullptr;
  cudaGetLastError();
}

// Give every job its factors back in allocations of its own (allocated and
// copied on the job's stream, after the batch's work).
void unpool(dfacto_batch* b) {
  if (b->main) cudaStreamSynchronize(b->main);
  for (BatchClass& C : b->cls) {
    for (size_t t = 0; t < C.jobs.size(); ++t) {
      dfacto_t* h = b->jobs[C.jobs[t]];
      if (!h) continue;
      for (int m = 0; m < 3; ++m) {
        const size_t bytes = elem_bytes(C.dtype) * (size_t)h->dims[m] * C.R;
        void* p = nullptr;
        if (dalloc(h, &p, bytes) == DFACTO_OK) {
          cudaMemcpyAsync(p, h->F[m], bytes, cudaMemcpyDeviceToDevice, h->stream);
          h->F[m] = p;
        } else {
          h->F[m] = nullptr;  // out of memory: the job has lost its factors
        }
      }
      h->batch = nullptr;
    }
  }
  for (dfacto_t* h : b->jobs)
    if (h) cudaStreamSynchronize(h->stream);
}

}  // namespace

void batch_forget(dfacto_batch* b, dfacto_t* h) {
  for (dfacto_t*& j : b->jobs)
    if (j == h) j = nullptr;
  b->broken = true;
}

}  // namespace dfacto

using namespace dfacto;

extern "C" {

void dfacto_batch_options_init(dfacto_batch_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->use_graph = 1;
  opt->autotune = 1;
}

dfacto_status dfacto_batch_create(dfacto_t* const* jobs, int32_t n, const dfacto_batch_options* opt_in,
                                  void* stream, dfacto_batch_t** out) {
  if (!out) return DFACTO_EINVAL;
  *out = nullptr;
  if (!jobs || n < 1 || n > 65536) return DFACTO_EINVAL;
  dfacto_batch_options opt;
  if (opt_in) opt = *opt_in;
  else dfacto_batch_options_init(&opt);
  for (int j = 0; j < n; ++j)
    if (!jobs[j] || jobs[j]->batch) return DFACTO_EINVAL;
  {
    std::vector<dfacto_t*> sorted(jobs, jobs + n);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return DFACTO_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DFACTO_ECUDA;
  for (int j = 0; j < n; ++j)
    if (jobs[j]->device != dev) return DFACTO_EINVAL;
  dfacto_batch* b = new (std::nothrow) dfacto_batch();
  if (!b) return DFACTO_ENOMEM;
  b->device = dev;
  b->opt = opt;
  b->user = static_cast<cudaStream_t>(stream);
  b->jobs.assign(jobs, jobs + n);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  auto bail = [&](dfacto_status st) {
    release(b);
    delete b;
    return st;
  };
  if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->side_ev, cudaEventDisableTiming) != cudaSuccess)
    return bail(DFACTO_ECUDA);
  for (dfacto_t* h : b->jobs)
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(DFACTO_ECUDA);

  // Rank classes: jobs with equal (R, factor type), in job order; a class is
  // closed before its nonzeros would pass kMaxNnz or its pool rows 2^31 - 1.
  const int64_t kRowLimit = (int64_t(1) << 31) - 1;
  for (int j = 0; j < n; ++j) {
    const dfacto_t* h = b->jobs[j];
    int k = -1;
    for (int c = (int)b->cls.size() - 1; c >= 0; --c) {
      const BatchClass& C = b->cls[c];
      if (C.R != h->R || C.dtype != h->dtype) continue;
      bool fits = C.nnz + h->nnz <= kMaxNnz;
      for (int m = 0; m < 3; ++m) fits = fits && C.rows[m] + h->dims[m] <= kRowLimit;
      if (fits) k = c;
      break;
    }
    if (k < 0) {
      b->cls.emplace_back();
      k = (int)b->cls.size() - 1;
      b->cls[k].R = h->R;
      b->cls[k].dtype = h->dtype;
    }
    BatchClass& C = b->cls[k];
    C.jobs.push_back(j);
    C.nnz_off.push_back(C.nnz);
    C.nnz += h->nnz;
    for (int m = 0; m < 3; ++m) {
      C.off[m].push_back(C.rows[m]);
      C.rows[m] += h->dims[m];
    }
  }

  dfacto_status st;
  for (BatchClass& C : b->cls) {
    const size_t es = elem_bytes(C.dtype);
    for (int m = 0; m < 3; ++m)
      if ((st = balloc(b, &C.F[m], es * (size_t)C.rows[m] * C.R)) != DFACTO_OK) return bail(st);
    for (int mode = 0; mode < 3; ++mode)
      if ((st = build_class_mode(b, C, mode)) != DFACTO_OK) return bail(st);
    // Walk configuration: the single-tensor default, then (optionally) tuned.
    C.cfg = choose_walk(C.R, C.dtype, C.nnz, C.m[0].nfib, 0, 0);
    C.cfg.kernel = 2;
    C.shape = multi_shape_id(C.cfg.vec, C.cfg.G);
    int min_seg = C.cfg.seg;
    int64_t min_P = (int64_t)C.segs() * C.cfg.seg;
    for (const WalkCfg& c : candidates(C)) {
      min_seg = std::min(min_seg, c.seg);
      min_P = std::min<int64_t>(min_P, (int64_t)kWalkWarps * (32 / c.G) * c.seg);
    }
    C.nseg_cap = (C.nnz + min_seg - 1) / min_seg;
    C.carry_cap = (C.nnz + min_P - 1) / min_P;
    for (int mode = 0; mode < 3; ++mode)
      if ((st = balloc(b, &C.m[mode].seg_fib, sizeof(int32_t) * (size_t)C.nseg_cap)) != DFACTO_OK)
        return bail(st);
    if ((st = balloc(b, &C.carry, sizeof(float) * 2 * (size_t)C.R * C.carry_cap)) != DFACTO_OK) return bail(st);
    if ((st = balloc(b, &C.carry_row, sizeof(int32_t) * 2 * (size_t)C.carry_cap)) != DFACTO_OK) return bail(st);
    if ((st = prepare_walk(b, C)) != DFACTO_OK) return bail(st);
  }
  if ((st = balloc(b, &b->d_scal, sizeof(double*) * n)) != DFACTO_OK) return bail(st);
  if ((st = balloc(b, &b->d_flags, sizeof(int32_t*) * n)) != DFACTO_OK) return bail(st);
  if ((st = balloc(b, &b->d_fits, sizeof(double) * n)) != DFACTO_OK) return bail(st);
  if ((st = balloc(b, &b->d_status, sizeof(int32_t) * n)) != DFACTO_OK) return bail(st);
  if ((st = balloc(b, &b->d_bad, sizeof(int32_t))) != DFACTO_OK) return bail(st);
  b->h_fits = new (std::nothrow) double[n]();
  b->h_status = new (std::nothrow) int32_t[n]();
  if (!b->h_fits || !b->h_status) return bail(DFACTO_ENOMEM);
  {
    std::vector<double*> sc(n);
    std::vector<int32_t*> fl(n);
    for (int j = 0; j < n; ++j) {
      sc[j] = b->jobs[j]->scal;
      fl[j] = b->jobs[j]->flags;
    }
    if (cudaMemcpy(b->d_scal, sc.data(), sizeof(double*) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_flags, fl.data(), sizeof(int32_t*) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemsetAsync(b->d_bad, 0, sizeof(int32_t), b->main) != cudaSuccess)
      return bail(DFACTO_ECUDA);
  }
  // Move the factors into the pools.
  for (BatchClass& C : b->cls) {
    const size_t es = elem_bytes(C.dtype);
    for (size_t t = 0; t < C.jobs.size(); ++t) {
      const dfacto_t* h = b->jobs[C.jobs[t]];
      for (int m = 0; m < 3; ++m)
        if (cudaMemcpyAsync(static_cast<char*>(C.F[m]) + es * (size_t)C.off[m][t] * C.R, h->F[m],
                            es * (size_t)h->dims[m] * C.R, cudaMemcpyDeviceToDevice, b->main) != cudaSuccess)
          return bail(DFACTO_ECUDA);
    }
  }
  if (cudaStreamSynchronize(b->main) != cudaSuccess) return bail(DFACTO_ECUDA);
  for (BatchClass& C : b->cls) {
    const size_t es = elem_bytes(C.dtype);
    for (size_t t = 0; t < C.jobs.size(); ++t) {
      dfacto_t* h = b->jobs[C.jobs[t]];
      for (int m = 0; m < 3; ++m) {
        dfree(h, h->F[m], es * (size_t)h->dims[m] * C.R);
        h->F[m] = static_cast<char*>(C.F[m]) + es * (size_t)C.off[m][t] * C.R;
      }
      h->batch = b;
    }
  }
  if ((st = build_dense_tables(b)) != DFACTO_OK) {
    unpool(b);
    return bail(st);
  }
  if (opt.autotune) {
    for (int k = 0; k < (int)b->cls.size(); ++k)
      if ((st = autotune_class(b, k)) != DFACTO_OK) {
        unpool(b);
        return bail(st);
      }
  }
  if (cudaStreamSynchronize(b->main) != cudaSuccess) {
    unpool(b);
    return bail(DFACTO_ECUDA);
  }
  *out = b;
  return DFACTO_OK;
}

void dfacto_batch_destroy(dfacto_batch_t* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  unpool(b);
  release(b);
  delete b;
}

dfacto_status dfacto_batch_mttkrp(dfacto_batch_t* b, int mode, float* const* out) {
  if (!b) return DFACTO_EINVAL;
  if (mode < 0 || mode > 2 || !out) return bfail(b, DFACTO_EINVAL, "dfacto_batch_mttkrp: bad arguments");
  for (size_t j = 0; j < b->jobs.size(); ++j)
    if (!out[j]) return bfail(b, DFACTO_EINVAL, "dfacto_batch_mttkrp: null output");
  dfacto_status st = enter(b);
  if (st != DFACTO_OK) return st;
  if ((st = batch_mttkrp_issue(b, mode, b->main, {})) != DFACTO_OK) return st;
  for (const BatchClass& C : b->cls)
    for (size_t t = 0; t < C.jobs.size(); ++t) {
      const dfacto_t* h = b->jobs[C.jobs[t]];
      DB_CUDA(b, cudaMemcpyAsync(out[C.jobs[t]], C.m[mode].N + (size_t)C.off[mode][t] * C.R,
                                 sizeof(float) * (size_t)h->dims[mode] * C.R, cudaMemcpyDeviceToDevice,
                                 b->main));
    }
  DB_CUDA(b, cudaEventRecord(b->fork_ev, b->main));
  DB_CUDA(b, cudaStreamWaitEvent(b->user, b->fork_ev, 0));
  return DFACTO_OK;
}

dfacto_status dfacto_batch_als_iter(dfacto_batch_t* b, double* fits) {
  if (!b) return DFACTO_EINVAL;
  dfacto_status st = enter(b);
  if (st != DFACTO_OK) return st;
  bool grams_known = true;
  for (dfacto_t* h : b->jobs)
    for (int m = 0; m < 3; ++m) grams_known = grams_known && h->gram_valid[m];
  if (!grams_known) drop_graph(b);  // factors changed outside the batch
  if (b->opt.use_graph && grams_known && !b->graph_ready) {
    // Capture one sweep.  Every host-side decision the sweep makes (Grams
    // known, walk shapes, buffer sizes) is fixed from here on.
    DB_CUDA(b, cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed));
    const long long before = g_launches.load();
    st = issue_sweep(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->main, &g);
    // Launches recorded during capture did not run: count them per replay.
    b->graph_kernels = g_launches.load() - before;
    g_launches.fetch_sub(b->graph_kernels);
    if (st != DFACTO_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
      drop_graph(b);
      return bcuda(b, e, "cudaGraphInstantiate");
    }
    b->graph_ready = true;
  }
  if (b->graph_ready) {
    DB_CUDA(b, cudaGraphLaunch(b->exec, b->main));
    g_launches.fetch_add(b->graph_kernels);
  } else if ((st = issue_sweep(b)) != DFACTO_OK) {
    return st;
  }
  ++b->sweeps;
  DB_CUDA(b, cudaEventRecord(b->fork_ev, b->main));
  DB_CUDA(b, cudaStreamWaitEvent(b->user, b->fork_ev, 0));
  if (!fits) return DFACTO_OK;
  const int n = (int)b->jobs.size();
  DB_CUDA(b, cudaMemcpyAsync(b->h_fits, b->d_fits, sizeof(double) * n, cudaMemcpyDeviceToHost, b->main));
  DB_CUDA(b, cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->main));
  DB_CUDA(b, cudaStreamSynchronize(b->main));
  bool singular = false, internal = false;
  for (int j = 0; j < n; ++j) {
    fits[j] = b->h_fits[j];
    singular = singular || (b->h_status[j] & 1);
    internal = internal || (b->h_status[j] & 2);
  }
  if (internal) return bfail(b, DFACTO_EINTERNAL, "internal consistency check failed");
  return singular ? DFACTO_ESINGULAR : DFACTO_OK;
}

dfacto_status dfacto_batch_sync(dfacto_batch_t* b) {
  if (!b) return DFACTO_EINVAL;
  DB_CUDA(b, cudaStreamSynchronize(b->main));
  return DFACTO_OK;
}

int32_t dfacto_batch_num_classes(const dfacto_batch_t* b) { return b ? (int32_t)b->cls.size() : 0; }

dfacto_status dfacto_batch_get_class(const dfacto_batch_t* b, int32_t k, dfacto_batch_class* out) {
  if (!b || !out || k < 0 || k >= (int32_t)b->cls.size()) return DFACTO_EINVAL;
  const BatchClass& C = b->cls[k];
  out->rank = C.R;
  out->factor_dtype = C.dtype;
  out->n_jobs = (int32_t)C.jobs.size();
  out->vec = C.cfg.vec;
  out->lanes = C.cfg.G;
  out->seg_nnz = C.cfg.seg;
  out->nnz = C.nnz;
  out->tuned_ms = C.tuned_ms;
  return DFACTO_OK;
}

const char* dfacto_batch_last_error(const dfacto_batch_t* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
