// noalloc.cu -- dfacto_mttkrp_noalloc: the MTTKRP of one mode for callers that
// must not allocate device memory.  Everything it needs besides the caller's
// inputs and output lives in one fixed device array defined in this file.
#include <mutex>

#include "mttkrp.cuh"

namespace dfacto {
namespace {

// Scratch of the allocation-free MTTKRP: segment starts and row carries.  Every
// GPU that loads the library holds this array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once with that
// device current (host code only knows the symbol, not its device address).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <int VEC, int G>
cudaError_t go(const MttkrpParams& a, int64_t ncta, size_t smem, cudaStream_t s) {
  auto k = mttkrp_walk<float, VEC, G, true>;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ncta, kWalkWarps * 32, smem, s>>>(a);
  DF_COUNT();
  return cudaGetLastError();
}

cudaError_t launch_rows_from_ptr(int vec, int G, const MttkrpParams& a, int64_t ncta, size_t smem,
                                 cudaStream_t s) {
#define DF_CASE(V, GG) \
  if (vec == V && G == GG) return go<V, GG>(a, ncta, smem, s);
  DF_CASE(1, 1) DF_CASE(1, 2) DF_CASE(1, 4) DF_CASE(1, 8) DF_CASE(1, 16) DF_CASE(1, 32)
  DF_CASE(2, 1) DF_CASE(2, 2) DF_CASE(2, 4) DF_CASE(2, 8) DF_CASE(2, 16) DF_CASE(2, 32)
  DF_CASE(4, 1) DF_CASE(4, 2) DF_CASE(4, 4) DF_CASE(4, 8) DF_CASE(4, 16) DF_CASE(4, 32)
  DF_CASE(8, 1) DF_CASE(8, 2) DF_CASE(8, 4) DF_CASE(8, 8) DF_CASE(8, 16)
#undef DF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace dfacto

using namespace dfacto;

extern "C" dfacto_status dfacto_mttkrp_noalloc(const dfacto_csr_view* csr, const float* F_in,
                                               const float* F_f, int32_t R, float* out,
                                               void* stream) {
  if (!csr || !out || R < 1 || R > 128 || (R > 32 && R % 4 != 0)) return DFACTO_EINVAL;
  const int64_t nnz = csr->nnz, nfib = csr->nfib, dim_o = csr->dim_o;
  if (nnz < 0 || nnz > kMaxNnz || nfib < 0 || nfib > nnz || dim_o < 1 || !csr->fiber_ptr)
    return DFACTO_EINVAL;
  if (nnz > 0 && (!csr->fiber_idx || !csr->nz_ptr || !csr->nz_idx || !csr->nz_val || !F_in || !F_f))
    return DFACTO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // Eight columns per lane where R allows it (R a multiple of 8: R / 8 lanes
  // per segment), fewer otherwise; the walk shape fixes the scratch per
  // nonzero stated in the header.
  const WalkCfg cfg = choose_walk(R, DFACTO_F32, nnz, nfib, 0, 8);
  const int segs = kWalkWarps * (32 / cfg.G);
  const int64_t P = (int64_t)segs * cfg.seg;
  const int64_t ncta = (nnz + P - 1) / P;
  const int64_t nseg = (nnz + cfg.seg - 1) / cfg.seg;

  // Scratch layout: seg_fib[nseg] | carry[ncta][2][R] | carry_row[ncta][2].
  const size_t off_carry = align256(sizeof(int32_t) * (size_t)nseg);
  const size_t off_rows = off_carry + align256(sizeof(float) * 2 * (size_t)R * ncta);
  const size_t need = off_rows + align256(sizeof(int32_t) * 2 * (size_t)ncta);
  if (need > kNoAllocScratchBytes) return DFACTO_ENOMEM;

  unsigned char* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return DFACTO_ECUDA;
  }
  int32_t* seg_fib = reinterpret_cast<int32_t*>(scratch);
  float* carry = reinterpret_cast<float*>(scratch + off_carry);
  int32_t* carry_row = reinterpret_cast<int32_t*>(scratch + off_rows);

  cudaError_t e = launch_segment_starts(csr->nz_ptr, nfib, nseg, cfg.seg, seg_fib, s);
  if (e == cudaSuccess && ncta > 0) {
    MttkrpParams a;
    a.fiber_ptr = csr->fiber_ptr;
    a.fiber_idx = csr->fiber_idx;
    a.fiber_row = nullptr;  // rows come from fiber_ptr
    a.nz_ptr = csr->nz_ptr;
    a.nz_idx = csr->nz_idx;
    a.nz_val = csr->nz_val;
    a.seg_fib = seg_fib;
    a.Fin = F_in;
    a.Ff = F_f;
    a.out = out;
    a.carry = carry;
    a.carry_row = carry_row;
    a.nnz = nnz;
    a.nfib = nfib;
    a.dim_o = dim_o;
    a.R = R;
    a.seg = cfg.seg;
    const size_t smem = sizeof(float) * (size_t)(2 * segs + 2 * kWalkWarps) * R;
    e = launch_rows_from_ptr(cfg.vec, cfg.G, a, ncta, smem, s);
  }
  if (e == cudaSuccess)
    e = launch_mttkrp_fixup(carry_row, carry, csr->fiber_ptr, csr->nz_ptr, out, R, P, ncta, dim_o,
                            /*bad=*/nullptr, s);  // no status word to report it through
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DFACTO_ENOMEM : DFACTO_ECUDA;
  }
  return DFACTO_OK;
}
