// mttkrp_f32.cu -- instantiations of the MTTKRP walk for float factors.
#include "mttkrp.cuh"

namespace dfacto {

template <int VEC, int G>
static cudaError_t go(const MttkrpParams& a, int64_t ncta, size_t smem, cudaStream_t s) {
  auto k = mttkrp_walk<float, VEC, G>;
  // Opt in to the dynamic shared memory this launch needs (the default limit
  // is 48 KB including the kernel's static shared memory).
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ncta, kWalkWarps * 32, smem, s>>>(a);
  DF_COUNT();
  return cudaGetLastError();
}

template <>
cudaError_t launch_walk<float>(int vec, int G, const MttkrpParams& a, int64_t ncta, size_t smem,
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

template <int VEC, int G>
static cudaError_t go2(const MttkrpParams& a, int64_t ncta, cudaStream_t s) {
  auto k = mttkrp_walk2<float, VEC, G>;
  const size_t smem = Walk2Shape<float, VEC, G>::smem_bytes(a.R);
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ncta, kWalkWarps * 32, smem, s>>>(a);
  DF_COUNT();
  return cudaGetLastError();
}

template <>
cudaError_t launch_walk2<float>(int vec, int G, const MttkrpParams& a, int64_t ncta, cudaStream_t s) {
#define DF_CASE(V, GG) \
  if (vec == V && G == GG) return go2<V, GG>(a, ncta, s);
  DF_CASE(1, 1) DF_CASE(1, 2) DF_CASE(1, 4) DF_CASE(1, 8) DF_CASE(1, 16) DF_CASE(1, 32)
  DF_CASE(2, 1) DF_CASE(2, 2) DF_CASE(2, 4) DF_CASE(2, 8) DF_CASE(2, 16) DF_CASE(2, 32)
  DF_CASE(4, 1) DF_CASE(4, 2) DF_CASE(4, 4) DF_CASE(4, 8) DF_CASE(4, 16) DF_CASE(4, 32)
  DF_CASE(8, 1) DF_CASE(8, 2) DF_CASE(8, 4) DF_CASE(8, 8) DF_CASE(8, 16)
#undef DF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace dfacto
