// batch_walk.cu -- instantiations of the batched MTTKRP walk (mttkrp.cuh).
#include "mttkrp.cuh"

namespace dfacto {

template <typename T>
cudaError_t launch_walk2_multi(const MultiWalkParams& mp, size_t smem, int grid, cudaStream_t s) {
  auto k = mttkrp_walk2_multi<T>;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  if (grid <= 0) return cudaSuccess;
  k<<<(unsigned)grid, kWalkWarps * 32, smem, s>>>(mp);
  DF_COUNT();
  return cudaGetLastError();
}

template cudaError_t launch_walk2_multi<float>(const MultiWalkParams&, size_t, int, cudaStream_t);
template cudaError_t launch_walk2_multi<__nv_bfloat16>(const MultiWalkParams&, size_t, int, cudaStream_t);

}  // namespace dfacto
