// scan.cu -- device-wide exclusive prefix sum of int32 values.
//
// Three kernels per level: per-tile totals, a (recursive) scan of the totals,
// and a per-tile scan that adds the tile's offset.  A tile is 256 threads x 16
// rounds; each round scans 256 consecutive values with warp shuffles, so every
// global access is coalesced.
#include "device.cuh"
#include "internal.h"

namespace dfacto {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanRounds = 16;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanRounds;

__global__ void __launch_bounds__(kScanThreads) tile_totals(const int32_t* __restrict__ in,
                                                           int64_t n, int32_t* __restrict__ tot) {
  __shared__ int32_t s_warp[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t acc = 0;
#pragma unroll 4
  for (int r = 0; r < kScanRounds; ++r) {
    int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t s = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) s += s_warp[w];
    tot[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kScanThreads) tile_scan(const int32_t* in, int32_t* out, int64_t n,
                                                         const int32_t* __restrict__ offsets) {
  __shared__ int32_t s_warp[kScanThreads / 32];
  __shared__ int32_t s_run;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (threadIdx.x == 0) s_run = offsets ? offsets[blockIdx.x] : 0;
  // all of the thread's values first (one load latency per tile, not one per
  // round); each value is read and written by this thread only, so in == out
  // is fine
  int32_t xs[kScanRounds];
#pragma unroll
  for (int r = 0; r < kScanRounds; ++r) {
    const int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
    xs[r] = (i < n) ? in[i] : 0;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kScanRounds; ++r) {
    const int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
    const int32_t x = xs[r];
    int32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int32_t wofs = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
      int32_t t = s_warp[w];
      wofs += (w < warp) ? t : 0;
      total += t;
    }
    const int32_t run = s_run;
    if (i < n) out[i] = run + wofs + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) s_run = run + total;
    // s_warp is rewritten next round only after every thread passed the
    // barrier above, and s_run is read next round after the first barrier.
  }
}

}  // namespace

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles == 1) {
    tile_scan<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr); DF_COUNT();
    return cudaGetLastError();
  }
  int32_t* tot = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&tot), sizeof(int32_t) * ntiles, s);
  if (e != cudaSuccess) return e;
  tile_totals<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tot); DF_COUNT();
  e = cudaGetLastError();
  if (e == cudaSuccess) e = exclusive_scan_i32(tot, tot, ntiles, s);
  if (e == cudaSuccess) {
    tile_scan<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, out, n, tot); DF_COUNT();
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaFreeAsync(tot, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace dfacto
