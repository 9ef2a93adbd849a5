// dual.cu -- the four trilinear terms the GD line search needs beyond the
// MTTKRP outputs:
//   T110 = <X, [[GA, GB, C ]]>,  T101 = <X, [[GA, B, GC]]>,
//   T011 = <X, [[A,  GB, GC]]>,  T111 = <X, [[GA, GB, GC]]>,
// all in one walk over the mode-1 CSR copy (rows i, fibers (i,k), entries j),
// organised like Algorithm 1 with two inputs per SpMV: per fiber
// vB = sum x B[j,:] and vG = sum x GB[j,:]; per row u1 = sum C[k,:] (*) vG,
// u2 = sum GC[k,:] (*) vB, u3 = sum GC[k,:] (*) vG; then T110 += GA[i,:].u1,
// T101 += GA[i,:].u2, T011 += A[i,:].u3, T111 += GA[i,:].u3.  Only scalars
// leave the walk, so rows split between segments need no carries.  Segment sums
// are FP32 (at most one segment of nonzeros), everything above is FP64.
//
// Range: T111 carries three gradient factors, and gradients reach 1e13 and
// more on large tensors (|F Gamma| grows with the product of two dimensions),
// so x * g^3 would overflow FP32.  Each gradient is therefore read scaled by
// 2^-e_n, its largest magnitude brought into [0.5, 1); the terms are divided
// by the product of their scales in FP64.  Powers of two scale exactly, so the
// result is the unscaled arithmetic wherever that did not overflow.
#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace dfacto {
namespace {

struct DualParams {
  const int32_t* fiber_idx;
  const int32_t* fiber_row;
  const int64_t* nz_ptr;
  const int32_t* nz_idx;
  const float* nz_val;
  const int32_t* seg_fib;
  const void* A;
  const void* B;
  const void* C;
  const float* GA;
  const float* GB;
  const float* GC;
  const float* gscale;  // [3] power-of-two scales of GA, GB, GC
  double* part;  // [ncta][4]
  int64_t nnz;
  int64_t nfib;
  int R;
  int seg;
};

template <typename T, int VEC, int G>
__global__ void __launch_bounds__(kWalkWarps * 32) dual_walk(const DualParams a) {
  constexpr int NG = 32 / G;
  constexpr int SEGS = kWalkWarps * NG;
  __shared__ double s_t[kWalkWarps][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, c = lane % G;
  const int gbase = g * G;
  const int col0 = c * VEC;
  const bool colok = col0 < a.R;
  const int sl = warp * NG + g;
  const int64_t p0 = ((int64_t)blockIdx.x * SEGS + sl) * a.seg;
  const int64_t p1 = min(p0 + a.seg, a.nnz);
  const bool active = p0 < a.nnz;
  const int R = a.R;
  const T* A = static_cast<const T*>(a.A);
  const T* B = static_cast<const T*>(a.B);
  const T* C = static_cast<const T*>(a.C);

  const float sA = a.gscale[0], sB = a.gscale[1], sC = a.gscale[2];
  float vB[VEC], vG[VEC], cf[VEC], gcf[VEC], u1[VEC], u2[VEC], u3[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) vB[q] = vG[q] = cf[q] = gcf[q] = u1[q] = u2[q] = u3[q] = 0.f;
  float t[4] = {0.f, 0.f, 0.f, 0.f};

  int64_t fib = 0, fend = 0;
  int row_cur = -1;
  auto load_fiber = [&](int64_t q) {
    fend = min(a.nz_ptr[q + 1], p1);
    row_cur = a.fiber_row[q];
    const int k = a.fiber_idx[q];
    if (colok) {
      VecIO<T, VEC>::load(C + (int64_t)k * R + col0, cf);
      VecIO<float, VEC>::load(a.GC + (int64_t)k * R + col0, gcf);
#pragma unroll
      for (int q = 0; q < VEC; ++q) gcf[q] *= sC;
    }
  };
  auto emit_row = [&]() {
    if (!colok) return;
    float ar[VEC], gar[VEC];
    VecIO<T, VEC>::load(A + (int64_t)row_cur * R + col0, ar);
    VecIO<float, VEC>::load(a.GA + (int64_t)row_cur * R + col0, gar);
#pragma unroll
    for (int q = 0; q < VEC; ++q) gar[q] *= sA;
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      t[0] = fmaf(gar[q], u1[q], t[0]);
      t[1] = fmaf(gar[q], u2[q], t[1]);
      t[2] = fmaf(ar[q], u3[q], t[2]);
      t[3] = fmaf(gar[q], u3[q], t[3]);
      u1[q] = u2[q] = u3[q] = 0.f;
    }
  };
  if (active) {
    fib = a.seg_fib[(int64_t)blockIdx.x * SEGS + sl];
    load_fiber(fib);
  }
  for (int64_t base = p0; base < p0 + a.seg; base += G) {
    const int64_t pl = base + c;
    const bool okl = pl < p1;
    const int my_in = okl ? __ldg(a.nz_idx + pl) : 0;
    const float my_x = okl ? __ldg(a.nz_val + pl) : 0.f;
#pragma unroll 1
    for (int u = 0; u < G; ++u) {
      const int j = __shfl_sync(kFull, my_in, gbase + u);
      const float x = __shfl_sync(kFull, my_x, gbase + u);
      const int64_t p = base + u;
      if (p < p1) {
        if (colok) {
          float b[VEC], gb[VEC];
          VecIO<T, VEC>::load(B + (int64_t)j * R + col0, b);
          VecIO<float, VEC>::load(a.GB + (int64_t)j * R + col0, gb);
#pragma unroll
          for (int q = 0; q < VEC; ++q) gb[q] *= sB;
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            vB[q] = fmaf(x, b[q], vB[q]);
            vG[q] = fmaf(x, gb[q], vG[q]);
          }
        }
        if (p + 1 == fend) {
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            u1[q] = fmaf(cf[q], vG[q], u1[q]);
            u2[q] = fmaf(gcf[q], vB[q], u2[q]);
            u3[q] = fmaf(gcf[q], vG[q], u3[q]);
            vB[q] = vG[q] = 0.f;
          }
          if (p + 1 < p1) {
            const int old_row = row_cur;
            ++fib;
            const int64_t save_fib = fib;
            // peek the next fiber's row before loading it
            const int next_row = a.fiber_row[save_fib];
            if (next_row != old_row) emit_row();
            load_fiber(save_fib);
          }
        }
      }
    }
  }
  if (active) emit_row();
  double td[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    td[k] = warp_sum((double)t[k]);
    if (lane == 0) s_t[warp][k] = td[k];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kWalkWarps; ++w) s += s_t[w][threadIdx.x];
    a.part[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
  }
}

// scal[kT110 + k] = sum over CTAs of part[b][k], k = 0..3 (fixed order:
// strided per-thread sums, then a fixed tree), divided by the term's scales.
__global__ void __launch_bounds__(256) dual_reduce(const double* __restrict__ part, int64_t ncta,
                                                   const float* __restrict__ gscale,
                                                   double* __restrict__ scal) {
  __shared__ double red[256];
  const double sA = gscale[0], sB = gscale[1], sC = gscale[2];
  const double unscale[4] = {1.0 / (sA * sB), 1.0 / (sA * sC), 1.0 / (sB * sC),
                             1.0 / (sA * sB * sC)};
  for (int k = 0; k < 4; ++k) {
    double v = 0.0;
    for (int64_t b = threadIdx.x; b < ncta; b += 256) v += part[b * 4 + k];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) scal[kT110 + k] = red[0] * unscale[k];
    __syncthreads();
  }
}

// Largest |g| of each gradient (as ordered bits of a non-negative float;
// atomicMax keeps it independent of the order), then scale[n] = 2^-e with
// max = m 2^e, m in [0.5, 1) (1 when the gradient is zero or not finite).
__global__ void grad_absmax(const float* __restrict__ g, int64_t n, unsigned* __restrict__ out) {
  unsigned m = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    m = max(m, __float_as_uint(fabsf(g[i])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void grad_scales(const unsigned* __restrict__ maxbits, float* __restrict__ scale) {
  const int n = threadIdx.x;
  if (n >= 3) return;
  const float m = __uint_as_float(maxbits[n]);
  float sc = 1.f;
  if (m > 0.f && isfinite(m)) {
    int e;
    frexpf(m, &e);        // m = f 2^e, f in [0.5, 1)
    sc = ldexpf(1.f, -e);  // 2^-e, exact
    if (sc == 0.f || !isfinite(sc)) sc = 1.f;
  }
  scale[n] = sc;
}

template <typename T, int VEC, int G>
cudaError_t go(const DualParams& a, int64_t ncta, cudaStream_t s) {
  dual_walk<T, VEC, G><<<(unsigned)ncta, kWalkWarps * 32, 0, s>>>(a); DF_COUNT();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch(int vec, int G, const DualParams& a, int64_t ncta, cudaStream_t s) {
#define DF_CASE(V, GG) \
  if (vec == V && G == GG) return go<T, V, GG>(a, ncta, s);
  DF_CASE(1, 1) DF_CASE(1, 2) DF_CASE(1, 4) DF_CASE(1, 8) DF_CASE(1, 16) DF_CASE(1, 32)
  DF_CASE(2, 1) DF_CASE(2, 2) DF_CASE(2, 4) DF_CASE(2, 8) DF_CASE(2, 16) DF_CASE(2, 32)
  DF_CASE(4, 1) DF_CASE(4, 2) DF_CASE(4, 4) DF_CASE(4, 8) DF_CASE(4, 16) DF_CASE(4, 32)
  DF_CASE(8, 1) DF_CASE(8, 2) DF_CASE(8, 4) DF_CASE(8, 8) DF_CASE(8, 16)
#undef DF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace

dfacto_status dual_pass(dfacto_t* h) {
  ModeCSR& M = h->m[0];
  dfacto_status st = ensure_segments(h, 0);
  if (st != DFACTO_OK) return st;
  const WalkCfg cfg = M.cfg;
  const int segs = kWalkWarps * (32 / cfg.G);
  const int64_t P = (int64_t)segs * cfg.seg;
  const int64_t ncta = (h->nnz + P - 1) / P;
  if ((st = grow_partials(h, ncta * 4)) != DFACTO_OK) return st;
  // Scales of the three gradients.
  unsigned* maxbits = h->gd_scratch;
  float* gscale = reinterpret_cast<float*>(h->gd_scratch + 4);
  DF_CUDA(h, cudaMemsetAsync(maxbits, 0, 3 * sizeof(unsigned), h->stream));
  for (int m = 0; m < 3; ++m) {
    const int64_t n = (int64_t)h->dims[m] * h->R;
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    grad_absmax<<<nb, 256, 0, h->stream>>>(h->grad[m], n, maxbits + m); DF_COUNT();
  }
  grad_scales<<<1, 32, 0, h->stream>>>(maxbits, gscale); DF_COUNT();
  if (ncta == 0) {
    DF_CUDA(h, cudaMemsetAsync(h->scal + kT110, 0, 4 * sizeof(double), h->stream));
    return DFACTO_OK;
  }
  DualParams a;
  a.fiber_idx = M.fiber_idx;
  a.fiber_row = M.fiber_row;
  a.nz_ptr = M.nz_ptr;
  a.nz_idx = M.nz_idx;
  a.nz_val = M.nz_val;
  a.seg_fib = M.seg_fib;
  a.A = h->F[0];
  a.B = h->F[1];
  a.C = h->F[2];
  a.GA = h->grad[0];
  a.GB = h->grad[1];
  a.GC = h->grad[2];
  a.gscale = gscale;
  a.part = h->partials;
  a.nnz = h->nnz;
  a.nfib = M.nfib;
  a.R = h->R;
  a.seg = cfg.seg;
  cudaError_t e = (h->dtype == DFACTO_BF16)
                      ? launch<__nv_bfloat16>(cfg.vec, cfg.G, a, ncta, h->stream)
                      : launch<float>(cfg.vec, cfg.G, a, ncta, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "dual_walk launch");
  dual_reduce<<<1, 256, 0, h->stream>>>(h->partials, ncta, gscale, h->scal); DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

}  // namespace dfacto
