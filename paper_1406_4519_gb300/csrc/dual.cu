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
#include "mttkrp.cuh"

namespace dfacto {
namespace {

struct DualParams {
  const int32_t* fiber_idx;
  const int32_t* fiber_row;
  const int64_t* nz_ptr;
  const int32_t* nz_idx;
  const float* nz_val;
  const int32_t* seg_fib;
  const uint32_t* end_bits;  // dual_walk2: bit p set iff nonzero p ends its fiber
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

// ---------------------------------------------------------------------------
// dual_walk2: the same four terms with the organisation of mttkrp_walk2: fiber
// ends from the end bitmask of the mode-1 copy, both fiber sums (vB, vG) parked
// in shared memory where a fiber ends, and the closed fibers folded CC at a
// time (their C and GC rows gathered together).  At most 8 values of each of
// the two gathered rows (B and GB) are in flight per lane.
// ---------------------------------------------------------------------------
template <int VEC>
struct Dual2Shape {
  static constexpr int NT = kWalkWarps * 32;
  static constexpr int U = 8 / VEC > 0 ? 8 / VEC : 1;  // capped by G below
  static constexpr int CC = 2;                           // fibers folded per round
};

template <typename T, int VEC, int G>
__global__ void __launch_bounds__(kWalkWarps * 32, 3) dual_walk2(const DualParams a) {
  constexpr int NG = 32 / G;
  constexpr int SEGS = kWalkWarps * NG;
  constexpr int NT = Dual2Shape<VEC>::NT;
  constexpr int U = G < Dual2Shape<VEC>::U ? G : Dual2Shape<VEC>::U;
  constexpr int CC = Dual2Shape<VEC>::CC < U ? Dual2Shape<VEC>::CC : U;
  extern __shared__ __align__(16) float vb[];  // 2U slots of NT x VEC parked sums
  __shared__ double s_t[kWalkWarps][4];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane / G, c = lane % G;
  const int gbase = g * G;
  const int col0 = c * VEC;
  const bool colok = col0 < a.R;
  const int sl = warp * NG + g;
  const int nnz = (int)a.nnz;
  const int p0 = (int)min(((int64_t)blockIdx.x * SEGS + sl) * a.seg, a.nnz);
  const int p1 = min(p0 + a.seg, nnz);
  const bool active = p0 < nnz;
  const int R = a.R;
  const T* __restrict__ A = static_cast<const T*>(a.A);
  const T* __restrict__ B = static_cast<const T*>(a.B);
  const T* __restrict__ C = static_cast<const T*>(a.C);
  const float sA = a.gscale[0], sB = a.gscale[1], sC = a.gscale[2];

  float vB[VEC], vG[VEC], u1[VEC], u2[VEC], u3[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) vB[e] = vG[e] = u1[e] = u2[e] = u3[e] = 0.f;
  float t[4] = {0.f, 0.f, 0.f, 0.f};
  int q = 0, row_cur = -1;
  if (active) {
    q = a.seg_fib[(int64_t)blockIdx.x * SEGS + sl];
    row_cur = a.fiber_row[q];
  }
  // Close row row_cur: T110 += GA.u1, T101 += GA.u2, T011 += A.u3, T111 += GA.u3.
  auto emit_row = [&]() {
    if (colok) {
      float ar[VEC], gar[VEC];
      VecIO<T, VEC>::load(A + (int64_t)row_cur * R + col0, ar);
      VecIO<float, VEC>::load(a.GA + (int64_t)row_cur * R + col0, gar);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float ga = gar[e] * sA;
        t[0] = fmaf(ga, u1[e], t[0]);
        t[1] = fmaf(ga, u2[e], t[1]);
        t[2] = fmaf(ar[e], u3[e], t[2]);
        t[3] = fmaf(ga, u3[e], t[3]);
      }
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) u1[e] = u2[e] = u3[e] = 0.f;
  };
  // Fold a closed fiber (row r, sums pB / pG, rows cf = C[k], gcf = GC[k]).
  auto fold = [&](int r, const float (&pB)[VEC], const float (&pG)[VEC], const float (&cf)[VEC],
                  const float (&gcf)[VEC]) {
    if (r != row_cur) {
      emit_row();
      row_cur = r;
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      u1[e] = fmaf(cf[e], pG[e], u1[e]);
      u2[e] = fmaf(gcf[e], pB[e], u2[e]);
      u3[e] = fmaf(gcf[e], pG[e], u3[e]);
    }
  };

  for (int base = p0; base < p0 + a.seg; base += G) {
    const int pl = base + c;
    const bool okl = pl < p1;
    const int my_in = okl ? __ldg(a.nz_idx + pl) : 0;
    const float my_x = okl ? __ldg(a.nz_val + pl) : 0.f;
    const uint32_t ebits =
        (active && base < p1) ? (__ldg(a.end_bits + (base >> 5)) >> (base & 31)) : 0u;
#pragma unroll
    for (int u0 = 0; u0 < G; u0 += U) {
      float b[U][VEC], gb[U][VEC];
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const int j = __shfl_sync(kFull, my_in, gbase + u0 + uu);
        if (colok && base + u0 + uu < p1) {
          VecIO<T, VEC>::load(B + (int64_t)j * R + col0, b[uu]);
          VecIO<float, VEC>::load(a.GB + (int64_t)j * R + col0, gb[uu]);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) b[uu][e] = gb[uu][e] = 0.f;
        }
      }
      int k = 0;
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const float x = __shfl_sync(kFull, my_x, gbase + u0 + uu);
        const int p = base + u0 + uu;
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          vB[e] = fmaf(x, b[uu][e], vB[e]);
          vG[e] = fmaf(x, gb[uu][e] * sB, vG[e]);
        }
        const bool end = p < p1 && ((ebits >> (u0 + uu)) & 1u);
        if (end) {
          smem_st<VEC, NT>(park_slot<VEC, NT>(vb, 2 * k, tid), vB);
          smem_st<VEC, NT>(park_slot<VEC, NT>(vb, 2 * k + 1, tid), vG);
#pragma unroll
          for (int e = 0; e < VEC; ++e) vB[e] = vG[e] = 0.f;
        }
        k += end ? 1 : 0;
      }
      for (int j0 = 0; j0 < k; j0 += CC) {
        int rj[CC];
        float cf[CC][VEC], gcf[CC][VEC];
#pragma unroll
        for (int j = 0; j < CC; ++j) {
          rj[j] = row_cur;
          if (j0 + j < k) {
            const int kk = __ldg(a.fiber_idx + q + j0 + j);
            rj[j] = __ldg(a.fiber_row + q + j0 + j);
            if (colok) {
              VecIO<T, VEC>::load(C + (int64_t)kk * R + col0, cf[j]);
              VecIO<float, VEC>::load(a.GC + (int64_t)kk * R + col0, gcf[j]);
            }
          }
          if (!(j0 + j < k && colok)) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) cf[j][e] = gcf[j][e] = 0.f;
          }
        }
#pragma unroll
        for (int j = 0; j < CC; ++j) {
          if (j0 + j < k) {
            float pB[VEC], pG[VEC];
            smem_ld<VEC, NT>(park_slot<VEC, NT>(vb, 2 * (j0 + j), tid), pB);
            smem_ld<VEC, NT>(park_slot<VEC, NT>(vb, 2 * (j0 + j) + 1, tid), pG);
#pragma unroll
            for (int e = 0; e < VEC; ++e) gcf[j][e] *= sC;
            fold(rj[j], pB, pG, cf[j], gcf[j]);
          }
        }
      }
      q += k;
    }
  }
  if (active) {
    // the fiber open at the segment end (its last nonzero lies beyond p1)
    if (!((__ldg(a.end_bits + ((p1 - 1) >> 5)) >> ((p1 - 1) & 31)) & 1u)) {
      const int kk = __ldg(a.fiber_idx + q);
      const int r = __ldg(a.fiber_row + q);
      float cf[VEC], gcf[VEC];
      if (colok) {
        VecIO<T, VEC>::load(C + (int64_t)kk * R + col0, cf);
        VecIO<float, VEC>::load(a.GC + (int64_t)kk * R + col0, gcf);
      } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) cf[e] = gcf[e] = 0.f;
      }
#pragma unroll
      for (int e = 0; e < VEC; ++e) gcf[e] *= sC;
      fold(r, vB, vG, cf, gcf);
    }
    emit_row();
  }
  double td[4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    td[kk] = warp_sum((double)t[kk]);
    if (lane == 0) s_t[warp][kk] = td[kk];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double sum = 0.0;
    for (int w = 0; w < kWalkWarps; ++w) sum += s_t[w][threadIdx.x];
    a.part[(size_t)blockIdx.x * 4 + threadIdx.x] = sum;
  }
}

template <int VEC, int G>
size_t dual2_smem() {
  constexpr int U = G < Dual2Shape<VEC>::U ? G : Dual2Shape<VEC>::U;
  return sizeof(float) * (size_t)2 * U * Dual2Shape<VEC>::NT * VEC;
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
cudaError_t go(const DualParams& a, int64_t ncta, cudaStream_t s, int kernel) {
  if (kernel == 2) {
    dual_walk2<T, VEC, G><<<(unsigned)ncta, kWalkWarps * 32, dual2_smem<VEC, G>(), s>>>(a);
  } else {
    dual_walk<T, VEC, G><<<(unsigned)ncta, kWalkWarps * 32, 0, s>>>(a);
  }
  DF_COUNT();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch(int vec, int G, const DualParams& a, int64_t ncta, cudaStream_t s, int kernel) {
#define DF_CASE(V, GG) \
  if (vec == V && G == GG) return go<T, V, GG>(a, ncta, s, kernel);
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
  // The mode-1 walk's segments; dual_walk2 keeps five accumulators and two
  // gathered rows per lane, so its lanes take at most four columns.  At a rank
  // that is not a multiple of four it walks zero-padded FP32 copies of the
  // factors and gradients at the rank rounded up, as the MTTKRP does (the zero
  // columns add nothing to the four terms).
  const int R = h->R;
  const int RP = walk_rank(R, h->opt.vec);
  const bool padded = RP != R;
  WalkCfg cfg = M.cfg;
  if (padded) {
    cfg = choose_walk(RP, DFACTO_F32, h->nnz, M.nfib, h->opt.seg_nnz, 0);
    cfg.kernel = M.cfg.kernel;
  }
  if (cfg.kernel == 2 && cfg.vec > 4) {
    cfg.vec = 4;
    int G = 1;
    while (G * 4 < RP) G <<= 1;
    cfg.G = G;
  }
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
  const void* Fm[3] = {h->F[0], h->F[1], h->F[2]};
  const float* Gm[3] = {h->grad[0], h->grad[1], h->grad[2]};
  if (padded) {
    const int64_t rows = (int64_t)h->dims[0] + h->dims[1] + h->dims[2];
    if (!h->pad_dual &&
        (st = dalloc(h, (void**)&h->pad_dual, sizeof(float) * 2 * (size_t)rows * RP)) != DFACTO_OK)
      return st;
    float* q = h->pad_dual;
    for (int m = 0; m < 3; ++m) {
      float* pf = q;
      float* pg = q + (size_t)h->dims[m] * RP;
      DF_CUDA(h, pad_factor_rows(h->F[m], h->dtype, h->dims[m], R, RP, pf, h->stream));
      DF_CUDA(h, pad_factor_rows(h->grad[m], DFACTO_F32, h->dims[m], R, RP, pg, h->stream));
      Fm[m] = pf;
      Gm[m] = pg;
      q += 2 * (size_t)h->dims[m] * RP;
    }
  }
  DualParams a;
  a.fiber_idx = M.fiber_idx;
  a.fiber_row = M.fiber_row;
  a.nz_ptr = M.nz_ptr;
  a.nz_idx = M.nz_idx;
  a.nz_val = M.nz_val;
  a.seg_fib = M.seg_fib;
  a.end_bits = M.end_bits;
  a.A = Fm[0];
  a.B = Fm[1];
  a.C = Fm[2];
  a.GA = Gm[0];
  a.GB = Gm[1];
  a.GC = Gm[2];
  a.gscale = gscale;
  a.part = h->partials;
  a.nnz = h->nnz;
  a.nfib = M.nfib;
  a.R = RP;
  a.seg = cfg.seg;
  cudaError_t e = (h->dtype == DFACTO_BF16 && !padded)
                      ? launch<__nv_bfloat16>(cfg.vec, cfg.G, a, ncta, h->stream, cfg.kernel)
                      : launch<float>(cfg.vec, cfg.G, a, ncta, h->stream, cfg.kernel);
  if (e != cudaSuccess) return cuda_fail(h, e, "dual_walk launch");
  dual_reduce<<<1, 256, 0, h->stream>>>(h->partials, ncta, gscale, h->scal); DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

}  // namespace dfacto
