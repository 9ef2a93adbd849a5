// joint.cu -- joint matrix completion and tensor factorization (Appendix F).
//
// A ratings matrix Y (users x items, observed entries Omega^Y) and the user x
// item x word tensor X share the user factor A and the item factor B:
//   f = 1/2 sum_{(i,j) in Omega^Y} (y_ij - a_i . b_j)^2 + mu 1/2 ||X - [[A,B,C]]||^2
//       + lambda 1/2 (||A||^2 + ||B||^2 + ||C||^2)                (Eq. joint-obj-fn)
// with lambda the handle's lambda_reg.  Every row of A has the system of
// Eq. grad-joint-A:
//   rhs_i = sum_{j in Omega_i} y_ij b_j + mu N_A[i],   N_A = X^1 (C kr B) (MTTKRP)
//   H_i   = sum_{j in Omega_i} b_j^T b_j + mu (C^T C * B^T B) + lambda I
// (B the same with the roles of A and B swapped; C with no ratings).  ALS sets
// a_i = rhs_i H_i^-1 row by row; GD takes grad_i = -rhs_i + a_i H_i for every
// row at the current point and searches along the ray.  The X^1 (C kr B) term
// is the library's MTTKRP (Algorithm 1), as the appendix says.
//
// The ratings are kept as two CSR copies (by user and by item), sorted with
// the library's radix sort: both kernels walk a row's ratings in ascending
// column order, so every sum has a fixed order.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "../../include/dfacto.h"
#include "device.cuh"
#include "internal.h"

namespace dfacto {

struct JointState {
  double mu = 0.0;
  int64_t nnzY = 0;
  int64_t* ptr[2] = {nullptr, nullptr};  // [dims[side] + 1]
  int32_t* col[2] = {nullptr, nullptr};  // [nnzY]: item (side 0) or user (side 1)
  float* val[2] = {nullptr, nullptr};    // [nnzY]
  double* base = nullptr;                // [R x R] mu Gamma + lambda I
  float* gam32 = nullptr;                // [R x R] Gamma
  double* ycoef = nullptr;               // [5] ratings quartic along the ray
  double* part = nullptr;                // block partials
  int64_t part_cap = 0;                  // doubles
};

namespace {

constexpr int kJT = 256;       // threads of the gradient and quartic kernels
constexpr int kJRowWarps = 4;  // warps of the ALS row kernel
constexpr int kJMaxBlocks = 152 * 8;

unsigned jgrid(int64_t rows, int warps) {
  const int64_t b = (rows + warps - 1) / warps;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kJMaxBlocks));
}

__global__ void ratings_in_range(const int32_t* __restrict__ yidx, int64_t n, int32_t I, int32_t J,
                                 int32_t* __restrict__ flag) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const int32_t i = yidx[t], j = yidx[n + t];
    bad |= (i < 0) | (i >= I) | (j < 0) | (j >= J);
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// key = (row << bits_col) | col for the CSR of `side` (row = user for side 0).
__global__ void rating_keys(const int32_t* __restrict__ yidx, int64_t n, int side, int bits_col,
                            uint64_t* __restrict__ key, uint32_t* __restrict__ perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const uint64_t row = (uint32_t)yidx[(int64_t)side * n + t];
    const uint64_t col = (uint32_t)yidx[(int64_t)(1 - side) * n + t];
    key[t] = (row << bits_col) | col;
    perm[t] = (uint32_t)t;
  }
}

__global__ void rating_scatter(const uint64_t* __restrict__ key, const uint32_t* __restrict__ perm,
                               const float* __restrict__ yval, int64_t n, int bits_col,
                               int32_t* __restrict__ col, float* __restrict__ val,
                               int32_t* __restrict__ dup) {
  const uint64_t mask = (uint64_t(1) << bits_col) - 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool d = false;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    col[t] = (int32_t)(key[t] & mask);
    val[t] = yval[perm[t]];
    d |= t > 0 && key[t] == key[t - 1];
  }
  if (__any_sync(kFull, d) && (threadIdx.x & 31) == 0) atomicOr(dup, 1);
}

// ptr[r] = first position whose row is >= r.
__global__ void rating_ptr(const uint64_t* __restrict__ key, int64_t n, int64_t rows, int bits_col,
                           int64_t* __restrict__ ptr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= rows; r += stride) {
    const uint64_t k = (uint64_t)r << bits_col;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (key[mid] < k) lo = mid + 1; else hi = mid;
    }
    ptr[r] = lo;
  }
}

__global__ void fill_ones(double* p, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 1.0;
}

// base = mu (Gf * Gi) + lambda I (FP64) and Gamma = Gf * Gi (FP32).
__global__ void joint_base(const double* __restrict__ Gf, const double* __restrict__ Gi, int R,
                           double mu, double lambda, double* __restrict__ base,
                           float* __restrict__ gam32) {
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const double g = Gf[e] * Gi[e];
    base[e] = mu * g + (e / R == e % R ? lambda : 0.0);
    gam32[e] = (float)g;
  }
}

__device__ __forceinline__ float ld_f(const float* p) { return *p; }
__device__ __forceinline__ float ld_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// ALS row update, one warp per row, lane l on column l (R <= 32):
// F[row] = rhs H^-1 with H = base + sum over the row's ratings of v^T v
// (Cholesky in FP64 shared memory; H is positive definite for lambda > 0).
template <typename T>
__global__ void __launch_bounds__(kJRowWarps * 32) joint_rows(
    const int64_t* __restrict__ yptr, const int32_t* __restrict__ ycol,
    const float* __restrict__ yval, const T* __restrict__ other, const float* __restrict__ N,
    const double* __restrict__ base, double mu, int64_t rows, int R, T* __restrict__ F,
    int32_t* __restrict__ bad_flag) {
  extern __shared__ double jsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int LD = R + 1;
  double* H = jsm + (size_t)warp * (R * LD + R);
  double* x = H + R * LD;
  const int64_t nw = (int64_t)gridDim.x * kJRowWarps;
  for (int64_t row = (int64_t)blockIdx.x * kJRowWarps + warp; row < rows; row += nw) {
    float hrow[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) hrow[m] = 0.f;
    double rhs = lane < R ? mu * (double)N[row * R + lane] : 0.0;
    if (yptr) {
      const int64_t p1 = yptr[row + 1];
      for (int64_t p = yptr[row]; p < p1; ++p) {
        const int64_t o = ycol[p];
        const float y = yval[p];
        const float v = lane < R ? ld_f(other + o * R + lane) : 0.f;
        rhs += (double)y * (double)v;
#pragma unroll
        for (int m = 0; m < 32; ++m) hrow[m] = fmaf(v, __shfl_sync(kFull, v, m), hrow[m]);
      }
    }
    if (lane < R) {
#pragma unroll
      for (int m = 0; m < 32; ++m)
        if (m < R) H[lane * LD + m] = base[lane * R + m] + (double)hrow[m];
      x[lane] = rhs;
    }
    __syncwarp();
    bool bad = false;
    for (int k = 0; k < R; ++k) {
      const double d = H[k * LD + k];
      bad |= !(d > 0.0);
      const double lkk = sqrt(fmax(d, 1e-300));
      __syncwarp();
      if (lane > k && lane < R) H[lane * LD + k] /= lkk;
      __syncwarp();
      if (lane > k && lane < R) {
        const double lik = H[lane * LD + k];
        for (int m = k + 1; m <= lane; ++m) H[lane * LD + m] -= lik * H[m * LD + k];
      }
      if (lane == k) H[k * LD + k] = lkk;
      __syncwarp();
    }
    if (lane == 0) {  // L L^T x = rhs
      for (int r = 0; r < R; ++r) {
        double s = x[r];
        for (int k = 0; k < r; ++k) s -= H[r * LD + k] * x[k];
        x[r] = s / H[r * LD + r];
      }
      for (int r = R - 1; r >= 0; --r) {
        double s = x[r];
        for (int k = r + 1; k < R; ++k) s -= H[k * LD + r] * x[k];
        x[r] = s / H[r * LD + r];
      }
      if (bad) atomicOr(bad_flag, 1);
    }
    __syncwarp();
    if (lane < R) st_elem(F + row * R + lane, (float)x[lane]);
    __syncwarp();
  }
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Block sum of per-thread doubles in a fixed order (into thread 0).
__device__ __forceinline__ double jblock_sum(double v, double* s) {
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = kJT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  const double t = s[0];
  __syncthreads();
  return t;
}

// GD gradient rows (Eq. grad-joint-A), one warp per row, lane l on column l:
//   g = mu (-N[row] + F[row] Gamma) + lambda F[row]
//       + sum over the row's ratings of (F[row] . v - y) v
// with per-block partials of ||g||^2, <g, N>, <F, N> (part[block][3]).
template <typename T>
__global__ void __launch_bounds__(kJT) joint_grad(
    const int64_t* __restrict__ yptr, const int32_t* __restrict__ ycol,
    const float* __restrict__ yval, const T* __restrict__ other, const float* __restrict__ N,
    const float* __restrict__ gam32, double mu, double lambda, int64_t rows, int R,
    const T* __restrict__ F, float* __restrict__ grad, double* __restrict__ part) {
  __shared__ float sg[32 * 32];
  __shared__ double red[kJT];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) sg[e] = gam32[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = kJT / 32;
  const int64_t nw = (int64_t)gridDim.x * W;
  double a_g2 = 0.0, a_gn = 0.0, a_fn = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * W + warp; row < rows; row += nw) {
    const float f = lane < R ? ld_f(F + row * R + lane) : 0.f;
    const float n = lane < R ? N[row * R + lane] : 0.f;
    float fg = 0.f;
    for (int m = 0; m < R; ++m) {
      const float fm = __shfl_sync(kFull, f, m);
      if (lane < R) fg = fmaf(fm, sg[m * R + lane], fg);
    }
    float g = (float)(mu * (double)(fg - n) + lambda * (double)f);
    if (yptr) {
      const int64_t p1 = yptr[row + 1];
      for (int64_t p = yptr[row]; p < p1; ++p) {
        const int64_t o = ycol[p];
        const float v = lane < R ? ld_f(other + o * R + lane) : 0.f;
        const float e = wsum(f * v) - yval[p];
        g = fmaf(e, v, g);
      }
    }
    if (lane < R) {
      grad[row * R + lane] = g;
      a_g2 += (double)g * g;
      a_gn += (double)g * n;
      a_fn += (double)f * n;
    }
  }
  const double v0 = jblock_sum(a_g2, red);
  const double v1 = jblock_sum(a_gn, red);
  const double v2 = jblock_sum(a_fn, red);
  if (threadIdx.x == 0) {
    part[(size_t)blockIdx.x * 3] = v0;
    part[(size_t)blockIdx.x * 3 + 1] = v1;
    part[(size_t)blockIdx.x * 3 + 2] = v2;
  }
}

// scal[kG2] += sum ||g||^2; scal[dst1] = <g, N> (T100, T010 or T001);
// scal[dst2] = <F, N> (T000, mode 0 only).
__global__ void __launch_bounds__(kJT) joint_grad_scalars(const double* __restrict__ part, int nb,
                                                         double* __restrict__ scal, int dst1, int dst2) {
  __shared__ double red[kJT];
  double v[3];
  for (int t = 0; t < 3; ++t) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += kJT) a += part[(size_t)b * 3 + t];
    v[t] = jblock_sum(a, red);
  }
  if (threadIdx.x == 0) {
    scal[kG2] += v[0];
    scal[dst1] = v[1];
    if (dst2 >= 0) scal[dst2] = v[2];
  }
}

// The ratings term along the ray theta - alpha grad, per user row (warp per
// row): r(alpha) = y - (a - alpha ga) . (b - alpha gb) = e0 + e1 alpha + e2 alpha^2
// and 1/2 r^2 has coefficients 1/2 e0^2, e0 e1, 1/2 e1^2 + e0 e2, e1 e2, 1/2 e2^2;
// per-block partials part[block][5].  With GA == nullptr only the first (the
// ratings loss at the current point) is formed.
template <typename T>
__global__ void __launch_bounds__(kJT) ratings_quartic(
    const int64_t* __restrict__ yptr, const int32_t* __restrict__ ycol,
    const float* __restrict__ yval, const T* __restrict__ A, const T* __restrict__ B,
    const float* __restrict__ GA, const float* __restrict__ GB, int64_t rows, int R,
    double* __restrict__ part) {
  __shared__ double red[kJT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = kJT / 32;
  const int64_t nw = (int64_t)gridDim.x * W;
  double c[5] = {0, 0, 0, 0, 0};
  for (int64_t row = (int64_t)blockIdx.x * W + warp; row < rows; row += nw) {
    const float a = lane < R ? ld_f(A + row * R + lane) : 0.f;
    const float ga = (GA && lane < R) ? GA[row * R + lane] : 0.f;
    const int64_t p1 = yptr[row + 1];
    for (int64_t p = yptr[row]; p < p1; ++p) {
      const int64_t o = ycol[p];
      const float b = lane < R ? ld_f(B + o * R + lane) : 0.f;
      const float gb = (GB && lane < R) ? GB[o * R + lane] : 0.f;
      const double u0 = (double)wsum(a * b);
      const double e0 = (double)yval[p] - u0;
      double e1 = 0.0, e2 = 0.0;
      if (GA) {
        e1 = (double)wsum(fmaf(a, gb, ga * b));
        e2 = -(double)wsum(ga * gb);
      }
      if (lane == 0) {
        c[0] += 0.5 * e0 * e0;
        c[1] += e0 * e1;
        c[2] += 0.5 * e1 * e1 + e0 * e2;
        c[3] += e1 * e2;
        c[4] += 0.5 * e2 * e2;
      }
    }
  }
  for (int k = 0; k < 5; ++k) {
    const double v = jblock_sum(c[k], red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 5 + k] = v;
  }
}

__global__ void __launch_bounds__(kJT) sum5(const double* __restrict__ part, int nb,
                                           double* __restrict__ out) {
  __shared__ double red[kJT];
  for (int k = 0; k < 5; ++k) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += kJT) a += part[(size_t)b * 5 + k];
    const double v = jblock_sum(a, red);
    if (threadIdx.x == 0) out[k] = v;
  }
}

// The joint objective at the current point: ratings loss ycoef[0], the tensor
// loss from the fit's pieces (lambda weights are 1), the ridge from the Grams.
__global__ void joint_objective_k(const double* __restrict__ ycoef, const double* __restrict__ GA,
                                  const double* __restrict__ GB, const double* __restrict__ GC, int R,
                                  double mu, double lambda, double* __restrict__ scal) {
  if (threadIdx.x != 0) return;
  double tr = 0.0;
  for (int r = 0; r < R; ++r) tr += GA[r * R + r] + GB[r * R + r] + GC[r * R + r];
  const double ft = 0.5 * (scal[kNormX2] - 2.0 * scal[kInner] + scal[kModelNorm2]);
  scal[kLoss] = ycoef[0] + mu * ft + 0.5 * lambda * tr;
}

dfacto_status grow_part(dfacto_t* h, int64_t doubles) {
  JointState* J = h->joint;
  if (doubles <= J->part_cap) return DFACTO_OK;
  if (J->part) dfree(h, J->part, sizeof(double) * (size_t)J->part_cap);
  J->part = nullptr;
  J->part_cap = 0;
  dfacto_status st = dalloc(h, reinterpret_cast<void**>(&J->part), sizeof(double) * (size_t)doubles);
  if (st == DFACTO_OK) J->part_cap = doubles;
  return st;
}

int bits_for(int64_t dim) {
  int b = 1;
  while (b < 40 && (int64_t(1) << b) < dim) ++b;
  return b;
}

template <typename T>
dfacto_status joint_rows_side(dfacto_t* h, int side) {
  JointState* J = h->joint;
  const int R = h->R;
  cudaStream_t s = h->stream;
  dfacto_status st;
  const int f = (side + 2) % 3, in = (side + 1) % 3;
  for (int m : {f, in})
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  joint_base<<<1, 256, 0, s>>>(h->gram[f], h->gram[in], R, J->mu, h->lambda_reg, J->base, J->gam32);
  DF_COUNT();
  if ((st = mttkrp_launch(h, side, h->N)) != DFACTO_OK) return st;
  const int64_t rows = h->dims[side];
  const size_t smem = sizeof(double) * (size_t)kJRowWarps * (R * (R + 1) + R);
  DF_CUDA(h, ensure_dynamic_smem(reinterpret_cast<const void*>(joint_rows<T>), smem));
  const bool rated = side < 2;
  joint_rows<T><<<jgrid(rows, kJRowWarps), kJRowWarps * 32, smem, s>>>(
      rated ? J->ptr[side] : nullptr, rated ? J->col[side] : nullptr,
      rated ? J->val[side] : nullptr, static_cast<const T*>(h->F[side == 0 ? 1 : 0]), h->N, J->base,
      J->mu, rows, R, static_cast<T*>(h->F[side]), h->flags + kFlagInternal);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  h->gram_valid[side] = false;
  return DFACTO_OK;
}

template <typename T>
dfacto_status joint_objective_T(dfacto_t* h) {
  JointState* J = h->joint;
  cudaStream_t s = h->stream;
  dfacto_status st;
  fill_ones<<<1, 128, 0, s>>>(h->lambda, h->R);
  DF_COUNT();
  if ((st = fit_direct(h)) != DFACTO_OK) return st;  // <X, Xhat>, ||Xhat||^2 (and the Grams)
  const unsigned nb = jgrid(h->dims[0], kJT / 32);
  if ((st = grow_part(h, (int64_t)nb * 5)) != DFACTO_OK) return st;
  ratings_quartic<T><<<nb, kJT, 0, s>>>(J->ptr[0], J->col[0], J->val[0],
                                       static_cast<const T*>(h->F[0]), static_cast<const T*>(h->F[1]),
                                       nullptr, nullptr, h->dims[0], h->R, J->part);
  DF_COUNT();
  sum5<<<1, kJT, 0, s>>>(J->part, (int)nb, J->ycoef);
  DF_COUNT();
  joint_objective_k<<<1, 32, 0, s>>>(J->ycoef, h->gram[0], h->gram[1], h->gram[2], h->R, J->mu,
                                     h->lambda_reg, h->scal);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

template <typename T>
dfacto_status joint_gd_T(dfacto_t* h) {
  JointState* J = h->joint;
  const int R = h->R;
  cudaStream_t s = h->stream;
  dfacto_status st;
  DF_CUDA(h, cudaMemsetAsync(h->scal + kG2, 0, sizeof(double), s));
  for (int side = 0; side < 3; ++side) {
    const int f = (side + 2) % 3, in = (side + 1) % 3;
    for (int m : {f, in})
      if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
    joint_base<<<1, 256, 0, s>>>(h->gram[f], h->gram[in], R, J->mu, h->lambda_reg, J->base,
                                 J->gam32);
    DF_COUNT();
    if ((st = mttkrp_launch(h, side, h->N)) != DFACTO_OK) return st;
    const int64_t rows = h->dims[side];
    const unsigned nb = jgrid(rows, kJT / 32);
    if ((st = grow_part(h, (int64_t)nb * 5)) != DFACTO_OK) return st;
    const bool rated = side < 2;
    joint_grad<T><<<nb, kJT, 0, s>>>(rated ? J->ptr[side] : nullptr, rated ? J->col[side] : nullptr,
                                     rated ? J->val[side] : nullptr,
                                     static_cast<const T*>(h->F[side == 0 ? 1 : 0]), h->N, J->gam32,
                                     J->mu, h->lambda_reg, rows, R, static_cast<const T*>(h->F[side]),
                                     h->grad[side], J->part);
    DF_COUNT();
    const int tlin = side == 0 ? kT100 : (side == 1 ? kT010 : kT001);
    joint_grad_scalars<<<1, kJT, 0, s>>>(J->part, (int)nb, h->scal, tlin, side == 0 ? kT000 : -1);
    DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
  }
  {  // the ratings quartic along the ray
    const unsigned nb = jgrid(h->dims[0], kJT / 32);
    if ((st = grow_part(h, (int64_t)nb * 5)) != DFACTO_OK) return st;
    ratings_quartic<T><<<nb, kJT, 0, s>>>(J->ptr[0], J->col[0], J->val[0],
                                         static_cast<const T*>(h->F[0]),
                                         static_cast<const T*>(h->F[1]), h->grad[0], h->grad[1],
                                         h->dims[0], R, J->part);
    DF_COUNT();
    sum5<<<1, kJT, 0, s>>>(J->part, (int)nb, J->ycoef);
    DF_COUNT();
  }
  if ((st = ray_matrices(h)) != DFACTO_OK) return st;
  if ((st = dual_pass(h)) != DFACTO_OK) return st;
  if ((st = line_search(h, J->mu, J->ycoef)) != DFACTO_OK) return st;
  return apply_step(h);
}

dfacto_status read_flags(dfacto_t* h) {
  DF_CUDA(h, cudaMemcpyAsync(h->host_scal, h->scal, sizeof(double) * kNumScalars,
                             cudaMemcpyDeviceToHost, h->stream));
  DF_CUDA(h, cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int32_t) * kNumFlags,
                             cudaMemcpyDeviceToHost, h->stream));
  DF_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->host_flags[kFlagInternal]) return fail(h, DFACTO_EINTERNAL, "joint row solve failed");
  return DFACTO_OK;
}

}  // namespace

void joint_free(dfacto_t* h) {
  JointState* J = h->joint;
  if (!J) return;
  for (int side = 0; side < 2; ++side)
    for (void* q : {(void*)J->ptr[side], (void*)J->col[side], (void*)J->val[side]})
      if (q) cudaFreeAsync(q, h->stream);
  for (void* q : {(void*)J->base, (void*)J->gam32, (void*)J->ycoef, (void*)J->part})
    if (q) cudaFreeAsync(q, h->stream);
  delete J;
  h->joint = nullptr;
}

}  // namespace dfacto

using namespace dfacto;

extern "C" {

dfacto_status dfacto_joint_set_ratings(dfacto_t* h, const int32_t* yidx, const float* yval,
                                       int64_t nnzY, double mu) {
  if (!h || nnzY < 0 || nnzY > kMaxNnz || (nnzY > 0 && (!yidx || !yval)) || !(mu >= 0.0))
    return DFACTO_EINVAL;
  if (h->R > 32) return fail(h, DFACTO_EINVAL, "the joint model takes R <= 32");
  if (h->batch) return fail(h, DFACTO_EINVAL, "handle is in a batch");
  cudaStream_t s = h->stream;
  joint_free(h);
  JointState* J = new (std::nothrow) JointState();
  if (!J) return DFACTO_ENOMEM;
  h->joint = J;
  J->mu = mu;
  J->nnzY = nnzY;
  const int R = h->R;
  dfacto_status st = DFACTO_OK;
  auto bail = [&](dfacto_status e) {
    joint_free(h);
    return e;
  };
  if ((st = dalloc(h, (void**)&J->base, sizeof(double) * R * R)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&J->gam32, sizeof(float) * R * R)) != DFACTO_OK) return bail(st);
  if ((st = dalloc(h, (void**)&J->ycoef, sizeof(double) * 8)) != DFACTO_OK) return bail(st);
  for (int side = 0; side < 2; ++side) {
    if ((st = dalloc(h, (void**)&J->ptr[side], sizeof(int64_t) * ((size_t)h->dims[side] + 1))) != DFACTO_OK)
      return bail(st);
    if ((st = dalloc(h, (void**)&J->col[side], sizeof(int32_t) * (size_t)nnzY)) != DFACTO_OK)
      return bail(st);
    if ((st = dalloc(h, (void**)&J->val[side], sizeof(float) * (size_t)nnzY)) != DFACTO_OK)
      return bail(st);
  }
  // the ratings on the device
  const int32_t* d_idx = yidx;
  const float* d_val = yval;
  int32_t* tmp_idx = nullptr;
  float* tmp_val = nullptr;
  uint64_t* k0 = nullptr;
  uint64_t* k1 = nullptr;
  uint32_t* v0 = nullptr;
  uint32_t* v1 = nullptr;
  auto cleanup = [&]() {
    for (void* q : {(void*)tmp_idx, (void*)tmp_val, (void*)k0, (void*)k1, (void*)v0, (void*)v1})
      if (q) cudaFreeAsync(q, s);
  };
  auto cuda_bail = [&](cudaError_t e, const char* what) {
    cleanup();
    st = cuda_fail(h, e, what);
    joint_free(h);
    return st;
  };
  cudaError_t e = cudaSuccess;
  if (nnzY > 0 && !is_device_ptr(yidx)) {
    if ((e = cudaMallocAsync((void**)&tmp_idx, sizeof(int32_t) * 2 * nnzY, s)) != cudaSuccess)
      return cuda_bail(e, "ratings copy");
    if ((e = cudaMemcpyAsync(tmp_idx, yidx, sizeof(int32_t) * 2 * nnzY, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_bail(e, "ratings copy");
    d_idx = tmp_idx;
  }
  if (nnzY > 0 && !is_device_ptr(yval)) {
    if ((e = cudaMallocAsync((void**)&tmp_val, sizeof(float) * nnzY, s)) != cudaSuccess)
      return cuda_bail(e, "ratings copy");
    if ((e = cudaMemcpyAsync(tmp_val, yval, sizeof(float) * nnzY, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_bail(e, "ratings copy");
    d_val = tmp_val;
  }
  if ((e = cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, s)) != cudaSuccess)
    return cuda_bail(e, "flags");
  if (nnzY > 0) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nnzY + 255) / 256, 152 * 32));
    ratings_in_range<<<g, 256, 0, s>>>(d_idx, nnzY, h->dims[0], h->dims[1], h->flags + kFlagRange);
    DF_COUNT();
    if ((e = cudaMallocAsync((void**)&k0, sizeof(uint64_t) * nnzY, s)) != cudaSuccess ||
        (e = cudaMallocAsync((void**)&k1, sizeof(uint64_t) * nnzY, s)) != cudaSuccess ||
        (e = cudaMallocAsync((void**)&v0, sizeof(uint32_t) * nnzY, s)) != cudaSuccess ||
        (e = cudaMallocAsync((void**)&v1, sizeof(uint32_t) * nnzY, s)) != cudaSuccess)
      return cuda_bail(e, "ratings sort buffers");
  }
  for (int side = 0; side < 2; ++side) {
    const int64_t rows = h->dims[side];
    const int bc = bits_for(h->dims[1 - side]), br = bits_for(rows);
    bool alt = false;
    if (nnzY > 0) {
      const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nnzY + 255) / 256, 152 * 32));
      rating_keys<<<g, 256, 0, s>>>(d_idx, nnzY, side, bc, k0, v0);
      DF_COUNT();
      if ((e = sort_pairs64(k0, v0, k1, v1, nnzY, 0, bc + br, s, &alt)) != cudaSuccess)
        return cuda_bail(e, "ratings sort");
      const uint64_t* ks = alt ? k1 : k0;
      const uint32_t* vs = alt ? v1 : v0;
      rating_scatter<<<g, 256, 0, s>>>(ks, vs, d_val, nnzY, bc, J->col[side], J->val[side],
                                       h->flags + kFlagDup);
      DF_COUNT();
      rating_ptr<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 256) / 256, 152 * 32)), 256, 0, s>>>(
          ks, nnzY, rows, bc, J->ptr[side]);
      DF_COUNT();
    } else {
      if ((e = cudaMemsetAsync(J->ptr[side], 0, sizeof(int64_t) * (rows + 1), s)) != cudaSuccess)
        return cuda_bail(e, "ratings pointers");
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_bail(e, "ratings build");
  }
  cleanup();
  int32_t flags[kNumFlags];
  if ((e = cudaMemcpyAsync(flags, h->flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_bail(e, "ratings check");
  if (flags[kFlagRange]) {
    joint_free(h);
    return fail(h, DFACTO_ERANGE, "a rating lies outside dims[0] x dims[1]");
  }
  if (flags[kFlagDup]) {
    joint_free(h);
    return fail(h, DFACTO_EDUP, "two ratings share (user, item)");
  }
  return DFACTO_OK;
}

dfacto_status dfacto_get_ratings_csr(dfacto_t* h, int side, dfacto_ratings_view* v) {
  if (!h || !v || side < 0 || side > 1) return DFACTO_EINVAL;
  if (!h->joint) return fail(h, DFACTO_EINVAL, "no ratings set");
  v->rows = h->dims[side];
  v->nnz = h->joint->nnzY;
  v->ptr = h->joint->ptr[side];
  v->col = h->joint->col[side];
  v->val = h->joint->val[side];
  return DFACTO_OK;
}

dfacto_status dfacto_joint_als_iter(dfacto_t* h, double* obj_out) {
  if (!h) return DFACTO_EINVAL;
  if (!h->joint) return fail(h, DFACTO_EINVAL, "no ratings set");
  if (!(h->lambda_reg > 0.0)) return fail(h, DFACTO_EINVAL, "the joint ALS needs lambda_reg > 0");
  DF_CUDA(h, cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, h->stream));
  dfacto_status st;
  for (int side = 0; side < 3; ++side) {
    st = h->dtype == DFACTO_BF16 ? joint_rows_side<__nv_bfloat16>(h, side) : joint_rows_side<float>(h, side);
    if (st != DFACTO_OK) return st;
  }
  if (!obj_out) return DFACTO_OK;
  st = h->dtype == DFACTO_BF16 ? joint_objective_T<__nv_bfloat16>(h) : joint_objective_T<float>(h);
  if (st != DFACTO_OK) return st;
  if ((st = read_flags(h)) != DFACTO_OK) return st;
  *obj_out = h->host_scal[kLoss];
  return DFACTO_OK;
}

dfacto_status dfacto_joint_gd_iter(dfacto_t* h, double* obj_out, double* alpha_out) {
  if (!h) return DFACTO_EINVAL;
  if (!h->joint) return fail(h, DFACTO_EINVAL, "no ratings set");
  dfacto_status st;
  for (int m = 0; m < 3; ++m)
    if (!h->grad[m] &&
        (st = dalloc(h, (void**)&h->grad[m], sizeof(float) * (size_t)h->dims[m] * h->R)) != DFACTO_OK)
      return st;
  DF_CUDA(h, cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, h->stream));
  st = h->dtype == DFACTO_BF16 ? joint_gd_T<__nv_bfloat16>(h) : joint_gd_T<float>(h);
  if (st != DFACTO_OK) return st;
  if (!obj_out && !alpha_out) return DFACTO_OK;
  if ((st = read_flags(h)) != DFACTO_OK) return st;
  if (obj_out) *obj_out = h->host_scal[kLoss];
  if (alpha_out) *alpha_out = h->host_scal[kStep];
  return h->host_flags[kFlagLsFail] ? DFACTO_ELSFAIL : DFACTO_OK;
}

dfacto_status dfacto_joint_objective(dfacto_t* h, double* obj_out) {
  if (!h || !obj_out) return DFACTO_EINVAL;
  if (!h->joint) return fail(h, DFACTO_EINVAL, "no ratings set");
  DF_CUDA(h, cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, h->stream));
  dfacto_status st =
      h->dtype == DFACTO_BF16 ? joint_objective_T<__nv_bfloat16>(h) : joint_objective_T<float>(h);
  if (st != DFACTO_OK) return st;
  if ((st = read_flags(h)) != DFACTO_OK) return st;
  *obj_out = h->host_scal[kLoss];
  return DFACTO_OK;
}

}  // extern "C"
