// dense.cu -- the R x R algebra and the row-wise passes around the MTTKRP:
// Grams (Eq. kr-product), the Gram-Hadamard solve of ALS (Eq.
// als-astep-sol-rw, pseudo-inverse of Eq. kr-pseudo as fallback), column
// normalisation and CP weights (Algorithm 2), the fit, and the GD gradient
// (Eq. gd-A), line search and update (Algorithm 5).
//
// Precision: factor rows are read in their storage type and multiplied in
// FP32; every reduction that feeds a Gram, a norm, the fit or the GD objective
// folds FP32 partials of at most kFold rows into FP64, and all R x R work is
// FP64.  Reductions use fixed per-block partials summed in block order, so
// results are bitwise reproducible.
#include <algorithm>
#include <cmath>

#include "device.cuh"
#include "internal.h"
#include "mttkrp.cuh"

namespace dfacto {

dfacto_status mttkrp_launch(dfacto_t* h, int mode, float* out);

namespace {

constexpr int kRowThreads = 256;
constexpr int kFold = 64;  // rows per FP32 partial before folding into FP64
constexpr int kMaxBlocks = 152 * 4;
constexpr int kMaxR = 128;

unsigned row_blocks(int64_t rows, int rows_per_block = 64) {
  int64_t b = (rows + rows_per_block - 1) / rows_per_block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kMaxBlocks));
}

// ---------------------------------------------------------------------------
// Cross Gram X^T Y of two rows x R matrices (X may equal Y), FP64 partial per
// block: part[block][R*R].  Rows are staged in shared memory as float tiles.
// ---------------------------------------------------------------------------
template <typename TX, typename TY, int PER>
__global__ void __launch_bounds__(kRowThreads) cross_gram_partials(const TX* __restrict__ X,
                                                                  const TY* __restrict__ Y,
                                                                  int64_t rows, int R,
                                                                  double* __restrict__ part) {
  extern __shared__ float tile[];  // [trows][R] X then [trows][R] Y
  const int trows = min(kFold, 4096 / R);
  float* tx = tile;
  float* ty = tile + (size_t)trows * R;
  const int RR = R * R;
  constexpr int per = PER;  // entries per thread: ceil(R*R / threads)
  double accd[PER];
#pragma unroll
  for (int q = 0; q < per; ++q) accd[q] = 0.0;
  const int64_t chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(rows, r0 + chunk);
  for (int64_t t0 = r0; t0 < r1; t0 += trows) {
    const int nt = (int)min((int64_t)trows, r1 - t0);
    for (int e = threadIdx.x; e < nt * R; e += kRowThreads) {
      tx[e] = ld_elem(X + t0 * R + e);
      ty[e] = ld_elem(Y + t0 * R + e);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < per; ++q) {
      const int ent = threadIdx.x + q * kRowThreads;
      if (ent < RR) {
        const int a = ent / R, b = ent % R;
        float s = 0.f;
        for (int i = 0; i < nt; ++i) s = fmaf(tx[i * R + a], ty[i * R + b], s);
        accd[q] += (double)s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < per; ++q) {
    const int ent = threadIdx.x + q * kRowThreads;
    if (ent < RR) part[(size_t)blockIdx.x * RR + ent] = accd[q];
  }
}

// out[e] = sum over blocks b (in order) of part[b][e]  (+ part^T if sym).
__global__ void reduce_partials(const double* __restrict__ part, int nblocks, int n, int R,
                                bool symmetrize, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * n + e];
    if (symmetrize) {
      const int a = e / R, c = e % R;
      const int et = c * R + a;
      for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * n + et];
    }
    out[e] = s;
  }
}

// ---------------------------------------------------------------------------
// Gamma = G_f * G_in + lambda_reg I and its inverse (or pseudo-inverse).
// One CTA, FP64 in shared memory.  Cholesky fails when a pivot drops to
// R * eps times its diagonal entry; then the cyclic Jacobi eigen-decomposition
// gives the pseudo-inverse with eigenvalue cutoff R * eps * max |w|.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gamma_inverse(const double* __restrict__ Gf,
                                                    const double* __restrict__ Gi, int R,
                                                    double lambda_reg, double* __restrict__ W,
                                                    float* __restrict__ W32,
                                                    int32_t* __restrict__ singular,
                                                    double* __restrict__ work) {
  double* A = work;               // [R][R] working copy / L
  double* B = work + R * R;       // [R][R] Linv or V
  double* d0 = work + 2 * R * R;  // [R] original diagonal / eigenvalues
  __shared__ int failed;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int RR = R * R;
  const double eps = 2.220446049250313e-16;
  for (int e = tid; e < RR; e += nt) {
    const int a = e / R, b = e % R;
    double g = Gf[e] * Gi[e];
    if (a == b) g += lambda_reg;
    A[e] = g;
  }
  if (tid == 0) failed = 0;
  __syncthreads();
  for (int a = tid; a < R; a += nt) d0[a] = A[a * R + a];
  __syncthreads();
  // Right-looking Cholesky, lower triangle.
  for (int j = 0; j < R; ++j) {
    if (tid == 0) {
      const double d = A[j * R + j];
      if (!(d0[j] > 0.0) || !(d > (double)R * eps * d0[j])) failed = 1;
      else A[j * R + j] = sqrt(d);
    }
    __syncthreads();
    if (failed) break;
    const double ljj = A[j * R + j];
    for (int i = j + 1 + tid; i < R; i += nt) A[i * R + j] /= ljj;
    __syncthreads();
    const int m = R - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) A[i * R + k] -= A[i * R + j] * A[k * R + j];
    }
    __syncthreads();
  }
  if (!failed) {
    // Linv by forward substitution, one column per thread.
    for (int c = tid; c < R; c += nt) {
      for (int i = 0; i < R; ++i) {
        double s = (i == c) ? 1.0 : 0.0;
        if (i >= c) {
          for (int k = c; k < i; ++k) s -= A[i * R + k] * B[k * R + c];
          B[i * R + c] = s / A[i * R + i];
        } else {
          B[i * R + c] = 0.0;
        }
      }
    }
    __syncthreads();
    // W = Linv^T Linv.
    for (int e = tid; e < RR; e += nt) {
      const int a = e / R, b = e % R;
      double s = 0.0;
      for (int k = max(a, b); k < R; ++k) s += B[k * R + a] * B[k * R + b];
      W[e] = s;
      W32[e] = (float)s;
    }
    return;
  }
  // Pseudo-inverse by cyclic Jacobi (Golub & Van Loan, Sec. 8.5).
  if (tid == 0) atomicOr(singular, 1);
  for (int e = tid; e < RR; e += nt) {
    const int a = e / R, b = e % R;
    double g = Gf[e] * Gi[e];
    if (a == b) g += lambda_reg;
    A[e] = g;
    B[e] = (a == b) ? 1.0 : 0.0;
  }
  __syncthreads();
  __shared__ double s_off, s_tot, s_c, s_s;
  for (int sweep = 0; sweep < 100; ++sweep) {
    if (tid == 0) {
      double off = 0.0, tot = 0.0;
      for (int e = 0; e < RR; ++e) {
        tot += A[e] * A[e];
        if (e / R != e % R) off += A[e] * A[e];
      }
      s_off = off;
      s_tot = tot;
    }
    __syncthreads();
    if (s_off <= 1e-30 * s_tot || s_off == 0.0) break;
    for (int p = 0; p < R - 1; ++p)
      for (int q = p + 1; q < R; ++q) {
        if (tid == 0) {
          const double apq = A[p * R + q];
          if (apq == 0.0) {
            s_c = 1.0;
            s_s = 0.0;
          } else {
            const double theta = (A[q * R + q] - A[p * R + p]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            s_c = 1.0 / sqrt(t * t + 1.0);
            s_s = t * s_c;
          }
        }
        __syncthreads();
        const double c = s_c, s = s_s;
        if (s != 0.0) {
          for (int k = tid; k < R; k += nt) {  // columns p, q
            const double akp = A[k * R + p], akq = A[k * R + q];
            A[k * R + p] = c * akp - s * akq;
            A[k * R + q] = s * akp + c * akq;
          }
          __syncthreads();
          for (int k = tid; k < R; k += nt) {  // rows p, q
            const double apk = A[p * R + k], aqk = A[q * R + k];
            A[p * R + k] = c * apk - s * aqk;
            A[q * R + k] = s * apk + c * aqk;
            const double vkp = B[k * R + p], vkq = B[k * R + q];
            B[k * R + p] = c * vkp - s * vkq;
            B[k * R + q] = s * vkp + c * vkq;
          }
        }
        __syncthreads();
      }
  }
  for (int a = tid; a < R; a += nt) d0[a] = A[a * R + a];
  __syncthreads();
  double wmax = 0.0;
  for (int a = 0; a < R; ++a) wmax = fmax(wmax, fabs(d0[a]));
  const double cut = (double)R * eps * wmax;
  for (int e = tid; e < RR; e += nt) {
    const int a = e / R, b = e % R;
    double s = 0.0;
    for (int k = 0; k < R; ++k)
      if (fabs(d0[k]) > cut) s += B[a * R + k] * B[b * R + k] / d0[k];
    W[e] = s;
    W32[e] = (float)s;
  }
}

// ---------------------------------------------------------------------------
// Row-wise passes: one warp per row, lane owns columns lane, lane+32, ...
// ---------------------------------------------------------------------------

// Fhat[o,:] = N[o,:] W; column sums of squares of Fhat -> part[block][R].
__global__ void __launch_bounds__(kRowThreads) als_colnorm_partials(const float* __restrict__ N,
                                                                   const float* __restrict__ W32,
                                                                   int64_t rows, int R,
                                                                   double* __restrict__ part) {
  extern __shared__ float sW[];  // [R][R]
  __shared__ double sacc[kRowThreads / 32][kMaxR];
  for (int e = threadIdx.x; e < R * R; e += kRowThreads) sW[e] = W32[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float accf[4] = {0.f, 0.f, 0.f, 0.f};
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
  int since = 0;
  const int64_t wstride = (int64_t)gridDim.x * (kRowThreads / 32);
  for (int64_t o = (int64_t)blockIdx.x * (kRowThreads / 32) + warp; o < rows; o += wstride) {
    float nrow[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) nrow[q] = (lane + 32 * q < R) ? N[o * R + lane + 32 * q] : 0.f;
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < R; ++k) {
      const float nk = __shfl_sync(kFull, nrow[k >> 5], k & 31);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (lane + 32 * q < R) f[q] = fmaf(nk, sW[k * R + lane + 32 * q], f[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) accf[q] = fmaf(f[q], f[q], accf[q]);
    if (++since == kFold) {
#pragma unroll
      for (int q = 0; q < 4; ++q) { accd[q] += accf[q]; accf[q] = 0.f; }
      since = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    accd[q] += accf[q];
    if (lane + 32 * q < R) sacc[warp][lane + 32 * q] = accd[q];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < R; col += kRowThreads) {
    double s = 0.0;
    for (int w = 0; w < kRowThreads / 32; ++w) s += sacc[w][col];
    part[(size_t)blockIdx.x * R + col] = s;
  }
}

// lambda[r] = sqrt(sum of partials); inv[r] = 1/lambda (0 -> leave column).
__global__ void finish_lambda(const double* __restrict__ part, int nblocks, int R,
                              double* __restrict__ lambda, float* __restrict__ inv) {
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * R + r];
    const double l = sqrt(s);
    lambda[r] = l;
    inv[r] = (l > 0.0) ? (float)(1.0 / l) : 1.0f;
  }
}

// F[o,:] = (N[o,:] W) / lambda, stored in T.  With ipart != null also
// accumulates sum_o F_stored[o,r] * N[o,r] (-> <X, Xhat> after a mode-3 update).
template <typename T>
__global__ void __launch_bounds__(kRowThreads) als_normalize(const float* __restrict__ N,
                                                            const float* __restrict__ W32,
                                                            const float* __restrict__ inv,
                                                            int64_t rows, int R, T* __restrict__ F,
                                                            double* __restrict__ ipart) {
  extern __shared__ float sW[];  // [R][R]
  __shared__ double sacc[kRowThreads / 32][kMaxR];
  for (int e = threadIdx.x; e < R * R; e += kRowThreads) sW[e] = W32[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float sc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) sc[q] = (lane + 32 * q < R) ? inv[lane + 32 * q] : 0.f;
  float accf[4] = {0.f, 0.f, 0.f, 0.f};
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
  int since = 0;
  const int64_t wstride = (int64_t)gridDim.x * (kRowThreads / 32);
  for (int64_t o = (int64_t)blockIdx.x * (kRowThreads / 32) + warp; o < rows; o += wstride) {
    float nrow[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) nrow[q] = (lane + 32 * q < R) ? N[o * R + lane + 32 * q] : 0.f;
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < R; ++k) {
      const float nk = __shfl_sync(kFull, nrow[k >> 5], k & 31);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (lane + 32 * q < R) f[q] = fmaf(nk, sW[k * R + lane + 32 * q], f[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = lane + 32 * q;
      if (col < R) {
        const float val = f[q] * sc[q];
        st_elem(F + o * R + col, val);
        if (ipart) accf[q] = fmaf(rt_elem(F, val), nrow[q], accf[q]);
      }
    }
    if (ipart && ++since == kFold) {
#pragma unroll
      for (int q = 0; q < 4; ++q) { accd[q] += accf[q]; accf[q] = 0.f; }
      since = 0;
    }
  }
  if (!ipart) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    accd[q] += accf[q];
    if (lane + 32 * q < R) sacc[warp][lane + 32 * q] = accd[q];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < R; col += kRowThreads) {
    double s = 0.0;
    for (int w = 0; w < kRowThreads / 32; ++w) s += sacc[w][col];
    ipart[(size_t)blockIdx.x * R + col] = s;
  }
}

// Fit from scalars and Grams (one thread block):
//   <X,Xhat> = sum_r lambda_r * ip[r];  ||Xhat||^2 = lambda^T (GA*GB*GC) lambda.
__global__ void fit_from_parts(const double* __restrict__ ipart, int nblocks, int R,
                               const double* __restrict__ lambda, const double* __restrict__ GA,
                               const double* __restrict__ GB, const double* __restrict__ GC,
                               double* __restrict__ scal) {
  __shared__ double s_ip[kMaxR];
  __shared__ double s_red[256];
  const int tid = threadIdx.x;
  for (int r = tid; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += ipart[(size_t)b * R + r];
    s_ip[r] = s;
  }
  double m = 0.0;
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int a = e / R, b = e % R;
    m += lambda[a] * lambda[b] * GA[e] * GB[e] * GC[e];
  }
  s_red[tid] = m;
  __syncthreads();
  if (tid == 0) {
    double nm2 = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) nm2 += s_red[t];
    double ip = 0.0;
    for (int r = 0; r < R; ++r) ip += lambda[r] * s_ip[r];
    const double nx2 = scal[kNormX2];
    double res2 = nx2 - 2.0 * ip + nm2;
    if (res2 < 0.0) res2 = 0.0;
    scal[kInner] = ip;
    scal[kModelNorm2] = nm2;
    scal[kFit] = nx2 > 0.0 ? 1.0 - sqrt(res2) / sqrt(nx2) : 0.0;
  }
}

// ---------------------------------------------------------------------------
// GD.
// ---------------------------------------------------------------------------

// grad[o,:] = -N[o,:] + F[o,:] Gamma (Gamma already holds + lambda_reg I).
// Scalar partials per block (FP64): [0] ||grad||^2, [1] sum grad*N, [2] sum F*N.
template <typename T>
__global__ void __launch_bounds__(kRowThreads) gd_gradient_rows(const float* __restrict__ N,
                                                               const T* __restrict__ F,
                                                               const float* __restrict__ Gam32,
                                                               int64_t rows, int R,
                                                               float* __restrict__ grad,
                                                               double* __restrict__ spart) {
  extern __shared__ float sG[];  // [R][R]
  __shared__ double sred[3][kRowThreads / 32];
  for (int e = threadIdx.x; e < R * R; e += kRowThreads) sG[e] = Gam32[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float af[3] = {0.f, 0.f, 0.f};
  double ad[3] = {0.0, 0.0, 0.0};
  int since = 0;
  const int64_t wstride = (int64_t)gridDim.x * (kRowThreads / 32);
  for (int64_t o = (int64_t)blockIdx.x * (kRowThreads / 32) + warp; o < rows; o += wstride) {
    float frow[4], nrow[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = lane + 32 * q;
      frow[q] = (col < R) ? ld_elem(F + o * R + col) : 0.f;
      nrow[q] = (col < R) ? N[o * R + col] : 0.f;
    }
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < R; ++k) {
      const float fk = __shfl_sync(kFull, frow[k >> 5], k & 31);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (lane + 32 * q < R) g[q] = fmaf(fk, sG[k * R + lane + 32 * q], g[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = lane + 32 * q;
      if (col < R) {
        const float gv = g[q] - nrow[q];
        grad[o * R + col] = gv;
        af[0] = fmaf(gv, gv, af[0]);
        af[1] = fmaf(gv, nrow[q], af[1]);
        af[2] = fmaf(frow[q], nrow[q], af[2]);
      }
    }
    if (++since == kFold) {
#pragma unroll
      for (int t = 0; t < 3; ++t) { ad[t] += af[t]; af[t] = 0.f; }
      since = 0;
    }
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    ad[t] += af[t];
    ad[t] = warp_sum(ad[t]);
    if (lane == 0) sred[t][warp] = ad[t];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kRowThreads / 32; ++w) s += sred[threadIdx.x][w];
    spart[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

// Gam = G_f * G_in + lambda_reg I in FP64 and FP32.
__global__ void hadamard_gamma(const double* __restrict__ Gf, const double* __restrict__ Gi, int R,
                               double lambda_reg, double* __restrict__ Gam,
                               float* __restrict__ Gam32) {
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double g = Gf[e] * Gi[e];
    if (e / R == e % R) g += lambda_reg;
    Gam[e] = g;
    Gam32[e] = (float)g;
  }
}

// Sum scalar partials [nblocks][k] in block order into scal[dst + i].
__global__ void reduce_scalars(const double* __restrict__ part, int nblocks, int k,
                               double* __restrict__ scal, int dst0, int dst1, int dst2) {
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * k + threadIdx.x];
    const int dst = threadIdx.x == 0 ? dst0 : (threadIdx.x == 1 ? dst1 : dst2);
    if (dst >= 0) scal[dst] = (dst == kG2) ? scal[dst] + s : s;
  }
}

// The GD objective along the search ray theta - alpha * grad (exact, FP64):
//   f(alpha) = 1/2 (||X||^2 - 2 P(alpha) + Q(alpha)) + 1/2 lambda_reg sum_n tr M_n(alpha)
//   P(alpha) = <X, [[A - aGA, B - aGB, C - aGC]]> = sum_S (-alpha)^|S| T_S
//   M_n(alpha) = P0_n - alpha P1_n + alpha^2 P2_n   (Gram of F_n - alpha G_n)
//   Q(alpha) = sum_rs prod_n M_n(alpha)_rs         (||[[.]]||^2, Eq. kr-product)
// Backtracking as specified in dfacto.h; one CTA.
__global__ void __launch_bounds__(256) gd_line_search(const double* __restrict__ mats, int R,
                                                     double lambda_reg, double* __restrict__ scal,
                                                     int32_t* __restrict__ lsfail) {
  __shared__ double red[256];
  __shared__ double s_q;
  const int tid = threadIdx.x;
  const int RR = R * R;
  auto Q = [&](double a) {
    double s = 0.0;
    for (int e = tid; e < RR; e += blockDim.x) {
      double p = 1.0;
      for (int n = 0; n < 3; ++n) {
        const double* P = mats + (size_t)n * 3 * RR;
        p *= P[e] - a * P[RR + e] + a * a * P[2 * RR + e];
      }
      s += p;
    }
    red[tid] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
      s_q = t;
    }
    __syncthreads();
    return s_q;
  };
  auto trace_sum = [&](double a) {
    double t = 0.0;
    for (int n = 0; n < 3; ++n) {
      const double* P = mats + (size_t)n * 3 * RR;
      for (int r = 0; r < R; ++r) {
        const int e = r * R + r;
        t += P[e] - a * P[RR + e] + a * a * P[2 * RR + e];
      }
    }
    return t;
  };
  const double nx2 = scal[kNormX2];
  const double t0 = scal[kT000];
  const double t1 = scal[kT100] + scal[kT010] + scal[kT001];
  const double t2 = scal[kT110] + scal[kT101] + scal[kT011];
  const double t3 = scal[kT111];
  auto f = [&](double a) {
    const double P = t0 - a * t1 + a * a * t2 - a * a * a * t3;
    double v = 0.5 * (nx2 - 2.0 * P + Q(a));
    if (lambda_reg != 0.0) v += 0.5 * lambda_reg * trace_sum(a);
    return v;
  };
  const double f0 = f(0.0);
  const double g2 = scal[kG2];
  const double prev = scal[kAlpha];
  double alpha = prev > 0.0 ? fmin(2.0 * prev, 1.0) : 1.0;
  bool ok = false;
  double fa = f0;
  for (int trial = 0; trial < 40; ++trial) {
    fa = f(alpha);
    if (fa <= f0 - 1e-4 * alpha * g2) {
      ok = true;
      break;
    }
    alpha *= 0.5;
  }
  if (tid == 0) {
    if (ok) {
      scal[kAlpha] = alpha;
      scal[kLoss] = fa;
      scal[kStep] = alpha;
    } else {
      atomicOr(lsfail, 1);
      scal[kLoss] = f0;
      scal[kStep] = 0.0;
    }
  }
}

// F <- F - step * grad (step read from device memory).
template <typename T>
__global__ void gd_update(T* __restrict__ F, const float* __restrict__ grad, int64_t n,
                          const double* __restrict__ scal) {
  const float a = (float)scal[kStep];
  if (a == 0.f) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    st_elem(F + t, ld_elem(F + t) - a * grad[t]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host orchestration.
// ---------------------------------------------------------------------------

namespace {

// Kernels that stage an R x R matrix in shared memory need the opt-in limit
// above 48 KB once R > 110.
template <typename K>
void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename TX, typename TY>
dfacto_status cross_gram(dfacto_t* h, const TX* X, const TY* Y, int64_t rows, double* out,
                         bool symmetrize) {
  const int R = h->R;
  const unsigned nb = row_blocks(rows, 256);
  const int trows = std::min(kFold, 4096 / R);
  const size_t smem = sizeof(float) * 2 * (size_t)trows * R;
  if ((int64_t)nb * R * R > h->partials_cap) return fail(h, DFACTO_EINTERNAL, "partials too small");
  const int per = (R * R + kRowThreads - 1) / kRowThreads;
  if (per <= 1) {
    cross_gram_partials<TX, TY, 1><<<nb, kRowThreads, smem, h->stream>>>(X, Y, rows, R, h->partials);
  } else if (per <= 4) {
    cross_gram_partials<TX, TY, 4><<<nb, kRowThreads, smem, h->stream>>>(X, Y, rows, R, h->partials);
  } else if (per <= 16) {
    cross_gram_partials<TX, TY, 16><<<nb, kRowThreads, smem, h->stream>>>(X, Y, rows, R, h->partials);
  } else {
    cross_gram_partials<TX, TY, 64><<<nb, kRowThreads, smem, h->stream>>>(X, Y, rows, R, h->partials);
  }
  DF_COUNT();
  reduce_partials<<<(R * R + 255) / 256, 256, 0, h->stream>>>(h->partials, (int)nb, R * R, R,
                                                               symmetrize, out); DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

template <typename T>
dfacto_status gram_T(dfacto_t* h, int m) {
  const T* F = static_cast<const T*>(h->F[m]);
  return cross_gram<T, T>(h, F, F, h->dims[m], h->gram[m], false);
}

}  // namespace

dfacto_status gram_of_factor(dfacto_t* h, int m) {
  dfacto_status st = (h->dtype == DFACTO_BF16) ? gram_T<__nv_bfloat16>(h, m) : gram_T<float>(h, m);
  if (st == DFACTO_OK) h->gram_valid[m] = true;
  return st;
}

namespace {

template <typename T>
dfacto_status als_mode_T(dfacto_t* h, int mode) {
  const ModeCSR& M = h->m[mode];
  const int R = h->R;
  cudaStream_t s = h->stream;
  dfacto_status st;
  for (int m : {M.f, M.in})
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  gamma_inverse<<<1, 256, 0, s>>>(h->gram[M.f], h->gram[M.in], R, h->lambda_reg, h->W, h->W32,
                                  h->flags + kFlagSingular, h->rr_work); DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  if ((st = mttkrp_launch(h, mode, h->N)) != DFACTO_OK) return st;
  const int64_t rows = M.dim_o;
  const unsigned nb = row_blocks(rows);
  const size_t smem = sizeof(float) * R * R;
  allow_smem(als_colnorm_partials, smem);
  allow_smem(als_normalize<T>, smem);
  als_colnorm_partials<<<nb, kRowThreads, smem, s>>>(h->N, h->W32, rows, R, h->partials); DF_COUNT();
  finish_lambda<<<1, 128, 0, s>>>(h->partials, (int)nb, R, h->lambda, h->inv_lambda); DF_COUNT();
  const bool last = (mode == 2);
  als_normalize<T><<<nb, kRowThreads, smem, s>>>(h->N, h->W32, h->inv_lambda, rows, R,
                                                 static_cast<T*>(h->F[mode]),
                                                 last ? h->partials : nullptr); DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  h->gram_valid[mode] = false;
  if (last) {
    // keep the <X,Xhat> partials: move them out of the way of the Gram below
    DF_CUDA(h, cudaMemcpyAsync(h->ipart, h->partials, sizeof(double) * nb * R,
                               cudaMemcpyDeviceToDevice, s));
    h->ipart_blocks = (int)nb;
  }
  return gram_of_factor(h, mode);
}

}  // namespace

dfacto_status als_mode(dfacto_t* h, int mode) {
  return h->dtype == DFACTO_BF16 ? als_mode_T<__nv_bfloat16>(h, mode) : als_mode_T<float>(h, mode);
}

dfacto_status als_fit(dfacto_t* h) {
  fit_from_parts<<<1, 256, 0, h->stream>>>(h->ipart, h->ipart_blocks, h->R, h->lambda, h->gram[0],
                                           h->gram[1], h->gram[2], h->scal); DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

// Fit of the current model without an ALS sweep: <X, Xhat> from a mode-3
// MTTKRP, sum_k sum_r lambda_r C[k,r] M3[k,r].
namespace {
template <typename T>
__global__ void __launch_bounds__(kRowThreads) rows_dot_partials(const float* __restrict__ N,
                                                                const T* __restrict__ F,
                                                                int64_t rows, int R,
                                                                double* __restrict__ part) {
  __shared__ double sacc[kRowThreads / 32][kMaxR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float accf[4] = {0.f, 0.f, 0.f, 0.f};
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
  int since = 0;
  const int64_t wstride = (int64_t)gridDim.x * (kRowThreads / 32);
  for (int64_t o = (int64_t)blockIdx.x * (kRowThreads / 32) + warp; o < rows; o += wstride) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = lane + 32 * q;
      if (col < R) accf[q] = fmaf(ld_elem(F + o * R + col), N[o * R + col], accf[q]);
    }
    if (++since == kFold) {
#pragma unroll
      for (int q = 0; q < 4; ++q) { accd[q] += accf[q]; accf[q] = 0.f; }
      since = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    accd[q] += accf[q];
    if (lane + 32 * q < R) sacc[warp][lane + 32 * q] = accd[q];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < R; col += kRowThreads) {
    double s = 0.0;
    for (int w = 0; w < kRowThreads / 32; ++w) s += sacc[w][col];
    part[(size_t)blockIdx.x * R + col] = s;
  }
}

template <typename T>
dfacto_status fit_direct_T(dfacto_t* h) {
  dfacto_status st;
  for (int m = 0; m < 3; ++m)
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  if ((st = mttkrp_launch(h, 2, h->N)) != DFACTO_OK) return st;
  const int64_t rows = h->dims[2];
  const unsigned nb = row_blocks(rows);
  rows_dot_partials<T><<<nb, kRowThreads, 0, h->stream>>>(h->N, static_cast<const T*>(h->F[2]),
                                                          rows, h->R, h->ipart); DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  h->ipart_blocks = (int)nb;
  return als_fit(h);
}
}  // namespace

dfacto_status fit_direct(dfacto_t* h) {
  return h->dtype == DFACTO_BF16 ? fit_direct_T<__nv_bfloat16>(h) : fit_direct_T<float>(h);
}

// ---------------------------------------------------------------------------
// GD step.
// ---------------------------------------------------------------------------

dfacto_status dual_pass(dfacto_t* h);  // dual.cu: T110, T101, T011, T111

namespace {

template <typename T>
dfacto_status gd_step_T(dfacto_t* h) {
  const int R = h->R;
  cudaStream_t s = h->stream;
  dfacto_status st;
  for (int m = 0; m < 3; ++m)
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  DF_CUDA(h, cudaMemsetAsync(h->scal + kG2, 0, sizeof(double), s));
  for (int mode = 0; mode < 3; ++mode) {
    const ModeCSR& M = h->m[mode];
    hadamard_gamma<<<1, 256, 0, s>>>(h->gram[M.f], h->gram[M.in], R, h->lambda_reg, h->W, h->W32); DF_COUNT();
    if ((st = mttkrp_launch(h, mode, h->N)) != DFACTO_OK) return st;
    const int64_t rows = M.dim_o;
    const unsigned nb = row_blocks(rows);
    allow_smem(gd_gradient_rows<T>, sizeof(float) * R * R);
    gd_gradient_rows<T><<<nb, kRowThreads, sizeof(float) * R * R, s>>>(
        h->N, static_cast<const T*>(h->F[mode]), h->W32, rows, R, h->grad[mode], h->partials); DF_COUNT();
    const int tlin = mode == 0 ? kT100 : (mode == 1 ? kT010 : kT001);
    reduce_scalars<<<1, 32, 0, s>>>(h->partials, (int)nb, 3, h->scal, kG2, tlin,
                                    mode == 0 ? kT000 : -1); DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
  }
  // R x R matrices of the polynomial: P0 = F^T F, P1 = F^T G + G^T F, P2 = G^T G.
  for (int m = 0; m < 3; ++m) {
    double* P = h->gd_mats + (size_t)m * 3 * R * R;
    DF_CUDA(h, cudaMemcpyAsync(P, h->gram[m], sizeof(double) * R * R, cudaMemcpyDeviceToDevice, s));
    if ((st = cross_gram<T, float>(h, static_cast<const T*>(h->F[m]), h->grad[m], h->dims[m],
                                   P + R * R, true)) != DFACTO_OK)
      return st;
    if ((st = cross_gram<float, float>(h, h->grad[m], h->grad[m], h->dims[m], P + 2 * R * R,
                                       false)) != DFACTO_OK)
      return st;
  }
  if ((st = dual_pass(h)) != DFACTO_OK) return st;
  gd_line_search<<<1, 256, 0, s>>>(h->gd_mats, R, h->lambda_reg, h->scal, h->flags + kFlagLsFail); DF_COUNT();
  for (int m = 0; m < 3; ++m) {
    const int64_t n = (int64_t)h->dims[m] * R;
    gd_update<T><<<row_blocks(n, 1024), 256, 0, s>>>(static_cast<T*>(h->F[m]), h->grad[m], n, h->scal); DF_COUNT();
    h->gram_valid[m] = false;
  }
  DF_CUDA(h, cudaGetLastError());
  for (int m = 0; m < 3; ++m)
    if ((st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  return DFACTO_OK;
}

}  // namespace

dfacto_status gd_step(dfacto_t* h) {
  return h->dtype == DFACTO_BF16 ? gd_step_T<__nv_bfloat16>(h) : gd_step_T<float>(h);
}

}  // namespace dfacto
