// dense.cu -- the R x R algebra and the row-wise passes around the MTTKRP:
// Grams (Eq. kr-product), the Gram-Hadamard solve of ALS (Eq.
// als-astep-sol-rw, pseudo-inverse of Eq. kr-pseudo as fallback), column
// normalisation and CP weights (Algorithm 2), the fit, and the GD gradient
// (Eq. gd-A), line search and update (Algorithm 5).
//
// Layout of the row passes: a block stages a tile of kTile rows in shared
// memory and each thread produces four consecutive columns of one row at a
// time; Grams use 4 x 4 register blocks over the staged rows.  These passes are
// bound by HBM (one read and one write of a dim x R matrix).
//
// Precision: factor rows are read in their storage type and multiplied in
// FP32; partial sums over at most kFoldTiles tiles of rows are FP32 and are
// folded into FP64 accumulators (GB300's FP64 rate is low, so the fold is kept
// rare), and all R x R work is FP64.  Every
// reduction runs over fixed per-block partials in a fixed order, so results
// are bitwise reproducible.
#include <algorithm>
#include <cmath>

#include "device.cuh"
#include "internal.h"
#include "mttkrp.cuh"

namespace dfacto {

dfacto_status mttkrp_launch(dfacto_t* h, int mode, float* out);

namespace {

constexpr int kT = 256;          // threads of the row-pass and Gram kernels
constexpr int kTile = 64;        // rows per staged tile
constexpr int kFoldTiles = 8;    // tiles summed in FP32 before folding into FP64
constexpr int kMaxBlocks = 152 * 4;
// Armijo trials of the GD line search (halvings of the step).  Each trial is an
// evaluation of the exact polynomial, so trials cost nothing; 100 halvings
// reach steps of 2^-100, far below the ~1e-14 that N(0,1) starting factors need
// on 1e6-row tensors (Gamma's diagonal ~ the product of two dimensions).
constexpr int kLineSearchTrials = 100;

unsigned row_blocks(int64_t rows) {
  const int64_t b = (rows + 4 * kTile - 1) / (4 * kTile);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kMaxBlocks));
}

// Rows [r0, r1) of block vb's share of `rows` (contiguous chunks over vgrid
// blocks).  Kernels take (vb, vgrid) = (blockIdx.x, gridDim.x) when launched
// for one tensor, or a block's position inside its job when launched for a
// batch of jobs.
__device__ __forceinline__ void block_rows(int64_t rows, int vb, int vgrid, int64_t& r0, int64_t& r1) {
  const int64_t chunk = (rows + vgrid - 1) / vgrid;
  r0 = min(rows, (int64_t)vb * chunk);
  r1 = min(rows, r0 + chunk);
}

// ---------------------------------------------------------------------------
// Deterministic reduction of per-block partials: part is [nb][n];
// out[e] = sum_b part[b][e] (+ part[b][e^T] when symmetrize, R x R entries).
// Block x takes 32 entries (one per lane); its eight warps take blocks
// b = w, w + 8, ... in order; the warp sums are added in warp order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reduce_partials_body(const double* __restrict__ part, int nb, int n,
                                                     int R, bool symmetrize, double* __restrict__ out,
                                                     int vb) {
  __shared__ double s[kT / 32][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = vb * 32 + lane;
  double acc = 0.0;
  if (e < n) {
    const int et = symmetrize ? (e % R) * R + e / R : e;
    for (int b = warp; b < nb; b += kT / 32) {
      acc += part[(size_t)b * n + e];
      if (symmetrize) acc += part[(size_t)b * n + et];
    }
  }
  s[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && e < n) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) t += s[w][lane];
    out[e] = t;
  }
}

__global__ void __launch_bounds__(kT) reduce_partials(const double* __restrict__ part, int nb, int n,
                                                      int R, bool symmetrize,
                                                      double* __restrict__ out) {
  reduce_partials_body(part, nb, n, R, symmetrize, out, blockIdx.x);
}

// Sum of the kT per-thread values v into thread 0 in a fixed order.
__device__ __forceinline__ double block_sum(double v, double* s) {
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  const double t = s[0];
  __syncthreads();
  return t;
}

// Four consecutive entries of a factor row in storage type T, widened.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const uint2 w = *reinterpret_cast<const uint2*>(p);
  return make_float4(bf16_lo(w.x), bf16_hi(w.x), bf16_lo(w.y), bf16_hi(w.y));
}

// Stage rows [t0, t0 + nt) of an n x R matrix into `tile` (row stride ld
// floats, columns R .. W-1 zero-filled).  Each thread owns a fixed (row offset,
// column) slot, computed once: four columns at a time when R % 4 == 0 (16-byte
// copies), one at a time otherwise.
template <typename T>
__device__ __forceinline__ void stage_tile(const T* __restrict__ M, int64_t t0, int nt, int R,
                                           float* __restrict__ tile, int ld, int W) {
  if ((R & 3) == 0) {
    const int R4 = R >> 2, per = kT / R4;
    const int i0 = threadIdx.x / R4, c = 4 * (threadIdx.x % R4);
    if ((int)threadIdx.x < per * R4)
      for (int i = i0; i < nt; i += per)
        *reinterpret_cast<float4*>(tile + i * ld + c) = ld4(M + (t0 + i) * R + c);
  } else {
    const int per = kT / W;
    const int i0 = threadIdx.x / W, c = threadIdx.x % W;
    if ((int)threadIdx.x < per * W)
      for (int i = i0; i < nt; i += per) tile[i * ld + c] = c < R ? ld_elem(M + (t0 + i) * R + c) : 0.f;
  }
}

// Row stride of a staged tile read row-wise by row_times: a multiple of four
// (16-byte aligned rows) shifted by four banks per row when R % 4 == 0.
__host__ __device__ __forceinline__ int row_ld(int R) { return (R & 3) == 0 ? R + 4 : R + 1; }

// ---------------------------------------------------------------------------
// Gram X^T Y (X may be Y) of rows x R matrices: per-block FP64 partials
// part[block][R*R].  Rows are staged as float tiles (columns padded to a
// multiple of 4 with zeros); thread (blk, grp) owns the 4 x 4 block blk of the
// result and the rows grp, grp + ngrp, ... of every tile.
// ---------------------------------------------------------------------------
template <typename TX, typename TY, bool SAME, int BPT>
__global__ void __launch_bounds__(kT) gram_tiles(const TX* __restrict__ X, const TY* __restrict__ Y,
                                                 int64_t rows, int R, double* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  const int R4 = (R + 3) / 4, W = 4 * R4;
  float* tx = sm;                                   // [kTile][W]
  float* ty = SAME ? sm : sm + (size_t)kTile * W;   // [kTile][W]
  const int nblk = R4 * R4;
  const int ngrp = nblk <= kT ? kT / nblk : 1;
  const int grp = nblk <= kT ? (int)threadIdx.x / nblk : 0;
  const bool owner = nblk <= kT ? ((int)threadIdx.x < ngrp * nblk) : true;
  double acc[BPT][16];
  float a32[BPT][16];
#pragma unroll
  for (int b = 0; b < BPT; ++b)
#pragma unroll
    for (int q = 0; q < 16; ++q) { acc[b][q] = 0.0; a32[b][q] = 0.f; }
  int64_t r0, r1;
  block_rows(rows, blockIdx.x, gridDim.x, r0, r1);
  int tiles = 0;
  for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
    const int nt = (int)min((int64_t)kTile, r1 - t0);
    stage_tile(X, t0, nt, R, tx, W, W);
    if (!SAME) stage_tile(Y, t0, nt, R, ty, W, W);
    __syncthreads();
    if (owner) {
#pragma unroll
      for (int b = 0; b < BPT; ++b) {
        const int blk = nblk <= kT ? (int)threadIdx.x % nblk : (int)threadIdx.x + b * kT;
        if (blk < nblk) {
          const int bi = blk / R4, bj = blk % R4;
          for (int i = grp; i < nt; i += ngrp) {
            const float4 xv = *reinterpret_cast<const float4*>(tx + i * W + 4 * bi);
            const float4 yv = *reinterpret_cast<const float4*>(ty + i * W + 4 * bj);
            const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int w = 0; w < 4; ++w) a32[b][u * 4 + w] = fmaf(xa[u], ya[w], a32[b][u * 4 + w]);
          }
        }
      }
    }
    if (++tiles == kFoldTiles || t0 + kTile >= r1) {
#pragma unroll
      for (int b = 0; b < BPT; ++b)
#pragma unroll
        for (int q = 0; q < 16; ++q) { acc[b][q] += (double)a32[b][q]; a32[b][q] = 0.f; }
      tiles = 0;
    }
    __syncthreads();
  }
  // Combine the row groups of each block in group order, write the partial.
  double* red = reinterpret_cast<double*>(sm);  // [kT][16] (fits the tile space)
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int blk = nblk <= kT ? (int)threadIdx.x % nblk : (int)threadIdx.x + b * kT;
#pragma unroll
    for (int q = 0; q < 16; ++q) red[threadIdx.x * 16 + q] = acc[b][q];
    __syncthreads();
    if (owner && grp == 0 && blk < nblk) {
      const int bi = blk / R4, bj = blk % R4;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        double t = 0.0;
        for (int gg = 0; gg < ngrp; ++gg) t += red[(gg * nblk + (nblk <= kT ? blk : (int)threadIdx.x)) * 16 + q];
        const int a = 4 * bi + q / 4, c = 4 * bj + q % 4;
        if (a < R && c < R) part[(size_t)blockIdx.x * R * R + a * R + c] = t;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Gamma = G_f * G_in + lambda_reg I and its inverse (or pseudo-inverse), one
// block, FP64.  Cholesky fails when a pivot drops to R * eps times its
// diagonal entry; then the cyclic Jacobi eigen-decomposition (Golub & Van
// Loan, Sec. 8.5) gives the pseudo-inverse with cutoff R * eps * max |w|.
// The (2R^2 + R)-double workspace is shared memory when it fits, else global.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void gamma_inverse_body(const double* __restrict__ Gf,
                                                   const double* __restrict__ Gi, int R,
                                                   double lambda_reg, double* __restrict__ W,
                                                   float* __restrict__ W32,
                                                   int32_t* __restrict__ singular,
                                                   double* __restrict__ gwork, bool in_smem) {
  extern __shared__ double swork[];
  double* work = in_smem ? swork : gwork;
  double* A = work;               // [R][R] working copy / L
  double* B = work + R * R;       // [R][R] Linv or V
  double* d0 = work + 2 * R * R;  // [R] original diagonal / eigenvalues
  __shared__ int failed;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int RR = R * R;
  const double eps = 2.220446049250313e-16;
  for (int e = tid; e < RR; e += nt) {
    double g = Gf[e] * Gi[e];
    if (e / R == e % R) g += lambda_reg;
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
    const double rjj = 1.0 / A[j * R + j];
    for (int i = j + 1 + tid; i < R; i += nt) A[i * R + j] *= rjj;
    __syncthreads();
    const int m = R - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) A[i * R + k] -= A[i * R + j] * A[k * R + j];
    }
    __syncthreads();
  }
  if (!failed) {
    // Linv by forward substitution, one column per thread (reciprocal
    // diagonal in d0).
    for (int a = tid; a < R; a += nt) d0[a] = 1.0 / A[a * R + a];
    __syncthreads();
    for (int c = tid; c < R; c += nt) {
      for (int i = 0; i < R; ++i) {
        if (i < c) {
          B[i * R + c] = 0.0;
        } else {
          double s = (i == c) ? 1.0 : 0.0;
          for (int k = c; k < i; ++k) s -= A[i * R + k] * B[k * R + c];
          B[i * R + c] = s * d0[i];
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
        const double c = s_c, sn = s_s;
        if (sn != 0.0) {
          for (int k = tid; k < R; k += nt) {  // columns p, q
            const double akp = A[k * R + p], akq = A[k * R + q];
            A[k * R + p] = c * akp - sn * akq;
            A[k * R + q] = sn * akp + c * akq;
          }
          __syncthreads();
          for (int k = tid; k < R; k += nt) {  // rows p, q and V
            const double apk = A[p * R + k], aqk = A[q * R + k];
            A[p * R + k] = c * apk - sn * aqk;
            A[q * R + k] = sn * apk + c * aqk;
            const double vkp = B[k * R + p], vkq = B[k * R + q];
            B[k * R + p] = c * vkp - sn * vkq;
            B[k * R + q] = sn * vkp + c * vkq;
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

__global__ void __launch_bounds__(256) gamma_inverse(const double* __restrict__ Gf,
                                                    const double* __restrict__ Gi, int R,
                                                    double lambda_reg, double* __restrict__ W,
                                                    float* __restrict__ W32,
                                                    int32_t* __restrict__ singular,
                                                    double* __restrict__ gwork, bool in_smem) {
  gamma_inverse_body(Gf, Gi, R, lambda_reg, W, W32, singular, gwork, in_smem);
}

// ---------------------------------------------------------------------------
// Row passes.  A block takes a contiguous chunk of rows in tiles of kTile; the
// tile of the input rows is staged (row stride R + 1) and thread t computes
// columns 4 (t % R4) .. +3 of rows t / R4, t / R4 + kT / R4, ... of the tile.
// ---------------------------------------------------------------------------

// Row r of a staged tile times the R x R matrix S (in shared memory): four
// consecutive output columns starting at 4 * cg.
__device__ __forceinline__ void row_times(const float* __restrict__ trow, const float* __restrict__ S,
                                          int R, int W, int cg, float (&o)[4]) {
  o[0] = o[1] = o[2] = o[3] = 0.f;
  for (int k = 0; k < R; ++k) {
    const float a = trow[k];
    const float4 w = *reinterpret_cast<const float4*>(S + k * W + 4 * cg);
    o[0] = fmaf(a, w.x, o[0]);
    o[1] = fmaf(a, w.y, o[1]);
    o[2] = fmaf(a, w.z, o[2]);
    o[3] = fmaf(a, w.w, o[3]);
  }
}

// Stage an R x R FP32 matrix with rows padded to W = 4 * R4 columns.
__device__ __forceinline__ void stage_rr(const float* __restrict__ M, int R, int W, float* S) {
  for (int e = threadIdx.x; e < R * W; e += kT) {
    const int k = e / W, c = e % W;
    S[e] = c < R ? M[k * R + c] : 0.f;
  }
}

// ALS pass A: Fh = N W (W = Gamma^{-1}) and per-block column sums of squares
// of Fh, colsq[block][R].
__device__ __forceinline__ void als_solve_rows_body(const float* __restrict__ N,
                                                    const float* __restrict__ W32, int64_t rows,
                                                    int R, float* __restrict__ Fh,
                                                    double* __restrict__ colsq, int vb, int vgrid) {
  extern __shared__ __align__(16) float sm[];
  const int R4 = (R + 3) / 4, W = 4 * R4;
  float* S = sm;                        // [R][W]
  float* tile = sm + (size_t)R * W;     // [kTile][row_ld(R)]
  const int ld = row_ld(R);
  __shared__ double red[kT];
  stage_rr(W32, R, W, S);
  const int cg = threadIdx.x % R4, rsub = threadIdx.x / R4, rstep = kT / R4;
  const bool active = rsub < rstep;
  double sq[4] = {0.0, 0.0, 0.0, 0.0};
  int64_t r0, r1;
  block_rows(rows, vb, vgrid, r0, r1);
  for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
    const int nt = (int)min((int64_t)kTile, r1 - t0);
    __syncthreads();
    stage_tile(N, t0, nt, R, tile, ld, R);
    __syncthreads();
    float s32[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
      for (int i = rsub; i < nt; i += rstep) {
        float o[4];
        row_times(tile + i * ld, S, R, W, cg, o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int col = 4 * cg + q;
          if (col < R) {
            Fh[(t0 + i) * R + col] = o[q];
            s32[q] = fmaf(o[q], o[q], s32[q]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) sq[q] += (double)s32[q];
  }
  // Column c is owned by the threads with cg = c / 4: add them in thread order.
  for (int c = 0; c < R; ++c) {
    const double v = (active && cg == c / 4) ? sq[c % 4] : 0.0;
    const double t = block_sum(v, red);
    if (threadIdx.x == 0) colsq[(size_t)vb * R + c] = t;
  }
}

__global__ void __launch_bounds__(kT) als_solve_rows(const float* __restrict__ N,
                                                     const float* __restrict__ W32, int64_t rows,
                                                     int R, float* __restrict__ Fh,
                                                     double* __restrict__ colsq) {
  als_solve_rows_body(N, W32, rows, R, Fh, colsq, blockIdx.x, gridDim.x);
}

// lambda[r] = sqrt(sum_b colsq[b][r]); inv[r] = 1/lambda (1 where lambda = 0).
// One block per column.
__device__ __forceinline__ void finish_lambda_body(const double* __restrict__ colsq, int nb, int R,
                                                   double* __restrict__ lambda,
                                                   float* __restrict__ inv, int r) {
  __shared__ double red[kT];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) v += colsq[(size_t)b * R + r];
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) {
    const double l = sqrt(t);
    lambda[r] = l;
    inv[r] = (l > 0.0) ? (float)(1.0 / l) : 1.0f;
  }
}

__global__ void __launch_bounds__(kT) finish_lambda(const double* __restrict__ colsq, int nb, int R,
                                                    double* __restrict__ lambda,
                                                    float* __restrict__ inv) {
  finish_lambda_body(colsq, nb, R, lambda, inv, blockIdx.x);
}

// ALS pass B: F = Fh / lambda stored in T; Gram partials of the stored values
// gpart[block][R*R]; with N != null also the scalar partial
// sum_{o,r} lambda_r F_stored[o,r] N[o,r] (= <X, Xhat> after the mode-3 update).
template <typename T, int BPT>
__device__ __forceinline__ void als_store_rows_body(const float* __restrict__ Fh,
                                                    const float* __restrict__ inv,
                                                    const double* __restrict__ lambda,
                                                    int64_t rows, int R, T* __restrict__ F,
                                                    double* __restrict__ gpart,
                                                    const float* __restrict__ N,
                                                    double* __restrict__ ipart, int vb, int vgrid) {
  extern __shared__ __align__(16) float sm[];
  const int R4 = (R + 3) / 4, W = 4 * R4;
  float* tile = sm;  // [kTile][W] stored values, zero-padded
  __shared__ double red[kT];
  const int nblk = R4 * R4;
  const int ngrp = nblk <= kT ? kT / nblk : 1;
  const int grp = nblk <= kT ? (int)threadIdx.x / nblk : 0;
  const bool owner = nblk <= kT ? ((int)threadIdx.x < ngrp * nblk) : true;
  double acc[BPT][16];  // BPT = 1 when R <= 64, else 4 blocks per thread
  float a32[BPT][16];
#pragma unroll
  for (int b = 0; b < BPT; ++b)
#pragma unroll
    for (int q = 0; q < 16; ++q) { acc[b][q] = 0.0; a32[b][q] = 0.f; }
  int tiles = 0;
  double ip = 0.0;
  int64_t r0, r1;
  block_rows(rows, vb, vgrid, r0, r1);
  for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
    const int nt = (int)min((int64_t)kTile, r1 - t0);
    __syncthreads();
    float ip32 = 0.f;
    {
      // thread slot: columns c .. c + CW - 1 of rows i0, i0 + per, ...
      const int CW = (R & 3) == 0 ? 4 : 1;
      const int ncol = (R & 3) == 0 ? (R >> 2) : W;
      const int per = kT / ncol;
      const int i0 = threadIdx.x / ncol, c = CW * (threadIdx.x % ncol);
      if ((int)threadIdx.x < per * ncol) {
        float sc[4], lm[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          sc[q] = (q < CW && c + q < R) ? inv[c + q] : 0.f;
          lm[q] = (N && q < CW && c + q < R) ? (float)lambda[c + q] : 0.f;
        }
        for (int i = i0; i < kTile; i += per) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (q >= CW) break;
            float v = 0.f;
            if (i < nt && c + q < R) {
              const int64_t g = (t0 + i) * R + c + q;
              const float x = Fh[g] * sc[q];
              st_elem(F + g, x);
              v = rt_elem(F, x);
              if (N) ip32 = fmaf(lm[q] * v, N[g], ip32);
            }
            tile[i * W + c + q] = v;
          }
        }
      }
    }
    ip += (double)ip32;
    __syncthreads();
    if (owner) {
#pragma unroll
      for (int b = 0; b < BPT; ++b) {
        const int blk = nblk <= kT ? (int)threadIdx.x % nblk : (int)threadIdx.x + b * kT;
        if (blk >= nblk) continue;
        const int bi = blk / R4, bj = blk % R4;
        for (int i = grp; i < nt; i += ngrp) {
          const float4 xv = *reinterpret_cast<const float4*>(tile + i * W + 4 * bi);
          const float4 yv = *reinterpret_cast<const float4*>(tile + i * W + 4 * bj);
          const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) a32[b][u * 4 + w] = fmaf(xa[u], ya[w], a32[b][u * 4 + w]);
        }
      }
    }
    if (++tiles == kFoldTiles || t0 + kTile >= r1) {
#pragma unroll
      for (int b = 0; b < BPT; ++b)
#pragma unroll
        for (int q = 0; q < 16; ++q) { acc[b][q] += (double)a32[b][q]; a32[b][q] = 0.f; }
      tiles = 0;
    }
  }
  if (N) {
    const double t = block_sum(ip, red);
    if (threadIdx.x == 0) ipart[vb] = t;
  }
  __syncthreads();
  double* rsm = reinterpret_cast<double*>(sm);  // [kT][16] over the tile space
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int blk = nblk <= kT ? (int)threadIdx.x % nblk : (int)threadIdx.x + b * kT;
#pragma unroll
    for (int q = 0; q < 16; ++q) rsm[threadIdx.x * 16 + q] = acc[b][q];
    __syncthreads();
    if (owner && grp == 0 && blk < nblk) {
      const int bi = blk / R4, bj = blk % R4;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        double t = 0.0;
        for (int gg = 0; gg < ngrp; ++gg)
          t += rsm[(gg * nblk + (nblk <= kT ? blk : (int)threadIdx.x)) * 16 + q];
        const int a = 4 * bi + q / 4, c = 4 * bj + q % 4;
        if (a < R && c < R) gpart[(size_t)vb * R * R + a * R + c] = t;
      }
    }
    __syncthreads();
  }
}

template <typename T, int BPT>
__global__ void __launch_bounds__(kT) als_store_rows(const float* __restrict__ Fh,
                                                     const float* __restrict__ inv,
                                                     const double* __restrict__ lambda,
                                                     int64_t rows, int R, T* __restrict__ F,
                                                     double* __restrict__ gpart,
                                                     const float* __restrict__ N,
                                                     double* __restrict__ ipart) {
  als_store_rows_body<T, BPT>(Fh, inv, lambda, rows, R, F, gpart, N, ipart, blockIdx.x, gridDim.x);
}

// Fit from scalars and Grams (one block):
//   <X,Xhat> = sum of ipart;  ||Xhat||^2 = lambda^T (GA*GB*GC) lambda.
__device__ __forceinline__ void fit_from_parts_body(const double* __restrict__ ipart, int nb, int R,
                                                    const double* __restrict__ lambda,
                                                    const double* __restrict__ GA,
                                                    const double* __restrict__ GB,
                                                    const double* __restrict__ GC,
                                                    double* __restrict__ scal) {
  __shared__ double red[kT];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) v += ipart[b];
  const double ip = block_sum(v, red);
  double m = 0.0;
  for (int e = threadIdx.x; e < R * R; e += kT) {
    const int a = e / R, b = e % R;
    m += lambda[a] * lambda[b] * GA[e] * GB[e] * GC[e];
  }
  const double nm2 = block_sum(m, red);
  if (threadIdx.x == 0) {
    const double nx2 = scal[kNormX2];
    double res2 = nx2 - 2.0 * ip + nm2;
    if (res2 < 0.0) res2 = 0.0;
    scal[kInner] = ip;
    scal[kModelNorm2] = nm2;
    scal[kFit] = nx2 > 0.0 ? 1.0 - sqrt(res2) / sqrt(nx2) : 0.0;
  }
}

__global__ void __launch_bounds__(kT) fit_from_parts(const double* __restrict__ ipart, int nb, int R,
                                                     const double* __restrict__ lambda,
                                                     const double* __restrict__ GA,
                                                     const double* __restrict__ GB,
                                                     const double* __restrict__ GC,
                                                     double* __restrict__ scal) {
  fit_from_parts_body(ipart, nb, R, lambda, GA, GB, GC, scal);
}

// <N, lambda-scaled F> partials for a fit without an ALS sweep.
template <typename T>
__global__ void __launch_bounds__(kT) rows_inner(const float* __restrict__ N, const T* __restrict__ F,
                                                 const double* __restrict__ lambda, int64_t rows,
                                                 int R, double* __restrict__ ipart) {
  __shared__ double red[kT];
  int64_t r0, r1;
  block_rows(rows, blockIdx.x, gridDim.x, r0, r1);
  double acc = 0.0;
  float a32 = 0.f;
  int since = 0;
  for (int64_t g = r0 * R + threadIdx.x; g < r1 * R; g += kT) {
    a32 = fmaf((float)lambda[g % R] * ld_elem(F + g), N[g], a32);
    if (++since == kTile) {
      acc += a32;
      a32 = 0.f;
      since = 0;
    }
  }
  acc += a32;
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) ipart[blockIdx.x] = t;
}

// ---------------------------------------------------------------------------
// GD.
// ---------------------------------------------------------------------------

// grad = -N + F Gamma (Gamma already holds + lambda_reg I); scalar partials
// per block: spart[block][3] = ||grad||^2, sum grad*N, sum F*N.
template <typename T>
__global__ void __launch_bounds__(kT) gd_gradient_rows(const float* __restrict__ N,
                                                       const T* __restrict__ F,
                                                       const float* __restrict__ Gam32,
                                                       int64_t rows, int R,
                                                       float* __restrict__ grad,
                                                       double* __restrict__ spart) {
  extern __shared__ __align__(16) float sm[];
  const int R4 = (R + 3) / 4, W = 4 * R4;
  float* S = sm;                     // [R][W]
  float* tile = sm + (size_t)R * W;  // [kTile][row_ld(R)] rows of F
  const int ld = row_ld(R);
  __shared__ double red[kT];
  stage_rr(Gam32, R, W, S);
  const int cg = threadIdx.x % R4, rsub = threadIdx.x / R4, rstep = kT / R4;
  const bool active = rsub < rstep;
  double ad[3] = {0.0, 0.0, 0.0};
  int64_t r0, r1;
  block_rows(rows, blockIdx.x, gridDim.x, r0, r1);
  for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
    const int nt = (int)min((int64_t)kTile, r1 - t0);
    __syncthreads();
    stage_tile(F, t0, nt, R, tile, ld, R);
    __syncthreads();
    float af[3] = {0.f, 0.f, 0.f};
    if (active) {
      for (int i = rsub; i < nt; i += rstep) {
        float o[4];
        row_times(tile + i * ld, S, R, W, cg, o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int col = 4 * cg + q;
          if (col < R) {
            const int64_t g = (t0 + i) * R + col;
            const float nv = N[g];
            const float gv = o[q] - nv;
            grad[g] = gv;
            af[0] = fmaf(gv, gv, af[0]);
            af[1] = fmaf(gv, nv, af[1]);
            af[2] = fmaf(tile[i * ld + col], nv, af[2]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) ad[t] += (double)af[t];
  }
  for (int t = 0; t < 3; ++t) {
    const double v = block_sum(ad[t], red);
    if (threadIdx.x == 0) spart[(size_t)blockIdx.x * 3 + t] = v;
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

// Sum the [nb][3] scalar partials of one mode (fixed order) and record them:
// ||grad||^2 accumulates into scal[kG2]; <grad, N> -> dst1; <F, N> -> dst2.
__global__ void __launch_bounds__(kT) gd_scalars(const double* __restrict__ spart, int nb,
                                                 double* __restrict__ scal, int dst1, int dst2) {
  __shared__ double red[kT];
  double v[3];
  for (int t = 0; t < 3; ++t) {
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += kT) a += spart[(size_t)b * 3 + t];
    v[t] = block_sum(a, red);
  }
  if (threadIdx.x == 0) {
    scal[kG2] += v[0];
    scal[dst1] = v[1];
    if (dst2 >= 0) scal[dst2] = v[2];
  }
}

// The GD objective along the search ray theta - alpha * grad (exact, FP64):
//   f(alpha) = 1/2 (||X||^2 - 2 P(alpha) + Q(alpha)) + 1/2 lambda_reg sum_n tr M_n(alpha)
//   P(alpha) = <X, [[A - aGA, B - aGB, C - aGC]]> = sum_S (-alpha)^|S| T_S
//   M_n(alpha) = P0_n - alpha P1_n + alpha^2 P2_n   (Gram of F_n - alpha G_n)
//   Q(alpha) = sum_rs prod_n M_n(alpha)_rs         (||[[.]]||^2, Eq. kr-product)
// f is a polynomial of degree 6 in alpha.

// Horner evaluation of c[0] + c[1] x + ... + c[n] x^n.
__device__ __forceinline__ double poly_eval(const double* c, int n, double x) {
  double v = c[n];
  for (int k = n - 1; k >= 0; --k) v = fma(v, x, c[k]);
  return v;
}

// The root of the monotone p (degree n) in [a, b], where p(a) and p(b) have
// opposite signs, by bisection down to adjacent doubles.
__device__ double bisect_root(const double* c, int n, double a, double b) {
  const double fa = poly_eval(c, n, a);
  for (int it = 0; it < 2200; ++it) {
    const double m = 0.5 * (a + b);
    if (m <= a || m >= b) break;
    const double fm = poly_eval(c, n, m);
    if (fm == 0.0) return m;
    if ((fm < 0.0) == (fa < 0.0)) a = m;
    else b = m;
  }
  return 0.5 * (a + b);
}

constexpr int kPolyMax = 5;  // degree of f'

// Real roots of p (coefficients c[0..n], 1 <= n <= kPolyMax, c[n] != 0) in the
// open interval (lo, hi), ascending, by the derivative sequence: the roots of
// p^(k+1) split (lo, hi) into pieces on which p^(k) is monotone, and each
// piece with a sign change holds exactly one root of p^(k), found by
// bisection.  Returns the count.
__device__ int poly_roots(const double* c, int n, double lo, double hi, double* roots) {
  double D[kPolyMax + 1][kPolyMax + 1];  // D[k] = k-th derivative, degree n - k
  for (int i = 0; i <= n; ++i) D[0][i] = c[i];
  for (int k = 1; k < n; ++k)
    for (int i = 0; i <= n - k; ++i) D[k][i] = D[k - 1][i + 1] * (double)(i + 1);
  double r[kPolyMax + 2];
  int nr = 0;
  {  // the (n-1)-th derivative is linear
    const double* L = D[n - 1];
    const double x = -L[0] / L[1];
    if (x > lo && x < hi) r[nr++] = x;
  }
  for (int k = n - 2; k >= 0; --k) {
    const double* P = D[k];
    const int deg = n - k;
    double pts[kPolyMax + 3];
    int np = 0;
    pts[np++] = lo;
    for (int i = 0; i < nr; ++i) pts[np++] = r[i];
    pts[np++] = hi;
    double nxt[kPolyMax + 2];
    int nn = 0;
    double va = poly_eval(P, deg, pts[0]);
    for (int i = 0; i + 1 < np; ++i) {
      const double vb = poly_eval(P, deg, pts[i + 1]);
      if (va == 0.0 && i > 0) {
        if (nn == 0 || nxt[nn - 1] != pts[i]) nxt[nn++] = pts[i];
      } else if ((va < 0.0 && vb > 0.0) || (va > 0.0 && vb < 0.0)) {
        nxt[nn++] = bisect_root(P, deg, pts[i], pts[i + 1]);
      }
      va = vb;
    }
    nr = nn;
    for (int i = 0; i < nn; ++i) r[i] = nxt[i];
  }
  for (int i = 0; i < nr; ++i) roots[i] = r[i];
  return nr;
}

// f(alpha) of the search ray, evaluated by a whole block of 256 threads (the
// model term Q block-reduced in a fixed order); every caller gets the same bits
// for the same alpha.
struct RayObjective {
  const double* mats;
  int R;
  double lambda_reg, mu;
  const double* ycoef;
  double nx2, t0, t1, t2, t3;
  __device__ RayObjective(const double* m, int r, double lam, const double* __restrict__ scal, double mu_,
                          const double* yc)
      : mats(m), R(r), lambda_reg(lam), mu(mu_), ycoef(yc) {
    nx2 = scal[kNormX2];
    t0 = scal[kT000];
    t1 = scal[kT100] + scal[kT010] + scal[kT001];
    t2 = scal[kT110] + scal[kT101] + scal[kT011];
    t3 = scal[kT111];
  }
  // called by all threads of the block; red: [blockDim.x] shared doubles
  __device__ double Q(double a, double* red, double* s_q) const {
    const int tid = threadIdx.x, RR = R * R;
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
      *s_q = t;
    }
    __syncthreads();
    return *s_q;
  }
  __device__ double trace_sum(double a) const {
    const int RR = R * R;
    double t = 0.0;
    for (int n = 0; n < 3; ++n) {
      const double* P = mats + (size_t)n * 3 * RR;
      for (int r = 0; r < R; ++r) {
        const int e = r * R + r;
        t += P[e] - a * P[RR + e] + a * a * P[2 * RR + e];
      }
    }
    return t;
  }
  __device__ double f(double a, double* red, double* s_q) const {
    const double P = t0 - a * t1 + a * a * t2 - a * a * a * t3;
    double v = 0.5 * mu * (nx2 - 2.0 * P + Q(a, red, s_q));
    if (lambda_reg != 0.0) v += 0.5 * lambda_reg * trace_sum(a);
    if (ycoef) v += ycoef[0] + a * (ycoef[1] + a * (ycoef[2] + a * (ycoef[3] + a * ycoef[4])));
    return v;
  }
};

// The backtracking trials all at once: block 0 evaluates f(0), block 1 + t the
// t-th trial step alpha0 / 2^t (alpha0 = min(2 alpha_prev, 1), or 1 at the
// first step), each as the single-block search would; fvals[1 + kLineSearchTrials].
__global__ void __launch_bounds__(256) gd_ray_values(const double* __restrict__ mats, int R,
                                                    double lambda_reg, const double* __restrict__ scal,
                                                    double mu, const double* __restrict__ ycoef,
                                                    double* __restrict__ fvals) {
  __shared__ double red[256];
  __shared__ double s_q;
  const RayObjective obj(mats, R, lambda_reg, scal, mu, ycoef);
  double a = 0.0;
  if (blockIdx.x > 0) {
    const double prev = scal[kAlpha];
    const double a0 = prev > 0.0 ? fmin(2.0 * prev, 1.0) : 1.0;
    a = ldexp(a0, -(int)(blockIdx.x - 1));  // exact: the halvings of the sequential search
  }
  const double v = obj.f(a, red, &s_q);
  if (threadIdx.x == 0) fvals[blockIdx.x] = v;
}

// One CTA.  exact == 0: backtracking as specified in dfacto.h.  exact == 1:
// the exact minimiser over alpha > 0 -- the coefficients of f are formed in
// FP64 from the same terms, the real roots of f' on (0, B] (B: Fujiwara's
// bound on the roots of f') are isolated, the local minima among them are
// evaluated in the factored form above, and the smallest is taken when it
// lowers f; when there is none (possible only through rounding of a
// degenerate ray), the step falls back to backtracking.
// The joint model of Appendix F weights the tensor term by mu and adds the
// ratings term, a quartic in alpha with coefficients ycoef[0..4] (nullable).
// The backtracking trials' values come from gd_ray_values (fvals).
__global__ void __launch_bounds__(256) gd_line_search(const double* __restrict__ mats, int R,
                                                     double lambda_reg, double* __restrict__ scal,
                                                     int32_t* __restrict__ lsfail, int exact,
                                                     double mu, const double* __restrict__ ycoef,
                                                     const double* __restrict__ fvals) {
  __shared__ double red[256];
  __shared__ double s_q;
  __shared__ double s_qc[256][7];
  __shared__ double s_cand[kPolyMax];
  __shared__ int s_ncand;
  const int tid = threadIdx.x;
  const int RR = R * R;
  const RayObjective obj(mats, R, lambda_reg, scal, mu, ycoef);
  auto f = [&](double a) { return obj.f(a, red, &s_q); };
  const double nx2 = obj.nx2, t0 = obj.t0, t1 = obj.t1, t2 = obj.t2, t3 = obj.t3;
  const double f0 = fvals[0];
  const double g2 = scal[kG2];
  bool ok = false;
  double alpha = 0.0, fa = f0;
  if (exact) {
    // coefficients of Q: per entry the product of three quadratics
    double q[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int e = tid; e < RR; e += blockDim.x) {
      double p[7] = {1, 0, 0, 0, 0, 0, 0};
      int deg = 0;
      for (int n = 0; n < 3; ++n) {
        const double* P = mats + (size_t)n * 3 * RR;
        const double u[3] = {P[e], -P[RR + e], P[2 * RR + e]};
        double np_[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i <= deg; ++i)
          for (int j = 0; j < 3; ++j) np_[i + j] += p[i] * u[j];
        deg += 2;
        for (int i = 0; i <= deg; ++i) p[i] = np_[i];
      }
      for (int k = 0; k < 7; ++k) q[k] += p[k];
    }
    for (int k = 0; k < 7; ++k) s_qc[tid][k] = q[k];
    __syncthreads();
    if (tid == 0) {
      double qc[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int i = 0; i < (int)blockDim.x; ++i)
        for (int k = 0; k < 7; ++k) qc[k] += s_qc[i][k];
      double tr[3] = {0, 0, 0};
      for (int n = 0; n < 3; ++n) {
        const double* P = mats + (size_t)n * 3 * RR;
        for (int r = 0; r < R; ++r) {
          tr[0] += P[r * R + r];
          tr[1] += P[RR + r * R + r];
          tr[2] += P[2 * RR + r * R + r];
        }
      }
      double c[7];
      c[0] = 0.5 * mu * (nx2 - 2.0 * t0 + qc[0]) + 0.5 * lambda_reg * tr[0];
      c[1] = 0.5 * mu * (2.0 * t1 + qc[1]) - 0.5 * lambda_reg * tr[1];
      c[2] = 0.5 * mu * (-2.0 * t2 + qc[2]) + 0.5 * lambda_reg * tr[2];
      c[3] = 0.5 * mu * (2.0 * t3 + qc[3]);
      c[4] = 0.5 * mu * qc[4];
      c[5] = 0.5 * mu * qc[5];
      c[6] = 0.5 * mu * qc[6];
      if (ycoef)
        for (int k = 0; k < 5; ++k) c[k] += ycoef[k];
      double d[kPolyMax + 1];
      for (int k = 0; k <= kPolyMax; ++k) d[k] = (double)(k + 1) * c[k + 1];
      int n = kPolyMax;
      while (n > 0 && d[n] == 0.0) --n;
      int nc = 0;
      if (n >= 1) {
        // Fujiwara's bound on |roots|: 2 max_i |d_{n-i} / d_n|^(1/i), last term halved
        double B = 0.0;
        for (int i = 1; i <= n; ++i) {
          double v = fabs(d[n - i] / d[n]);
          if (i == n) v *= 0.5;
          B = fmax(B, pow(v, 1.0 / i));
        }
        B = 2.0 * B;
        if (isfinite(B) && B > 0.0) {
          double roots[kPolyMax];
          const int nr = poly_roots(d, n, 0.0, B * (1.0 + 1e-12), roots);
          for (int i = 0; i < nr; ++i) {
            // a local minimum: f' changes from negative to positive
            const double lo = i == 0 ? 0.0 : roots[i - 1];
            const double hi = i + 1 < nr ? roots[i + 1] : 2.0 * B + 1.0;
            const double left = poly_eval(d, n, 0.5 * (lo + roots[i]));
            const double right = poly_eval(d, n, 0.5 * (roots[i] + hi));
            if (left < 0.0 && right > 0.0 && roots[i] > 0.0) s_cand[nc++] = roots[i];
          }
        }
      }
      s_ncand = nc;
    }
    __syncthreads();
    const int nc = s_ncand;
    for (int i = 0; i < nc; ++i) {
      const double a = s_cand[i];
      const double v = f(a);  // all threads (block-wide Q)
      if (v < fa) {  // fa starts at f(0): only a decrease is taken
        ok = true;
        fa = v;
        alpha = a;
      }
    }
  }
  if (!ok) {
    const double prev = scal[kAlpha];
    alpha = prev > 0.0 ? fmin(2.0 * prev, 1.0) : 1.0;
    for (int trial = 0; trial < kLineSearchTrials; ++trial) {
      fa = fvals[1 + trial];  // f(alpha), alpha = alpha0 / 2^trial
      if (fa <= f0 - 1e-4 * alpha * g2) {
        ok = true;
        break;
      }
      alpha *= 0.5;
    }
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

// ---------------------------------------------------------------------------
// Row passes for R <= 32, one thread per row.  Pass 1 (colnorm_rows) computes
// the column sums of squares of N Gamma^{-1} without storing it; pass 2
// (scale_store_rows) recomputes N Gamma^{-1} row by row (same arithmetic, same
// order, so the same values), scales by 1/lambda, stores F, and forms the Gram
// of the stored values (and the fit's inner product on the last mode).  Each
// pass reads N once: 4R + s R bytes per row over both passes instead of a
// write and a read of N Gamma^{-1} in between.  Gamma^{-1} sits in shared
// memory as RT x RT (zero-padded), read by broadcast.
// ---------------------------------------------------------------------------
// Blocks of a row pass: one per 256-row tile up to one full wave (two
// resident blocks per SM at 128 registers), so that large passes run as one
// balanced wave of equal chunks.
constexpr int kPassWave = 152 * 2;

int pass_blocks(int64_t rows) {
  const int64_t tiles = (rows + kT - 1) / kT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, kPassWave));
}

// Row r of N (R columns) zero-padded to RT.
template <int RT>
__device__ __forceinline__ void load_row(const float* __restrict__ N, int64_t r, int R, float (&n)[RT]) {
  const float* p = N + r * R;
  if ((R & 3) == 0) {
#pragma unroll
    for (int c4 = 0; c4 < RT / 4; ++c4) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4 * c4 < R) v = __ldg(reinterpret_cast<const float4*>(p) + c4);
      n[4 * c4] = v.x; n[4 * c4 + 1] = v.y; n[4 * c4 + 2] = v.z; n[4 * c4 + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < RT; ++c) n[c] = c < R ? __ldg(p + c) : 0.f;
  }
}

// Columns [c0, c0 + CW) of o = n W (W: RT x RT in shared memory, row k holds
// the coefficients of n[k]); k ascends, so every caller gets the same values.
template <int RT, int CW>
__device__ __forceinline__ void row_solve(const float (&n)[RT], const float* __restrict__ Ws, int c0,
                                          float (&o)[CW]) {
#pragma unroll
  for (int c = 0; c < CW; ++c) o[c] = 0.f;
#pragma unroll
  for (int k = 0; k < RT; ++k) {
    const float a = n[k];
#pragma unroll
    for (int c4 = 0; c4 < CW / 4; ++c4) {
      const float4 w = reinterpret_cast<const float4*>(Ws + k * RT + c0)[c4];
      o[4 * c4] = fmaf(a, w.x, o[4 * c4]);
      o[4 * c4 + 1] = fmaf(a, w.y, o[4 * c4 + 1]);
      o[4 * c4 + 2] = fmaf(a, w.z, o[4 * c4 + 2]);
      o[4 * c4 + 3] = fmaf(a, w.w, o[4 * c4 + 3]);
    }
  }
}

template <int RT>
__device__ __forceinline__ void stage_w(const float* __restrict__ W32, int R, float* Ws) {
  for (int e = threadIdx.x; e < RT * RT; e += kT) {
    const int k = e / RT, c = e % RT;
    Ws[e] = (k < R && c < R) ? W32[k * R + c] : 0.f;
  }
}

// Output columns are produced CW = min(RT, 16) at a time (fewer live registers).
// The Gram partials use NGRP groups of NBLK threads (one 4 x 4 block each);
// when NBLK does not divide kT (RT = 12: 28 groups of 9) the last kT % NBLK
// threads add nothing.
template <int RT>
struct PassShape {
  static constexpr int CW = RT < 16 ? RT : 16;
  static constexpr int LD = RT + 4;  // tile row stride (16-byte aligned rows)
  static constexpr int NB4 = RT / 4, NBLK = NB4 * NB4, NGRP = kT / NBLK;
};

// Rows [t0, t0 + nt) of an R-column row-major matrix (one contiguous run of
// nt * R floats) into tile rows of stride LD, with coalesced 16-byte loads when
// R % 4 == 0.  Columns R .. RT-1 of the tile are left as they are (zero).
template <int LD>
__device__ __forceinline__ void tile_load(const float* __restrict__ M, int64_t t0, int nt, int R,
                                          float* __restrict__ tile) {
  const float* src = M + t0 * R;
  const int total = nt * R;
  if ((R & 3) == 0) {
    for (int e4 = threadIdx.x; e4 < (total >> 2); e4 += kT) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src) + e4);
      const int e = 4 * e4, r = e / R, c = e - r * R;
      *reinterpret_cast<float4*>(tile + r * LD + c) = v;
    }
  } else {
    for (int e = threadIdx.x; e < total; e += kT) {
      const int r = e / R, c = e - r * R;
      tile[r * LD + c] = __ldg(src + e);
    }
  }
}

// tile_load issued as 16-byte asynchronous copies (cp.async, committed as one
// group) for R % 4 == 0: the caller overlaps the copy of the next tile with
// the work on the current one and waits with cp_async_wait<n>() (at most n
// groups still in flight) followed by a barrier.
template <int LD>
__device__ __forceinline__ void tile_load_async(const float* __restrict__ M, int64_t t0, int nt,
                                                int R, float* __restrict__ tile) {
  const float* src = M + t0 * R;
  const int total4 = (nt * R) >> 2;
  for (int e4 = threadIdx.x; e4 < total4; e4 += kT) {
    const int e = 4 * e4, r = e / R, c = e - r * R;
    const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + r * LD + c);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + e) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// The tensor-core form of the row passes (RT = 16 or 32) keeps W split into
// TF32 heads and tails, rows padded to RT + 8 (conflict-free fragment loads).
template <int RT>
constexpr bool row_pass_tc() { return RT == 16 || RT == 32; }
template <int RT>
constexpr int row_pass_wstride() { return RT + 8; }
template <int RT>
constexpr size_t row_pass_w_floats() {
  return row_pass_tc<RT>() ? 2 * (size_t)RT * row_pass_wstride<RT>() : (size_t)RT * RT;
}

// Shared memory of the double-buffered row passes: W and two tiles.
template <int RT>
constexpr size_t row_pass_smem() {
  return sizeof(float) * (row_pass_w_floats<RT>() + 2 * (size_t)kT * (RT + 4));
}

// Tile t of a row pass in buffer t & 1: for R % 4 == 0 the next tile's copy is
// issued before this one is waited for; otherwise the tile is loaded here.
// Callers issue the first tile (row_pass_prefetch) before their loop, and call
// this after a barrier that ends all use of the other buffer.
template <int LD>
__device__ __forceinline__ void row_pass_prefetch(const float* __restrict__ M, int64_t r0, int64_t r1,
                                                  int R, float* __restrict__ tiles) {
  if ((R & 3) == 0 && r0 < r1) tile_load_async<LD>(M, r0, (int)min((int64_t)kT, r1 - r0), R, tiles);
}
template <int LD>
__device__ __forceinline__ float* row_pass_tile(const float* __restrict__ M, int64_t t0, int64_t r1,
                                                int R, float* __restrict__ tiles, int buf) {
  float* tile = tiles + (size_t)buf * kT * LD;
  if ((R & 3) == 0) {
    const int64_t tn = t0 + kT;
    if (tn < r1) {
      tile_load_async<LD>(M, tn, (int)min((int64_t)kT, r1 - tn), R, tiles + (size_t)(buf ^ 1) * kT * LD);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
  } else {
    tile_load<LD>(M, t0, (int)min((int64_t)kT, r1 - t0), R, tile);
  }
  return tile;
}

// Tile rows (already rounded to T) back to rows [t0, t0 + nt) of an R-column
// matrix in storage type T, with coalesced 16-byte stores where the layout
// allows (FP32: R % 4 == 0; BF16: R % 8 == 0).
template <int LD>
__device__ __forceinline__ void tile_store(const float* __restrict__ tile, int64_t t0, int nt, int R,
                                           float* __restrict__ M) {
  float* dst = M + t0 * R;
  const int total = nt * R;
  if ((R & 3) == 0) {
    for (int e4 = threadIdx.x; e4 < (total >> 2); e4 += kT) {
      const int e = 4 * e4, r = e / R, c = e - r * R;
      reinterpret_cast<float4*>(dst)[e4] = *reinterpret_cast<const float4*>(tile + r * LD + c);
    }
  } else {
    for (int e = threadIdx.x; e < total; e += kT) {
      const int r = e / R, c = e - r * R;
      dst[e] = tile[r * LD + c];
    }
  }
}
template <int LD>
__device__ __forceinline__ void tile_store(const float* __restrict__ tile, int64_t t0, int nt, int R,
                                           __nv_bfloat16* __restrict__ M) {
  __nv_bfloat16* dst = M + t0 * R;
  const int total = nt * R;
  if ((R & 7) == 0) {
    for (int e8 = threadIdx.x; e8 < (total >> 3); e8 += kT) {
      const int e = 8 * e8, r = e / R, c = e - r * R;
      const float* q = tile + r * LD + c;
      uint4 w;
      w.x = (__float_as_uint(q[0]) >> 16) | (__float_as_uint(q[1]) & 0xffff0000u);
      w.y = (__float_as_uint(q[2]) >> 16) | (__float_as_uint(q[3]) & 0xffff0000u);
      w.z = (__float_as_uint(q[4]) >> 16) | (__float_as_uint(q[5]) & 0xffff0000u);
      w.w = (__float_as_uint(q[6]) >> 16) | (__float_as_uint(q[7]) & 0xffff0000u);
      reinterpret_cast<uint4*>(dst)[e8] = w;  // values are BF16-exact: the high halves
    }
  } else {
    for (int e = threadIdx.x; e < total; e += kT) {
      const int r = e / R, c = e - r * R;
      st_elem(dst + e, tile[r * LD + c]);
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form of the row passes for RT = 16 and 32.  The products
// N W (rows x RT times RT x RT) and the Gram of the stored factor (RT x RT
// over the rows) are dense contractions: they run as mma.sync m16n8k8 with
// TF32 operands, every FP32 operand split into a TF32 head and a TF32 tail
// (x = h + l) and each product formed as l h' + h l' + h h' (the dropped l l'
// term and the tail's rounding are below 2^-21 of the product).  Each k-step
// of eight starts from a zero accumulator and is added to an FP32 register
// sum with round-to-nearest adds (the tensor unit's own accumulation is not
// rounded to nearest, so long accumulator chains inside it drift); the Gram's
// FP32 sums are folded into FP64 after every tile.  The result has the
// accuracy of the FP32 FMA form at a fraction of its instructions, which
// leaves the passes bound by their HBM traffic.  Warp w takes tile rows
// [32w, 32w + 32) for N W, and output block w of the Gram.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& h, uint32_t& l) {
  h = to_tf32(x);
  l = to_tf32(x - __uint_as_float(h));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// d += a b from split operands: tails first, heads last.
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
  mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
  mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}

// W (R x R, zero-padded to RT x RT) split into heads Wh and tails Wl, row
// stride row_pass_wstride<RT>().
template <int RT>
__device__ __forceinline__ void stage_w_split(const float* __restrict__ W32, int R, uint32_t* Wh,
                                              uint32_t* Wl) {
  constexpr int WS = row_pass_wstride<RT>();
  for (int e = threadIdx.x; e < RT * WS; e += kT) {
    const int k = e / WS, c = e % WS;
    const float w = (k < R && c < R) ? W32[k * R + c] : 0.f;
    split_tf32(w, Wh[e], Wl[e]);
  }
}

// o = rows [m0, m0 + 16) of the tile times W: o[n][0..3] is the mma output
// fragment of columns [8n, 8n + 8) (rows m0 + gid and m0 + gid + 8, columns
// 8n + 2 tig and 8n + 2 tig + 1, gid = lane / 4, tig = lane % 4).
template <int RT>
__device__ __forceinline__ void tc_rows_times_w(const float* __restrict__ tile, int m0,
                                                const uint32_t* __restrict__ Wh,
                                                const uint32_t* __restrict__ Wl,
                                                float (&o)[RT / 8][4]) {
  constexpr int LD = RT + 4, WS = row_pass_wstride<RT>(), KS = RT / 8;
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  uint32_t ah[KS][4], al[KS][4];
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const float* r0 = tile + (m0 + gid) * LD + 8 * k + tig;
    const float* r1 = r0 + 8 * LD;
    split_tf32(r0[0], ah[k][0], al[k][0]);
    split_tf32(r1[0], ah[k][1], al[k][1]);
    split_tf32(r0[4], ah[k][2], al[k][2]);
    split_tf32(r1[4], ah[k][3], al[k][3]);
  }
#pragma unroll
  for (int n = 0; n < RT / 8; ++n) {
    o[n][0] = o[n][1] = o[n][2] = o[n][3] = 0.f;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const int e0 = (8 * k + tig) * WS + 8 * n + gid, e1 = e0 + 4 * WS;
      float t[4] = {0.f, 0.f, 0.f, 0.f};
      mma3(t, ah[k], al[k], Wh[e0], Wh[e1], Wl[e0], Wl[e1]);
#pragma unroll
      for (int j = 0; j < 4; ++j) o[n][j] += t[j];
    }
  }
}

// Per-warp Gram on the tensor cores: g += X[rows]^T Y[rows] over the 32 tile
// rows [row0, row0 + 32) (four k-steps of eight rows; tiles of row stride
// RT + 4).  g[i][j] is the mma output fragment of the 16 x 8 block at rows
// [16 i, +16) and columns [8 j, +8).
template <int RT>
__device__ __forceinline__ void warp_gram_acc(const float* __restrict__ X, const float* __restrict__ Y,
                                              int row0, float (&g)[RT / 16][RT / 8][4]) {
  constexpr int LD = RT + 4, MB = RT / 16, NS = RT / 8;
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const float* x0 = X + (row0 + 8 * ks + tig) * LD;
    const float* x1 = x0 + 4 * LD;
    const float* y0 = Y + (row0 + 8 * ks + tig) * LD;
    const float* y1 = y0 + 4 * LD;
    uint32_t ah[MB][4], al[MB][4], bh[NS][2], bl[NS][2];
#pragma unroll
    for (int i = 0; i < MB; ++i) {
      split_tf32(x0[16 * i + gid], ah[i][0], al[i][0]);
      split_tf32(x0[16 * i + gid + 8], ah[i][1], al[i][1]);
      split_tf32(x1[16 * i + gid], ah[i][2], al[i][2]);
      split_tf32(x1[16 * i + gid + 8], ah[i][3], al[i][3]);
    }
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      split_tf32(y0[8 * j + gid], bh[j][0], bl[j][0]);
      split_tf32(y1[8 * j + gid], bh[j][1], bl[j][1]);
    }
#pragma unroll
    for (int i = 0; i < MB; ++i)
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        mma3(t, ah[i], al[i], bh[j][0], bh[j][1], bl[j][0], bl[j][1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) g[i][j][q] += t[q];
      }
  }
}

// The warps' Grams added in FP64 in warp order, through `scratch`
// (kT / 32 * RT * RT floats): warps [0, nw) into gpart[vb][R*R], and with
// gpart2 warps [nw, 2 nw) into gpart2[vb][R*R].  Called by all threads after
// the last use of `scratch` as a tile.
template <int RT>
__device__ __forceinline__ void fold_warp_grams(const float (&g)[RT / 16][RT / 8][4], float* scratch,
                                                int R, double* __restrict__ gpart, int vb,
                                                int nw = kT / 32, double* __restrict__ gpart2 = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < RT / 16; ++i)
#pragma unroll
    for (int j = 0; j < RT / 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = 16 * i + gid + (q >> 1) * 8, c = 8 * j + 2 * tig + (q & 1);
        scratch[(warp * RT + a) * RT + c] = g[i][j][q];
      }
  __syncthreads();
  for (int e = threadIdx.x; e < RT * RT; e += kT) {
    const int a = e / RT, c = e % RT;
    if (a < R && c < R) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += (double)scratch[w * RT * RT + e];
      gpart[(size_t)vb * R * R + a * R + c] = t;
      if (gpart2) {
        double t2 = 0.0;
        for (int w = nw; w < 2 * nw; ++w) t2 += (double)scratch[w * RT * RT + e];
        gpart2[(size_t)vb * R * R + a * R + c] = t2;
      }
    }
  }
  __syncthreads();
}

template <int RT>
__device__ __forceinline__ void zero_gram(float (&g)[RT / 16][RT / 8][4]) {
#pragma unroll
  for (int i = 0; i < RT / 16; ++i)
#pragma unroll
    for (int j = 0; j < RT / 8; ++j) g[i][j][0] = g[i][j][1] = g[i][j][2] = g[i][j][3] = 0.f;
}

// Pass 1, tensor-core form: colsq[vb][c] = sum over the block's rows of
// (N W)[row, c]^2.  Each lane sums the squares of its fragment entries in
// FP32; lanes are added by shuffles, warps in FP64 in warp order.
template <int RT>
__device__ __forceinline__ void colnorm_rows_tc(const float* __restrict__ N,
                                                const float* __restrict__ W32, int64_t rows, int R,
                                                double* __restrict__ colsq, int vb, int vgrid) {
  constexpr int LD = RT + 4, WS = row_pass_wstride<RT>(), NS = RT / 8;
  extern __shared__ __align__(16) float row_smem[];
  uint32_t* Wh = reinterpret_cast<uint32_t*>(row_smem);
  uint32_t* Wl = Wh + RT * WS;
  float* tiles = row_smem + row_pass_w_floats<RT>();
  __shared__ float s_part[kT / 32][RT];
  stage_w_split<RT>(W32, R, Wh, Wl);
  for (int e = threadIdx.x; e < 2 * kT * LD; e += kT) tiles[e] = 0.f;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
  int64_t r0, r1;
  block_rows(rows, vb, vgrid, r0, r1);
  float sq[NS][2];
#pragma unroll
  for (int n = 0; n < NS; ++n) sq[n][0] = sq[n][1] = 0.f;
  __syncthreads();
  row_pass_prefetch<LD>(N, r0, r1, R, tiles);
  int buf = 0;
  for (int64_t t0 = r0; t0 < r1; t0 += kT, buf ^= 1) {
    const int nt = (int)min((int64_t)kT, r1 - t0);
    __syncthreads();
    const float* tile = row_pass_tile<LD>(N, t0, r1, R, tiles, buf);
    __syncthreads();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int m0 = 32 * warp + 16 * mt;
      if (m0 >= nt) break;  // warp-uniform
      float o[NS][4];
      tc_rows_times_w<RT>(tile, m0, Wh, Wl, o);
      const bool v0 = m0 + gid < nt, v1 = m0 + gid + 8 < nt;
#pragma unroll
      for (int n = 0; n < NS; ++n) {
        if (v0) { sq[n][0] = fmaf(o[n][0], o[n][0], sq[n][0]); sq[n][1] = fmaf(o[n][1], o[n][1], sq[n][1]); }
        if (v1) { sq[n][0] = fmaf(o[n][2], o[n][2], sq[n][0]); sq[n][1] = fmaf(o[n][3], o[n][3], sq[n][1]); }
      }
    }
  }
  // lanes with equal tig hold the same columns: add over gid
#pragma unroll
  for (int n = 0; n < NS; ++n)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float v = sq[n][j];
      v += __shfl_xor_sync(kFull, v, 4);
      v += __shfl_xor_sync(kFull, v, 8);
      v += __shfl_xor_sync(kFull, v, 16);
      if (gid == 0) s_part[warp][8 * n + 2 * tig + j] = v;
    }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += kT) {
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t += (double)s_part[w][c];
    colsq[(size_t)vb * R + c] = t;
  }
}

// Pass 2, tensor-core form: F[row] = (N W)[row] * inv stored in T, the Gram
// partials of the stored values gpart[vb][R*R], and with with_ip the fit's
// inner product ipart[vb] = sum lambda_c F_stored[row, c] N[row, c].  Each
// warp replaces its 32 tile rows by their stored values and adds their outer
// products to its own FP32 Gram (every 16 x 8 block of it, as four k-steps of
// eight rows); the tile is then written to F with coalesced stores.  At the
// end the warps' Grams are added in FP64, in warp order.
template <typename T, int RT>
__device__ __forceinline__ void scale_store_rows_tc(const float* __restrict__ N,
                                                    const float* __restrict__ W32,
                                                    const float* __restrict__ inv,
                                                    const double* __restrict__ lambda, int64_t rows,
                                                    int R, T* __restrict__ F,
                                                    double* __restrict__ gpart, bool with_ip,
                                                    double* __restrict__ ipart, int vb, int vgrid) {
  constexpr int LD = RT + 4, WS = row_pass_wstride<RT>(), NS = RT / 8, MB = RT / 16;
  extern __shared__ __align__(16) float row_smem[];
  uint32_t* Wh = reinterpret_cast<uint32_t*>(row_smem);
  uint32_t* Wl = Wh + RT * WS;
  float* tiles = row_smem + row_pass_w_floats<RT>();
  __shared__ float s_sc[RT], s_lm[RT];
  __shared__ double red[kT];
  stage_w_split<RT>(W32, R, Wh, Wl);
  for (int c = threadIdx.x; c < RT; c += kT) {
    s_sc[c] = c < R ? inv[c] : 0.f;
    s_lm[c] = (with_ip && c < R) ? (float)lambda[c] : 0.f;
  }
  for (int e = threadIdx.x; e < 2 * kT * LD; e += kT) tiles[e] = 0.f;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
  float g[MB][NS][4];  // this warp's Gram: block (i, j) = rows [16 i, +16) x cols [8 j, +8)
  zero_gram<RT>(g);
  double ip = 0.0;
  int64_t r0, r1;
  block_rows(rows, vb, vgrid, r0, r1);
  __syncthreads();
  row_pass_prefetch<LD>(N, r0, r1, R, tiles);
  int buf = 0;
  for (int64_t t0 = r0; t0 < r1; t0 += kT, buf ^= 1) {
    const int nt = (int)min((int64_t)kT, r1 - t0);
    __syncthreads();
    float* tile = row_pass_tile<LD>(N, t0, r1, R, tiles, buf);
    __syncthreads();
    float ip32 = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int m0 = 32 * warp + 16 * mt;
      float o[NS][4];
      tc_rows_times_w<RT>(tile, m0, Wh, Wl, o);
      __syncwarp();  // every lane has read its operands from these rows
#pragma unroll
      for (int n = 0; n < NS; ++n)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int row = m0 + gid + (j >> 1) * 8, col = 8 * n + 2 * tig + (j & 1);
          float* cell = tile + row * LD + col;
          const float x = o[n][j] * s_sc[col];
          const float v = (col < R && row < nt) ? rt_elem(F, x) : 0.f;
          ip32 = fmaf(s_lm[col] * v, *cell, ip32);
          *cell = v;
        }
    }
    ip += (double)ip32;
    __syncwarp();  // the warp's rows hold the stored values
    warp_gram_acc<RT>(tile, tile, 32 * warp, g);
    __syncthreads();
    tile_store<LD>(tile, t0, nt, R, F);
  }
  if (with_ip) {
    const double t = block_sum(ip, red);
    if (threadIdx.x == 0) ipart[vb] = t;
  }
  fold_warp_grams<RT>(g, tiles, R, gpart, vb);  // NW x RT x RT floats <= 2 kT LD floats
}

// Pass 1: colsq[vb][c] = sum over the block's rows of (N W)[row, c]^2.  A tile
// of kT rows is loaded into shared memory with coalesced loads; thread t then
// takes row t of the tile.  Each thread sums its rows in FP32; the block adds
// the threads in FP64, in thread order.
template <int RT>
__device__ __forceinline__ void colnorm_rows_body(const float* __restrict__ N,
                                                  const float* __restrict__ W32, int64_t rows, int R,
                                                  double* __restrict__ colsq, int vb, int vgrid) {
  if constexpr (row_pass_tc<RT>()) {
    colnorm_rows_tc<RT>(N, W32, rows, R, colsq, vb, vgrid);
    return;
  }
  using PS = PassShape<RT>;
  constexpr int CW = PS::CW, LD = PS::LD;
  static_assert(LD >= RT + 1, "the tile doubles as the FP64 reduction area");
  extern __shared__ __align__(16) float row_smem[];  // row_pass_smem<RT>() bytes
  float* Ws = row_smem;
  float* tiles = row_smem + row_pass_w_floats<RT>();
  stage_w<RT>(W32, R, Ws);
  for (int e = threadIdx.x; e < 2 * kT * LD; e += kT) tiles[e] = 0.f;
  int64_t r0, r1;
  block_rows(rows, vb, vgrid, r0, r1);
  float sq[RT];
#pragma unroll
  for (int c = 0; c < RT; ++c) sq[c] = 0.f;
  __syncthreads();
  row_pass_prefetch<LD>(N, r0, r1, R, tiles);
  int buf = 0;
  for (int64_t t0 = r0; t0 < r1; t0 += kT, buf ^= 1) {
    const int nt = (int)min((int64_t)kT, r1 - t0);
    __syncthreads();
    const float* tile = row_pass_tile<LD>(N, t0, r1, R, tiles, buf);
    __syncthreads();
    if ((int)threadIdx.x < nt) {
      float n[RT];
#pragma unroll
      for (int c4 = 0; c4 < RT / 4; ++c4) {
        const float4 v = *reinterpret_cast<const float4*>(tile + threadIdx.x * LD + 4 * c4);
        n[4 * c4] = v.x; n[4 * c4 + 1] = v.y; n[4 * c4 + 2] = v.z; n[4 * c4 + 3] = v.w;
      }
#pragma unroll
      for (int h = 0; h < RT / CW; ++h) {
        float o[CW];
        row_solve<RT, CW>(n, Ws, h * CW, o);
#pragma unroll
        for (int c = 0; c < CW; ++c) sq[h * CW + c] = fmaf(o[c], o[c], sq[h * CW + c]);
      }
    }
  }
  __syncthreads();
  float* red = tiles;  // [kT][RT + 1]
#pragma unroll
  for (int c = 0; c < RT; ++c) red[threadIdx.x * (RT + 1) + c] = sq[c];
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += kT) {
    double t = 0.0;
    for (int i = 0; i < kT; ++i) t += (double)red[i * (RT + 1) + c];
    colsq[(size_t)vb * R + c] = t;
  }
}

// Pass 2: F[row] = (N W)[row] * inv stored in T; Gram partials of the stored
// values gpart[vb][R*R]: a tile of kT rows is loaded into shared memory with
// coalesced loads, thread t replaces row t of the tile by its stored values,
// the tile is written to F with coalesced stores, and thread (grp, blk) adds
// the outer products of the 4 x 4 block blk over rows grp, grp + NGRP, ... in
// FP32; the groups are added in FP64, in group order.  With with_ip also
// ipart[vb] = sum lambda_c F_stored[row, c] N[row, c] (the fit's inner
// product after the last mode).
template <typename T, int RT>
__device__ __forceinline__ void scale_store_rows_body(const float* __restrict__ N,
                                                      const float* __restrict__ W32,
                                                      const float* __restrict__ inv,
                                                      const double* __restrict__ lambda, int64_t rows,
                                                      int R, T* __restrict__ F,
                                                      double* __restrict__ gpart, bool with_ip,
                                                      double* __restrict__ ipart, int vb, int vgrid) {
  if constexpr (row_pass_tc<RT>()) {
    scale_store_rows_tc<T, RT>(N, W32, inv, lambda, rows, R, F, gpart, with_ip, ipart, vb, vgrid);
    return;
  }
  using PS = PassShape<RT>;
  constexpr int CW = PS::CW, LD = PS::LD, NB4 = PS::NB4, NBLK = PS::NBLK, NGRP = PS::NGRP;
  extern __shared__ __align__(16) float row_smem[];  // row_pass_smem<RT>() bytes
  float* Ws = row_smem;
  float* tiles = row_smem + row_pass_w_floats<RT>();
  __shared__ float s_sc[RT], s_lm[RT];
  __shared__ double red[kT];
  stage_w<RT>(W32, R, Ws);
  for (int c = threadIdx.x; c < RT; c += kT) {
    s_sc[c] = c < R ? inv[c] : 0.f;
    s_lm[c] = (with_ip && c < R) ? (float)lambda[c] : 0.f;
  }
  for (int e = threadIdx.x; e < 2 * kT * LD; e += kT) tiles[e] = 0.f;
  const int blk = threadIdx.x % NBLK, grp = threadIdx.x / NBLK;
  const int bi = blk / NB4, bj = blk % NB4;
  float a32[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) a32[q] = 0.f;
  double ip = 0.0;
  int64_t r0, r1;
  block_rows(rows, vb, vgrid, r0, r1);
  __syncthreads();
  row_pass_prefetch<LD>(N, r0, r1, R, tiles);
  int buf = 0;
  for (int64_t t0 = r0; t0 < r1; t0 += kT, buf ^= 1) {
    const int nt = (int)min((int64_t)kT, r1 - t0);
    __syncthreads();
    float* tile = row_pass_tile<LD>(N, t0, r1, R, tiles, buf);
    __syncthreads();
    float ip32 = 0.f;
    float* trow = tile + threadIdx.x * LD;
    if ((int)threadIdx.x < nt) {
      float n[RT];
#pragma unroll
      for (int c4 = 0; c4 < RT / 4; ++c4) {
        const float4 v = *reinterpret_cast<const float4*>(trow + 4 * c4);
        n[4 * c4] = v.x; n[4 * c4 + 1] = v.y; n[4 * c4 + 2] = v.z; n[4 * c4 + 3] = v.w;
      }
#pragma unroll
      for (int h = 0; h < RT / CW; ++h) {
        float o[CW];
        row_solve<RT, CW>(n, Ws, h * CW, o);
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int col = h * CW + c;
          const float x = o[c] * s_sc[col];
          const float v = col < R ? rt_elem(F, x) : 0.f;
          ip32 = fmaf(s_lm[col] * v, n[col], ip32);
          o[c] = v;
        }
#pragma unroll
        for (int c4 = 0; c4 < CW / 4; ++c4)
          *reinterpret_cast<float4*>(trow + h * CW + 4 * c4) =
              make_float4(o[4 * c4], o[4 * c4 + 1], o[4 * c4 + 2], o[4 * c4 + 3]);
      }
    } else {
#pragma unroll
      for (int c4 = 0; c4 < NB4; ++c4)
        *reinterpret_cast<float4*>(trow + 4 * c4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    ip += (double)ip32;
    __syncthreads();
    tile_store<LD>(tile, t0, nt, R, F);
    for (int i = grp; grp < NGRP && i < nt; i += NGRP) {
      const float4 xv = *reinterpret_cast<const float4*>(tile + i * LD + 4 * bi);
      const float4 yv = *reinterpret_cast<const float4*>(tile + i * LD + 4 * bj);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) a32[u * 4 + w] = fmaf(xa[u], ya[w], a32[u * 4 + w]);
    }
  }
  if (with_ip) {
    const double t = block_sum(ip, red);
    if (threadIdx.x == 0) ipart[vb] = t;
  }
  // Add the groups of each block in group order, four entries at a time
  // through the tile ([kT][4] doubles = 8 KB <= the tile's kT * LD floats).
  __syncthreads();
  double* rsm = reinterpret_cast<double*>(tiles);
  for (int q0 = 0; q0 < 16; q0 += 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) rsm[threadIdx.x * 4 + q] = (double)a32[q0 + q];
    __syncthreads();
    if (grp == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double t = 0.0;
        for (int gg = 0; gg < NGRP; ++gg) t += rsm[(gg * NBLK + blk) * 4 + q];
        const int e = q0 + q;
        const int a = 4 * bi + e / 4, c = 4 * bj + e % 4;
        if (a < R && c < R) gpart[(size_t)vb * R * R + a * R + c] = t;
      }
    }
    __syncthreads();
  }
}

// Tile rows of a factor in storage type T (BF16 widened), coalesced 16-byte
// loads where the layout allows.
template <int LD>
__device__ __forceinline__ void tile_load_T(const float* __restrict__ M, int64_t t0, int nt, int R,
                                            float* __restrict__ tile) {
  tile_load<LD>(M, t0, nt, R, tile);
}
template <int LD>
__device__ __forceinline__ void tile_load_T(const __nv_bfloat16* __restrict__ M, int64_t t0, int nt,
                                            int R, float* __restrict__ tile) {
  const __nv_bfloat16* src = M + t0 * R;
  const int total = nt * R;
  if ((R & 7) == 0) {
    for (int e8 = threadIdx.x; e8 < (total >> 3); e8 += kT) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(src) + e8);
      const int e = 8 * e8, r = e / R, c = e - r * R;
      float* q = tile + r * LD + c;
      q[0] = bf16_lo(w.x); q[1] = bf16_hi(w.x); q[2] = bf16_lo(w.y); q[3] = bf16_hi(w.y);
      q[4] = bf16_lo(w.z); q[5] = bf16_hi(w.z); q[6] = bf16_lo(w.w); q[7] = bf16_hi(w.w);
    }
  } else {
    for (int e = threadIdx.x; e < total; e += kT) {
      const int r = e / R, c = e - r * R;
      tile[r * LD + c] = ld_elem(src + e);
    }
  }
}

// Sum the per-thread 4 x 4 block partials a32 of the groups of each block in
// group order (FP64, four entries at a time through `scratch`, >= kT * 4
// doubles) and store block vb's R x R partial at gpart[vb][R*R].
template <int RT>
__device__ __forceinline__ void store_gram_partial(const float (&a32)[16], double* scratch, int R,
                                                   double* __restrict__ gpart, int vb) {
  using PS = PassShape<RT>;
  constexpr int NB4 = PS::NB4, NBLK = PS::NBLK, NGRP = PS::NGRP;
  const int blk = threadIdx.x % NBLK, grp = threadIdx.x / NBLK;
  const int bi = blk / NB4, bj = blk % NB4;
  for (int q0 = 0; q0 < 16; q0 += 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) scratch[threadIdx.x * 4 + q] = (double)a32[q0 + q];
    __syncthreads();
    if (grp == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double t = 0.0;
        for (int gg = 0; gg < NGRP; ++gg) t += scratch[(gg * NBLK + blk) * 4 + q];
        const int e = q0 + q;
        const int a = 4 * bi + e / 4, c = 4 * bj + e % 4;
        if (a < R && c < R) gpart[(size_t)vb * R * R + a * R + c] = t;
      }
    }
    __syncthreads();
  }
}

// GD, one pass per mode for R <= 32: grad = -N + F Gamma (Gamma already holds
// + lambda_reg I) stored, with the partials of the line search's matrices
// P2 = grad^T grad (gg) and F^T grad (fg, symmetrised later into P1) and the
// scalars spart[vb][3] = ||grad||^2, sum grad * N, sum F * N.  Tiles of kT rows
// of N and F are staged with coalesced loads; thread t forms row t of grad
// (F row t times Gamma, same arithmetic order as the other row passes) into
// the N tile, which is then stored with coalesced stores.  Dynamic shared
// memory: Gamma (RT x RT) and two tiles.
// Tensor-core form of gd_rows for RT = 16 and 32 (the split TF32 products of
// the ALS row passes): each warp forms the gradient of its 32 tile rows from
// F Gamma; then warp w < 4 adds G^T G and warp w + 4 adds F^T G over the rows
// of warps w and w + 4 (one Gram per warp keeps the registers), and the warps'
// partials are added in FP64 in warp order.  Dynamic shared memory: Gamma
// split into heads and tails, and two tiles.
template <typename T, int RT>
__device__ __forceinline__ void gd_rows_tc(const float* __restrict__ N, const T* __restrict__ F,
                                           const float* __restrict__ Gam32, int64_t rows, int R,
                                           float* __restrict__ grad, double* __restrict__ gpart_gg,
                                           double* __restrict__ gpart_fg,
                                           double* __restrict__ spart) {
  constexpr int LD = RT + 4, WS = row_pass_wstride<RT>(), NS = RT / 8, MB = RT / 16;
  extern __shared__ __align__(16) float dyn[];
  uint32_t* Wh = reinterpret_cast<uint32_t*>(dyn);
  uint32_t* Wl = Wh + RT * WS;
  float* tN = dyn + row_pass_w_floats<RT>();  // [kT * LD] N, then grad
  float* tF = tN + kT * LD;                   // [kT * LD] F
  __shared__ double red[kT];
  stage_w_split<RT>(Gam32, R, Wh, Wl);
  for (int e = threadIdx.x; e < 2 * kT * LD; e += kT) tN[e] = 0.f;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
  constexpr int HW = kT / 64;  // warps per Gram
  float g[MB][NS][4];  // G^T G (warps < HW) or F^T G (warps >= HW)
  zero_gram<RT>(g);
  const bool is_gg = warp < HW;
  const int wr = is_gg ? warp : warp - HW;  // rows of warps wr and wr + HW
  double ad[3] = {0.0, 0.0, 0.0};
  int64_t r0, r1;
  block_rows(rows, blockIdx.x, gridDim.x, r0, r1);
  for (int64_t t0 = r0; t0 < r1; t0 += kT) {
    const int nt = (int)min((int64_t)kT, r1 - t0);
    __syncthreads();
    tile_load<LD>(N, t0, nt, R, tN);
    tile_load_T<LD>(F, t0, nt, R, tF);
    __syncthreads();
    if ((int)threadIdx.x >= nt) {  // rows past the tile's end add nothing
      for (int c = 0; c < RT; ++c) {
        tN[threadIdx.x * LD + c] = 0.f;
        tF[threadIdx.x * LD + c] = 0.f;
      }
    }
    __syncwarp();
    float af[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int m0 = 32 * warp + 16 * mt;
      float o[NS][4];
      tc_rows_times_w<RT>(tF, m0, Wh, Wl, o);
#pragma unroll
      for (int n = 0; n < NS; ++n)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int row = m0 + gid + (j >> 1) * 8, col = 8 * n + 2 * tig + (j & 1);
          float* cell = tN + row * LD + col;
          const float nv = *cell;
          const float gv = o[n][j] - nv;  // 0 in padding rows and columns
          af[0] = fmaf(gv, gv, af[0]);
          af[1] = fmaf(gv, nv, af[1]);
          af[2] = fmaf(tF[row * LD + col], nv, af[2]);
          *cell = gv;
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) ad[t] += (double)af[t];
    __syncthreads();  // every warp's gradient rows are in tN
    warp_gram_acc<RT>(is_gg ? tN : tF, tN, 32 * wr, g);
    warp_gram_acc<RT>(is_gg ? tN : tF, tN, 32 * (wr + HW), g);
    tile_store<LD>(tN, t0, nt, R, grad);
  }
  for (int t = 0; t < 3; ++t) {
    const double v = block_sum(ad[t], red);
    if (threadIdx.x == 0) spart[(size_t)blockIdx.x * 3 + t] = v;
  }
  fold_warp_grams<RT>(g, tN, R, gpart_gg, blockIdx.x, HW, gpart_fg);
}

template <typename T, int RT>
__global__ void __launch_bounds__(kT, 2) gd_rows(const float* __restrict__ N, const T* __restrict__ F,
                                                 const float* __restrict__ Gam32, int64_t rows, int R,
                                                 float* __restrict__ grad,
                                                 double* __restrict__ gpart_gg,
                                                 double* __restrict__ gpart_fg,
                                                 double* __restrict__ spart) {
  if constexpr (row_pass_tc<RT>()) {
    gd_rows_tc<T, RT>(N, F, Gam32, rows, R, grad, gpart_gg, gpart_fg, spart);
    return;
  }
  using PS = PassShape<RT>;
  constexpr int CW = PS::CW, LD = PS::LD, NB4 = PS::NB4, NBLK = PS::NBLK, NGRP = PS::NGRP;
  extern __shared__ __align__(16) float dyn[];
  float* Ws = dyn;                    // [RT * RT]
  float* tN = Ws + RT * RT;           // [kT * LD] N, then grad
  float* tF = tN + kT * LD;           // [kT * LD] F
  __shared__ double red[kT];
  stage_w<RT>(Gam32, R, Ws);
  for (int e = threadIdx.x; e < 2 * kT * LD; e += kT) tN[e] = 0.f;
  const int blk = threadIdx.x % NBLK, grp = threadIdx.x / NBLK;
  const int bi = blk / NB4, bj = blk % NB4;
  float agg[16], afg[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) agg[q] = afg[q] = 0.f;
  double ad[3] = {0.0, 0.0, 0.0};
  int64_t r0, r1;
  block_rows(rows, blockIdx.x, gridDim.x, r0, r1);
  for (int64_t t0 = r0; t0 < r1; t0 += kT) {
    const int nt = (int)min((int64_t)kT, r1 - t0);
    __syncthreads();
    tile_load<LD>(N, t0, nt, R, tN);
    tile_load_T<LD>(F, t0, nt, R, tF);
    __syncthreads();
    float af[3] = {0.f, 0.f, 0.f};
    if ((int)threadIdx.x < nt) {
      float* nrow = tN + threadIdx.x * LD;
      float f[RT];
#pragma unroll
      for (int c4 = 0; c4 < RT / 4; ++c4) {
        const float4 v = *reinterpret_cast<const float4*>(tF + threadIdx.x * LD + 4 * c4);
        f[4 * c4] = v.x; f[4 * c4 + 1] = v.y; f[4 * c4 + 2] = v.z; f[4 * c4 + 3] = v.w;
      }
#pragma unroll
      for (int h = 0; h < RT / CW; ++h) {
        float o[CW];
        row_solve<RT, CW>(f, Ws, h * CW, o);
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          const int col = h * CW + c;
          const float nv = nrow[col];
          const float gv = o[c] - nv;  // 0 in the padding columns
          af[0] = fmaf(gv, gv, af[0]);
          af[1] = fmaf(gv, nv, af[1]);
          af[2] = fmaf(f[col], nv, af[2]);
          nrow[col] = gv;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) ad[t] += (double)af[t];
    __syncthreads();
    tile_store<LD>(tN, t0, nt, R, grad);
    for (int i = grp; grp < NGRP && i < nt; i += NGRP) {
      const float4 gx = *reinterpret_cast<const float4*>(tN + i * LD + 4 * bi);
      const float4 gy = *reinterpret_cast<const float4*>(tN + i * LD + 4 * bj);
      const float4 fx = *reinterpret_cast<const float4*>(tF + i * LD + 4 * bi);
      const float ga[4] = {gx.x, gx.y, gx.z, gx.w}, gb[4] = {gy.x, gy.y, gy.z, gy.w};
      const float fa[4] = {fx.x, fx.y, fx.z, fx.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          agg[u * 4 + w] = fmaf(ga[u], gb[w], agg[u * 4 + w]);
          afg[u * 4 + w] = fmaf(fa[u], gb[w], afg[u * 4 + w]);
        }
    }
  }
  for (int t = 0; t < 3; ++t) {
    const double v = block_sum(ad[t], red);
    if (threadIdx.x == 0) spart[(size_t)blockIdx.x * 3 + t] = v;
  }
  __syncthreads();
  double* scratch = reinterpret_cast<double*>(tN);
  store_gram_partial<RT>(agg, scratch, R, gpart_gg, blockIdx.x);
  store_gram_partial<RT>(afg, scratch, R, gpart_fg, blockIdx.x);
}

// GD update for R <= 32: F <- F - step * grad (step = scal[kStep], 0 after a
// failed search), stored in T, with the Gram partials of the stored factor
// (the Gram the next step needs).  Same staging as gd_rows.
template <typename T, int RT>
__global__ void __launch_bounds__(kT, 2) gd_update_gram(T* __restrict__ F, const float* __restrict__ grad,
                                                        const double* __restrict__ scal, int64_t rows,
                                                        int R, double* __restrict__ gpart) {
  using PS = PassShape<RT>;
  constexpr int LD = PS::LD, NB4 = PS::NB4, NBLK = PS::NBLK, NGRP = PS::NGRP;
  extern __shared__ __align__(16) float dyn[];
  float* tF = dyn;             // [kT * LD]
  float* tG = tF + kT * LD;    // [kT * LD]
  const float step = (float)scal[kStep];
  for (int e = threadIdx.x; e < 2 * kT * LD; e += kT) tF[e] = 0.f;
  const int blk = threadIdx.x % NBLK, grp = threadIdx.x / NBLK;
  const int bi = blk / NB4, bj = blk % NB4;
  float a32[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) a32[q] = 0.f;
  float g[RT / 16 > 0 ? RT / 16 : 1][RT / 8][4];  // tensor-core Gram (RT = 16, 32)
  if constexpr (row_pass_tc<RT>()) zero_gram<RT>(g);
  int64_t r0, r1;
  block_rows(rows, blockIdx.x, gridDim.x, r0, r1);
  for (int64_t t0 = r0; t0 < r1; t0 += kT) {
    const int nt = (int)min((int64_t)kT, r1 - t0);
    __syncthreads();
    tile_load_T<LD>(F, t0, nt, R, tF);
    tile_load<LD>(grad, t0, nt, R, tG);
    __syncthreads();
    if ((int)threadIdx.x < nt) {
      float* frow = tF + threadIdx.x * LD;
      const float* grow = tG + threadIdx.x * LD;
      for (int c = 0; c < R; ++c) frow[c] = rt_elem(F, frow[c] - step * grow[c]);
    } else {  // rows past the tile's end add nothing to the Gram
      float* frow = tF + threadIdx.x * LD;
      for (int c = 0; c < RT; ++c) frow[c] = 0.f;
    }
    __syncthreads();
    tile_store<LD>(tF, t0, nt, R, F);
    if constexpr (row_pass_tc<RT>()) {
      warp_gram_acc<RT>(tF, tF, 32 * (threadIdx.x >> 5), g);  // rows >= nt are zero
    } else {
      for (int i = grp; grp < NGRP && i < nt; i += NGRP) {
        const float4 xv = *reinterpret_cast<const float4*>(tF + i * LD + 4 * bi);
        const float4 yv = *reinterpret_cast<const float4*>(tF + i * LD + 4 * bj);
        const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w) a32[u * 4 + w] = fmaf(xa[u], ya[w], a32[u * 4 + w]);
      }
    }
  }
  __syncthreads();
  if constexpr (row_pass_tc<RT>())
    fold_warp_grams<RT>(g, tF, R, gpart, blockIdx.x);
  else
    store_gram_partial<RT>(a32, reinterpret_cast<double*>(tF), R, gpart, blockIdx.x);
}

// Opt a kernel in to `Bytes` of dynamic shared memory (above the default
// 48 KB) on the current device (once per kernel and device).
template <auto Kernel, size_t Bytes>
cudaError_t opt_in_smem() {
  return ensure_dynamic_smem(reinterpret_cast<const void*>(Kernel), Bytes);
}

template <int RT>
__global__ void __launch_bounds__(kT, 2) colnorm_rows(const float* __restrict__ N,
                                                   const float* __restrict__ W32, int64_t rows, int R,
                                                   double* __restrict__ colsq) {
  colnorm_rows_body<RT>(N, W32, rows, R, colsq, blockIdx.x, gridDim.x);
}

template <typename T, int RT>
__global__ void __launch_bounds__(kT, 2) scale_store_rows(const float* __restrict__ N,
                                                       const float* __restrict__ W32,
                                                       const float* __restrict__ inv,
                                                       const double* __restrict__ lambda,
                                                       int64_t rows, int R, T* __restrict__ F,
                                                       double* __restrict__ gpart, bool with_ip,
                                                       double* __restrict__ ipart) {
  scale_store_rows_body<T, RT>(N, W32, inv, lambda, rows, R, F, gpart, with_ip, ipart, blockIdx.x,
                               gridDim.x);
}

// ---------------------------------------------------------------------------
// Batched launches: one launch per step for every job of a rank class.  Each
// block finds its job and its position inside the job and runs the per-job
// body with that position, so every job gets exactly what its own launch
// would compute.
// ---------------------------------------------------------------------------

// Job of block b: the last j with begin[j] <= b.
__device__ __forceinline__ int job_of_block(const int32_t* __restrict__ begin, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) gamma_inverse_batch(const DenseJob* __restrict__ jobs, int R,
                                                          bool in_smem) {
  const DenseJob& J = jobs[blockIdx.x];
  gamma_inverse_body(J.Gf, J.Gi, R, J.lambda_reg, J.W, J.W32, J.singular, J.rr_work, in_smem);
}

__global__ void __launch_bounds__(kT) als_solve_rows_batch(const DenseJob* __restrict__ jobs,
                                                           const int32_t* __restrict__ begin, int n,
                                                           int R) {
  const int j = job_of_block(begin, n, blockIdx.x);
  const DenseJob& J = jobs[j];
  als_solve_rows_body(J.N, J.W32, J.rows, R, J.Fh, J.partials, blockIdx.x - begin[j], J.nb);
}

template <int RT>
__global__ void __launch_bounds__(kT, 2) colnorm_rows_batch(const DenseJob* __restrict__ jobs,
                                                         const int32_t* __restrict__ begin, int n,
                                                         int R) {
  const int j = job_of_block(begin, n, blockIdx.x);
  const DenseJob& J = jobs[j];
  colnorm_rows_body<RT>(J.N, J.W32, J.rows, R, J.partials, blockIdx.x - begin[j], J.nb);
}

template <typename T, int RT>
__global__ void __launch_bounds__(kT, 2) scale_store_rows_batch(const DenseJob* __restrict__ jobs,
                                                             const int32_t* __restrict__ begin, int n,
                                                             int R, bool last) {
  const int j = job_of_block(begin, n, blockIdx.x);
  const DenseJob& J = jobs[j];
  scale_store_rows_body<T, RT>(J.N, J.W32, J.inv_lambda, J.lambda, J.rows, R, static_cast<T*>(J.F),
                               J.partials, last, J.ipart, blockIdx.x - begin[j], J.nb);
}

__global__ void __launch_bounds__(kT) finish_lambda_batch(const DenseJob* __restrict__ jobs, int R) {
  const DenseJob& J = jobs[blockIdx.x / R];
  finish_lambda_body(J.partials, J.nb, R, J.lambda, J.inv_lambda, blockIdx.x % R);
}

template <typename T, int BPT>
__global__ void __launch_bounds__(kT) als_store_rows_batch(const DenseJob* __restrict__ jobs,
                                                           const int32_t* __restrict__ begin, int n,
                                                           int R, bool last) {
  const int j = job_of_block(begin, n, blockIdx.x);
  const DenseJob& J = jobs[j];
  als_store_rows_body<T, BPT>(J.Fh, J.inv_lambda, J.lambda, J.rows, R, static_cast<T*>(J.F),
                              J.partials, last ? J.N : nullptr, J.ipart, blockIdx.x - begin[j], J.nb);
}

__global__ void __launch_bounds__(kT) reduce_partials_batch(const DenseJob* __restrict__ jobs, int R,
                                                            int per_job) {
  const DenseJob& J = jobs[blockIdx.x / per_job];
  reduce_partials_body(J.partials, J.nb, R * R, R, false, J.gram_out, blockIdx.x % per_job);
}

__global__ void __launch_bounds__(kT) fit_from_parts_batch(const DenseJob* __restrict__ jobs, int R) {
  const DenseJob& J = jobs[blockIdx.x];
  fit_from_parts_body(J.ipart, J.nb, R, J.lambda, J.GA, J.GB, J.GC, J.scal);
}

}  // namespace

// Blocks of one job's row passes inside a batch: at least 1024 * 32 / RT rows
// per block (many jobs fill the GPU together; a block's fixed costs -- staging
// Gamma^{-1}, its column and R x R partial sums -- are then paid per about
// 32K row-columns of work; narrow rows get proportionally more rows).
int dense_row_blocks(int64_t rows, int R) {
  if (R > 32) return (int)row_blocks(rows);
  const int RT = R <= 8 ? 8 : (R <= 12 ? 12 : (R <= 16 ? 16 : 32));
  const int64_t per = 1024 * 32 / RT;
  const int64_t b = (rows + per - 1) / per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, kMaxBlocks));
}

// ---------------------------------------------------------------------------
// Host orchestration.
// ---------------------------------------------------------------------------

namespace {

// Kernels that stage R x R matrices or row tiles need the opt-in shared memory
// limit for large R.
template <typename K>
void allow_smem(K kernel, size_t bytes) {
  // a failure shows up as the launch error that follows
  ensure_dynamic_smem(reinterpret_cast<const void*>(kernel), bytes);
}

size_t tile_bytes(int R, int copies) {
  const int W = 4 * ((R + 3) / 4);
  return std::max(sizeof(float) * (size_t)kTile * W * copies, sizeof(double) * kT * 16);
}

size_t solve_bytes(int R) {
  const int W = 4 * ((R + 3) / 4);
  return sizeof(float) * ((size_t)R * W + (size_t)kTile * row_ld(R));
}

template <typename TX, typename TY, bool SAME>
dfacto_status cross_gram(dfacto_t* h, const TX* X, const TY* Y, int64_t rows, double* out,
                         bool symmetrize) {
  const int R = h->R;
  const int R4 = (R + 3) / 4;
  const unsigned nb = row_blocks(rows);
  if ((int64_t)nb * R * R > h->partials_cap) return fail(h, DFACTO_EINTERNAL, "partials too small");
  const size_t smem = tile_bytes(R, SAME ? 1 : 2);
  if (R4 * R4 <= kT) {
    allow_smem(gram_tiles<TX, TY, SAME, 1>, smem);
    gram_tiles<TX, TY, SAME, 1><<<nb, kT, smem, h->stream>>>(X, Y, rows, R, h->partials);
  } else {
    allow_smem(gram_tiles<TX, TY, SAME, 4>, smem);
    gram_tiles<TX, TY, SAME, 4><<<nb, kT, smem, h->stream>>>(X, Y, rows, R, h->partials);
  }
  DF_COUNT();
  reduce_partials<<<(R * R + 31) / 32, kT, 0, h->stream>>>(h->partials, (int)nb, R * R, R, symmetrize,
                                                           out);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

template <typename T>
dfacto_status gram_T(dfacto_t* h, int m) {
  const T* F = static_cast<const T*>(h->F[m]);
  return cross_gram<T, T, true>(h, F, F, h->dims[m], h->gram[m], false);
}

dfacto_status launch_gamma_inverse(dfacto_t* h, const double* Gf, const double* Gi) {
  const int R = h->R;
  const size_t need = sizeof(double) * (2 * (size_t)R * R + R);
  const bool in_smem = need <= 48 * 1024;
  gamma_inverse<<<1, 256, in_smem ? need : 0, h->stream>>>(Gf, Gi, R, h->lambda_reg, h->W, h->W32,
                                                           h->flags + kFlagSingular, h->rr_work,
                                                           in_smem);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

}  // namespace

dfacto_status gram_of_factor(dfacto_t* h, int m) {
  dfacto_status st = (h->dtype == DFACTO_BF16) ? gram_T<__nv_bfloat16>(h, m) : gram_T<float>(h, m);
  if (st == DFACTO_OK) h->gram_valid[m] = true;
  return st;
}

namespace {

// The row passes of one mode for R <= 32 (one thread per row).
template <typename T, int RT>
dfacto_status als_post_rows(dfacto_t* h, int mode, float* N) {
  const int R = h->R;
  cudaStream_t s = h->stream;
  const int64_t rows = h->m[mode].dim_o;
  const int nb = pass_blocks(rows);
  const bool last = (mode == 2);
  constexpr size_t smem = row_pass_smem<RT>();
  DF_CUDA(h, (opt_in_smem<colnorm_rows<RT>, smem>()));
  DF_CUDA(h, (opt_in_smem<scale_store_rows<T, RT>, smem>()));
  colnorm_rows<RT><<<nb, kT, smem, s>>>(N, h->W32, rows, R, h->partials);
  DF_COUNT();
  finish_lambda<<<R, kT, 0, s>>>(h->partials, nb, R, h->lambda, h->inv_lambda);
  DF_COUNT();
  scale_store_rows<T, RT><<<nb, kT, smem, s>>>(N, h->W32, h->inv_lambda, h->lambda, rows, R,
                                               static_cast<T*>(h->F[mode]), h->partials, last, h->ipart);
  DF_COUNT();
  reduce_partials<<<(R * R + 31) / 32, kT, 0, s>>>(h->partials, nb, R * R, R, false, h->gram[mode]);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  h->gram_valid[mode] = true;
  if (last) h->ipart_blocks = nb;
  return DFACTO_OK;
}

template <typename T>
dfacto_status als_post_T(dfacto_t* h, int mode, float* N) {
  const ModeCSR& M = h->m[mode];
  const int R = h->R;
  const int R4 = (R + 3) / 4;
  cudaStream_t s = h->stream;
  if (R <= 8) return als_post_rows<T, 8>(h, mode, N);
  if (R <= 12) return als_post_rows<T, 12>(h, mode, N);
  if (R <= 16) return als_post_rows<T, 16>(h, mode, N);
  if (R <= 32) return als_post_rows<T, 32>(h, mode, N);
  const int64_t rows = M.dim_o;
  const unsigned nb = row_blocks(rows);
  const size_t smem_a = solve_bytes(R);
  allow_smem(als_solve_rows, smem_a);
  als_solve_rows<<<nb, kT, smem_a, s>>>(N, h->W32, rows, R, h->Fh, h->partials);
  DF_COUNT();
  finish_lambda<<<R, kT, 0, s>>>(h->partials, (int)nb, R, h->lambda, h->inv_lambda);
  DF_COUNT();
  const bool last = (mode == 2);
  const size_t smem_b = tile_bytes(R, 1);
  T* F = static_cast<T*>(h->F[mode]);
  if (R4 * R4 <= kT) {
    allow_smem(als_store_rows<T, 1>, smem_b);
    als_store_rows<T, 1><<<nb, kT, smem_b, s>>>(h->Fh, h->inv_lambda, h->lambda, rows, R, F,
                                                h->partials, last ? N : nullptr, h->ipart);
  } else {
    allow_smem(als_store_rows<T, 4>, smem_b);
    als_store_rows<T, 4><<<nb, kT, smem_b, s>>>(h->Fh, h->inv_lambda, h->lambda, rows, R, F,
                                                h->partials, last ? N : nullptr, h->ipart);
  }
  DF_COUNT();
  reduce_partials<<<(R * R + 31) / 32, kT, 0, s>>>(h->partials, (int)nb, R * R, R, false,
                                                   h->gram[mode]);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  h->gram_valid[mode] = true;
  if (last) h->ipart_blocks = (int)nb;
  return DFACTO_OK;
}

}  // namespace

// Steps of Algorithm 2 for one mode before the MTTKRP: the Grams of the other
// two factors (when not already known) and Gamma^{-1}.
dfacto_status als_pre(dfacto_t* h, int mode) {
  const ModeCSR& M = h->m[mode];
  dfacto_status st;
  for (int m : {M.f, M.in})
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  return launch_gamma_inverse(h, h->gram[M.f], h->gram[M.in]);
}

// Steps after the MTTKRP N of this mode: N Gamma^{-1}, normalisation, store,
// and the Gram of the new factor (plus the fit's inner product on mode 3).
dfacto_status als_post(dfacto_t* h, int mode, float* N) {
  return h->dtype == DFACTO_BF16 ? als_post_T<__nv_bfloat16>(h, mode, N) : als_post_T<float>(h, mode, N);
}

// One mode of Algorithm 2.  Gamma^{-1} depends only on the other two factors,
// so it runs on the handle's auxiliary stream beside the MTTKRP; the row
// passes wait for both.
dfacto_status als_mode(dfacto_t* h, int mode) {
  dfacto_status st;
  if (h->aux) {
    DF_CUDA(h, cudaEventRecord(h->aux_fork, h->stream));
    DF_CUDA(h, cudaStreamWaitEvent(h->aux, h->aux_fork, 0));
    cudaStream_t main = h->stream;
    h->stream = h->aux;
    st = als_pre(h, mode);
    h->stream = main;
    cudaError_t e = cudaEventRecord(h->aux_join, h->aux);
    if (st == DFACTO_OK) st = mttkrp_launch(h, mode, h->N);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->aux_join, 0);
    if (e != cudaSuccess && st == DFACTO_OK) return cuda_fail(h, e, "auxiliary stream join");
  } else {
    st = als_pre(h, mode);
    if (st == DFACTO_OK) st = mttkrp_launch(h, mode, h->N);
  }
  if (st == DFACTO_OK) st = als_post(h, mode, h->N);
  return st;
}

dfacto_status als_fit(dfacto_t* h) {
  fit_from_parts<<<1, kT, 0, h->stream>>>(h->ipart, h->ipart_blocks, h->R, h->lambda, h->gram[0],
                                          h->gram[1], h->gram[2], h->scal);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

// Fit of the current model without an ALS sweep: <X, Xhat> from a mode-3
// MTTKRP, sum_k sum_r lambda_r C[k,r] M3[k,r].
namespace {
template <typename T>
dfacto_status fit_direct_T(dfacto_t* h) {
  dfacto_status st;
  for (int m = 0; m < 3; ++m)
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  if ((st = mttkrp_launch(h, 2, h->N)) != DFACTO_OK) return st;
  const int64_t rows = h->dims[2];
  const unsigned nb = row_blocks(rows);
  rows_inner<T><<<nb, kT, 0, h->stream>>>(h->N, static_cast<const T*>(h->F[2]), h->lambda, rows,
                                          h->R, h->ipart);
  DF_COUNT();
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

// One GD step for R <= 32 with the fused row passes (gd_rows, gd_update_gram).
template <typename T, int RT>
dfacto_status gd_step_rows(dfacto_t* h) {
  const int R = h->R;
  cudaStream_t s = h->stream;
  dfacto_status st;
  for (int m = 0; m < 3; ++m)
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  DF_CUDA(h, cudaMemsetAsync(h->scal + kG2, 0, sizeof(double), s));
  constexpr int LD = PassShape<RT>::LD;
  const size_t smem_rows = sizeof(float) * (row_pass_w_floats<RT>() + 2 * (size_t)kT * LD);
  const size_t smem_upd = sizeof(float) * 2 * (size_t)kT * LD;
  allow_smem(gd_rows<T, RT>, smem_rows);
  allow_smem(gd_update_gram<T, RT>, smem_upd);
  for (int mode = 0; mode < 3; ++mode) {
    const ModeCSR& M = h->m[mode];
    hadamard_gamma<<<1, 256, 0, s>>>(h->gram[M.f], h->gram[M.in], R, h->lambda_reg, h->W, h->W32);
    DF_COUNT();
    if ((st = mttkrp_launch(h, mode, h->N)) != DFACTO_OK) return st;
    const int64_t rows = M.dim_o;
    const int nb = pass_blocks(rows);
    const int64_t RR = (int64_t)R * R;
    if ((st = grow_partials(h, 2 * nb * RR + 3 * nb)) != DFACTO_OK) return st;
    double* gg = h->partials;
    double* fg = h->partials + nb * RR;
    double* sp = h->partials + 2 * nb * RR;
    double* P = h->gd_mats + (size_t)mode * 3 * RR;
    gd_rows<T, RT><<<nb, kT, smem_rows, s>>>(h->N, static_cast<const T*>(h->F[mode]), h->W32, rows, R,
                                             h->grad[mode], gg, fg, sp);
    DF_COUNT();
    // P0 = F^T F (known), P1 = F^T G + G^T F, P2 = G^T G
    DF_CUDA(h, cudaMemcpyAsync(P, h->gram[mode], sizeof(double) * RR, cudaMemcpyDeviceToDevice, s));
    reduce_partials<<<(R * R + 31) / 32, kT, 0, s>>>(fg, nb, R * R, R, true, P + RR);
    DF_COUNT();
    reduce_partials<<<(R * R + 31) / 32, kT, 0, s>>>(gg, nb, R * R, R, false, P + 2 * RR);
    DF_COUNT();
    const int tlin = mode == 0 ? kT100 : (mode == 1 ? kT010 : kT001);
    gd_scalars<<<1, kT, 0, s>>>(sp, nb, h->scal, tlin, mode == 0 ? kT000 : -1);
    DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
  }
  if ((st = dual_pass(h)) != DFACTO_OK) return st;
  if ((st = line_search(h, 1.0, nullptr)) != DFACTO_OK) return st;
  for (int m = 0; m < 3; ++m) {
    const int64_t rows = h->dims[m];
    const int nb = pass_blocks(rows);
    gd_update_gram<T, RT><<<nb, kT, smem_upd, s>>>(static_cast<T*>(h->F[m]), h->grad[m], h->scal,
                                                  rows, R, h->partials);
    DF_COUNT();
    reduce_partials<<<(R * R + 31) / 32, kT, 0, s>>>(h->partials, nb, R * R, R, false, h->gram[m]);
    DF_COUNT();
    h->gram_valid[m] = true;
  }
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

template <typename T>
dfacto_status gd_step_T(dfacto_t* h) {
  const int R = h->R;
  cudaStream_t s = h->stream;
  dfacto_status st;
  if (R <= 8) return gd_step_rows<T, 8>(h);
  if (R <= 12) return gd_step_rows<T, 12>(h);
  if (R <= 16) return gd_step_rows<T, 16>(h);
  if (R <= 32) return gd_step_rows<T, 32>(h);
  for (int m = 0; m < 3; ++m)
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
  DF_CUDA(h, cudaMemsetAsync(h->scal + kG2, 0, sizeof(double), s));
  for (int mode = 0; mode < 3; ++mode) {
    const ModeCSR& M = h->m[mode];
    hadamard_gamma<<<1, 256, 0, s>>>(h->gram[M.f], h->gram[M.in], R, h->lambda_reg, h->W, h->W32);
    DF_COUNT();
    if ((st = mttkrp_launch(h, mode, h->N)) != DFACTO_OK) return st;
    const int64_t rows = M.dim_o;
    const unsigned nb = row_blocks(rows);
    const size_t smem = solve_bytes(R);
    allow_smem(gd_gradient_rows<T>, smem);
    gd_gradient_rows<T><<<nb, kT, smem, s>>>(h->N, static_cast<const T*>(h->F[mode]), h->W32, rows,
                                             R, h->grad[mode], h->partials);
    DF_COUNT();
    const int tlin = mode == 0 ? kT100 : (mode == 1 ? kT010 : kT001);
    gd_scalars<<<1, kT, 0, s>>>(h->partials, (int)nb, h->scal, tlin, mode == 0 ? kT000 : -1);
    DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
  }
  // R x R matrices of the polynomial: P0 = F^T F, P1 = F^T G + G^T F, P2 = G^T G.
  for (int m = 0; m < 3; ++m) {
    double* P = h->gd_mats + (size_t)m * 3 * R * R;
    DF_CUDA(h, cudaMemcpyAsync(P, h->gram[m], sizeof(double) * R * R, cudaMemcpyDeviceToDevice, s));
    if ((st = cross_gram<T, float, false>(h, static_cast<const T*>(h->F[m]), h->grad[m], h->dims[m],
                                          P + R * R, true)) != DFACTO_OK)
      return st;
    if ((st = cross_gram<float, float, true>(h, h->grad[m], h->grad[m], h->dims[m], P + 2 * R * R,
                                             false)) != DFACTO_OK)
      return st;
  }
  if ((st = dual_pass(h)) != DFACTO_OK) return st;
  if ((st = line_search(h, 1.0, nullptr)) != DFACTO_OK) return st;
  for (int m = 0; m < 3; ++m) {
    const int64_t n = (int64_t)h->dims[m] * R;
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, kMaxBlocks * 4));
    gd_update<T><<<nb, 256, 0, s>>>(static_cast<T*>(h->F[m]), h->grad[m], n, h->scal);
    DF_COUNT();
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

namespace {
template <typename T>
dfacto_status ray_matrices_T(dfacto_t* h) {
  const int R = h->R;
  cudaStream_t s = h->stream;
  dfacto_status st;
  for (int m = 0; m < 3; ++m) {
    if (!h->gram_valid[m] && (st = gram_of_factor(h, m)) != DFACTO_OK) return st;
    double* P = h->gd_mats + (size_t)m * 3 * R * R;
    DF_CUDA(h, cudaMemcpyAsync(P, h->gram[m], sizeof(double) * R * R, cudaMemcpyDeviceToDevice, s));
    if ((st = cross_gram<T, float, false>(h, static_cast<const T*>(h->F[m]), h->grad[m], h->dims[m],
                                          P + R * R, true)) != DFACTO_OK)
      return st;
    if ((st = cross_gram<float, float, true>(h, h->grad[m], h->grad[m], h->dims[m], P + 2 * R * R,
                                             false)) != DFACTO_OK)
      return st;
  }
  return DFACTO_OK;
}

template <typename T>
dfacto_status apply_step_T(dfacto_t* h) {
  const int R = h->R;
  for (int m = 0; m < 3; ++m) {
    const int64_t n = (int64_t)h->dims[m] * R;
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, kMaxBlocks * 4));
    gd_update<T><<<nb, 256, 0, h->stream>>>(static_cast<T*>(h->F[m]), h->grad[m], n, h->scal);
    DF_COUNT();
    h->gram_valid[m] = false;
  }
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}
}  // namespace

dfacto_status ray_matrices(dfacto_t* h) {
  return h->dtype == DFACTO_BF16 ? ray_matrices_T<__nv_bfloat16>(h) : ray_matrices_T<float>(h);
}

dfacto_status line_search(dfacto_t* h, double mu, const double* ycoef) {
  if (!h->ls_vals) {
    const dfacto_status st =
        dalloc(h, reinterpret_cast<void**>(&h->ls_vals), sizeof(double) * (1 + kLineSearchTrials));
    if (st != DFACTO_OK) return st;
  }
  gd_ray_values<<<1 + kLineSearchTrials, 256, 0, h->stream>>>(h->gd_mats, h->R, h->lambda_reg, h->scal,
                                                             mu, ycoef, h->ls_vals);
  DF_COUNT();
  gd_line_search<<<1, 256, 0, h->stream>>>(h->gd_mats, h->R, h->lambda_reg, h->scal,
                                           h->flags + kFlagLsFail, h->opt.line_search, mu, ycoef,
                                           h->ls_vals);
  DF_COUNT();
  DF_CUDA(h, cudaGetLastError());
  return DFACTO_OK;
}

dfacto_status apply_step(dfacto_t* h) {
  return h->dtype == DFACTO_BF16 ? apply_step_T<__nv_bfloat16>(h) : apply_step_T<float>(h);
}

cudaError_t batch_gamma_inverse(const DenseJob* jobs, int n, int R, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t need = sizeof(double) * (2 * (size_t)R * R + R);
  const bool in_smem = need <= 48 * 1024;
  gamma_inverse_batch<<<n, 256, in_smem ? need : 0, s>>>(jobs, R, in_smem);
  DF_COUNT();
  return cudaGetLastError();
}

namespace {
template <int RT>
cudaError_t batch_post_rows(const DenseJob* jobs, const int32_t* begin, int n, int total_blocks,
                            int R, int dtype, bool last, cudaStream_t s) {
  constexpr size_t smem = row_pass_smem<RT>();
  cudaError_t e = opt_in_smem<colnorm_rows_batch<RT>, smem>();
  if (e == cudaSuccess) e = opt_in_smem<scale_store_rows_batch<__nv_bfloat16, RT>, smem>();
  if (e == cudaSuccess) e = opt_in_smem<scale_store_rows_batch<float, RT>, smem>();
  if (e != cudaSuccess) return e;
  colnorm_rows_batch<RT><<<total_blocks, kT, smem, s>>>(jobs, begin, n, R);
  DF_COUNT();
  finish_lambda_batch<<<n * R, kT, 0, s>>>(jobs, R);
  DF_COUNT();
  if (dtype == DFACTO_BF16)
    scale_store_rows_batch<__nv_bfloat16, RT><<<total_blocks, kT, smem, s>>>(jobs, begin, n, R, last);
  else
    scale_store_rows_batch<float, RT><<<total_blocks, kT, smem, s>>>(jobs, begin, n, R, last);
  DF_COUNT();
  const int per_job = (R * R + 31) / 32;
  reduce_partials_batch<<<n * per_job, kT, 0, s>>>(jobs, R, per_job);
  DF_COUNT();
  return cudaGetLastError();
}
}  // namespace

cudaError_t batch_als_post(const DenseJob* jobs, const int32_t* begin, int n, int total_blocks, int R,
                           int dtype, bool last, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (R <= 32) {
    if (R <= 8) return batch_post_rows<8>(jobs, begin, n, total_blocks, R, dtype, last, s);
    if (R <= 12) return batch_post_rows<12>(jobs, begin, n, total_blocks, R, dtype, last, s);
    if (R <= 16) return batch_post_rows<16>(jobs, begin, n, total_blocks, R, dtype, last, s);
    return batch_post_rows<32>(jobs, begin, n, total_blocks, R, dtype, last, s);
  }
  const int R4 = (R + 3) / 4;
  const size_t smem_a = solve_bytes(R);
  allow_smem(als_solve_rows_batch, smem_a);
  als_solve_rows_batch<<<total_blocks, kT, smem_a, s>>>(jobs, begin, n, R);
  DF_COUNT();
  finish_lambda_batch<<<n * R, kT, 0, s>>>(jobs, R);
  DF_COUNT();
  const size_t smem_b = tile_bytes(R, 1);
  auto store = [&](auto kernel) {
    allow_smem(kernel, smem_b);
    kernel<<<total_blocks, kT, smem_b, s>>>(jobs, begin, n, R, last);
    DF_COUNT();
  };
  if (dtype == DFACTO_BF16) {
    if (R4 * R4 <= kT) store(als_store_rows_batch<__nv_bfloat16, 1>);
    else store(als_store_rows_batch<__nv_bfloat16, 4>);
  } else {
    if (R4 * R4 <= kT) store(als_store_rows_batch<float, 1>);
    else store(als_store_rows_batch<float, 4>);
  }
  const int per_job = (R * R + 31) / 32;
  reduce_partials_batch<<<n * per_job, kT, 0, s>>>(jobs, R, per_job);
  DF_COUNT();
  return cudaGetLastError();
}

cudaError_t batch_fit(const DenseJob* jobs, int n, int R, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fit_from_parts_batch<<<n, kT, 0, s>>>(jobs, R);
  DF_COUNT();
  return cudaGetLastError();
}

}  // namespace dfacto
