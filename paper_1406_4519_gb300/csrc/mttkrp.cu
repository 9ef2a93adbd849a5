// mttkrp.cu -- host side of the MTTKRP: configuration, launch, and the carry
// fix-up kernel that finishes rows spanning several CTAs and zero-fills rows
// with no nonzeros.
#include <algorithm>

#include "mttkrp.cuh"

namespace dfacto {
namespace {

constexpr int kFixThreads = 256;
constexpr int kFixWarps = kFixThreads / 32;
constexpr int kAheadCols = 32;  // carry values per lane a warp loads before adding them

// One block per CTA c (grid-stride): if c's last partial run belongs to a row r
// that starts inside c, add up r's partials from CTAs c .. c_last in CTA order
// (eight warps take interleaved entries, then their sums are added in warp
// order) and store N[r, :].  Then all blocks zero the rows without fibers.
// `bad` (nullable) is set when a carry entry does not name the row it should.
// CPL = columns per lane (R <= 32 * CPL); a warp keeps 32 / CPL entries in
// flight, which bounds the time of the longest row (a heavy row of a
// power-law mode spans over a thousand CTAs).
template <int CPL>
__global__ void __launch_bounds__(kFixThreads) mttkrp_fixup(
    const int32_t* __restrict__ carry_row, const float* __restrict__ carry,
    const int64_t* __restrict__ fiber_ptr, const int64_t* __restrict__ nz_ptr, float* __restrict__ out,
    int R, int64_t P, int64_t ncta, int64_t dim_o, int32_t* __restrict__ bad) {
  __shared__ float part[kFixWarps][128];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t c = blockIdx.x; c < ncta; c += gridDim.x) {
    const int k = carry_row[2 * c + 1] >= 0 ? 1 : 0;
    const int r = carry_row[2 * c + k];
    if (r < 0) continue;
    const int64_t rb = nz_ptr[fiber_ptr[r]];
    if (rb < c * P) continue;  // r started in an earlier CTA, which owns it
    const int64_t re = nz_ptr[fiber_ptr[r + 1]];
    const int64_t clast = (re - 1) / P;
    const int64_t ne = clast - c + 1;
    float s[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) s[q] = 0.f;
    // Warp w adds entries w, w + 8, w + 16, ... in that order; kAhead of them
    // are loaded before the adds so that their loads overlap.
    constexpr int kAhead = kAheadCols / CPL;
    for (int64_t j0 = warp; j0 < ne; j0 += (int64_t)kAhead * kFixWarps) {
      float t[kAhead][CPL];
#pragma unroll
      for (int u = 0; u < kAhead; ++u) {
        const int64_t j = j0 + (int64_t)u * kFixWarps;
        const int64_t entry = (j == 0) ? (2 * c + k) : (2 * (c + j));
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
          const int col = lane + 32 * q;
          t[u][q] = (j < ne && col < R) ? carry[entry * R + col] : 0.f;
        }
      }
      // Entries past the end hold +0 and are added too (no branch between the
      // loads and the adds); only the sign of a zero sum can differ.
#pragma unroll
      for (int u = 0; u < kAhead; ++u)
#pragma unroll
        for (int q = 0; q < CPL; ++q) s[q] += t[u][q];
      if (lane < kAhead) {
        const int64_t j = j0 + (int64_t)lane * kFixWarps;
        if (bad && j > 0 && j < ne && carry_row[2 * (c + j)] != r) atomicOr(bad, 1);
      }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int col = lane + 32 * q;
      if (col < R) part[warp][col] = s[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const int col = lane + 32 * q;
        if (col < R) {
          float t = 0.f;
          for (int w = 0; w < kFixWarps; ++w) t += part[w][col];
          out[(int64_t)r * R + col] = t;
        }
      }
    }
    __syncthreads();
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < dim_o; o += stride) {
    if (fiber_ptr[o] == fiber_ptr[o + 1]) {
      float* row = out + o * R;
      for (int col = 0; col < R; ++col) row[col] = 0.f;
    }
  }
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }

// Rows of an R-column matrix (storage type T) as FP32 rows of RP >= R columns,
// the extra columns zero.
template <typename T>
__global__ void pad_rows(const T* __restrict__ src, int64_t rows, int R, int RP, float* __restrict__ dst) {
  const int64_t n = rows * RP;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t r = e / RP;
    const int c = (int)(e - r * RP);
    dst[e] = c < R ? to_float(src[r * R + c]) : 0.f;
  }
}

// The first R of every RP columns back to rows of R columns.
__global__ void unpad_rows(const float* __restrict__ src, int64_t rows, int R, int RP, float* __restrict__ dst) {
  const int64_t n = rows * R;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t r = e / R;
    const int c = (int)(e - r * R);
    dst[e] = src[r * RP + c];
  }
}

unsigned rows_grid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

}  // namespace

int walk_rank(int R, int vec_opt) {
  return (vec_opt == 0 && R > 2 && R % 4 != 0) ? (R + 3) / 4 * 4 : R;
}

cudaError_t pad_factor_rows(const void* src, int src_dtype, int64_t rows, int R, int RP, float* dst,
                            cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (src_dtype == DFACTO_BF16)
    pad_rows<__nv_bfloat16><<<rows_grid(rows * RP), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(src),
                                                                   rows, R, RP, dst);
  else
    pad_rows<float><<<rows_grid(rows * RP), 256, 0, s>>>(static_cast<const float*>(src), rows, R, RP, dst);
  DF_COUNT();
  return cudaGetLastError();
}

cudaError_t launch_mttkrp_fixup(const int32_t* carry_row, const float* carry,
                                const int64_t* fiber_ptr, const int64_t* nz_ptr, float* out, int R,
                                int64_t P, int64_t ncta, int64_t dim_o, int32_t* bad,
                                cudaStream_t s) {
  const int64_t zero_blocks = (dim_o + kFixThreads - 1) / kFixThreads;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(std::max(ncta, zero_blocks), 152 * 16));
  if (R <= 32)
    mttkrp_fixup<1><<<(unsigned)blocks, kFixThreads, 0, s>>>(carry_row, carry, fiber_ptr, nz_ptr, out,
                                                              R, P, ncta, dim_o, bad);
  else if (R <= 64)
    mttkrp_fixup<2><<<(unsigned)blocks, kFixThreads, 0, s>>>(carry_row, carry, fiber_ptr, nz_ptr, out,
                                                              R, P, ncta, dim_o, bad);
  else
    mttkrp_fixup<kMaxColsPerLane><<<(unsigned)blocks, kFixThreads, 0, s>>>(
        carry_row, carry, fiber_ptr, nz_ptr, out, R, P, ncta, dim_o, bad);
  DF_COUNT();
  return cudaGetLastError();
}

WalkCfg choose_walk(int R, int dtype, int64_t nnz, int64_t nfib, int seg_opt, int vec_opt) {
  (void)nnz;
  (void)nfib;
  WalkCfg c;
  // Default: one 16-byte load per lane and factor row (4 FP32 or 8 BF16
  // columns), measured fastest on the 50M-nonzero power-law workload at
  // R = 16 and 32.
  int vec = vec_opt > 0 ? vec_opt : (dtype == DFACTO_BF16 ? 8 : 4);
  while (vec > 1 && (R % vec) != 0) vec >>= 1;
  int G = next_pow2((R + vec - 1) / vec);
  while (G > 32 && vec < 8 && (R % (vec * 2)) == 0) {
    vec *= 2;
    G = next_pow2((R + vec - 1) / vec);
  }
  c.vec = vec;
  c.G = G;
  c.kernel = 2;  // fiber ends from the end bitmask (faster on every measured shape)
  int seg = seg_opt > 0 ? seg_opt : 128;
  seg = std::max(32, (seg + 31) / 32 * 32);
  c.seg = seg;
  return c;
}

dfacto_status mttkrp_launch(dfacto_t* h, int mode, float* out) {
  ModeCSR& M = h->m[mode];
  // At a rank that is not a multiple of four the walk runs on zero-padded FP32
  // copies of the two gathered factors at the padded rank RP (one 16-byte
  // gather per lane: R = 10 walks 3 of 4 lanes per group instead of 5 of 8
  // with 8-byte gathers, measured 1.45x faster) and its output is copied back
  // to R columns; an explicit lane width keeps the unpadded walk.  Both walks
  // pad alike, so they still compute the same sums in the same order.
  const int R = h->R;
  const int RP = walk_rank(R, h->opt.vec);
  const bool padded = RP != R;
  WalkCfg cfg = M.cfg;
  if (padded) {
    cfg = choose_walk(RP, DFACTO_F32, h->nnz, M.nfib, h->opt.seg_nnz, 0);
    cfg.kernel = M.cfg.kernel;
  }
  dfacto_status st = ensure_segments(h, mode);
  if (st != DFACTO_OK) return st;
  const int segs = kWalkWarps * (32 / cfg.G);
  const int64_t P = (int64_t)segs * cfg.seg;
  const int64_t ncta = (h->nnz + P - 1) / P;
  if (ncta > h->carry_cap || RP > h->carry_rank) {
    if (h->carry) dfree(h, h->carry, sizeof(float) * 2 * (size_t)h->carry_rank * h->carry_cap);
    if (h->carry_row) dfree(h, h->carry_row, sizeof(int32_t) * 2 * (size_t)h->carry_cap);
    h->carry = nullptr;
    h->carry_row = nullptr;
    const int64_t cap = std::max(ncta, h->carry_cap);
    const int rank = std::max(RP, h->carry_rank);
    h->carry_cap = 0;
    h->carry_rank = 0;
    st = dalloc(h, reinterpret_cast<void**>(&h->carry), sizeof(float) * 2 * (size_t)rank * cap);
    if (st == DFACTO_OK)
      st = dalloc(h, reinterpret_cast<void**>(&h->carry_row), sizeof(int32_t) * 2 * (size_t)cap);
    if (st != DFACTO_OK) return st;
    h->carry_cap = cap;
    h->carry_rank = rank;
  }
  const void* Fin = h->F[M.in];
  const void* Ff = h->F[M.f];
  float* wout = out;
  if (padded) {
    const int64_t maxdim = std::max<int64_t>(h->dims[0], std::max<int64_t>(h->dims[1], h->dims[2]));
    const size_t bytes = sizeof(float) * (size_t)maxdim * RP;
    for (float** q : {&h->pad_in, &h->pad_f, &h->pad_out})
      if (!*q && (st = dalloc(h, reinterpret_cast<void**>(q), bytes)) != DFACTO_OK) return st;
    DF_CUDA(h, pad_factor_rows(Fin, h->dtype, h->dims[M.in], R, RP, h->pad_in, h->stream));
    DF_CUDA(h, pad_factor_rows(Ff, h->dtype, h->dims[M.f], R, RP, h->pad_f, h->stream));
    Fin = h->pad_in;
    Ff = h->pad_f;
    wout = h->pad_out;
  }
  MttkrpParams a;
  a.fiber_ptr = M.fiber_ptr;
  a.fiber_idx = M.fiber_idx;
  a.fiber_row = M.fiber_row;
  a.nz_ptr = M.nz_ptr;
  a.nz_idx = M.nz_idx;
  a.nz_val = M.nz_val;
  a.seg_fib = M.seg_fib;
  a.end_bits = M.end_bits;
  a.Fin = Fin;
  a.Ff = Ff;
  a.out = wout;
  a.carry = h->carry;
  a.carry_row = h->carry_row;
  a.nnz = h->nnz;
  a.nfib = M.nfib;
  a.dim_o = M.dim_o;
  a.R = RP;
  a.seg = cfg.seg;
  if (ncta > 0) {
    const size_t smem = sizeof(float) * (size_t)(2 * segs + 2 * kWalkWarps) * RP;
    cudaError_t e;
    if (cfg.kernel == 2)
      e = (h->dtype == DFACTO_BF16 && !padded) ? launch_walk2<__nv_bfloat16>(cfg.vec, cfg.G, a, ncta, h->stream)
                                               : launch_walk2<float>(cfg.vec, cfg.G, a, ncta, h->stream);
    else
      e = (h->dtype == DFACTO_BF16 && !padded)
              ? launch_walk<__nv_bfloat16>(cfg.vec, cfg.G, a, ncta, smem, h->stream)
              : launch_walk<float>(cfg.vec, cfg.G, a, ncta, smem, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "mttkrp_walk launch");
  }
  DF_CUDA(h, launch_mttkrp_fixup(h->carry_row, h->carry, M.fiber_ptr, M.nz_ptr, wout, RP, P, ncta,
                                 M.dim_o, h->flags + kFlagInternal, h->stream));
  if (padded) {
    unpad_rows<<<rows_grid(M.dim_o * R), 256, 0, h->stream>>>(h->pad_out, M.dim_o, R, RP, out);
    DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
  }
  return DFACTO_OK;
}

}  // namespace dfacto
