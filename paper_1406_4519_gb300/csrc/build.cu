// build.cu -- COO -> flattened CSR copies on the device (Sec. 3, Lemmas 3-4).
//
// For each mode n the nonzeros are sorted by the key (o, f, in), o = axis n,
// f = axis n+2, in = axis n+1: this is the row order of (X^{n+1})^T (row index
// f + o*dim_f in 0-based form of the proof of Lemma 4) with ascending columns
// inside each row.  Maximal runs of equal (o, f) are the nonzero rows of
// (X^{n+1})^T, i.e. the fibers; their starts give nz_ptr, their f gives
// col(M^r) and their o gives row(M^r) (fiber_ptr, empty rows kept).
//
// The sort is a least-significant-digit radix sort with 8- or 9-bit digits
// written for this library: per-tile digit histograms, a device-wide scan, and
// a stable scatter that ranks equal digits inside a warp with
// __match_any_sync.  Keys of up to 64 bits sort in one run with the nonzero's
// value as payload; wider (o, f, in) keys take two stable runs (first by `in`,
// then by (o, f)) with the nonzero's position as payload.  The fiber-end
// bitmask of the walk comes out of the same pass that flags the fiber starts.
//
// The three modes are sorted as a chain m, m + 1, m + 2.  Mode m's sorted
// order is lexicographic in (m, m + 2, m + 1); mode m + 1 wants
// (m + 1, m, m + 2), which is that order with axis m + 1 moved to the front,
// so a stable sort by mode m + 1's row axis o alone yields it (equal o keep
// their (f, in) order).  For 64-bit keys the next mode's key is a bit rotation
// of the sorted key (every axis is in it), and its sort reads only the o bits.
#include <algorithm>

#include "device.cuh"
#include "internal.h"
#include "mttkrp.cuh"

namespace dfacto {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int64_t kSortTile = (int64_t)kSortThreads * kSortRounds;
constexpr int kMaxDigitBits = 9;  // digits of 8 or 9 bits (256 or 512 bins)

int nbits_for(int64_t dim) {  // bits needed for values 0 .. dim-1
  int b = 0;
  while (b < 63 && (int64_t(1) << b) < dim) ++b;
  return b;
}

__global__ void check_range(const int32_t* __restrict__ idx, int64_t nnz, int32_t d0, int32_t d1,
                            int32_t d2, int32_t* __restrict__ flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += stride) {
    const int32_t i = idx[t], j = idx[nnz + t], k = idx[2 * nnz + t];
    bad |= (i < 0) | (i >= d0) | (j < 0) | (j >= d1) | (k < 0) | (k >= d2);
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// ||X||^2: squares and partial sums in FP64, one partial per block.
__global__ void sumsq_partials(const float* __restrict__ val, int64_t n, double* __restrict__ part) {
  __shared__ double s[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const double x = val[t];
    acc += x * x;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_partials(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];  // fixed order: deterministic
    *out = t;
  }
}

__device__ __forceinline__ uint64_t shl64(uint64_t x, int b) { return b >= 64 ? 0ull : x << b; }
__device__ __forceinline__ uint64_t shr64(uint64_t x, int b) { return b >= 64 ? 0ull : x >> b; }
__device__ __forceinline__ uint64_t low64(uint64_t x, int b) { return b >= 64 ? x : x & ((1ull << b) - 1ull); }

// Composite 64-bit key (o << (bf + bi)) | (f << bi) | in with the value's bits
// as payload.
__global__ void make_keys64_val(const int32_t* __restrict__ idx, const float* __restrict__ val,
                                int64_t nnz, int ao, int af, int ai, int bf, int bi,
                                uint64_t* __restrict__ key, uint32_t* __restrict__ vbits) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += stride) {
    const uint64_t o = (uint32_t)idx[ao * nnz + t], f = (uint32_t)idx[af * nnz + t],
                   in = (uint32_t)idx[ai * nnz + t];
    key[t] = shl64(o, bf + bi) | shl64(f, bi) | in;
    vbits[t] = __float_as_uint(val[t]);
  }
}

// Key of the next mode of the chain from a sorted key of this one (in place):
// (o, f, in) with widths (bo, bf, bi) becomes (in, o, f), i.e. the next mode's
// (o, f, in) with widths (bi, bo, bf).
__global__ void rotate_keys(uint64_t* __restrict__ key, int64_t n, int bo, int bf, int bi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const uint64_t k = key[p];
    const uint64_t o = shr64(k, bf + bi), f = low64(shr64(k, bi), bf), in = low64(k, bi);
    key[p] = shl64(in, bo + bf) | shl64(o, bf) | f;
  }
}

// First run of a wide key: sort by `in` alone.
__global__ void make_keys_in(const int32_t* __restrict__ idx, int64_t nnz, int ai,
                             uint64_t* __restrict__ key, uint32_t* __restrict__ perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += stride) {
    key[t] = (uint32_t)idx[ai * nnz + t];
    perm[t] = (uint32_t)t;
  }
}

// Second run of a wide key: (o << bf) | f of the element now at position p.
__global__ void make_keys_of(const int32_t* __restrict__ idx, int64_t nnz, int ao, int af, int bf,
                             const uint32_t* __restrict__ perm, uint64_t* __restrict__ key) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int64_t t = perm[p];
    key[p] = ((uint64_t)(uint32_t)idx[ao * nnz + t] << bf) | (uint32_t)idx[af * nnz + t];
  }
}

// Chained run: key (o << bf) | f of the element at position p of the previous
// mode's sorted order, whose permutation `chain` is carried along as payload.
__global__ void make_keys_chain(const int32_t* __restrict__ idx, int64_t nnz, int ao, int af, int bf,
                                const uint32_t* __restrict__ chain, uint64_t* __restrict__ key,
                                uint32_t* __restrict__ perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const uint32_t t = chain[p];
    key[p] = ((uint64_t)(uint32_t)idx[ao * nnz + t] << bf) | (uint32_t)idx[af * nnz + t];
    perm[p] = t;
  }
}

// Per-tile digit counts, written digit-major: cnt[d * ntiles + tile] (scanned
// into output offsets afterwards), and tile-major: lcnt[tile * D + d] (kept
// for the tile's own digit order in radix_scatter).  A digit is BITS bits of
// the key from `shift`, masked by dmask (the last digit of a range may be
// narrower).  Each warp counts into its own counters: one add of 32 when the
// warp's 32 digits are equal (the high digits of power-law indices), else one
// shared-memory atomic per lane; the warps' counters are added at the end.
template <int BITS>
__global__ void __launch_bounds__(kSortThreads) radix_hist(const uint64_t* __restrict__ key,
                                                          int64_t n, int shift, uint32_t dmask,
                                                          int32_t* __restrict__ cnt,
                                                          int32_t* __restrict__ lcnt, int64_t ntiles) {
  constexpr int D = 1 << BITS;
  constexpr int W = kSortThreads / 32;
  __shared__ int32_t s_cnt[W][D];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < D; d += 32) s_cnt[warp][d] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  // all of the thread's keys first (independent loads in flight together)
  int dg[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    dg[r] = i < n ? (int)((key[i] >> shift) & dmask) : D;
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int d = dg[r];
    const int d0 = __shfl_sync(kFull, d, 0);
    if (__all_sync(kFull, d == d0)) {
      if (lane == 0 && d0 < D) s_cnt[warp][d0] += 32;
    } else if (d < D) {
      atomicAdd(&s_cnt[warp][d], 1);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int d = threadIdx.x; d < D; d += kSortThreads) {
    int32_t c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += s_cnt[w][d];
    cnt[(int64_t)d * ntiles + blockIdx.x] = c;
    lcnt[(int64_t)blockIdx.x * D + d] = c;
  }
}

// Stable scatter of one tile.  Warp w holds the tile's elements
// [512 w, 512 w + 512) (round r, lane l: element 512 w + 32 r + l), so the
// order (warp, round, lane) is the tile's element order.  Each warp ranks its
// own elements against its own digit counters (no block barrier per round);
// one pass over the digits then turns the warps' counts into offsets of the
// tile's digit-ordered layout in shared memory, and thread t copies out
// positions t, t + 256, ...: consecutive threads write consecutive positions
// of one digit's output run, so the writes are coalesced runs.
constexpr int kSortWarps = kSortThreads / 32;
template <int BITS>
constexpr size_t scatter_smem() {
  return (sizeof(uint64_t) + sizeof(uint32_t)) * kSortTile +
         sizeof(int32_t) * (kSortWarps + 2) * ((size_t)1 << BITS);
}

template <int BITS>
__global__ void __launch_bounds__(kSortThreads, 3) radix_scatter(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, uint32_t dmask,
    const int32_t* __restrict__ ofs, const int32_t* __restrict__ lcnt, int64_t ntiles) {
  constexpr int D = 1 << BITS;
  constexpr int DPT = D / kSortThreads;  // digits per thread in the digit passes
  constexpr int kPerWarp = kSortTile / kSortWarps;
  extern __shared__ __align__(16) unsigned char sort_smem[];  // scatter_smem<BITS>() bytes
  uint64_t* s_key = reinterpret_cast<uint64_t*>(sort_smem);              // [kSortTile]
  uint32_t* s_val = reinterpret_cast<uint32_t*>(s_key + kSortTile);       // [kSortTile]
  int32_t* s_cnt = reinterpret_cast<int32_t*>(s_val + kSortTile);         // [kSortWarps][D]
  int32_t* s_lstart = s_cnt + kSortWarps * D;                             // [D]
  int32_t* s_gofs = s_lstart + D;                                         // [D]
  __shared__ int32_t s_wsum[kSortWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const int tn = (int)min((int64_t)kSortTile, n - base);
  const int64_t wbase = base + (int64_t)warp * kPerWarp + lane;
  // the warp's keys, all loads in flight together (the payloads are read when
  // they are placed)
  uint64_t k[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = wbase + 32 * r;
    k[r] = i < n ? kin[i] : 0;
  }
  int32_t* wcnt = s_cnt + warp * D;
#pragma unroll
  for (int q = 0; q < D / 32; ++q) wcnt[lane + 32 * q] = 0;
  __syncwarp();
  // rank of each element among the warp's equal digits before it (< 512: two
  // ranks per register)
  uint32_t lr[kSortRounds / 2];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const bool ok = wbase + 32 * r < n;
    const int d = ok ? (int)((k[r] >> shift) & dmask) : D;
    const unsigned peers = __match_any_sync(kFull, d);
    const int rank = __popc(peers & lt);
    const int c = ok ? wcnt[d] : 0;
    if (r & 1) lr[r / 2] |= (uint32_t)(c + rank) << 16;
    else lr[r / 2] = (uint32_t)(c + rank);
    __syncwarp();
    if (ok && rank == 0) wcnt[d] = c + __popc(peers);
    __syncwarp();
  }
  {  // the tile's digit starts: exclusive scan of its counts, thread t owns
     // digits [DPT t, DPT t + DPT)
    const int d0 = DPT * threadIdx.x;
    int c[DPT];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      c[j] = lcnt[(int64_t)blockIdx.x * D + d0 + j];
      sum += c[j];
    }
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();  // also: every warp's counts are final
    int run = x - sum;
    for (int w = 0; w < warp; ++w) run += s_wsum[w];
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = d0 + j;
      s_lstart[d] = run;
      s_gofs[d] = ofs[(int64_t)d * ntiles + blockIdx.x];
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {  // warp w's first position of digit d
        const int32_t cw = s_cnt[w * D + d];
        s_cnt[w * D + d] = run;
        run += cw;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    if (wbase + 32 * r < n) {
      const int d = (int)((k[r] >> shift) & dmask);
      const int lp = wcnt[d] + (int)((lr[r / 2] >> (16 * (r & 1))) & 0xffffu);
      s_key[lp] = k[r];
      s_val[lp] = vin[wbase + 32 * r];
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < tn; p += kSortThreads) {
    const uint64_t key = s_key[p];
    const int d = (int)((key >> shift) & dmask);
    const int64_t gp = (int64_t)s_gofs[d] + (p - s_lstart[d]);
    kout[gp] = key;
    vout[gp] = s_val[p];
  }
}

// After the sort: fiber-start flags, duplicate detection, nz_idx and nz_val,
// and the fiber-end bitmask (bit p of end_bits set iff nonzero p is the last
// of its fiber: p is the last nonzero or p + 1 starts a new fiber; one ballot
// per warp of 32 consecutive positions).
// narrow: key = (o,f,in) packed with `in` in the low bi bits.
// wide:   key = (o,f) packed; `in` comes from the COO through perm.
// With val_payload the payload holds the value's bits (narrow keys), else the
// nonzero's position in the COO.
__global__ void segment_flags(const uint64_t* __restrict__ key, const uint32_t* __restrict__ perm,
                              int64_t n, int bi, bool wide, bool val_payload,
                              const int32_t* __restrict__ idx, int ai,
                              const float* __restrict__ val, int32_t* __restrict__ head,
                              int32_t* __restrict__ nz_idx, float* __restrict__ nz_val,
                              uint32_t* __restrict__ end_bits, int32_t* __restrict__ dup_flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32
  const int lane = threadIdx.x & 31;
  bool dup = false;
  // warp-uniform loop: the warp's lanes take 32 consecutive positions from p0
  for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); p0 < n; p0 += stride) {
    const int64_t p = p0 + lane;
    bool endb = false;
    if (p < n) {
      const uint64_t k = key[p];
      const uint32_t pl = perm[p];
      int32_t in;
      uint64_t fkey;
      if (wide) {
        in = idx[ai * n + pl];
        fkey = k;
      } else {
        in = (int32_t)low64(k, bi);
        fkey = shr64(k, bi);
      }
      int32_t h = 1;
      if (p > 0) {
        const uint64_t kp = key[p - 1];
        if (wide) {
          if (kp == k) {
            h = 0;
            dup |= (idx[ai * n + perm[p - 1]] == in);
          }
        } else {
          const uint64_t fp = (bi >= 64) ? 0 : (kp >> bi);
          h = (fp != fkey);
          dup |= (kp == k);
        }
      }
      if (p + 1 >= n) {
        endb = true;
      } else {
        const uint64_t kn = key[p + 1];
        endb = wide ? (kn != k) : (shr64(kn, bi) != fkey);
      }
      head[p] = h;
      nz_idx[p] = in;
      nz_val[p] = val_payload ? __uint_as_float(pl) : val[pl];
    }
    const unsigned bits = __ballot_sync(kFull, endb);
    if (lane == 0) end_bits[p0 >> 5] = bits;
  }
  if (__any_sync(kFull, dup) && lane == 0) atomicOr(dup_flag, 1);
}

__global__ void scatter_fibers(const uint64_t* __restrict__ key, const uint32_t* __restrict__ perm,
                               int64_t n, int bf, int bi, bool wide, const int32_t* __restrict__ head,
                               const int32_t* __restrict__ fid, int64_t* __restrict__ nz_ptr,
                               int32_t* __restrict__ fiber_idx, int32_t* __restrict__ fiber_row,
                               int64_t nfib) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    if (!head[p]) continue;
    const uint64_t k = key[p];
    const uint64_t of = wide ? k : ((bi >= 64) ? 0 : (k >> bi));
    const uint64_t fmask = (bf >= 64) ? ~0ull : ((1ull << bf) - 1ull);
    const int32_t q = fid[p];
    nz_ptr[q] = p;
    fiber_idx[q] = (int32_t)(of & fmask);
    fiber_row[q] = (int32_t)((bf >= 64) ? 0 : (of >> bf));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) nz_ptr[nfib] = n;
}

// fiber_ptr[r] = number of fibers whose row is < r (lower bound in fiber_row).
__global__ void row_pointers(const int32_t* __restrict__ fiber_row, int64_t nfib, int64_t dim_o,
                             int64_t* __restrict__ fiber_ptr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= dim_o; r += stride) {
    int64_t lo = 0, hi = nfib;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (fiber_row[mid] < r) lo = mid + 1; else hi = mid;
    }
    fiber_ptr[r] = lo;
  }
}

// end_bits: bit e set for the last nonzero e of every fiber, from nz_ptr (the
// batched tensors' concatenated copies; a tensor's own build sets the bits in
// segment_flags).
__global__ void fiber_end_bits(const int64_t* __restrict__ nz_ptr, int64_t nfib,
                               uint32_t* __restrict__ bits) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nfib; q += stride) {
    const int64_t e = nz_ptr[q + 1] - 1;
    atomicOr(bits + (e >> 5), 1u << (e & 31));
  }
}

// seg_fib[s] = the fiber holding nonzero s*seg: the last q with nz_ptr[q] <= s*seg.
__global__ void segment_starts(const int64_t* __restrict__ nz_ptr, int64_t nfib, int64_t nseg,
                               int64_t seg, int32_t* __restrict__ seg_fib) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += stride) {
    const int64_t p = s * seg;
    int64_t lo = 0, hi = nfib;  // find first q with nz_ptr[q] > p, in [1, nfib]
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (nz_ptr[mid] <= p) lo = mid + 1; else hi = mid;
    }
    seg_fib[s] = (int32_t)(lo - 1);
  }
}

unsigned grid_for(int64_t n, int threads = 256, int64_t cap = 152 * 32) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

// One radix pass of BITS-bit digits from `shift` (digits masked to the sort's
// top bit): counts, scan, scatter.
template <int BITS>
cudaError_t radix_pass(const uint64_t* ki, const uint32_t* vi, uint64_t* ko, uint32_t* vo, int64_t n,
                       int shift, int hi_bit, int32_t* cnt, int64_t ntiles, cudaStream_t s) {
  constexpr int D = 1 << BITS;
  const int w = std::min(BITS, hi_bit - shift);
  const uint32_t dmask = (w >= 32) ? 0xffffffffu : ((1u << w) - 1u);
  int32_t* lcnt = cnt + (int64_t)D * ntiles;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(radix_scatter<BITS>),
                                      scatter_smem<BITS>());
  if (e != cudaSuccess) return e;
  radix_hist<BITS><<<(unsigned)ntiles, kSortThreads, 0, s>>>(ki, n, shift, dmask, cnt, lcnt, ntiles);
  DF_COUNT();
  e = cudaGetLastError();
  if (e == cudaSuccess) e = exclusive_scan_i32(cnt, cnt, (int64_t)D * ntiles, s);
  if (e == cudaSuccess) {
    radix_scatter<BITS><<<(unsigned)ntiles, kSortThreads, scatter_smem<BITS>(), s>>>(
        ki, vi, ko, vo, n, shift, dmask, cnt, lcnt, ntiles);
    DF_COUNT();
    e = cudaGetLastError();
  }
  return e;
}

// Digit passes for an nbits-wide range: the fewest passes of at most
// kMaxDigitBits bits, of equal width (at least 8).
void radix_plan(int nbits, int* passes, int* bits) {
  if (nbits <= 0) {
    *passes = 0;
    *bits = 8;
    return;
  }
  int p = (nbits + kMaxDigitBits - 1) / kMaxDigitBits;
  int b = (nbits + p - 1) / p;
  if (b < 8) {
    b = 8;
    p = (nbits + 7) / 8;
  }
  *passes = p;
  *bits = b;
}
int radix_passes(int nbits) {
  int p, b;
  radix_plan(nbits, &p, &b);
  return p;
}

// Digit-count scratch of a sort of n pairs (int32 entries): enough for every
// digit width.
int64_t radix_scratch_entries(int64_t n) {
  return 2 * ((int64_t)1 << kMaxDigitBits) * ((n + kSortTile - 1) / kSortTile);
}

// Stable LSD radix sort of (key, val) pairs by bits [lo_bit, hi_bit), digits
// from lo_bit up (the order of keys equal in those bits is kept), in the
// passes of radix_plan.  The result is left in (k0, v0) or (k1, v1); *in_alt
// tells which.  `scratch` (radix_scratch_entries(n) entries) may be null: the
// sort then allocates its own.
cudaError_t radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                       int lo_bit, int hi_bit, cudaStream_t s, bool* in_alt,
                       int32_t* scratch = nullptr) {
  *in_alt = false;
  const int nbits = hi_bit - lo_bit;
  if (n <= 1 || nbits <= 0) return cudaSuccess;
  int passes, bits;
  radix_plan(nbits, &passes, &bits);
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  int32_t* cnt = scratch;
  cudaError_t e = cudaSuccess;
  if (!cnt) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&cnt), sizeof(int32_t) * radix_scratch_entries(n), s);
    if (e != cudaSuccess) return e;
  }
  uint64_t *ki = k0, *ko = k1;
  uint32_t *vi = v0, *vo = v1;
  for (int pass = 0; pass < passes && e == cudaSuccess; ++pass) {
    const int shift = lo_bit + bits * pass;
    e = (bits == 8) ? radix_pass<8>(ki, vi, ko, vo, n, shift, hi_bit, cnt, ntiles, s)
                    : radix_pass<9>(ki, vi, ko, vo, n, shift, hi_bit, cnt, ntiles, s);
    std::swap(ki, ko);
    std::swap(vi, vo);
    *in_alt = !*in_alt;
  }
  cudaError_t e2 = scratch ? cudaSuccess : cudaFreeAsync(cnt, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace

cudaError_t sort_pairs64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                         int lo_bit, int hi_bit, cudaStream_t s, bool* in_alt) {
  return radix_sort(k0, v0, k1, v1, n, lo_bit, hi_bit, s, in_alt);
}

cudaError_t launch_segment_starts(const int64_t* nz_ptr, int64_t nfib, int64_t nseg, int64_t seg,
                                  int32_t* seg_fib, cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  segment_starts<<<grid_for(nseg), 256, 0, s>>>(nz_ptr, nfib, nseg, seg, seg_fib);
  DF_COUNT();
  return cudaGetLastError();
}

cudaError_t launch_fiber_end_bits(const int64_t* nz_ptr, int64_t nfib, int64_t nnz, uint32_t* bits,
                                  cudaStream_t s) {
  const size_t words = (size_t)((nnz + 31) / 32);
  if (words == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(uint32_t) * words, s);
  if (e != cudaSuccess || nfib <= 0) return e;
  fiber_end_bits<<<grid_for(nfib), 256, 0, s>>>(nz_ptr, nfib, bits);
  DF_COUNT();
  return cudaGetLastError();
}

dfacto_status ensure_segments(dfacto_t* h, int mode) {
  ModeCSR& M = h->m[mode];
  const int seg = M.cfg.seg;
  if (M.seg_fib && M.seg_fib_for == seg) return DFACTO_OK;
  if (M.seg_fib) {
    dfree(h, M.seg_fib, sizeof(int32_t) * (size_t)std::max<int64_t>(M.nseg, 1));
    M.seg_fib = nullptr;
  }
  M.nseg = (h->nnz + seg - 1) / seg;
  dfacto_status st = dalloc(h, reinterpret_cast<void**>(&M.seg_fib),
                            sizeof(int32_t) * (size_t)std::max<int64_t>(M.nseg, 1));
  if (st != DFACTO_OK) return st;
  if (M.nseg > 0) {
    segment_starts<<<grid_for(M.nseg), 256, 0, h->stream>>>(M.nz_ptr, M.nfib, M.nseg, seg, M.seg_fib); DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
  }
  M.seg_fib_for = seg;
  return DFACTO_OK;
}

dfacto_status build_modes(dfacto_t* h, const int32_t* d_idx, const float* d_val) {
  cudaStream_t s = h->stream;
  const int64_t n = h->nnz;
  DF_CUDA(h, cudaMemsetAsync(h->flags, 0, sizeof(int32_t) * kNumFlags, s));
  if (n > 0) {
    check_range<<<grid_for(n), 256, 0, s>>>(d_idx, n, h->dims[0], h->dims[1], h->dims[2],
                                            h->flags + kFlagRange); DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
    DF_CUDA(h, cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int32_t) * kNumFlags,
                               cudaMemcpyDeviceToHost, s));
    DF_CUDA(h, cudaStreamSynchronize(s));
    if (h->host_flags[kFlagRange]) return fail(h, DFACTO_ERANGE, "a coordinate lies outside dims");
  }
  // ||X||^2 once (FP64).
  {
    const unsigned nb = grid_for(n, 256, 1024);
    sumsq_partials<<<nb, 256, 0, s>>>(d_val, n, h->partials); DF_COUNT();
    sum_partials<<<1, 32, 0, s>>>(h->partials, (int)nb, h->scal + kNormX2); DF_COUNT();
    DF_CUDA(h, cudaGetLastError());
  }

  uint64_t *k0 = nullptr, *k1 = nullptr;
  uint32_t *v0 = nullptr, *v1 = nullptr;
  int32_t *head = nullptr, *fid = nullptr, *sort_cnt = nullptr;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  cudaError_t e = cudaSuccess;
  auto cleanup = [&]() {
    if (k0) cudaFreeAsync(k0, s);
    if (k1) cudaFreeAsync(k1, s);
    if (v0) cudaFreeAsync(v0, s);
    if (v1) cudaFreeAsync(v1, s);
    if (head) cudaFreeAsync(head, s);
    if (fid) cudaFreeAsync(fid, s);
    if (sort_cnt) cudaFreeAsync(sort_cnt, s);
  };
  if (n > 0) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&k0), sizeof(uint64_t) * nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&k1), sizeof(uint64_t) * nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&v0), sizeof(uint32_t) * nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&v1), sizeof(uint32_t) * nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&head), sizeof(int32_t) * nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&fid), sizeof(int32_t) * nn, s);
    if (e == cudaSuccess)
      e = cudaMallocAsync(reinterpret_cast<void**>(&sort_cnt), sizeof(int32_t) * radix_scratch_entries(n), s);
    if (e != cudaSuccess) {
      cleanup();
      cudaGetLastError();
      return fail(h, e == cudaErrorMemoryAllocation ? DFACTO_ENOMEM : DFACTO_ECUDA,
                  std::string("build scratch allocation: ") + cudaGetErrorString(e));
    }
  }

  // Mode order of the sorts (the chain of the header): the start is the mode
  // that minimises the total number of digit passes; with 64-bit keys every
  // start costs the same full sort, and each later mode sorts its o bits only.
  int bits[3];
  for (int a = 0; a < 3; ++a) bits[a] = nbits_for(h->dims[a]);
  const bool narrow = bits[0] + bits[1] + bits[2] <= 64;
  auto o_passes = [&](int m) { return radix_passes(bits[m]); };
  auto full_passes = [&](int m) {
    const int bo = bits[m], bf = bits[(m + 2) % 3], bi = bits[(m + 1) % 3];
    return narrow ? radix_passes(bo + bf + bi) : radix_passes(bi) + radix_passes(bo + bf);
  };
  int start = 2, best = 1 << 30;
  for (int m = 2; m >= 0; --m) {
    const int c = full_passes(m) + o_passes((m + 1) % 3) + o_passes((m + 2) % 3);
    if (c < best) {
      best = c;
      start = m;
    }
  }
  // The previous mode's sorted (key, payload) arrays and key widths.
  uint64_t* prev_k = nullptr;
  uint32_t* prev_v = nullptr;
  int prev_bo = 0, prev_bf = 0, prev_bi = 0;

  for (int step = 0; step < 3; ++step) {
    const int mode = (start + step) % 3;
    ModeCSR& M = h->m[mode];
    M.o = mode;
    M.in = (mode + 1) % 3;
    M.f = (mode + 2) % 3;
    M.dim_o = h->dims[M.o];
    const int bo = nbits_for(h->dims[M.o]), bf = nbits_for(h->dims[M.f]),
              bi = nbits_for(h->dims[M.in]);
    const bool chained = prev_k != nullptr;
    // wide: the sorted key holds (o, f) only, the payload is the COO position
    // and `in` and the value are read through it
    const bool wide = !narrow;
    dfacto_status st = DFACTO_OK;
    st = dalloc(h, reinterpret_cast<void**>(&M.fiber_ptr), sizeof(int64_t) * (size_t)(M.dim_o + 1));
    if (st == DFACTO_OK) st = dalloc(h, reinterpret_cast<void**>(&M.nz_idx), sizeof(int32_t) * nn);
    if (st == DFACTO_OK) st = dalloc(h, reinterpret_cast<void**>(&M.nz_val), sizeof(float) * nn);
    if (st != DFACTO_OK) {
      cleanup();
      return st;
    }
    if (n == 0) {
      M.nfib = 0;
      st = dalloc(h, reinterpret_cast<void**>(&M.nz_ptr), sizeof(int64_t));
      if (st == DFACTO_OK) st = dalloc(h, reinterpret_cast<void**>(&M.fiber_idx), sizeof(int32_t));
      if (st == DFACTO_OK) st = dalloc(h, reinterpret_cast<void**>(&M.fiber_row), sizeof(int32_t));
      if (st == DFACTO_OK) st = dalloc(h, reinterpret_cast<void**>(&M.end_bits), sizeof(uint32_t));
      if (st != DFACTO_OK) return st;
      DF_CUDA(h, cudaMemsetAsync(M.nz_ptr, 0, sizeof(int64_t), s));
      DF_CUDA(h, cudaMemsetAsync(M.fiber_ptr, 0, sizeof(int64_t) * (size_t)(M.dim_o + 1), s));
      continue;
    }
    bool alt = false, alt2 = false;
    // The sort runs on (kin, vin) with (kalt, valt) as its ping-pong partner.
    uint64_t* kin = k0;
    uint32_t* vin = v0;
    if (chained) {
      kin = prev_k;
      vin = prev_v;
    }
    uint64_t* kalt = (kin == k0) ? k1 : k0;
    uint32_t* valt = (vin == v0) ? v1 : v0;
    if (narrow && !chained) {
      make_keys64_val<<<grid_for(n), 256, 0, s>>>(d_idx, d_val, n, M.o, M.f, M.in, bf, bi, kin, vin);
      DF_COUNT();
      e = cudaGetLastError();
      if (e == cudaSuccess) e = radix_sort(kin, vin, kalt, valt, n, 0, bo + bf + bi, s, &alt, sort_cnt);
    } else if (narrow) {
      // the previous order ascends in this mode's (f, in): sort the o bits
      rotate_keys<<<grid_for(n), 256, 0, s>>>(kin, n, prev_bo, prev_bf, prev_bi);
      DF_COUNT();
      e = cudaGetLastError();
      if (e == cudaSuccess) e = radix_sort(kin, vin, kalt, valt, n, bf + bi, bo + bf + bi, s, &alt, sort_cnt);
    } else if (chained) {
      // previous payload = COO positions in an order ascending in this mode's
      // (f, in): key (o, f), sort the o bits
      make_keys_chain<<<grid_for(n), 256, 0, s>>>(d_idx, n, M.o, M.f, bf, vin, kalt, valt);
      DF_COUNT();
      e = cudaGetLastError();
      std::swap(kin, kalt);
      std::swap(vin, valt);
      if (e == cudaSuccess) e = radix_sort(kin, vin, kalt, valt, n, bf, bo + bf, s, &alt, sort_cnt);
    } else {
      make_keys_in<<<grid_for(n), 256, 0, s>>>(d_idx, n, M.in, kin, vin); DF_COUNT();
      e = cudaGetLastError();
      if (e == cudaSuccess) e = radix_sort(kin, vin, kalt, valt, n, 0, bi, s, &alt, sort_cnt);
      if (alt) {
        std::swap(kin, kalt);
        std::swap(vin, valt);
      }
      if (e == cudaSuccess) {
        make_keys_of<<<grid_for(n), 256, 0, s>>>(d_idx, n, M.o, M.f, bf, vin, kin); DF_COUNT();
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = radix_sort(kin, vin, kalt, valt, n, 0, bo + bf, s, &alt2, sort_cnt);
      alt = alt2;
    }
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(h, e, "radix sort");
    }
    if (alt) {
      std::swap(kin, kalt);
      std::swap(vin, valt);
    }
    const uint64_t* key = kin;
    const uint32_t* perm = vin;
    prev_k = kin;
    prev_v = vin;
    prev_bo = bo;
    prev_bf = bf;
    prev_bi = bi;
    st = dalloc(h, reinterpret_cast<void**>(&M.end_bits), sizeof(uint32_t) * (size_t)((n + 31) / 32));
    if (st != DFACTO_OK) {
      cleanup();
      return st;
    }
    segment_flags<<<grid_for(n), 256, 0, s>>>(key, perm, n, bi, wide, narrow, d_idx, M.in, d_val,
                                             head, M.nz_idx, M.nz_val, M.end_bits,
                                             h->flags + kFlagDup); DF_COUNT();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan_i32(head, fid, n, s);
    int32_t last[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[0], fid + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], head + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(h, e, "fiber segmentation");
    }
    M.nfib = (int64_t)last[0] + last[1];
    st = dalloc(h, reinterpret_cast<void**>(&M.nz_ptr), sizeof(int64_t) * (size_t)(M.nfib + 1));
    if (st == DFACTO_OK)
      st = dalloc(h, reinterpret_cast<void**>(&M.fiber_idx), sizeof(int32_t) * (size_t)M.nfib);
    if (st == DFACTO_OK)
      st = dalloc(h, reinterpret_cast<void**>(&M.fiber_row), sizeof(int32_t) * (size_t)M.nfib);
    if (st != DFACTO_OK) {
      cleanup();
      return st;
    }
    scatter_fibers<<<grid_for(n), 256, 0, s>>>(key, perm, n, bf, bi, wide, head, fid, M.nz_ptr,
                                              M.fiber_idx, M.fiber_row, M.nfib); DF_COUNT();
    row_pointers<<<grid_for(M.dim_o + 1), 256, 0, s>>>(M.fiber_row, M.nfib, M.dim_o, M.fiber_ptr); DF_COUNT();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(h, e, "fiber arrays");
    }
  }
  cleanup();
  DF_CUDA(h, cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int32_t) * kNumFlags,
                             cudaMemcpyDeviceToHost, s));
  DF_CUDA(h, cudaStreamSynchronize(s));
  if (h->host_flags[kFlagDup]) return fail(h, DFACTO_EDUP, "two nonzeros share a coordinate");
  return DFACTO_OK;
}

}  // namespace dfacto
