// mttkrp.cuh -- the fused two-SpMV MTTKRP of DFacTo (Algorithm 1), batched
// over all R columns.
//
// For mode n and every output row o:
//   N[o, :] = sum over fibers q = (o, f) of  F_f[f, :] (*) v_q,
//   v_q     = sum over nonzeros (in, x) of fiber q of  x * F_in[in, :],
// where v_q is row q of value(M^r) for all r at once (first SpMV, (Xhat)^T b_r)
// and the outer sum is the second SpMV, M^r c_r.  v_q never leaves registers.
//
// Work split (GB300): the nonzero stream is cut into segments of `seg`
// nonzeros, independent of row and fiber boundaries, so heavy (power-law)
// rows and fibers are spread over many lanes.  A group of G lanes walks one
// segment; each lane owns VEC consecutive columns and gathers them with one
// vector load per factor row.  The group's lanes fetch G upcoming (in, x)
// pairs with one coalesced load and pass them around by shuffles.  Splitting
// inside a fiber is exact because the second SpMV is linear in v.
//
// A row finished inside a segment is stored directly.  A segment's first and
// last rows may continue into neighbouring segments: their partial sums go to
// shared memory and are merged in segment order, first inside each warp, then
// across the CTA's warps.  Rows that continue beyond the CTA's range are left
// as per-CTA carries that mttkrp_fixup adds up in CTA order.  Every sum
// therefore has a fixed order: results are bitwise reproducible.
#pragma once

#include "device.cuh"
#include "internal.h"

namespace dfacto {

struct MttkrpParams {
  const int64_t* fiber_ptr;
  const int32_t* fiber_idx;
  const int32_t* fiber_row;
  const int64_t* nz_ptr;
  const int32_t* nz_idx;
  const float* nz_val;
  const int32_t* seg_fib;
  const uint32_t* end_bits;  // bit p set iff nonzero p ends its fiber (walk2)
  const void* Fin;
  const void* Ff;
  float* out;
  float* carry;       // [ncta][2][R]
  int32_t* carry_row; // [ncta][2]
  int64_t nnz;
  int64_t nfib;
  int64_t dim_o;
  int R;
  int seg;
};

constexpr int kMaxColsPerLane = 4;  // R <= 128 in the CTA merge (lane-strided columns)

// Merge a sequence of (row, partial) entries into runs of equal rows, in order.
// flush(row, vals, is_first, is_last) is called once per run; is_first/is_last
// say whether the run contains the first/last valid entry.  Executed by one
// full warp; lane handles columns lane, lane+32, ...
template <typename Flush>
__device__ __forceinline__ void merge_runs(const int32_t* rows, const float* vals, int count, int R,
                                           int lane, Flush&& flush) {
  int run_row = -1;
  bool run_first = true;
  float run[kMaxColsPerLane];
#pragma unroll
  for (int k = 0; k < kMaxColsPerLane; ++k) run[k] = 0.f;
  for (int e = 0; e < count; ++e) {
    const int row = rows[e];
    if (row < 0) continue;
    if (row != run_row) {
      if (run_row >= 0) {
        flush(run_row, run, run_first, false);
        run_first = false;
      }
      run_row = row;
#pragma unroll
      for (int k = 0; k < kMaxColsPerLane; ++k) run[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kMaxColsPerLane; ++k) {
      const int col = lane + 32 * k;
      if (col < R) run[k] += vals[(size_t)e * R + col];
    }
  }
  if (run_row >= 0) flush(run_row, run, run_first, true);
}

// Merge the segment slots of one CTA (s_row/s_val: [SEGS * 2] entries), first
// inside each warp, then across warps; store complete rows and leave the CTA's
// partial first/last rows as carries.  Called by all threads after the walk.
template <int SEGS, int NG>
__device__ __forceinline__ void mttkrp_merge_cta(const MttkrpParams& a, int cta, int32_t* s_row,
                                                 float* s_val, int32_t* w_row, float* w_val, int lane,
                                                 int warp, int64_t cta_p0, int64_t cta_p1) {
  const int R = a.R;
  // Level 1: each warp merges its NG segments.  Runs strictly inside the
  // warp's range are complete rows.
  {
    if (lane == 0) { w_row[warp * 2] = -1; w_row[warp * 2 + 1] = -1; }
    __syncwarp();
    merge_runs(s_row + warp * NG * 2, s_val + (size_t)warp * NG * 2 * R, NG * 2, R, lane,
               [&](int row, const float (&run)[kMaxColsPerLane], bool first, bool last) {
                 const int k = first ? 0 : (last ? 1 : -1);
                 if (k < 0) {
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) a.out[(int64_t)row * R + col] = run[q];
                   }
                 } else {
                   if (lane == 0) w_row[warp * 2 + k] = row;
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) w_val[(size_t)(warp * 2 + k) * R + col] = run[q];
                   }
                 }
               });
  }
  __syncthreads();

  // Level 2: warp 0 merges the warps.  The CTA's first run may have started in
  // an earlier CTA, its last run may continue in a later one.
  if (warp == 0) {
    int first_row = -1, last_row = -1;
    for (int e = 0; e < kWalkWarps * 2; ++e) {
      const int r = w_row[e];
      if (r >= 0) { if (first_row < 0) first_row = r; last_row = r; }
    }
    bool first_partial = false, last_partial = false;
    if (first_row >= 0) {
      // rows of the first and last run: where do they begin and end?
      const int64_t fb = a.fiber_ptr[first_row];
      const int64_t le = a.fiber_ptr[last_row + 1];
      first_partial = a.nz_ptr[fb] < cta_p0;
      last_partial = a.nz_ptr[le] > cta_p1;
    }
    if (lane == 0) {
      a.carry_row[cta * 2] = -1;
      a.carry_row[cta * 2 + 1] = -1;
    }
    __syncwarp();
    merge_runs(w_row, w_val, kWalkWarps * 2, R, lane,
               [&](int row, const float (&run)[kMaxColsPerLane], bool first, bool last) {
                 const bool partial = (first && first_partial) || (last && last_partial);
                 if (!partial) {
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) a.out[(int64_t)row * R + col] = run[q];
                   }
                 } else {
                   const int k = (first && first_partial) ? 0 : 1;
                   if (lane == 0) a.carry_row[cta * 2 + k] = row;
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) a.carry[((int64_t)cta * 2 + k) * R + col] = run[q];
                   }
                 }
               });
  }
}

// Row of fiber q from row(M^r) alone: the largest r < dim_o with
// fiber_ptr[r] <= q (empty rows have fiber_ptr[r] == fiber_ptr[r + 1]).
__device__ __forceinline__ int row_of_fiber(const int64_t* fiber_ptr, int64_t dim_o, int64_t q) {
  int64_t lo = 0, hi = dim_o - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (fiber_ptr[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return (int)lo;
}

// Row of fiber q given the row r0 of an earlier fiber (rows ascend with q).
__device__ __forceinline__ int row_after(const int64_t* fiber_ptr, int r0, int64_t q) {
  int r = r0;
  while (__ldg(fiber_ptr + r + 1) <= q) ++r;
  return r;
}

// kRowsFromPtr: take each fiber's row from fiber_ptr instead of the fiber_row
// array (for callers that pass only the CSR arrays of dfacto_csr_view).
template <typename T, int VEC, int G, bool kRowsFromPtr = false>
__global__ void __launch_bounds__(kWalkWarps * 32) mttkrp_walk(const MttkrpParams a) {
  constexpr int NG = 32 / G;
  constexpr int SEGS = kWalkWarps * NG;
  extern __shared__ float smem[];
  float* s_val = smem;                          // [SEGS * 2][R]
  float* w_val = smem + (size_t)SEGS * 2 * a.R; // [kWalkWarps * 2][R]
  __shared__ int32_t s_row[SEGS * 2];
  __shared__ int32_t w_row[kWalkWarps * 2];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / G, c = lane % G;
  const int gbase = g * G;
  const int col0 = c * VEC;
  const bool colok = col0 < a.R;
  const int sl = warp * NG + g;  // segment index inside the CTA
  const int64_t cta_p0 = (int64_t)blockIdx.x * SEGS * a.seg;
  const int64_t cta_p1 = min(cta_p0 + (int64_t)SEGS * a.seg, a.nnz);
  const int64_t p0 = cta_p0 + (int64_t)sl * a.seg;
  const int64_t p1 = min(p0 + a.seg, a.nnz);
  const bool active = p0 < a.nnz;
  const T* __restrict__ Fin = static_cast<const T*>(a.Fin);
  const T* __restrict__ Ff = static_cast<const T*>(a.Ff);
  const int R = a.R;

  float v[VEC], acc[VEC], ffc[VEC];
#pragma unroll
  for (int k = 0; k < VEC; ++k) { v[k] = 0.f; acc[k] = 0.f; ffc[k] = 0.f; }

  int64_t fib = 0, fend = 0, fend_next = 0;
  int row_cur = -1, row_next = -1, f_next = 0;
  if (active) {
    fib = a.seg_fib[(int64_t)blockIdx.x * SEGS + sl];
    fend = min(a.nz_ptr[fib + 1], p1);
    if constexpr (kRowsFromPtr) row_cur = row_of_fiber(a.fiber_ptr, a.dim_o, fib);
    else row_cur = a.fiber_row[fib];
    if (colok) VecIO<T, VEC>::load(Ff + (int64_t)a.fiber_idx[fib] * R + col0, ffc);
    if (fib + 1 < a.nfib) {
      fend_next = a.nz_ptr[fib + 2];
      f_next = a.fiber_idx[fib + 1];
      if constexpr (kRowsFromPtr) row_next = row_after(a.fiber_ptr, row_cur, fib + 1);
      else row_next = a.fiber_row[fib + 1];
    }
  }

  auto put_slot = [&](int k, int row, const float (&val)[VEC]) {
    if (c == 0) s_row[sl * 2 + k] = row;
    if (colok) {
#pragma unroll
      for (int q = 0; q < VEC; ++q) s_val[(size_t)(sl * 2 + k) * R + col0 + q] = val[q];
    }
  };
  bool head_open = true;

  for (int64_t base = p0; base < p0 + a.seg; base += G) {
    const int64_t pl = base + c;
    const bool okl = pl < p1;
    const int my_in = okl ? __ldg(a.nz_idx + pl) : 0;
    const float my_x = okl ? __ldg(a.nz_val + pl) : 0.f;
    // Row gathers are issued U at a time before any is used (memory-level
    // parallelism), U * VEC <= 32 registers.
    constexpr int U = (G < 32 / VEC) ? G : (32 / VEC);
#pragma unroll
    for (int u0 = 0; u0 < G; u0 += U) {
      float fin[U][VEC];
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const int in = __shfl_sync(kFull, my_in, gbase + u0 + uu);
        if (colok && base + u0 + uu < p1) {
          VecIO<T, VEC>::load(Fin + (int64_t)in * R + col0, fin[uu]);
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) fin[uu][q] = 0.f;
        }
      }
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const float x = __shfl_sync(kFull, my_x, gbase + u0 + uu);
        const int64_t p = base + u0 + uu;
        if (p < p1) {
#pragma unroll
          for (int q = 0; q < VEC; ++q) v[q] = fmaf(x, fin[uu][q], v[q]);
          if (p + 1 == fend) {  // the fiber (or its part in this segment) ends
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
              acc[q] = fmaf(v[q], ffc[q], acc[q]);
              v[q] = 0.f;
            }
            if (p + 1 < p1) {  // next fiber starts inside this segment
              ++fib;
              fend = min(fend_next, p1);
              if (row_next != row_cur) {
                if (head_open) {
                  put_slot(0, row_cur, acc);
                  head_open = false;
                } else if (colok) {
                  VecIO<float, VEC>::store(a.out + (int64_t)row_cur * R + col0, acc);
                }
#pragma unroll
                for (int q = 0; q < VEC; ++q) acc[q] = 0.f;
                row_cur = row_next;
              }
              if (colok) VecIO<T, VEC>::load(Ff + (int64_t)f_next * R + col0, ffc);
              if (fib + 1 < a.nfib) {
                fend_next = __ldg(a.nz_ptr + fib + 2);
                f_next = __ldg(a.fiber_idx + fib + 1);
                if constexpr (kRowsFromPtr) row_next = row_after(a.fiber_ptr, row_cur, fib + 1);
                else row_next = __ldg(a.fiber_row + fib + 1);
              }
            }
          }
        }
      }
    }
  }

  // Segment slots: 0 = head row partial, 1 = tail row partial (-1 = none).
  if (!active) {
    if (c == 0) { s_row[sl * 2] = -1; s_row[sl * 2 + 1] = -1; }
  } else if (head_open) {
    put_slot(0, row_cur, acc);
    if (c == 0) s_row[sl * 2 + 1] = -1;
  } else {
    put_slot(1, row_cur, acc);
  }
  __syncthreads();

  // Level 1: each warp merges its NG segments.  Runs strictly inside the
  // warp's range are complete rows.
  {
    if (lane == 0) { w_row[warp * 2] = -1; w_row[warp * 2 + 1] = -1; }
    __syncwarp();
    merge_runs(s_row + warp * NG * 2, s_val + (size_t)warp * NG * 2 * R, NG * 2, R, lane,
               [&](int row, const float (&run)[kMaxColsPerLane], bool first, bool last) {
                 const int k = first ? 0 : (last ? 1 : -1);
                 if (k < 0) {
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) a.out[(int64_t)row * R + col] = run[q];
                   }
                 } else {
                   if (lane == 0) w_row[warp * 2 + k] = row;
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) w_val[(size_t)(warp * 2 + k) * R + col] = run[q];
                   }
                 }
               });
  }
  __syncthreads();

  // Level 2: warp 0 merges the warps.  The CTA's first run may have started in
  // an earlier CTA, its last run may continue in a later one.
  if (warp == 0) {
    int first_row = -1, last_row = -1;
    for (int e = 0; e < kWalkWarps * 2; ++e) {
      const int r = w_row[e];
      if (r >= 0) { if (first_row < 0) first_row = r; last_row = r; }
    }
    bool first_partial = false, last_partial = false;
    if (first_row >= 0) {
      // rows of the first and last run: where do they begin and end?
      const int64_t fb = a.fiber_ptr[first_row];
      const int64_t le = a.fiber_ptr[last_row + 1];
      first_partial = a.nz_ptr[fb] < cta_p0;
      last_partial = a.nz_ptr[le] > cta_p1;
    }
    if (lane == 0) {
      a.carry_row[blockIdx.x * 2] = -1;
      a.carry_row[blockIdx.x * 2 + 1] = -1;
    }
    __syncwarp();
    merge_runs(w_row, w_val, kWalkWarps * 2, R, lane,
               [&](int row, const float (&run)[kMaxColsPerLane], bool first, bool last) {
                 const bool partial = (first && first_partial) || (last && last_partial);
                 if (!partial) {
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) a.out[(int64_t)row * R + col] = run[q];
                   }
                 } else {
                   const int k = (first && first_partial) ? 0 : 1;
                   if (lane == 0) a.carry_row[blockIdx.x * 2 + k] = row;
#pragma unroll
                   for (int q = 0; q < kMaxColsPerLane; ++q) {
                     const int col = lane + 32 * q;
                     if (col < R) a.carry[((int64_t)blockIdx.x * 2 + k) * R + col] = run[q];
                   }
                 }
               });
  }
}

// ---------------------------------------------------------------------------
// mttkrp_walk2: the same walk with fiber ends taken from a bitmask and fibers
// closed in batches.  Per sub-batch of U steps a group
//   (1) gathers the U F_in rows,
//   (2) accumulates v over the U nonzeros; where a bit of end_bits marks the
//       last nonzero of a fiber, v is parked in a per-lane shared-memory slot
//       and restarted (no branch on fiber metadata in this loop),
//   (3) closes the k <= U fibers that ended: loads their f and row, issues all
//       k F_f gathers at once, then folds v_j (*) F_f[f_j] into the row sums.
// The merge of rows shared between segments, warps and CTAs is the one of
// mttkrp_walk.
// ---------------------------------------------------------------------------
// A thread's VEC parked floats in shared memory.  Slot k of thread tid holds
// them as VEC/4 float4 chunks, chunk q at ((k * VEC/4 + q) * NT + tid) * 4, so
// that a warp's accesses to one chunk are consecutive 16-byte words (no bank
// conflicts); VEC < 4 keeps the VEC floats together at (k * NT + tid) * VEC.
template <int VEC, int NT>
__device__ __forceinline__ float* park_slot(float* vb, int k, int tid) {
  if constexpr (VEC % 4 == 0) return vb + ((size_t)k * (VEC / 4) * NT + tid) * 4;
  else return vb + ((size_t)k * NT + tid) * VEC;
}
template <int VEC, int NT>
__device__ __forceinline__ void smem_st(float* p, const float (&v)[VEC]) {
  if constexpr (VEC % 4 == 0) {
#pragma unroll
    for (int e = 0; e < VEC; e += 4)
      *reinterpret_cast<float4*>(p + (size_t)(e / 4) * NT * 4) =
          make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) p[e] = v[e];
  }
}
template <int VEC, int NT>
__device__ __forceinline__ void smem_ld(const float* p, float (&v)[VEC]) {
  if constexpr (VEC % 4 == 0) {
#pragma unroll
    for (int e = 0; e < VEC; e += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + (size_t)(e / 4) * NT * 4);
      v[e] = t.x; v[e + 1] = t.y; v[e + 2] = t.z; v[e + 3] = t.w;
    }
  } else if constexpr (VEC == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) v[e] = p[e];
  }
}

// Fibers closed per round of the fiber-closing pass (fewer predicated-off
// slots when fibers are long; a sub-batch closes at most U).
constexpr int kCloseChunk = 4;

// Gathers in flight per lane of the walk shape (VEC, G): at most 16 gathered
// values (U * VEC <= 16); more leave the kernel short of registers (spills) at
// the budget of Walk2Shape.
__host__ __device__ constexpr int walk2_gathers(int vec, int G) { return G < 16 / vec ? G : 16 / vec; }
// Per-lane shared-memory slots for parked fiber sums.
__host__ __device__ constexpr int walk2_park_slots(int vec, int G) { return walk2_gathers(vec, G); }
// Dynamic shared memory of the walk at rank R: segment and warp partial rows
// for the merge, then the park slots.
inline size_t walk2_smem_bytes(int vec, int G, int R) {
  return sizeof(float) * ((size_t)(2 * kWalkWarps * (32 / G) + 2 * kWalkWarps) * R +
                          (size_t)kWalkWarps * 32 * walk2_park_slots(vec, G) * vec);
}

template <typename T, int VEC, int G>
struct Walk2Shape {
  static constexpr int NG = 32 / G;
  static constexpr int SEGS = kWalkWarps * NG;
  static constexpr int U = walk2_gathers(VEC, G);
  // Resident CTAs per SM the register budget is cut for: the kernel is bound by
  // the latency of its gathers and its L1 traffic, so occupancy pays more than
  // a few registers: 80 registers (3 CTAs) for eight-column lanes, 64 (4 CTAs)
  // for narrower ones.
  static constexpr int MIN_BLOCKS = VEC >= 8 ? 3 : 4;
  static size_t smem_bytes(int R) { return walk2_smem_bytes(VEC, G, R); }
};

// The walk of CTA `cta` of one MTTKRP (shared by the single-tensor kernel and
// the batched one).  smem holds Walk2Shape::smem_bytes(R) bytes; s_row and
// w_row hold SEGS * 2 and kWalkWarps * 2 entries.
template <typename T, int VEC, int G>
__device__ __forceinline__ void walk2_cta(const MttkrpParams& a, int cta, float* smem,
                                          int32_t* s_row, int32_t* w_row) {
  using Shape = Walk2Shape<T, VEC, G>;
  constexpr int NG = Shape::NG, SEGS = Shape::SEGS, U = Shape::U;
  constexpr int NT = kWalkWarps * 32;
  const int R = a.R;
  float* s_val = smem;                           // [SEGS * 2][R]
  float* w_val = smem + (size_t)SEGS * 2 * R;    // [kWalkWarps * 2][R]
  float* vb = w_val + (size_t)kWalkWarps * 2 * R;  // U slots of NT x VEC parked fiber sums

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane / G, c = lane % G;
  const int gbase = g * G;
  const int col0 = c * VEC;
  const bool colok = col0 < R;
  const int sl = warp * NG + g;
  // Positions fit in int: nnz <= kMaxNnz and seg <= kMaxSeg keep p0 + seg + G
  // below 2^31 (the bounds are formed in 64 bits first).
  const int nnz = (int)a.nnz;
  const int cta_p0 = (int)min((int64_t)cta * SEGS * a.seg, a.nnz);
  const int cta_p1 = (int)min((int64_t)cta_p0 + (int64_t)SEGS * a.seg, a.nnz);
  const int p0 = (int)min((int64_t)cta_p0 + (int64_t)sl * a.seg, a.nnz);
  const int p1 = min(p0 + a.seg, nnz);
  const bool active = p0 < nnz;
  const T* __restrict__ Fin = static_cast<const T*>(a.Fin);
  const T* __restrict__ Ff = static_cast<const T*>(a.Ff);

  float v[VEC], acc[VEC];
#pragma unroll
  for (int k = 0; k < VEC; ++k) { v[k] = 0.f; acc[k] = 0.f; }
  int q = 0;          // fiber holding the current nonzero
  int row_cur = -1;
  if (active) {
    q = a.seg_fib[(int64_t)cta * SEGS + sl];
    row_cur = a.fiber_row[q];
  }
  bool head_open = true;
  auto put_slot = [&](int k, int row, const float (&val)[VEC]) {
    if (c == 0) s_row[sl * 2 + k] = row;
    if (colok) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) s_val[(size_t)(sl * 2 + k) * R + col0 + e] = val[e];
    }
  };
  // Fold w = vv (*) ff of a fiber of row r into the row sums (emitting the
  // previous row when r starts a new one).
  auto fold = [&](int r, const float (&vv)[VEC], const float (&ff)[VEC]) {
    if (r != row_cur) {
      if (head_open) {
        put_slot(0, row_cur, acc);
        head_open = false;
      } else if (colok) {
        VecIO<float, VEC>::store(a.out + (int64_t)row_cur * R + col0, acc);
      }
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = 0.f;
      row_cur = r;
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = fmaf(vv[e], ff[e], acc[e]);
  };

  for (int base = p0; base < p0 + a.seg; base += G) {
    const int pl = base + c;
    const bool okl = pl < p1;
    const int my_in = okl ? __ldg(a.nz_idx + pl) : 0;
    const float my_x = okl ? __ldg(a.nz_val + pl) : 0.f;
    // end bits of the batch's G positions (base is a multiple of G, G | 32);
    // a batch starting at or past p1 has none, and its word may lie past the
    // end of end_bits ((nnz + 31) / 32 words) in the last segment
    const uint32_t ebits = (active && base < p1) ? (__ldg(a.end_bits + (base >> 5)) >> (base & 31)) : 0u;
#pragma unroll
    for (int u0 = 0; u0 < G; u0 += U) {
      float fin[U][VEC];
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const int in = __shfl_sync(kFull, my_in, gbase + u0 + uu);
        if (colok && base + u0 + uu < p1) {
          VecIO<T, VEC>::load(Fin + (int64_t)in * R + col0, fin[uu]);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) fin[uu][e] = 0.f;
        }
      }
      int k = 0;  // fibers closed in this sub-batch
#pragma unroll
      for (int uu = 0; uu < U; ++uu) {
        const float x = __shfl_sync(kFull, my_x, gbase + u0 + uu);
        const int p = base + u0 + uu;
#pragma unroll
        for (int e = 0; e < VEC; ++e) v[e] = fmaf(x, fin[uu][e], v[e]);
        const bool end = p < p1 && ((ebits >> (u0 + uu)) & 1u);
        if (end) {
          smem_st<VEC, NT>(park_slot<VEC, NT>(vb, k, tid), v);
#pragma unroll
          for (int e = 0; e < VEC; ++e) v[e] = 0.f;
        }
        k += end ? 1 : 0;
      }
      // Close the k fibers q .. q + k - 1, CC at a time (the F_f gathers of a
      // round are issued together).
      constexpr int CC = kCloseChunk < U ? kCloseChunk : U;
      for (int j0 = 0; j0 < k; j0 += CC) {
        int fj[CC], rj[CC];
#pragma unroll
        for (int j = 0; j < CC; ++j) {
          fj[j] = 0;
          rj[j] = row_cur;
          if (j0 + j < k) {
            fj[j] = __ldg(a.fiber_idx + q + j0 + j);
            rj[j] = __ldg(a.fiber_row + q + j0 + j);
          }
        }
        float ff[CC][VEC];
#pragma unroll
        for (int j = 0; j < CC; ++j) {
          if (j0 + j < k && colok) {
            VecIO<T, VEC>::load(Ff + (int64_t)fj[j] * R + col0, ff[j]);
          } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) ff[j][e] = 0.f;
          }
        }
#pragma unroll
        for (int j = 0; j < CC; ++j) {
          if (j0 + j < k) {
            float vv[VEC];
            smem_ld<VEC, NT>(park_slot<VEC, NT>(vb, j0 + j, tid), vv);
            fold(rj[j], vv, ff[j]);
          }
        }
      }
      q += k;
    }
  }
  // The fiber open at the segment end (if its last nonzero lies beyond p1).
  if (active && !((__ldg(a.end_bits + ((p1 - 1) >> 5)) >> ((p1 - 1) & 31)) & 1u)) {
    const int f = __ldg(a.fiber_idx + q);
    const int r = __ldg(a.fiber_row + q);
    float ff[VEC];
    if (colok) VecIO<T, VEC>::load(Ff + (int64_t)f * R + col0, ff);
    else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) ff[e] = 0.f;
    }
    fold(r, v, ff);
  }

  // Segment slots: 0 = head row partial, 1 = tail row partial (-1 = none).
  if (!active) {
    if (c == 0) { s_row[sl * 2] = -1; s_row[sl * 2 + 1] = -1; }
  } else if (head_open) {
    put_slot(0, row_cur, acc);
    if (c == 0) s_row[sl * 2 + 1] = -1;
  } else {
    put_slot(1, row_cur, acc);
  }
  __syncthreads();
  mttkrp_merge_cta<SEGS, NG>(a, cta, s_row, s_val, w_row, w_val, lane, warp, cta_p0, cta_p1);
}

template <typename T, int VEC, int G>
__global__ void __launch_bounds__(kWalkWarps * 32, (Walk2Shape<T, VEC, G>::MIN_BLOCKS))
    mttkrp_walk2(const MttkrpParams a) {
  using Shape = Walk2Shape<T, VEC, G>;
  extern __shared__ __align__(16) float smem[];
  __shared__ int32_t s_row[Shape::SEGS * 2];
  __shared__ int32_t w_row[kWalkWarps * 2];
  walk2_cta<T, VEC, G>(a, blockIdx.x, smem, s_row, w_row);
}

// ---------------------------------------------------------------------------
// Batched MTTKRP: the jobs of a batch that share (R, factor type) form one
// block-diagonal tensor (a "rank class": indices offset per job, factors
// pooled), so a class is one walk.  mttkrp_walk2_multi walks up to
// kMaxClasses classes in one persistent launch: block b takes the virtual CTAs
// b, b + gridDim.x, ... of the concatenated class ranges, and each class runs
// the walk shape its autotuned (VEC, G) selects.  The per-class parameters stay
// in the kernel's parameter space (__grid_constant__).
// ---------------------------------------------------------------------------
constexpr int kMaxClasses = 4;

// Walk shapes compiled into the batched kernel: (VEC, G) by id.
constexpr int kMultiShapes = 6;
__host__ __device__ constexpr int multi_shape_vec(int id) { return id < 3 ? 4 : 8; }
__host__ __device__ constexpr int multi_shape_G(int id) {
  return id == 0 ? 2 : id == 1 ? 4 : id == 2 ? 8 : id == 3 ? 1 : id == 4 ? 2 : 4;
}
inline int multi_shape_id(int vec, int G) {
  for (int i = 0; i < kMultiShapes; ++i)
    if (multi_shape_vec(i) == vec && multi_shape_G(i) == G) return i;
  return -1;
}
constexpr int kMultiMaxSegs = kWalkWarps * 32;  // SEGS of the G = 1 shape

struct MultiWalkParams {
  MttkrpParams p[kMaxClasses];
  int shape[kMaxClasses];          // multi shape id of each class
  int cta_begin[kMaxClasses + 1];  // virtual CTAs [cta_begin[c], cta_begin[c + 1]) walk class c
  int nclass;
};

template <typename T>
__global__ void __launch_bounds__(kWalkWarps * 32, 3)
    mttkrp_walk2_multi(const __grid_constant__ MultiWalkParams mp) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int32_t s_row[kMultiMaxSegs * 2];
  __shared__ int32_t w_row[kWalkWarps * 2];
  const int total = mp.cta_begin[mp.nclass];
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
      if (k < mp.nclass && v >= mp.cta_begin[k]) c = k;
    const MttkrpParams& a = mp.p[c];
    const int cta = v - mp.cta_begin[c];
    __syncthreads();  // the previous virtual CTA's merge is done with shared memory
    switch (mp.shape[c]) {
      case 0: walk2_cta<T, multi_shape_vec(0), multi_shape_G(0)>(a, cta, smem, s_row, w_row); break;
      case 1: walk2_cta<T, multi_shape_vec(1), multi_shape_G(1)>(a, cta, smem, s_row, w_row); break;
      case 2: walk2_cta<T, multi_shape_vec(2), multi_shape_G(2)>(a, cta, smem, s_row, w_row); break;
      case 3: walk2_cta<T, multi_shape_vec(3), multi_shape_G(3)>(a, cta, smem, s_row, w_row); break;
      case 4: walk2_cta<T, multi_shape_vec(4), multi_shape_G(4)>(a, cta, smem, s_row, w_row); break;
      default: walk2_cta<T, multi_shape_vec(5), multi_shape_G(5)>(a, cta, smem, s_row, w_row); break;
    }
  }
}

// Launch the batched walk (defined in the batch instantiation units).
template <typename T>
cudaError_t launch_walk2_multi(const MultiWalkParams& mp, size_t smem, int grid, cudaStream_t s);

// Launchers of the carry fix-up (mttkrp.cu) and of the segment-start search
// (build.cu), shared with the allocation-free entry point.
cudaError_t launch_mttkrp_fixup(const int32_t* carry_row, const float* carry,
                                const int64_t* fiber_ptr, const int64_t* nz_ptr, float* out, int R,
                                int64_t P, int64_t ncta, int64_t dim_o, int32_t* bad,
                                cudaStream_t s);
cudaError_t launch_segment_starts(const int64_t* nz_ptr, int64_t nfib, int64_t nseg, int64_t seg,
                                  int32_t* seg_fib, cudaStream_t s);
// Zero bits[(nnz + 31) / 32] and set the bit of the last nonzero of every fiber.
cudaError_t launch_fiber_end_bits(const int64_t* nz_ptr, int64_t nfib, int64_t nnz, uint32_t* bits,
                                  cudaStream_t s);

// Launch one walk configuration (defined in the instantiation units).
template <typename T>
cudaError_t launch_walk(int vec, int G, const MttkrpParams& a, int64_t ncta, size_t smem,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_walk2(int vec, int G, const MttkrpParams& a, int64_t ncta, cudaStream_t s);

}  // namespace dfacto
