// mttkrp_stage.cu -- the MTTKRP walk with factor rows staged in shared memory
// by bulk asynchronous copies (walk = 3; FP32 factors, R % 4 == 0, R <= 32).
//
// Same sums as mttkrp_walk2 with one lane group of 32 lanes per segment (lane c
// owns column c): v (row q of value(M^r), all r) accumulates x * F_in[in, :]
// over the nonzeros of fiber q in order, and each closed fiber folds
// v (*) F_f[f, :] into its row (Sec. 3, Algorithm 1; Lemma 2).  What differs is
// how the gathered rows arrive: every warp walks its segment in batches of 32
// nonzeros, and for each batch lane j issues a bulk copy of F_in[in_j, :] into
// the warp's shared-memory ring (and, where nonzero j ends a fiber, a copy of
// F_f[f, :]), all completing on one mbarrier of the ring slot.  Two batches are
// in flight per warp while the previous one is folded, so the number of rows
// in flight no longer costs registers, and the per-nonzero bookkeeping (end
// bit, x, fiber row) is uniform across the warp.
//
// Every mbarrier wait is bounded: after kWaitLimit polls the warp records a
// timeout in a device flag (read by the host as DFACTO_ETIMEOUT) and stops
// issuing and folding; CTAs that start later see the flag and leave at once.
// Measured on the 50M-nonzero power-law tensor at R = 32 this walk is about
// six times slower than mttkrp_walk2 (one bulk copy per 128-byte row is far
// slower than register gathers served by L1/L2), so it is an option only.
#include "mttkrp.cuh"

namespace dfacto {
namespace {

constexpr int kStageBatch = 32;               // nonzeros per batch (one per lane)
constexpr uint32_t kWaitLimit = 1u << 20;     // mbarrier polls before giving up (~40 ms)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// One arrival that also announces `bytes` of copies completing on the barrier.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Non-blocking test of whether the phase of `bar` with the given parity is done.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase of `bar` with the given parity (polls, then polls
// with a short sleep); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (it >= 64) __nanosleep(32);
  }
  return false;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// One ring slot of a warp: the batch's F_in rows then its F_f rows.
struct StageSlot {
  float x = 0.f;        // lane j: value of nonzero j of the batch
  int32_t frow = 0;     // lane j (ends only): output row of the fiber ending at j
  uint32_t ends = 0;    // bit j: nonzero j ends its fiber
  int32_t n = 0;        // valid nonzeros in the batch
};

__global__ void __launch_bounds__(kWalkWarps * 32, 1)
    mttkrp_stage(const MttkrpParams a, int32_t* __restrict__ timeout_flag) {
  constexpr int SEGS = kWalkWarps;  // one segment per warp
  constexpr int NT = kWalkWarps * 32;
  extern __shared__ __align__(128) float dsm[];
  __shared__ __align__(8) uint64_t bars[kWalkWarps][2];
  __shared__ int32_t s_row[SEGS * 2];
  __shared__ int32_t w_row[kWalkWarps * 2];
  (void)NT;
  const int R = a.R;
  const uint32_t row_bytes = (uint32_t)R * 4u;
  const size_t slot_floats = (size_t)2 * kStageBatch * R;
  float* ring = dsm;                                             // [warp][2 slots][2][32][R]
  float* s_val = dsm + (size_t)kWalkWarps * 2 * slot_floats;     // [SEGS * 2][R]
  float* w_val = s_val + (size_t)SEGS * 2 * R;                   // [kWalkWarps * 2][R]

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cta = blockIdx.x;
  // After a timeout anywhere in this launch the remaining CTAs leave at once
  // (with empty carries, so that the fix-up touches nothing of theirs); one
  // thread reads the flag so that the whole CTA takes the same branch.
  __shared__ int32_t s_quit;
  if (threadIdx.x == 0) s_quit = *reinterpret_cast<volatile int32_t*>(timeout_flag);
  __syncthreads();
  if (s_quit != 0) {
    if (threadIdx.x == 0) {
      a.carry_row[cta * 2] = -1;
      a.carry_row[cta * 2 + 1] = -1;
    }
    return;
  }
  if (lane == 0) {
    mbar_init(&bars[warp][0], 1);
    mbar_init(&bars[warp][1], 1);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  const int nnz = (int)a.nnz;
  const int cta_p0 = (int)min((int64_t)cta * SEGS * a.seg, a.nnz);
  const int cta_p1 = (int)min((int64_t)cta_p0 + (int64_t)SEGS * a.seg, a.nnz);
  const int p0 = (int)min((int64_t)cta_p0 + (int64_t)warp * a.seg, a.nnz);
  const int p1 = min(p0 + a.seg, nnz);
  const bool active = p0 < nnz;
  const bool colok = lane < R;
  const float* __restrict__ Fin = static_cast<const float*>(a.Fin);
  const float* __restrict__ Ff = static_cast<const float*>(a.Ff);
  const unsigned lt = (1u << lane) - 1u;

  float v = 0.f, acc = 0.f;
  int q = 0, row_cur = -1;
  if (active) {
    q = a.seg_fib[(int64_t)cta * SEGS + warp];
    row_cur = a.fiber_row[q];
  }
  bool head_open = true;
  auto put_slot = [&](int k, int row, float val) {
    if (lane == 0) s_row[warp * 2 + k] = row;
    if (colok) s_val[(size_t)(warp * 2 + k) * R + lane] = val;
  };
  auto fold = [&](int r, float vv, float ff) {
    if (r != row_cur) {
      if (head_open) {
        put_slot(0, row_cur, acc);
        head_open = false;
      } else if (colok) {
        a.out[(int64_t)row_cur * R + lane] = acc;
      }
      acc = 0.f;
      row_cur = r;
    }
    acc = fmaf(vv, ff, acc);
  };

  const int nb = active ? (p1 - p0 + kStageBatch - 1) / kStageBatch : 0;
  int q_issue = q;  // fiber holding the first nonzero of the next batch issued
  bool ok = true;

  // Issue batch b into ring slot s (the slot's previous batch is consumed).
  auto issue = [&](int b, int s, StageSlot& st) {
    if (!ok) return;  // after a timeout nothing more is issued
    const int base = p0 + b * kStageBatch;  // a multiple of 32: segments start on seg % 32 == 0
    const int p = base + lane;
    const bool okp = p < p1;
    const int in = okp ? __ldg(a.nz_idx + p) : 0;
    st.x = okp ? __ldg(a.nz_val + p) : 0.f;
    st.n = min(kStageBatch, p1 - base);
    const uint32_t valid = st.n >= 32 ? ~0u : ((1u << st.n) - 1u);
    st.ends = __ldg(a.end_bits + (base >> 5)) & valid;
    const bool is_end = (st.ends >> lane) & 1u;
    const int rank = __popc(st.ends & lt);
    int f = 0;
    st.frow = 0;
    if (is_end) {
      f = __ldg(a.fiber_idx + q_issue + rank);
      st.frow = __ldg(a.fiber_row + q_issue + rank);
    }
    q_issue += __popc(st.ends);
    float* slot = ring + ((size_t)warp * 2 + s) * slot_floats;
    // the copies overwrite rows the generic proxy read in the previous round
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive_expect(&bars[warp][s], (uint32_t)(st.n + __popc(st.ends)) * row_bytes);
    __syncwarp();
    if (okp) bulk_copy(slot + (size_t)lane * R, Fin + (int64_t)in * R, row_bytes, &bars[warp][s]);
    if (is_end)
      bulk_copy(slot + (size_t)(kStageBatch + rank) * R, Ff + (int64_t)f * R, row_bytes, &bars[warp][s]);
  };

  // Fold the batch held in ring slot s.
  uint32_t phase0 = 0, phase1 = 0;
  auto consume = [&](int s, const StageSlot& st, uint32_t& phase) {
    if (!ok) return;
    if (!mbar_wait(&bars[warp][s], phase)) {
      ok = false;
      if (lane == 0) atomicExch(timeout_flag, 1);
      return;
    }
    phase ^= 1u;
    const float* slot = ring + ((size_t)warp * 2 + s) * slot_floats;
#pragma unroll 8
    for (int j = 0; j < kStageBatch; ++j) {
      if (j >= st.n) break;
      const float x = __shfl_sync(kFull, st.x, j);
      const float fv = colok ? slot[(size_t)j * R + lane] : 0.f;
      v = fmaf(x, fv, v);
      if ((st.ends >> j) & 1u) {
        const int k = __popc(st.ends & ((1u << j) - 1u));
        const int r = __shfl_sync(kFull, st.frow, j);
        const float ff = colok ? slot[(size_t)(kStageBatch + k) * R + lane] : 0.f;
        fold(r, v, ff);
        v = 0.f;
      }
    }
    q += __popc(st.ends);
    __syncwarp();
  };

  StageSlot s0, s1;
  if (nb > 0) issue(0, 0, s0);
  if (nb > 1) issue(1, 1, s1);
  for (int b = 0; b < nb; b += 2) {
    consume(0, s0, phase0);
    if (b + 2 < nb) issue(b + 2, 0, s0);
    if (b + 1 < nb) {
      consume(1, s1, phase1);
      if (b + 3 < nb) issue(b + 3, 1, s1);
    }
  }
  (void)ok;

  // The fiber open at the segment end (if its last nonzero lies beyond p1).
  if (active && !((__ldg(a.end_bits + ((p1 - 1) >> 5)) >> ((p1 - 1) & 31)) & 1u)) {
    const int f = __ldg(a.fiber_idx + q);
    const int r = __ldg(a.fiber_row + q);
    const float ff = colok ? __ldg(Ff + (int64_t)f * R + lane) : 0.f;
    fold(r, v, ff);
  }
  if (!active) {
    if (lane == 0) { s_row[warp * 2] = -1; s_row[warp * 2 + 1] = -1; }
  } else if (head_open) {
    put_slot(0, row_cur, acc);
    if (lane == 0) s_row[warp * 2 + 1] = -1;
  } else {
    put_slot(1, row_cur, acc);
  }
  __syncthreads();
  mttkrp_merge_cta<SEGS, 1>(a, cta, s_row, s_val, w_row, w_val, lane, warp, cta_p0, cta_p1);
}

}  // namespace

size_t stage_smem_bytes(int R) {
  return sizeof(float) * ((size_t)kWalkWarps * 2 * 2 * kStageBatch * R + (size_t)(2 * kWalkWarps + 2 * kWalkWarps) * R);
}

bool stage_supported(int dtype, int R) { return dtype == DFACTO_F32 && R <= 32 && (R % 4) == 0; }

cudaError_t launch_walk_stage(const MttkrpParams& a, int64_t ncta, int32_t* timeout_flag, cudaStream_t s) {
  if (!(a.R <= 32 && (a.R % 4) == 0 && (a.seg % kStageBatch) == 0)) return cudaErrorInvalidValue;
  // bulk copies need 16-byte aligned rows (R % 4 == 0) and bases
  if (((reinterpret_cast<uintptr_t>(a.Fin) | reinterpret_cast<uintptr_t>(a.Ff)) & 15) != 0)
    return cudaErrorMisalignedAddress;
  const size_t smem = stage_smem_bytes(a.R);
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(mttkrp_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  mttkrp_stage<<<(unsigned)ncta, kWalkWarps * 32, smem, s>>>(a, timeout_flag);
  DF_COUNT();
  return cudaGetLastError();
}

}  // namespace dfacto
