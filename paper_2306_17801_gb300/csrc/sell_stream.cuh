// Streaming SpMV over the sliced-ELL copy (sell.cuh): the matrix streams
// through shared memory by bulk copies while the FMAs run.
//
// Why: on GB300 the float64 SpMV needs the float64 pipe (one FMA per stored
// entry, two lanes per SM per cycle) and HBM (12 bytes per stored entry) for
// about the same time.  When every warp both loads its slice and computes on
// it, a warp waiting for its float64 turn holds back its next loads, and the
// two resources take turns instead of overlapping.  Here one producer warp per
// CTA keeps a ring of stages filled with the column indices and values of the
// CTA's next slices (cp.async.bulk, completed on mbarriers), and the consumer
// warps only gather x and run the FMAs, reading the entries from shared memory.
//
// Work split: CTA c owns the slices [part[c], part[c+1]) (contiguous, so its
// entries are one contiguous range of the col and val arrays), chosen on the
// host so that every CTA streams about the same number of entries.  The host
// also cuts each CTA's range into stages of whole consecutive slices holding
// at most kStageEntries entries (the stage table: first slice, end slice,
// first entry, entry count), so the producer never searches.  Consumer warp w
// takes the CTA's slices w, w + NW, w + 2 NW, ... whatever stage they fall in,
// so every warp gets the same share of slices.  A slice must fit in one stage:
// width <= kStageEntries / 32.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "kernels_common.cuh"
#include "sell.cuh"

namespace apcg {
namespace dev {

constexpr int kStreamConsumers = 16;                        // consumer warps per CTA
constexpr int kStreamThreads = 32 * (kStreamConsumers + 1);  // plus one producer warp
constexpr int kStages = 4;
constexpr int kStageEntries = 4096;
constexpr int kStreamMaxWidth = kStageEntries / 32;

// Dynamic shared memory of one CTA: the col and val rings.
template <class TV>
constexpr size_t stream_smem_bytes() {
  return (size_t)kStages * kStageEntries * (sizeof(int32_t) + sizeof(TV));
}

// Barriers and stage descriptors (static shared memory of the kernel).
struct StreamBars {
  uint64_t full[kStages];   // producer arrival + copied bytes
  uint64_t empty[kStages];  // one arrival per consumer warp
  int4 meta[kStages];       // first slice, end slice, first entry, entry count; x < 0 ends the stream
};

// The host-built work split of the streaming SpMV.
struct StreamPlan {
  const int32_t* part = nullptr;    // [grid + 1] first slice of each CTA
  const int32_t* stage_ptr = nullptr;  // [grid + 1] first stage of each CTA
  const int4* stages = nullptr;     // stage table
};

// Apply epi(row, (A x)[row], x[row]) to every row of the CTA's slices.  All
// threads of the block (kStreamThreads) call it together.  Returns false in
// every thread of a warp whose bounded wait ran out (the caller flags the
// solve); the block's later barriers are still reached by every thread.
template <class T, class TV, class Epi>
__device__ __forceinline__ bool sell_spmv_stream(const SellView<TV>& A, const StreamPlan& P, const T* __restrict__ x,
                                                 unsigned char* dyn, StreamBars& B, Epi epi) {
  constexpr int G = 4;  // gathers issued before their FMAs
  int32_t* const scol = reinterpret_cast<int32_t*>(dyn);
  TV* const sval = reinterpret_cast<TV*>(dyn + (size_t)kStages * kStageEntries * sizeof(int32_t));
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&B.full[st], 1);
      mbar_init(&B.empty[st], kStreamConsumers);
    }
    mbar_init_fence();
  }
  __syncthreads();
  bool ok = true;
  if (warp == kStreamConsumers) {
    // ---- producer warp: lanes fetch 32 stage descriptors at a time, lane 0 issues
    const int32_t t0 = __ldg(P.stage_ptr + blockIdx.x), t1 = __ldg(P.stage_ptr + blockIdx.x + 1);
    int stage = 0;
    uint32_t round = 0;
    int32_t last_round[kStages];
#pragma unroll
    for (int st = 0; st < kStages; ++st) last_round[st] = -1;
    bool ended = false;
    for (int32_t t = t0; !ended; t += 32) {
      const int4 mine = (t + lane < t1) ? __ldg(P.stages + t + lane) : make_int4(-1, -1, 0, 0);
      for (int j = 0; j < 32 && !ended; ++j) {
        int4 m;
        m.x = __shfl_sync(kFull, mine.x, j);
        m.y = __shfl_sync(kFull, mine.y, j);
        m.z = __shfl_sync(kFull, mine.z, j);
        m.w = __shfl_sync(kFull, mine.w, j);
        bool go = true;
        if (lane == 0) {
          if (round > 0) go = mbar_wait(&B.empty[stage], (round - 1) & 1u);
          if (go) {
            B.meta[stage] = m;
            if (m.x >= 0 && m.w > 0) {
              const uint32_t cnt = (uint32_t)m.w;  // a multiple of 32
              mbar_arrive_expect_tx(&B.full[stage], cnt * (uint32_t)(sizeof(int32_t) + sizeof(TV)));
              bulk_g2s(scol + stage * kStageEntries, A.col + m.z, cnt * (uint32_t)sizeof(int32_t), &B.full[stage]);
              bulk_g2s(sval + stage * kStageEntries, A.val + m.z, cnt * (uint32_t)sizeof(TV), &B.full[stage]);
            } else {
              mbar_arrive(&B.full[stage]);  // the end of the stream, or slices of empty rows
            }
            last_round[stage] = (int32_t)round;
          }
        }
        go = __shfl_sync(kFull, go, 0);
        if (!go) {
          ok = false;
          ended = true;
        } else if (m.x < 0) {
          ended = true;
        } else if (++stage == kStages) {
          stage = 0;
          ++round;
        }
      }
    }
    // Every copy this warp issued has landed before the block moves on (normally at once:
    // the consumers waited for each of them).
    if (lane == 0) {
#pragma unroll
      for (int st = 0; st < kStages; ++st)
        if (last_round[st] >= 0 && !mbar_wait(&B.full[st], (uint32_t)last_round[st] & 1u)) ok = false;
    }
    ok = __shfl_sync(kFull, ok, 0);
  } else {
    // ---- consumer warps: slices s0 + warp + k NW, slice offsets fetched one slice ahead
    const int32_t s1 = __ldg(P.part + blockIdx.x + 1);
    int32_t sl = __ldg(P.part + blockIdx.x) + warp;
    int32_t b_next = 0, e_next = 0;
    if (sl < s1) {
      b_next = __ldg(A.sptr + sl);
      e_next = __ldg(A.sptr + sl + 1);
    }
    int stage = 0;
    uint32_t round = 0;
    for (;;) {
      if (!mbar_wait(&B.full[stage], round & 1u)) {
        ok = false;
        break;
      }
      const int4 m = B.meta[stage];
      if (m.x < 0) break;
      const int32_t* cs = scol + stage * kStageEntries;
      const TV* vs = sval + stage * kStageEntries;
      while (sl < m.y) {
        const int32_t b0 = b_next - m.z;
        const int32_t width = (e_next - b_next) >> 5;
        const int32_t row = sl * 32 + lane;
        const int32_t sn = sl + kStreamConsumers;
        if (sn < s1) {
          b_next = __ldg(A.sptr + sn);
          e_next = __ldg(A.sptr + sn + 1);
        }
        const T x_own = row < A.n ? ld_ro(x + row) : T(0);
        const int32_t* cp = cs + b0 + lane;
        const TV* vp = vs + b0 + lane;
        T acc = T(0);
        int32_t k = 0;
        for (; k + G <= width; k += G) {  // whole groups: gathers first, then their FMAs
          T xv[G];
#pragma unroll
          for (int g = 0; g < G; ++g) xv[g] = ld_ro(x + cp[32 * (k + g)]);
#pragma unroll
          for (int g = 0; g < G; ++g) acc = fma((T)vp[32 * (k + g)], xv[g], acc);
        }
        for (; k < width; ++k) acc = fma((T)vp[32 * k], ld_ro(x + cp[32 * k]), acc);  // no FMA predicated off
        if (row < A.n) epi(row, acc, x_own);
        sl = sn;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.empty[stage]);
      if (++stage == kStages) {
        stage = 0;
        ++round;
      }
    }
  }
  return ok;
}

}  // namespace dev
}  // namespace apcg
