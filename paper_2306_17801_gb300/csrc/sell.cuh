// Sliced-ELL layout of a CSR matrix, and the SpMV over it.
//
// The plan converts the caller's CSR matrix once into slices of 32
// consecutive rows stored column-major: entry k of row 32 s + l sits at
// sptr[s] + 32 k + l, each slice padded to its longest row (padding: value 0,
// column = the row itself, or 0 past the last row).  Row order is unchanged,
// so vectors keep their layout.  Why: on GB300 a float64 FMA costs one warp
// instruction on a pipe that retires two lanes per SM per cycle, so the SpMV
// must keep all 32 lanes busy on every FMA.  In this layout lane l owns row
// 32 s + l and loads its own entries with fully coalesced accesses; a slice of
// rows with w entries costs exactly w FMA instructions, whatever w is (the
// CSR warp tiles of spmv.cuh leave lanes idle when rows straddle chunks, as
// 27-point rows do).  Stencil slices carry almost no padding.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "apcg.h"
#include "kernels_common.cuh"

namespace apcg {
namespace dev {

// How the column of a stored entry is found (the SpMV's CF argument):
//   kColIndex:   a 32-bit index per entry (A.col);
//   kColOff16:   a 16-bit offset from the row per entry (A.dcol), for
//                matrices whose entries all lie within 32767 of the diagonal;
//   kColPattern: one list of offsets from the row per slice (A.poff), shared
//                by its 32 rows.  Entry k of every row of slice s has the
//                column row + poff[sptr[s] / 32 + k]; a row without that
//                offset stores the value 0 there.  Built where each row's
//                columns increase and the union of a slice's offsets is
//                (nearly) as short as its longest row -- stencil matrices,
//                whose rows differ only where the grid ends.  No column bytes
//                stream from memory at all.
enum ColFormat : int { kColIndex = 0, kColOff16 = 1, kColPattern = 2 };
static_assert(kColIndex == APCG_COLS_INDEX && kColOff16 == APCG_COLS_OFFSET16 && kColPattern == APCG_COLS_PATTERN,
              "the column formats are reported by their APCG_COLS_* values");

template <class TV>
struct SellView {
  int32_t n = 0;        // rows
  int32_t nslices = 0;  // ceil(n / 32)
  const int32_t* __restrict__ sptr = nullptr;  // [nslices + 1] entry offsets (multiples of 32)
  const int32_t* __restrict__ col = nullptr;   // [sptr[nslices]] column indices, or
  const int16_t* __restrict__ dcol = nullptr;  // [sptr[nslices]] column - row (kColOff16), or
  const int32_t* __restrict__ poff = nullptr;  // [sptr[nslices] / 32] per-slice column offsets (kColPattern)
  const TV* __restrict__ val = nullptr;        // [sptr[nslices]]
  int32_t long_rows = 0;  // 0: one entry at a time; else the group size G of the grouped path (8 or 9)
  int32_t stage_cap = 0;  // float32 offset-list SpMV: slices of at most this many entries per row are staged
                          // in shared memory (0: none)
  uint32_t stage_tx_extra = 0;  // test hook: bytes each staged copy is expected to move beyond what it moves
                                // (nonzero makes every wait on the copies run out; 0 in normal use)
};

template <class TV>
__host__ __device__ inline int col_format(const SellView<TV>& A) {
  return A.poff ? kColPattern : A.dcol ? kColOff16 : kColIndex;
}

// Column of entry k of this lane's row in the given format (see ColFormat).
template <int CF>
__device__ __forceinline__ int32_t sell_column(const int32_t* cp, const int16_t* dp, const int32_t* op, int32_t k,
                                               int32_t row, int32_t last) {
  if constexpr (CF == kColIndex) {
    return ld_stream(cp + 32 * k);
  } else if constexpr (CF == kColOff16) {
    return row + (int32_t)ld_stream(dp + 32 * k);
  } else {
    return min(max(row + __ldg(op + k), 0), last);
  }
}

// Apply epi(row, (A x)[row], x[row]) for every row; warps of the grid take
// slices in a grid-stride loop.  Values TV are widened to T, the type of x
// and of the row sums.  All 32 lanes must call this function together.
// LONG selects the grouped path for long rows (it needs more registers, so
// short-row matrices use a separate instance); G is its group size, the
// entries per lane loaded before their FMAs.  A group that runs past the
// slice width still issues its predicated FMAs, and on GB300 every float64
// warp instruction costs pipe time, so the plan picks the G that wastes the
// fewest (27-point rows: G = 9, three whole groups, against 32 slots for 27
// entries with G = 8; measured 228 against 256 us per launch at 160^3).
// CF selects the column format (ColFormat).  The sums are the same in all
// three: each row adds its entries in its CSR order, plus exact zeros.  In the
// pattern format an offset that a row lacks may point outside [0, n) (at the
// edges of the grid, or past the last row); its column is clamped into range,
// where it multiplies the stored 0.
template <bool OWN_X, bool LONG, class T, int G = 8, int CF = kColIndex, class TV, class Epi>
__device__ __forceinline__ void sell_spmv(const SellView<TV>& A, const T* __restrict__ x, Epi epi) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int32_t b_next = 0, e_next = 0;
  if (gwarp < A.nslices) {
    b_next = __ldg(A.sptr + gwarp);
    e_next = __ldg(A.sptr + gwarp + 1);
  }
  for (int64_t s = gwarp; s < A.nslices; s += nwarps) {
    const int32_t base = b_next, end = e_next;
    if (s + nwarps < A.nslices) {
      b_next = __ldg(A.sptr + s + nwarps);
      e_next = __ldg(A.sptr + s + nwarps + 1);
    }
    const int32_t row = (int32_t)(s * 32 + lane);
    T x_own = T(0);
    if (OWN_X && row < A.n) x_own = ld_ro(x + row);
    const int32_t* cp = CF == kColIndex ? A.col + base + lane : nullptr;
    const int16_t* dp = CF == kColOff16 ? A.dcol + base + lane : nullptr;
    const int32_t* op = CF == kColPattern ? A.poff + (base >> 5) : nullptr;
    const int32_t last = A.n - 1;
    const TV* vp = A.val + base + lane;
    const int32_t width = (end - base) >> 5;
    T acc = T(0);
    if (LONG) {
      // Long rows: groups of G entries per lane -- all column/value loads of a
      // group, then its gathers, then its FMAs.  The width is the same for the
      // 32 lanes of a slice, so every predicate below is uniform.
      if constexpr (sizeof(T) == 4) {
        // float32: whole groups without predicates, the pointers advanced
        // once per group (constant load offsets), then one predicated partial
        // group (160^3 27-point refinement about 3.5% faster; the float64
        // kernels, bound by the float64 pipe rather than by issue, came out
        // about 1% slower this way and keep the form below).
        int32_t k = 0;
        for (; k + G <= width; k += G) {
          int32_t j[G];
          TV a[G];
          T xv[G];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            j[g] = sell_column<CF>(cp, dp, op, g, row, last);
            a[g] = ld_stream(vp + 32 * g);
          }
#pragma unroll
          for (int g = 0; g < G; ++g) xv[g] = ld_ro(x + j[g]);
#pragma unroll
          for (int g = 0; g < G; ++g) acc = fma((T)a[g], xv[g], acc);
          if (CF == kColIndex) cp += 32 * G;
          if (CF == kColOff16) dp += 32 * G;
          if (CF == kColPattern) op += G;
          vp += 32 * G;
        }
        if (k < width) {
          const int32_t left = width - k;
          int32_t j[G];
          TV a[G];
          T xv[G];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const bool ok = g < left;
            j[g] = ok ? sell_column<CF>(cp, dp, op, g, row, last) : 0;
            a[g] = ok ? ld_stream(vp + 32 * g) : TV(0);
          }
#pragma unroll
          for (int g = 0; g < G; ++g) xv[g] = (g < left) ? ld_ro(x + j[g]) : T(0);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (g < left) acc = fma((T)a[g], xv[g], acc);
        }
      } else {
        // float64: every group predicated.  Measured faster than whole groups
        // plus single entries for the rest (27-point: 256 vs 285 us per launch
        // at 160^3).
        for (int32_t k = 0; k < width; k += G) {
          int32_t j[G];
          TV a[G];
          T xv[G];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const bool ok = k + g < width;
            j[g] = ok ? sell_column<CF>(cp, dp, op, k + g, row, last) : 0;
            a[g] = ok ? ld_stream(vp + 32 * (k + g)) : TV(0);
          }
#pragma unroll
          for (int g = 0; g < G; ++g) xv[g] = (k + g < width) ? ld_ro(x + j[g]) : T(0);
#pragma unroll
          for (int g = 0; g < G; ++g)
            if (k + g < width) acc = fma((T)a[g], xv[g], acc);
        }
      }
    } else {
      // Short rows (5- and 7-point stencils): one entry at a time (measured
      // faster: fewer registers, more resident warps).
      for (int32_t k = 0; k < width; ++k) {
        const int32_t j = sell_column<CF>(cp, dp, op, k, row, last);
        const TV a = ld_stream(vp + 32 * k);
        acc = fma((T)a, ld_ro(x + j), acc);
      }
    }
    if (row < A.n) epi(row, acc, x_own);
  }
}

// ---------------------------------------------------------------- staged float32 SpMV
//
// The float32 SpMV over per-slice offset lists streams 4 bytes per entry and
// is bound by how many bytes each SM keeps in flight: with the values held in
// registers, 48 registers per thread leave five blocks per SM, each warp with
// one group of loads outstanding.  The staged form moves each warp's next
// slice of values into shared memory with one bulk copy (the TMA engine,
// cp.async.bulk, completion counted on an mbarrier) while the warp works on
// the current slice, so a whole slice per warp is in flight without using
// registers.  Every wait on an mbarrier is bounded.

constexpr int kStageMaxWidth = 27;                // entries per row of the widest staged slice
constexpr uint32_t kStageSpinLimit = 1u << 16;    // try_wait polls before a wait gives up (about 0.16 s)
constexpr int kStageBarrierBytes = 128;           // mbarriers at the front of the dynamic shared memory

// Dynamic shared memory of the staged K1: two slice buffers and two mbarriers per warp.
__host__ __device__ constexpr int stage_smem_bytes(int cap, int warps) {
  return kStageBarrierBytes + warps * 2 * cap * 32 * (int)sizeof(float);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// Bulk copy of bytes (a multiple of 16; both addresses 16-byte aligned) from global to shared memory,
// completing a transaction of that many bytes on bar (one arrival by the calling thread, which announces
// bytes + extra: extra is 0 except under the test hook SellView::stage_tx_extra).
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                             uint32_t extra) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes + extra)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok)
               : "r"(bar), "r"(parity)
               : "memory");
  return ok != 0;
}

// Waits until bar completes the phase of the given parity; false after kStageSpinLimit polls.  A poll
// that finds the phase still open suspends the thread for a time the hardware chooses (about 2.5 us on
// GB300), so a wait that runs out takes about 0.16 s.  Bounding the wait by a clock read instead made the
// staged SpMV 45 us per launch slower (the compiler then scheduled the whole loop differently).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < kStageSpinLimit; ++i)
    if (mbar_try_wait(a, parity)) return true;
  return false;
}

// sell_spmv for float32 values and kColPattern with the values staged as above.  stage holds this warp's two
// buffers of A.stage_cap * 32 floats, bars its two mbarriers.  Slices wider than A.stage_cap read their
// values from global memory.  A wait that gives up sets *fail to fail_code, lets the warp's copies in flight
// land (bounded again) and ends the warp's sweep.  All 32 lanes must call this function together.
template <bool OWN_X, int G, class Epi>
__device__ __forceinline__ void sell_spmv_staged(const SellView<float>& A, const float* __restrict__ x, float* stage,
                                                 uint64_t* bars, int32_t* fail, int32_t fail_code, Epi epi) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int32_t cap_entries = A.stage_cap * 32;
  const int32_t last = A.n - 1;
  if (lane == 0) {
    mbar_init(&bars[0]);
    mbar_init(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // slice offsets of the current, the next and the one after (loaded a sweep step ahead)
  int32_t b_cur = 0, e_cur = 0, b_nx = 0, e_nx = 0, b_far = 0, e_far = 0;
  if (gwarp < A.nslices) {
    b_cur = __ldg(A.sptr + gwarp);
    e_cur = __ldg(A.sptr + gwarp + 1);
  }
  if (gwarp + nwarps < A.nslices) {
    b_nx = __ldg(A.sptr + gwarp + nwarps);
    e_nx = __ldg(A.sptr + gwarp + nwarps + 1);
  }
  uint32_t parity = 0u;   // bit b: parity of buffer b's next phase
  uint32_t pending = 0u;  // bit b: a copy into buffer b has been issued and not waited for
  int buf = 0;            // buffer of the current slice
  bool cur_staged = gwarp < A.nslices && e_cur > b_cur && e_cur - b_cur <= cap_entries;
  if (cur_staged) {
    if (lane == 0) bulk_to_smem(stage, A.val + b_cur, (uint32_t)(e_cur - b_cur) * 4u, &bars[0], A.stage_tx_extra);
    pending |= 1u;
  }
  bool failed = false;
  for (int64_t s = gwarp; s < A.nslices; s += nwarps) {
    // the next slice's values into the other buffer (its previous contents were consumed before the
    // __syncwarp that ended the last step)
    const bool has_next = s + nwarps < A.nslices;
    const bool nx_staged = has_next && e_nx > b_nx && e_nx - b_nx <= cap_entries;
    if (nx_staged) {
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bulk_to_smem(stage + (buf ^ 1) * cap_entries, A.val + b_nx, (uint32_t)(e_nx - b_nx) * 4u, &bars[buf ^ 1],
                     A.stage_tx_extra);
      }
      pending |= 1u << (buf ^ 1);
    }
    if (s + 2 * nwarps < A.nslices) {
      b_far = __ldg(A.sptr + s + 2 * nwarps);
      e_far = __ldg(A.sptr + s + 2 * nwarps + 1);
    }
    const int32_t row = (int32_t)(s * 32 + lane);
    float x_own = 0.f;
    if (OWN_X && row < A.n) x_own = ld_ro(x + row);
    const int32_t* op = A.poff + (b_cur >> 5);
    const int32_t width = (e_cur - b_cur) >> 5;
    const float* sv;
    if (cur_staged) {
      const bool ok = mbar_wait(&bars[buf], (parity >> buf) & 1u);
      if (!__all_sync(kFull, ok)) {  // the copy stays pending, with its phase's parity
        failed = true;
        break;
      }
      parity ^= 1u << buf;
      pending &= ~(1u << buf);
      sv = stage + buf * cap_entries + lane;
    } else {
      sv = A.val + b_cur + lane;
    }
    float acc = 0.f;
    int32_t k = 0;
    for (; k + G <= width; k += G) {
      int32_t j[G];
      float xv[G];
#pragma unroll
      for (int g = 0; g < G; ++g) j[g] = min(max(row + __ldg(op + k + g), 0), last);
#pragma unroll
      for (int g = 0; g < G; ++g) xv[g] = ld_ro(x + j[g]);
#pragma unroll
      for (int g = 0; g < G; ++g) acc = fmaf(sv[32 * (k + g)], xv[g], acc);
    }
    for (; k < width; ++k) acc = fmaf(sv[32 * k], ld_ro(x + min(max(row + __ldg(op + k), 0), last)), acc);
    if (row < A.n) epi(row, acc, x_own);
    __syncwarp();
    buf ^= 1;
    b_cur = b_nx;
    e_cur = e_nx;
    b_nx = b_far;
    e_nx = e_far;
    cur_staged = nx_staged;
  }
  if (failed) {
    if (lane == 0) atomicMax(fail, fail_code);
    // let the copies still in flight land before the shared memory goes away
    for (int b = 0; b < 2; ++b)
      if (pending & (1u << b)) (void)mbar_wait(&bars[b], (parity >> b) & 1u);
  }
}

}  // namespace dev
}  // namespace apcg
