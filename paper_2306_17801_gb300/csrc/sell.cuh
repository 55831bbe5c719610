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

#include "kernels_common.cuh"

namespace apcg {
namespace dev {

template <class TV>
struct SellView {
  int32_t n = 0;        // rows
  int32_t nslices = 0;  // ceil(n / 32)
  const int32_t* __restrict__ sptr = nullptr;  // [nslices + 1] entry offsets (multiples of 32)
  const int32_t* __restrict__ col = nullptr;   // [sptr[nslices]] column indices, or
  const int16_t* __restrict__ dcol = nullptr;  // [sptr[nslices]] column - row (the D16 instances)
  const TV* __restrict__ val = nullptr;        // [sptr[nslices]]
  int32_t long_rows = 0;  // 0: one entry at a time; else the group size G of the grouped path (8 or 9)
};

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
// D16: the column of an entry is read as a 16-bit offset from its row
// (A.dcol) instead of a 32-bit index (A.col): 2 bytes per entry less, for
// matrices whose entries all lie within 32767 of the diagonal (the plan
// checks).  The sums are the same.
template <bool OWN_X, bool LONG, class T, int G = 8, bool D16 = false, class TV, class Epi>
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
    const int32_t* cp = D16 ? nullptr : A.col + base + lane;
    const int16_t* dp = D16 ? A.dcol + base + lane : nullptr;
    const TV* vp = A.val + base + lane;
    const int32_t width = (end - base) >> 5;
    T acc = T(0);
    if (LONG) {
      // Long rows: groups of G entries per lane -- all column/value loads of a
      // group, then its gathers, then its FMAs; the last group is predicated
      // (the width is the same for the 32 lanes of a slice, so the predicate
      // is uniform).  Measured faster than whole groups plus single entries
      // for the rest (27-point: 256 vs 285 us per launch at 160^3).
      for (int32_t k = 0; k < width; k += G) {
        int32_t j[G];
        TV a[G];
        T xv[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const bool ok = k + g < width;
          j[g] = ok ? (D16 ? row + (int32_t)ld_stream(dp + 32 * (k + g)) : ld_stream(cp + 32 * (k + g))) : 0;
          a[g] = ok ? ld_stream(vp + 32 * (k + g)) : TV(0);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) xv[g] = (k + g < width) ? ld_ro(x + j[g]) : T(0);
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (k + g < width) acc = fma((T)a[g], xv[g], acc);
      }
    } else {
      // Short rows (5- and 7-point stencils): one entry at a time (measured
      // faster: fewer registers, more resident warps).
      for (int32_t k = 0; k < width; ++k) {
        const int32_t j = D16 ? row + (int32_t)ld_stream(dp + 32 * k) : ld_stream(cp + 32 * k);
        const TV a = ld_stream(vp + 32 * k);
        acc = fma((T)a, ld_ro(x + j), acc);
      }
    }
    if (row < A.n) epi(row, acc, x_own);
  }
}

}  // namespace dev
}  // namespace apcg
