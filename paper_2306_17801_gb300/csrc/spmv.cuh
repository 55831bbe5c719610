// CSR sparse matrix-vector product, warp-tile form.
//
// A warp owns a tile of 32 consecutive rows.  The tile's nonzeros are one
// contiguous range [rowptr[r0], rowptr[r0+32]) of col/val, so the warp streams
// it in chunks of 32*U entries with fully coalesced loads (lane l reads entry
// c + 32u + l), gathers x[col] for each entry, and parks the value/x pairs in
// shared memory; then each lane accumulates its own row with one fused
// multiply-add per nonzero, in storage order.  On GB300 the float64 pipe
// (two lanes per SM per cycle) rather than HBM bounds a float64 SpMV, so the
// kernel spends exactly one FMA per nonzero and none on padding.  Loads are
// issued in phases -- all column indices and values of a chunk, then all
// gathers of x -- so that every lane keeps 2U independent requests in
// flight, and the row bounds of the warp's next tile are fetched while the
// current tile is processed.  The x gathers go through the read-only L1 path;
// col/val are loaded with the streaming (evict-first) cache operator.  A row's
// result does not depend on the tile shape: its terms are always fused in
// storage order.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels_common.cuh"

namespace apcg {
namespace dev {

// Per-warp staging buffer: 32 * U matrix values and 32 * U gathered x values.
template <int U, class T>
struct SpmvSmem {
  T buf[2 * 32 * U];
};

// Apply `epi(row, value, x_own)` for every row handled by this warp, where
// x_own = x[row] (square matrices only: pass OWN_X = false otherwise, x_own
// is then 0).  Matrix values have type TV and are widened to the vector type
// T, in which the row sums are formed (float32 values times float64 x is
// exact widening).  Warps of the whole grid take 32-row tiles in a
// grid-stride loop.  All 32 lanes must call this function together.
template <int U, bool OWN_X, class T, class TV = T, class Epi>
__device__ __forceinline__ void spmv_warp_tiles(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                const TV* __restrict__ val, const T* __restrict__ x, int32_t nrows,
                                                T* __restrict__ wbuf, Epi epi) {
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;
  const int64_t ntiles = ((int64_t)nrows + 31) >> 5;
  auto bounds = [&](int64_t tile, int32_t& rs, int32_t& re) {
    const int64_t row = tile * 32 + lane;
    const int32_t rlo = row < nrows ? (int32_t)row : nrows;
    const int32_t rhi = row < nrows ? (int32_t)row + 1 : nrows;
    rs = __ldg(rowptr + rlo);
    re = __ldg(rowptr + rhi);
  };
  int32_t rs_next = 0, re_next = 0;
  if (gwarp < ntiles) bounds(gwarp, rs_next, re_next);
  for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
    const int32_t rs = rs_next, re = re_next;
    const int32_t row = (int32_t)(tile * 32 + lane);
    T x_own = T(0);
    if (OWN_X && row < nrows) x_own = ld_ro(x + row);
    if (tile + nwarps < ntiles) bounds(tile + nwarps, rs_next, re_next);
    const int32_t base = __shfl_sync(kFull, rs, 0);
    const int32_t end = __shfl_sync(kFull, re, 31);
    T acc = T(0);
    for (int32_t c = base; c < end; c += 32 * U) {
      int32_t j[U];
      TV a[U];
      T xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t e = c + u * 32 + lane;
        const bool ok = e < end;
        j[u] = ok ? ld_stream(col + e) : -1;
        a[u] = ok ? ld_stream(val + e) : TV(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = j[u] >= 0 ? ld_ro(x + j[u]) : T(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        wbuf[u * 32 + lane] = (T)a[u];
        wbuf[32 * U + u * 32 + lane] = xv[u];
      }
      __syncwarp();
      const int32_t lo = (rs > c ? rs : c) - c;
      const int32_t hi = (re < c + 32 * U ? re : c + 32 * U) - c;
      for (int32_t k = lo; k < hi; ++k) acc = fma(wbuf[k], wbuf[32 * U + k], acc);
      __syncwarp();
    }
    if (row < nrows) epi(row, acc, x_own);
  }
}

}  // namespace dev
}  // namespace apcg
