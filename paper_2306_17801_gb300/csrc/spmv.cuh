// CSR sparse matrix-vector product, warp-tile form.
//
// A warp owns a tile of 32 consecutive rows.  The tile's nonzeros are one
// contiguous range [rowptr[r0], rowptr[r0+32]) of col/val, so the warp streams
// it in chunks of 32*U entries with fully coalesced loads (lane l reads entry
// c + 32u + l), forms the products val * x[col] and parks them in shared
// memory; then each lane adds up the products of its own row in storage
// order.  The x gathers go through the read-only L1 path; col/val are loaded
// with an evict-first hint so that they stream through L2 without displacing
// the vectors.  Every row sum is accumulated in storage order, one rounded
// product at a time, with no fused multiply-add, so the result of a row does
// not depend on the tile shape.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels_common.cuh"

namespace apcg {
namespace dev {

// Per-warp staging buffer: 32 * U values of T.
template <int U, class T>
struct SpmvSmem {
  T buf[32 * U];
};

// Apply `epi(row, value)` for every row handled by this warp.  Warps of the
// whole grid take 32-row tiles in a grid-stride loop.  All 32 lanes must call
// this function together.
template <int U, class T, class Epi>
__device__ __forceinline__ void spmv_warp_tiles(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                const T* __restrict__ val, const T* __restrict__ x, int32_t nrows,
                                                T* __restrict__ wbuf, Epi epi) {
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;
  const int64_t ntiles = ((int64_t)nrows + 31) >> 5;
  for (int64_t tile = gwarp; tile < ntiles; tile += nwarps) {
    const int32_t row = (int32_t)(tile * 32 + lane);
    const int32_t rlo = row < nrows ? row : nrows;
    const int32_t rhi = row < nrows ? row + 1 : nrows;
    const int32_t rs = __ldg(rowptr + rlo);
    const int32_t re = __ldg(rowptr + rhi);
    const int32_t base = __shfl_sync(kFull, rs, 0);
    const int32_t end = __shfl_sync(kFull, re, 31);
    T acc = T(0);
    for (int32_t c = base; c < end; c += 32 * U) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t e = c + u * 32 + lane;
        T prod = T(0);
        if (e < end) {
          const int32_t j = ld_stream(col + e);
          const T a = ld_stream(val + e);
          prod = a * ld_ro(x + j);
        }
        wbuf[u * 32 + lane] = prod;
      }
      __syncwarp();
      const int32_t lo = (rs > c ? rs : c) - c;
      const int32_t hi = (re < c + 32 * U ? re : c + 32 * U) - c;
      for (int32_t k = lo; k < hi; ++k) acc += wbuf[k];
      __syncwarp();
    }
    if (row < nrows) epi(row, acc);
  }
}

}  // namespace dev
}  // namespace apcg
