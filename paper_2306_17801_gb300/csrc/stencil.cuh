// Matrix-free constant-coefficient stencil operator (device side).
//
// The Laplace problems of Sec. 4.1 are stencils on a structured grid; the
// paper's JAX comparison (Sec. 4.4) applies the operator as a convolution.
// Here a stencil of up to 27 terms on an nx x ny x nz grid (x fastest) is
// applied without any matrix array: row i of S x is
//   sum over k of w_k x[i + dx_k + nx (dy_k + ny dz_k)],
// a term whose neighbour lies outside the grid being dropped (Dirichlet
// boundary by elimination, as in the assembled stencil matrices).  The terms
// are kept in ascending order of their linear offset -- the column order of
// an assembled row -- and each is one FMA into the row sum, so a row costs the
// same float64 instructions as its sliced-ELL row while the SpMV reads only x
// and writes only y (no value or column arrays: 12 bytes per nonzero less).
// Out-of-grid terms multiply a zero instead of branching, which leaves the
// row sum unchanged bit for bit.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels_common.cuh"

namespace apcg {
namespace dev {

constexpr int kMaxStencilTerms = 27;

struct StencilView {
  int32_t nx = 0, ny = 0, nz = 0;
  int32_t npts = 0;                 // number of terms (<= 27)
  int32_t n = 0;                    // nx ny nz
  int8_t dx[kMaxStencilTerms] = {};  // term offsets, ascending linear offset
  int8_t dy[kMaxStencilTerms] = {};
  int8_t dz[kMaxStencilTerms] = {};
  int32_t lin[kMaxStencilTerms] = {};  // dx + nx (dy + ny dz)
  double w[kMaxStencilTerms] = {};     // weights
  float wf[kMaxStencilTerms] = {};     // weights rounded to float (float32 solves)
};

template <class T>
__device__ __forceinline__ T stencil_weight(const StencilView& S, int k);
template <>
__device__ __forceinline__ double stencil_weight<double>(const StencilView& S, int k) {
  return S.w[k];
}
template <>
__device__ __forceinline__ float stencil_weight<float>(const StencilView& S, int k) {
  return S.wf[k];
}

// Apply epi(row, (S x)[row], x[row]) for every row.  Work items are 32
// consecutive rows of one x-line (segment seg of line (iy, iz)); warps take
// items in a grid-stride loop and lane l owns row 32 seg + l of the item, so
// every term's loads are coalesced.  A warp walks its items by mixed-radix
// increments of (seg, iy, iz) -- no integer division per row, which in float32
// solves would cost more than the arithmetic -- and the y/z bounds of every
// term are uniform across the warp.  NP > 0 fixes the number of terms at
// compile time (no loop overhead, no predicated FMA); NP = 0 reads it from S.
// Each row adds its terms in ascending order whatever the walk.
template <int NP, bool OWN_X, class T, class Epi>
__device__ __forceinline__ void stencil_spmv(const StencilView& S, const T* __restrict__ x, Epi epi) {
  const int32_t nx = S.nx, ny = S.ny, nz = S.nz;
  const int32_t segs = (nx + 31) >> 5;
  const int64_t nitems = (int64_t)segs * ny * nz;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // position of the first item and the increment of one grid stride, in (seg, iy, iz)
  int32_t seg = (int32_t)(w0 % segs), iy, iz;
  {
    const int64_t t = w0 / segs;
    iy = (int32_t)(t % ny);
    iz = (int32_t)(t / ny);
  }
  const int32_t dseg = (int32_t)(nw % segs);
  int32_t dy, dz;
  {
    const int64_t t = nw / segs;
    dy = (int32_t)(t % ny);
    dz = (int32_t)(t / ny);  // may exceed nz: the walk then ends after one item
  }
  const int np = NP > 0 ? NP : S.npts;
  for (int64_t item = w0; item < nitems; item += nw) {
    const int32_t ix = (seg << 5) + lane;
    const int32_t r = ix + nx * (iy + ny * iz);
    if (ix < nx) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < (NP > 0 ? NP : kMaxStencilTerms); ++k) {
        if (NP == 0 && k >= np) break;
        const bool in = (unsigned)(ix + S.dx[k]) < (unsigned)nx && (unsigned)(iy + S.dy[k]) < (unsigned)ny &&
                        (unsigned)(iz + S.dz[k]) < (unsigned)nz;
        const T xv = in ? ld_ro(x + r + S.lin[k]) : T(0);
        acc = fma(stencil_weight<T>(S, k), xv, acc);
      }
      epi(r, acc, OWN_X ? ld_ro(x + r) : T(0));
    }
    // advance by one grid stride: seg += dseg, carry into iy, then into iz
    seg += dseg;
    int32_t carry = seg >= segs;
    seg -= carry ? segs : 0;
    iy += dy + carry;
    carry = iy >= ny;
    iy -= carry ? ny : 0;
    iz += dz + carry;
  }
}

}  // namespace dev
}  // namespace apcg
