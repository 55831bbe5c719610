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

// Apply epi(row, (S x)[row], x[row]) for every row; threads of the grid take
// rows in a grid-stride loop (consecutive threads, consecutive rows, so every
// term's loads are coalesced).  NP > 0 fixes the number of terms at compile
// time (no loop overhead, no predicated FMA); NP = 0 reads it from S.
template <int NP, bool OWN_X, class T, class Epi>
__device__ __forceinline__ void stencil_spmv(const StencilView& S, const T* __restrict__ x, Epi epi) {
  const int32_t n = S.n, nx = S.nx, ny = S.ny, nz = S.nz;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t r = (int32_t)i;
    const int32_t ix = r % nx, t = r / nx;
    const int32_t iy = t % ny, iz = t / ny;
    T acc = T(0);
    if (NP > 0) {
#pragma unroll
      for (int k = 0; k < (NP > 0 ? NP : 1); ++k) {
        const bool in = (unsigned)(ix + S.dx[k]) < (unsigned)nx && (unsigned)(iy + S.dy[k]) < (unsigned)ny &&
                        (unsigned)(iz + S.dz[k]) < (unsigned)nz;
        const T xv = in ? ld_ro(x + r + S.lin[k]) : T(0);
        acc = fma(stencil_weight<T>(S, k), xv, acc);
      }
    } else {
      for (int k = 0; k < S.npts; ++k) {
        const bool in = (unsigned)(ix + S.dx[k]) < (unsigned)nx && (unsigned)(iy + S.dy[k]) < (unsigned)ny &&
                        (unsigned)(iz + S.dz[k]) < (unsigned)nz;
        const T xv = in ? ld_ro(x + r + S.lin[k]) : T(0);
        acc = fma(stencil_weight<T>(S, k), xv, acc);
      }
    }
    epi(r, acc, OWN_X ? ld_ro(x + r) : T(0));
  }
}

}  // namespace dev
}  // namespace apcg
