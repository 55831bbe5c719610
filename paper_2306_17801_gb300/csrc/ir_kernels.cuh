// Kernels of mixed-precision iterative refinement (ir.cu): the float64 outer
// residual fused with the float32 inner set-up, the float64 update, and the
// float32 Jacobi diagonal.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cg_internal.hpp"
#include "kernels_common.cuh"
#include "sell.cuh"
#include "stencil.cuh"

namespace apcg {
namespace ir {

constexpr int kThreads = 256;

struct IrState {
  double rnorm2;  // ||b - A x||^2 of the latest outer residual
  double bnorm2;  // ||b||^2
  unsigned int ticket;
  int32_t pad;
};

// dinv32 = 1 / diag(A) in float32, from values of type TV rounded to float
// entry by entry; flags a missing, zero or non-finite diagonal entry.
template <class TV>
__global__ void jacobi32_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const TV* __restrict__ val, int32_t n, float* __restrict__ dinv, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float d = 0.0f;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == (int32_t)i) d += (float)val[e];
    const bool bad = !(d != 0.0f) || !isfinite(d);
    if (bad) atomicOr(err, kDevErrBadDiagonal);
    dinv[i] = bad ? 0.0f : 1.0f / d;
  }
}

struct ResidualArgs {
  int32_t n;
  const double* b;
  const double* x;
  float* r32;
  float* p32;
  float* d32;
  const float* dinv32;
  IrState* ost;
  double* opartials;  // [2 * kMaxPartials]
  CgState* ist;       // inner state block
  float* ipartials;   // [2 * kMaxPartials] (the inner core's partials)
  float rtol_inner;
  int32_t max_inner, inner_k;
  int32_t hist_len;   // inner alpha/beta to record in this correction (the core's history arrays)
};

// r = b - A x in float64 (values TV widened to double), ||r||^2 and ||b||^2 in
// float64; then the inner set-up in float32: r32 = (float) r, p = z = D32^-1 r32,
// d = 0, rho = (r32, z), (r32, r32) and the inner tolerance.
// spmv(epi) applies the float64 operator to x with the given row epilogue.
template <class Spmv>
__device__ __forceinline__ void residual_body(const ResidualArgs& a, Spmv spmv) {
  __shared__ double red64[2 * kThreads];
  __shared__ float red32[2 * kThreads];
  double v64[2] = {0.0, 0.0};
  float v32[2] = {0.0f, 0.0f};
  spmv([&](int32_t i, double ax, double) {
    const double bi = __ldg(a.b + i);
    const double ri = bi - ax;
    v64[0] = fma(ri, ri, v64[0]);
    v64[1] = fma(bi, bi, v64[1]);
    const float rf = (float)ri;
    const float zf = __ldg(a.dinv32 + i) * rf;
    a.r32[i] = rf;
    a.p32[i] = zf;
    a.d32[i] = 0.0f;
    v32[0] = fmaf(rf, zf, v32[0]);
    v32[1] = fmaf(rf, rf, v32[1]);
  });
  double t64[2];
  if (dev::grid_sum_last<2>(v64, a.opartials, &a.ost->ticket, red64, t64) && threadIdx.x == 0) {
    a.ost->rnorm2 = t64[0];
    a.ost->bnorm2 = t64[1];
  }
  float t32[2];
  if (dev::grid_sum_last<2>(v32, a.ipartials, &a.ist->ticket, red32, t32) && threadIdx.x == 0) {
    CgState* st = a.ist;
    st->rho = t32[0];
    st->rr = t32[1];
    st->bnorm2 = t32[1];
    const float tol = a.rtol_inner * sqrtf(t32[1]);
    st->tol = tol;
    st->iter = 0;
    st->max_it = a.max_inner;
    st->check_every = a.inner_k;
    st->hist_len = a.hist_len;
    st->body_runs = 0;
    st->alpha = st->beta = st->gamma = st->rho_new = 0.0;
    st->done = (sqrtf(t32[1]) <= tol) ? kDoneConverged : 0;
  }
}

template <bool LONG, class TV, int CF>
__global__ void __launch_bounds__(kThreads) residual_kernel(ResidualArgs a, dev::SellView<TV> A) {
  residual_body(a, [&](auto epi) { dev::sell_spmv<false, LONG, double, 8, CF>(A, a.x, epi); });
}

// The same on a stencil operator (float64 weights).
template <int NP>
__global__ void __launch_bounds__(kThreads) residual_stencil_kernel(ResidualArgs a, dev::StencilView S) {
  residual_body(a, [&](auto epi) { dev::stencil_spmv<NP, false, double>(S, a.x, epi); });
}

// y[0..n) = v (float32).
__global__ void __launch_bounds__(kThreads) fill32_kernel(float* __restrict__ y, int64_t n, float v) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = v;
}

// x += (double) d.
__global__ void __launch_bounds__(kThreads) update_kernel(double* __restrict__ x, const float* __restrict__ d,
                                                          int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = n / 4;
  double2* x2 = reinterpret_cast<double2*>(x);
  const float4* d4 = reinterpret_cast<const float4*>(d);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 dd = __ldg(d4 + i);
    double2 a = x2[2 * i], b = x2[2 * i + 1];
    a.x += (double)dd.x;
    a.y += (double)dd.y;
    b.x += (double)dd.z;
    b.y += (double)dd.w;
    x2[2 * i] = a;
    x2[2 * i + 1] = b;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int64_t i = n4 * 4; i < n; ++i) x[i] += (double)d[i];
}

}  // namespace ir
}  // namespace apcg
