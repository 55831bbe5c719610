// Matrix-free stencil operators (host side): creation and validation of the
// term list, y = S x, and the accessors the CG plan uses (stencil.cuh holds
// the device side and the reasons for the design).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "stencil.cuh"

struct apcg_stencil_s {
  apcg::dev::StencilView v;
  double center = 0.0;  // weight of the (0,0,0) term, 0 if there is none
};

namespace apcg {
namespace {

constexpr int kThreads = 256;

template <int NP>
__global__ void __launch_bounds__(kThreads) stencil_apply_kernel(dev::StencilView S, const double* __restrict__ x,
                                                                 double* __restrict__ y) {
  dev::stencil_spmv<NP, false, double>(S, x, [&](int32_t i, double s, double) { y[i] = s; });
}

apcg_status launch_apply(apcg_ctx ctx, const dev::StencilView& S, const double* x, double* y) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stencil_apply_kernel<7>, kThreads, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t want = ((int64_t)S.n + kThreads - 1) / kThreads;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * ctx_num_sms(ctx)));
  cudaStream_t s = ctx->stream;
  switch (S.npts) {
    case 5: stencil_apply_kernel<5><<<g, kThreads, 0, s>>>(S, x, y); break;
    case 7: stencil_apply_kernel<7><<<g, kThreads, 0, s>>>(S, x, y); break;
    case 9: stencil_apply_kernel<9><<<g, kThreads, 0, s>>>(S, x, y); break;
    case 27: stencil_apply_kernel<27><<<g, kThreads, 0, s>>>(S, x, y); break;
    default: stencil_apply_kernel<0><<<g, kThreads, 0, s>>>(S, x, y); break;
  }
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return APCG_OK;
}

}  // namespace

const dev::StencilView& stencil_view(const apcg_stencil_s* S) { return S->v; }
double stencil_center(const apcg_stencil_s* S) { return S->center; }

}  // namespace apcg

using namespace apcg;

extern "C" {

apcg_status apcg_stencil_create(int32_t nx, int32_t ny, int32_t nz, int32_t npts, const int32_t* offsets,
                                const double* weights, apcg_stencil* out) {
  APCG_CHECK(out && offsets && weights, "NULL argument");
  APCG_CHECK(nx >= 1 && ny >= 1 && nz >= 1, "grid dimensions must be >= 1");
  const int64_t n = (int64_t)nx * ny * nz;
  APCG_CHECK(n <= INT32_MAX, "grid of %lld points exceeds the int32 row range", (long long)n);
  APCG_CHECK(npts >= 1 && npts <= dev::kMaxStencilTerms, "npts must be in 1..%d", dev::kMaxStencilTerms);
  struct Term {
    int32_t dx, dy, dz;
    int64_t lin;
    double w;
  };
  std::vector<Term> t((size_t)npts);
  for (int32_t k = 0; k < npts; ++k) {
    const int32_t dx = offsets[3 * k], dy = offsets[3 * k + 1], dz = offsets[3 * k + 2];
    APCG_CHECK(std::abs(dx) <= 127 && std::abs(dy) <= 127 && std::abs(dz) <= 127, "term %d: offsets exceed +-127", k);
    APCG_CHECK(std::isfinite(weights[k]), "term %d: weight is not finite", k);
    t[k] = Term{dx, dy, dz, (int64_t)dx + (int64_t)nx * ((int64_t)dy + (int64_t)ny * dz), weights[k]};
    APCG_CHECK(std::llabs(t[k].lin) <= INT32_MAX, "term %d: linear offset exceeds the int32 range", k);
  }
  // Ascending linear offset: the column order of an assembled row (offsets are
  // unique per term, so the order is total).
  std::stable_sort(t.begin(), t.end(), [](const Term& a, const Term& b) { return a.lin < b.lin; });
  for (int32_t k = 1; k < npts; ++k)
    APCG_CHECK(!(t[k].dx == t[k - 1].dx && t[k].dy == t[k - 1].dy && t[k].dz == t[k - 1].dz),
               "offset (%d,%d,%d) appears twice", t[k].dx, t[k].dy, t[k].dz);
  apcg_stencil S = new apcg_stencil_s();
  S->v.nx = nx;
  S->v.ny = ny;
  S->v.nz = nz;
  S->v.npts = npts;
  S->v.n = (int32_t)n;
  for (int32_t k = 0; k < npts; ++k) {
    S->v.dx[k] = (int8_t)t[k].dx;
    S->v.dy[k] = (int8_t)t[k].dy;
    S->v.dz[k] = (int8_t)t[k].dz;
    S->v.lin[k] = (int32_t)t[k].lin;
    S->v.w[k] = t[k].w;
    S->v.wf[k] = (float)t[k].w;
    if (t[k].dx == 0 && t[k].dy == 0 && t[k].dz == 0) S->center = t[k].w;
  }
  *out = S;
  return APCG_OK;
}

apcg_status apcg_stencil_destroy(apcg_stencil S) {
  APCG_CHECK(S, "stencil is NULL");
  delete S;
  return APCG_OK;
}

apcg_status apcg_stencil_apply_async(apcg_ctx ctx_in, apcg_stencil S, apcg_vec x, apcg_vec y) {
  APCG_CHECK(S && x && y, "NULL argument");
  APCG_CHECK(x->dtype == APCG_F64 && y->dtype == APCG_F64, "x and y must be float64");
  APCG_CHECK(x->n == S->v.n && y->n == S->v.n, "x/y length differs from the grid size %d", S->v.n);
  APCG_CHECK(x->dptr != y->dptr || S->v.n == 0, "x and y must not alias");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.read(x->id).write(y->id);
  APCG_TRY(op.begin());
  if (S->v.n > 0) APCG_TRY(launch_apply(ctx, S->v, static_cast<const double*>(x->dptr), static_cast<double*>(y->dptr)));
  return op.finish();
}

}  // extern "C"
