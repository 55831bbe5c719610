// Mixed-precision iterative refinement around a float32 Jacobi-PCG.
//
// The paper's solver is float64 CG (Sec. 4.2).  This extension keeps float64
// only where accuracy needs it -- the outer residual r = b - A x, the update
// x += d and the convergence norm -- and runs the inner Jacobi-PCG on A d = r
// entirely in float32 (float32 matrix values, vectors, FMAs and
// accumulation), which halves the bytes of every inner iteration and moves
// its arithmetic off GB300's scarce float64 pipe.  Outer loop:
//   r = b - A x (float64);  stop if ||r|| <= max(rtol ||b||, atol)
//   inner: float32 PCG on A32 d = (float) r from d = 0 to rtol_inner ||(float) r||
//   x += (double) d
// The outer residual kernel also sets up the inner solve, so each correction
// is one residual kernel, one inner graph launch (k iterations per body of a
// conditional while node, the float32 instance of the CG core) and one update
// kernel; the host reads two norms once per correction.  Both the outer and
// the inner SpMV read the plan's sliced-ELL copy of the matrix (one column
// array; float64 values for the outer residual unless the float32 values are
// exact copies, float32 values for the inner solve).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "apcg_internal.hpp"
#include "cg_core.hpp"
#include "cg_internal.hpp"
#include "ir_kernels.cuh"
#include "sell.hpp"

using apcg::ir::IrState;
using apcg::ir::kThreads;

struct apcg_ir_plan_s {
  apcg_ctx ctx = nullptr;
  apcg_ir_opts opts{};
  int32_t n = 0;
  int64_t nnz = 0;
  apcg_id id_a64 = 0, id_a32 = 0, id = 0;
  apcg::dev::SellView<double> A64;  // outer residual values (nslices == 0 when absent)
  apcg::dev::SellView<float> A32;   // inner values (also the outer ones when A64 is absent)
  apcg::dev::StencilView S;         // or a stencil operator (S.n > 0): float64 weights outside, float32 inside
  apcg::CgCore<float> core;         // inner solver; its x is d32
  float* d32 = nullptr;
  IrState* ost = nullptr;
  double* opartials = nullptr;
  char* ws = nullptr;
  int grid_res = 1, grid_upd = 1;
  bool outer64 = false;
  int64_t padded = 0;  // stored entries of the sliced-ELL copy
  void* host_state = nullptr;  // pinned: IrState followed by CgState
};

namespace apcg {
namespace {

void ir_destroy(apcg_ir_plan P) {
  if (!P) return;
  core_release_graph(P->core);
  if (P->core.cap_stream) cudaStreamDestroy(P->core.cap_stream);
  if (P->ws) {
    {
      std::lock_guard<std::mutex> g(global_mutex());
      reg_forget_memory(P->ws);
    }
    cudaFreeAsync(P->ws, P->ctx->stream);
  }
  if (P->host_state) {
    cudaStreamSynchronize(P->ctx->stream);
    cudaFreeHost(P->host_state);
  }
  delete P;
}

// The outer residual and the set-up of the inner solve (its tolerance rtol_inner ||r32||, at most max_inner
// iterations).
apcg_status launch_residual(apcg_ir_plan P, const double* b, const double* x, cudaStream_t s, double rtol_inner,
                            int32_t max_inner, int32_t hist_len = 0) {
  ir::ResidualArgs a;
  a.n = P->n;
  a.b = b;
  a.x = x;
  a.r32 = P->core.r;
  a.p32 = P->core.p;
  a.d32 = P->d32;
  a.dinv32 = P->core.dinv;
  a.ost = P->ost;
  a.opartials = P->opartials;
  a.ist = P->core.st;
  a.ipartials = P->core.partials;
  a.rtol_inner = rtol_inner;
  a.max_inner = max_inner;
  a.inner_k = P->core.k;
  a.hist_len = hist_len;
  if (P->S.n > 0) {
    const int g = P->grid_res;
    switch (P->S.npts) {
      case 5: ir::residual_stencil_kernel<5><<<g, kThreads, 0, s>>>(a, P->S); break;
      case 7: ir::residual_stencil_kernel<7><<<g, kThreads, 0, s>>>(a, P->S); break;
      case 9: ir::residual_stencil_kernel<9><<<g, kThreads, 0, s>>>(a, P->S); break;
      case 27: ir::residual_stencil_kernel<27><<<g, kThreads, 0, s>>>(a, P->S); break;
      default: ir::residual_stencil_kernel<0><<<g, kThreads, 0, s>>>(a, P->S); break;
    }
    APCG_CUDA(cudaGetLastError());
    return APCG_OK;
  }
  const bool lg = P->A32.long_rows != 0;
  const bool pat = P->A32.poff != nullptr;
#define APCG_RES(L, TV, V) \
  (pat ? ir::residual_kernel<L, TV, dev::kColPattern><<<P->grid_res, kThreads, 0, s>>>(a, V) \
       : ir::residual_kernel<L, TV, dev::kColIndex><<<P->grid_res, kThreads, 0, s>>>(a, V))
  if (P->outer64)
    lg ? APCG_RES(true, double, P->A64) : APCG_RES(false, double, P->A64);
  else
    lg ? APCG_RES(true, float, P->A32) : APCG_RES(false, float, P->A32);
#undef APCG_RES
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

}  // namespace
}  // namespace apcg

using namespace apcg;

extern "C" {

apcg_status apcg_ir_opts_default(apcg_ir_opts* o) {
  APCG_CHECK(o, "opts is NULL");
  memset(o, 0, sizeof(*o));
  o->rtol = 1e-10;
  o->atol = 0.0;
  o->max_outer = 50;
  o->max_inner = 1000;
  o->rtol_inner = 1e-4f;
  o->inner_check_every = 1;
  return APCG_OK;
}

apcg_status apcg_ir_plan_create(apcg_ctx ctx_in, apcg_mat A64, apcg_mat A32, const apcg_ir_opts* opts,
                                apcg_ir_plan* out) {
  APCG_CHECK(out && (A64 || A32), "NULL argument (give A64, A32 or both)");
  APCG_CHECK(!A64 || (A64->dtype == APCG_F64 && A64->nrows == A64->ncols), "A64 must be square float64");
  APCG_CHECK(!A32 || (A32->dtype == APCG_F32 && A32->nrows == A32->ncols), "A32 must be square float32");
  if (A64 && A32)
    APCG_CHECK(A64->nrows == A32->nrows && A64->nnz == A32->nnz && A64->rowptr == A32->rowptr && A64->col == A32->col,
               "A64 and A32 must share one CSR structure (same rowptr and col arrays)");
  apcg_ir_opts o;
  if (opts)
    o = *opts;
  else
    apcg_ir_opts_default(&o);
  if (o.max_outer <= 0) o.max_outer = 50;
  if (o.max_inner <= 0) o.max_inner = 1000;
  if (!(o.rtol_inner > 0.0f)) o.rtol_inner = 1e-4f;
  if (o.inner_check_every < 1) o.inner_check_every = 1;
  APCG_CHECK(o.rtol >= 0.0 && o.atol >= 0.0, "tolerances must be non-negative");
  APCG_CHECK(o.history_len >= 0, "history_len must be >= 0");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  const apcg_mat_s& S = A64 ? *A64 : *A32;
  std::unique_ptr<apcg_ir_plan_s, void (*)(apcg_ir_plan)> P(new apcg_ir_plan_s(), ir_destroy);
  P->ctx = ctx;
  P->opts = o;
  P->n = S.nrows;
  P->nnz = S.nnz;
  P->id_a64 = A64 ? A64->id : 0;
  P->id_a32 = A32 ? A32->id : 0;
  P->outer64 = A64 != nullptr;
  CgCore<float>& c = P->core;
  c.n = P->n;
  c.k = o.inner_check_every;
  c.max_it = o.max_inner;
  c.hist_len = 0;
  const int sms = ctx_num_sms(ctx);
  core_configure(c, S.nnz, sms);
  P->grid_res = c.grid_spmv;
  P->grid_upd = std::max(1, std::min(sms * 8, (int)((P->n / 4 + kThreads - 1) / kThreads)));
  SellLayout L;
  APCG_TRY(csr_layout(ctx, &S, true, &L));
  // Columns: per-slice offset lists where the slices' rows share them (no column stream: 4 of the float32
  // SpMV's 8 bytes per entry), else 32-bit indices even where 16-bit offsets would fit: the float32 inner SpMV
  // is bound by HBM at six blocks per SM, and the offset form's extra registers cost it one (160^3 27-point
  // refinement: 108.8 against 107.8 ms).
  // Workspace: sliced-ELL (sptr, col, float32 values, float64 values if A64), dinv32, r, p, w, z, d,
  // partials and states.
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nv = up(sizeof(float) * (size_t)(P->n > 0 ? P->n : 1));
  const size_t nsptr = up(sizeof(int32_t) * ((size_t)L.nslices + 1));
  const size_t ncol = up(sizeof(int32_t) * (size_t)std::max<int64_t>(L.pattern ? L.padded / 32 : L.padded, 1));
  const size_t nv32 = up(sizeof(float) * (size_t)std::max<int64_t>(L.padded, 1));
  const size_t nv64 = A64 ? up(sizeof(double) * (size_t)std::max<int64_t>(L.padded, 1)) : 0;
  const size_t nip = up(sizeof(float) * dev::kMaxPartials * 3);
  const size_t nop = up(sizeof(double) * dev::kMaxPartials * 2);
  const size_t nst = up(sizeof(CgState)) + up(sizeof(IrState));
  const size_t nh = up(sizeof(double) * (size_t)std::max(o.history_len, 1));
  const size_t total = nsptr + ncol + nv32 + nv64 + 6 * nv + nip + nop + nst + 2 * nh;
  char* ws = nullptr;
  APCG_TRY(dev_alloc_async((void**)&ws, total, ctx->stream));
  P->ws = ws;
  char* q = ws;
  int32_t* sptr = reinterpret_cast<int32_t*>(q);
  q += nsptr;
  int32_t* scol = L.pattern ? nullptr : reinterpret_cast<int32_t*>(q);
  int32_t* spat = L.pattern ? reinterpret_cast<int32_t*>(q) : nullptr;
  q += ncol;
  float* sval32 = reinterpret_cast<float*>(q);
  q += nv32;
  double* sval64 = A64 ? reinterpret_cast<double*>(q) : nullptr;
  q += nv64;
  c.dinv = reinterpret_cast<float*>(q);
  c.r = reinterpret_cast<float*>(q + nv);
  c.p = reinterpret_cast<float*>(q + 2 * nv);
  c.w = reinterpret_cast<float*>(q + 3 * nv);
  c.z = reinterpret_cast<float*>(q + 4 * nv);
  P->d32 = reinterpret_cast<float*>(q + 5 * nv);
  q += 6 * nv;
  c.partials = reinterpret_cast<float*>(q);
  P->opartials = reinterpret_cast<double*>(q + nip);
  c.st = reinterpret_cast<CgState*>(q + nip + nop);
  P->ost = reinterpret_cast<IrState*>(q + nip + nop + up(sizeof(CgState)));
  c.alpha_h = reinterpret_cast<double*>(q + nip + nop + nst);
  c.beta_h = reinterpret_cast<double*>(q + nip + nop + nst + nh);
  APCG_CUDA(cudaMemsetAsync(q, 0, nip + nop + nst, ctx->stream));
  APCG_CUDA(cudaMallocHost(&P->host_state, sizeof(IrState) + sizeof(CgState)));
  {
    std::lock_guard<std::mutex> g(global_mutex());
    P->id = register_memory(ws, total);
  }
  APCG_TRY(ensure_scratch(ctx));
  OpScope op(ctx);
  op.read(P->id_a64).read(P->id_a32).write(P->id);
  APCG_TRY(op.begin());
  APCG_CUDA(cudaMemcpyAsync(sptr, L.d_sptr, sizeof(int32_t) * ((size_t)L.nslices + 1), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  if (A32)
    APCG_TRY(sell_fill<float, float>(ctx->stream, L, sptr, S.rowptr, S.col, static_cast<const float*>(A32->val),
                                     scol, nullptr, spat, sval32));
  else
    APCG_TRY(sell_fill<double, float>(ctx->stream, L, sptr, S.rowptr, S.col, static_cast<const double*>(A64->val),
                                      scol, nullptr, spat, sval32));
  if (A64)
    APCG_TRY(sell_fill<double, double>(ctx->stream, L, sptr, S.rowptr, S.col, static_cast<const double*>(A64->val),
                                       nullptr, nullptr, nullptr, sval64));
  P->A32.n = P->A64.n = P->n;
  P->A32.nslices = L.nslices;
  P->A32.sptr = sptr;
  P->A32.col = scol;
  P->A32.poff = spat;
  P->A32.val = sval32;
  if (A64) {
    P->A64.nslices = L.nslices;
    P->A64.sptr = sptr;
    P->A64.col = scol;
    P->A64.poff = spat;
    P->A64.val = sval64;
  }
  P->A32.long_rows = P->A64.long_rows = L.long_rows;
  // float32 offset-list SpMV of long rows: stage each warp's next slice of values in shared memory
  P->A32.stage_cap = (L.pattern && L.long_rows) ? std::min(L.max_width, dev::kStageMaxWidth) : 0;
  P->padded = L.padded;
  c.A = P->A32;
  core_configure(c, S.nnz, sms);  // the SpMV kernel instance depends on the row length
  P->grid_res = c.grid_spmv;
  if (P->n > 0) {
    const int g = std::max(1, std::min(sms * 8, (int)((P->n + kThreads - 1) / kThreads)));
    if (A32)
      ir::jacobi32_kernel<float><<<g, kThreads, 0, ctx->stream>>>(S.rowptr, S.col, static_cast<const float*>(A32->val),
                                                                  P->n, c.dinv, ctx->scratch.dev_error);
    else
      ir::jacobi32_kernel<double><<<g, kThreads, 0, ctx->stream>>>(
          S.rowptr, S.col, static_cast<const double*>(A64->val), P->n, c.dinv, ctx->scratch.dev_error);
    APCG_CUDA(cudaGetLastError());
    count_kernels(1);
  }
  APCG_TRY(op.finish());
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));
  counters().host_syncs++;
  APCG_TRY(ctx_check_device_error(ctx));
  APCG_TRY(core_build_graph(c, P->d32, ctx->stream));
  *out = P.release();
  return APCG_OK;
}

apcg_status apcg_ir_plan_create_stencil(apcg_ctx ctx_in, apcg_stencil St, const apcg_ir_opts* opts,
                                        apcg_ir_plan* out) {
  APCG_CHECK(out && St, "NULL argument");
  const double center = stencil_center(St);
  if (!(center != 0.0) || !std::isfinite(center) || !((float)center != 0.0f) || !std::isfinite((float)center))
    return set_error(APCG_ERR_BAD_DIAGONAL, "Jacobi: the stencil's centre weight is missing, zero or not finite");
  apcg_ir_opts o;
  if (opts)
    o = *opts;
  else
    apcg_ir_opts_default(&o);
  if (o.max_outer <= 0) o.max_outer = 50;
  if (o.max_inner <= 0) o.max_inner = 1000;
  if (!(o.rtol_inner > 0.0f)) o.rtol_inner = 1e-4f;
  if (o.inner_check_every < 1) o.inner_check_every = 1;
  APCG_CHECK(o.rtol >= 0.0 && o.atol >= 0.0, "tolerances must be non-negative");
  APCG_CHECK(o.history_len >= 0, "history_len must be >= 0");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  std::unique_ptr<apcg_ir_plan_s, void (*)(apcg_ir_plan)> P(new apcg_ir_plan_s(), ir_destroy);
  P->ctx = ctx;
  P->opts = o;
  P->S = stencil_view(St);
  P->n = P->S.n;
  P->nnz = (int64_t)P->S.npts * P->S.n;
  P->outer64 = true;
  CgCore<float>& c = P->core;
  c.n = P->n;
  c.k = o.inner_check_every;
  c.max_it = o.max_inner;
  c.hist_len = 0;
  c.S = P->S;
  const int sms = ctx_num_sms(ctx);
  core_configure(c, P->nnz, sms);
  P->grid_res = c.grid_spmv;
  P->grid_upd = std::max(1, std::min(sms * 8, (int)((P->n / 4 + kThreads - 1) / kThreads)));
  // Workspace: dinv32, r, p, w, z, d (float32); partials and states.
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nv = up(sizeof(float) * (size_t)(P->n > 0 ? P->n : 1));
  const size_t nip = up(sizeof(float) * dev::kMaxPartials * 3);
  const size_t nop = up(sizeof(double) * dev::kMaxPartials * 2);
  const size_t nst = up(sizeof(CgState)) + up(sizeof(IrState));
  const size_t nh = up(sizeof(double) * (size_t)std::max(o.history_len, 1));
  const size_t total = 6 * nv + nip + nop + nst + 2 * nh;
  char* ws = nullptr;
  APCG_TRY(dev_alloc_async((void**)&ws, total, ctx->stream));
  P->ws = ws;
  c.dinv = reinterpret_cast<float*>(ws);
  c.r = reinterpret_cast<float*>(ws + nv);
  c.p = reinterpret_cast<float*>(ws + 2 * nv);
  c.w = reinterpret_cast<float*>(ws + 3 * nv);
  c.z = reinterpret_cast<float*>(ws + 4 * nv);
  P->d32 = reinterpret_cast<float*>(ws + 5 * nv);
  char* q = ws + 6 * nv;
  c.partials = reinterpret_cast<float*>(q);
  P->opartials = reinterpret_cast<double*>(q + nip);
  c.st = reinterpret_cast<CgState*>(q + nip + nop);
  P->ost = reinterpret_cast<IrState*>(q + nip + nop + up(sizeof(CgState)));
  c.alpha_h = reinterpret_cast<double*>(q + nip + nop + nst);
  c.beta_h = reinterpret_cast<double*>(q + nip + nop + nst + nh);
  APCG_CUDA(cudaMemsetAsync(q, 0, nip + nop + nst, ctx->stream));
  APCG_CUDA(cudaMallocHost(&P->host_state, sizeof(IrState) + sizeof(CgState)));
  {
    std::lock_guard<std::mutex> g(global_mutex());
    P->id = register_memory(ws, total);
  }
  OpScope op(ctx);
  op.write(P->id);
  APCG_TRY(op.begin());
  if (P->n > 0) {
    const int g = std::max(1, std::min(sms * 8, (int)((P->n + kThreads - 1) / kThreads)));
    ir::fill32_kernel<<<g, kThreads, 0, ctx->stream>>>(c.dinv, P->n, 1.0f / (float)center);
    APCG_CUDA(cudaGetLastError());
    count_kernels(1);
  }
  APCG_TRY(op.finish());
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));
  counters().host_syncs++;
  APCG_TRY(core_build_graph(c, P->d32, ctx->stream));
  *out = P.release();
  return APCG_OK;
}

apcg_status apcg_ir_plan_solve(apcg_ir_plan P, apcg_vec b, apcg_vec x, apcg_ir_result* res) {
  APCG_CHECK(P && b && x && res, "NULL argument");
  APCG_CHECK(b->dtype == APCG_F64 && x->dtype == APCG_F64, "b and x must be float64");
  APCG_CHECK(b->n == P->n && x->n == P->n, "b/x length differs from the matrix size %d", P->n);
  APCG_CHECK(b->dptr != x->dptr || P->n == 0, "b and x must not alias");
  cudaStream_t s = P->ctx->stream;
  const double* bp = static_cast<const double*>(b->dptr);
  double* xp = static_cast<double*>(x->dptr);
  OpScope op(P->ctx);
  op.read(P->id_a64).read(P->id_a32).read(b->id).rw(x->id).rw(P->id);
  APCG_TRY(op.begin());
  IrState* ho = static_cast<IrState*>(P->host_state);
  CgState* hi = reinterpret_cast<CgState*>(static_cast<char*>(P->host_state) + sizeof(IrState));
  memset(res, 0, sizeof(*res));
  int64_t launches = 0;
  apcg_status st = APCG_OK;
  const int32_t H = P->opts.history_len;
  if (H > 0) {  // entries the first correction does not reach stay NaN (all bits set)
    cudaError_t e = cudaMemsetAsync(P->core.alpha_h, 0xff, sizeof(double) * H, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->core.beta_h, 0xff, sizeof(double) * H, s);
    if (e != cudaSuccess) st = cuda_error(e, "history reset", __FILE__, __LINE__);
  }
  for (int32_t k = 0; st == APCG_OK; ++k) {
    st = launch_residual(P, bp, xp, s, P->opts.rtol_inner, P->core.max_it, k == 0 ? H : 0);
    if (st != APCG_OK) break;
    launches += 1;
    cudaError_t e = cudaMemcpyAsync(ho, P->ost, sizeof(IrState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hi, P->core.st, sizeof(CgState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "refinement state read", __FILE__, __LINE__);
      break;
    }
    counters().d2h_copies += 2;
    counters().host_syncs++;
    const double rn = std::sqrt(ho->rnorm2), bn = std::sqrt(ho->bnorm2);
    res->rel_res = bn > 0.0 ? rn / bn : rn;
    if (!std::isfinite(rn)) {
      res->reason = APCG_BREAKDOWN;
      break;
    }
    if (rn <= std::max(P->opts.rtol * bn, P->opts.atol)) {
      res->reason = APCG_CONVERGED;
      break;
    }
    if (k == P->opts.max_outer) {
      res->reason = APCG_NOT_CONVERGED;
      break;
    }
    if (hi->done) {  // the float32 right-hand side vanished: no further progress possible
      res->reason = APCG_NOT_CONVERGED;
      break;
    }
    e = cudaGraphLaunch(P->core.exec, s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "inner graph launch", __FILE__, __LINE__);
      break;
    }
    counters().graph_launches++;
    const int g = P->grid_upd;
    ir::update_kernel<<<g, kThreads, 0, s>>>(xp, P->d32, P->n);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      st = cuda_error(e, "update launch", __FILE__, __LINE__);
      break;
    }
    launches += 1;
    // the inner iteration count of this correction, read with the next outer residual
    e = cudaMemcpyAsync(hi, P->core.st, sizeof(CgState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "inner state read", __FILE__, __LINE__);
      break;
    }
    counters().d2h_copies++;
    res->inner_total += hi->iter;
    if (k == 0) res->inner_first = hi->iter;
    launches += (int64_t)hi->body_runs * 3 * P->core.body;
    res->outer = k + 1;
    if (hi->done == kDoneTimeout) {  // a bounded wait in the staged SpMV ran out: the correction is not usable
      res->reason = APCG_BREAKDOWN;
      st = set_error(APCG_ERR_TIMEOUT, "a bounded device wait ran out (staged float32 SpMV)");
      break;
    }
  }
  if (st == APCG_OK && H > 0 && (P->opts.alpha_hist || P->opts.beta_hist)) {
    cudaError_t e = cudaSuccess;
    if (P->opts.alpha_hist)
      e = cudaMemcpyAsync(P->opts.alpha_hist, P->core.alpha_h, sizeof(double) * H, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && P->opts.beta_hist)
      e = cudaMemcpyAsync(P->opts.beta_hist, P->core.beta_h, sizeof(double) * H, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "history read", __FILE__, __LINE__);
    counters().d2h_copies += 2;
    counters().host_syncs++;
  }
  res->kernel_launches = launches;
  count_kernels(launches);
  apcg_status st2 = op.finish();
  return st != APCG_OK ? st : st2;
}

apcg_status apcg_ir_plan_inner_spmv(apcg_ir_plan P, apcg_vec p32, apcg_vec w32, double* gamma) {
  APCG_CHECK(P && p32 && w32, "NULL argument");
  APCG_CHECK(p32->dtype == APCG_F32 && w32->dtype == APCG_F32, "p and w must be float32");
  APCG_CHECK(p32->n == P->n && w32->n == P->n, "p/w length differs from the matrix size %d", P->n);
  APCG_CHECK(p32->dptr != w32->dptr || P->n == 0, "p and w must not alias");
  if (gamma) *gamma = 0.0;
  if (P->n == 0) return APCG_OK;
  cudaStream_t s = P->ctx->stream;
  OpScope op(P->ctx);
  op.read(P->id_a64).read(P->id_a32).read(p32->id).write(w32->id).rw(P->id);
  APCG_TRY(op.begin());
  // the inner solve's K1 instance, reading p32 and writing w32 in place of the plan's p and w; a cleared
  // state block (not done, no history, ticket 0) so that it runs its whole sweep and its last block only
  // forms gamma and alpha in the state
  CgCore<float> c = P->core;
  c.p = static_cast<float*>(p32->dptr);
  c.w = static_cast<float*>(w32->dptr);
  APCG_CUDA(cudaMemsetAsync(c.st, 0, sizeof(CgState), s));
  apcg_status st = core_k1(c, P->d32, s, false);
  count_kernels(1);
  CgState hs;
  if (st == APCG_OK) {
    cudaError_t e = cudaMemcpyAsync(P->host_state, c.st, sizeof(CgState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "state read", __FILE__, __LINE__);
    memcpy(&hs, P->host_state, sizeof(hs));
    counters().d2h_copies++;
    counters().host_syncs++;
  }
  apcg_status st2 = op.finish();
  APCG_TRY(st);
  if (hs.done == kDoneTimeout) return set_error(APCG_ERR_TIMEOUT, "a bounded device wait ran out (staged float32 SpMV)");
  if (gamma) *gamma = hs.gamma;
  return st2;
}

apcg_status apcg_ir_plan_profile(apcg_ir_plan P, apcg_vec b, apcg_vec x, int32_t iters, float* ms) {
  APCG_CHECK(P && b && x, "NULL argument");
  APCG_CHECK(b->dtype == APCG_F64 && x->dtype == APCG_F64, "b and x must be float64");
  APCG_CHECK(b->n == P->n && x->n == P->n, "b/x length differs from the matrix size %d", P->n);
  APCG_CHECK(iters >= 1 && ms, "iters must be >= 1 and ms non-NULL");
  APCG_CHECK(P->n > 0, "empty system");
  cudaStream_t s = P->ctx->stream;
  OpScope op(P->ctx);
  op.read(P->id_a64).read(P->id_a32).read(b->id).read(x->id).rw(P->id);
  APCG_TRY(op.begin());
  cudaEvent_t ev[5];
  for (auto& e : ev) APCG_CUDA(cudaEventCreate(&e));
  float tot[4] = {0.f, 0.f, 0.f, 0.f};
  // no inner tolerance and no cap: every inner iteration runs
  cudaEventRecord(ev[0], s);
  apcg_status st = launch_residual(P, static_cast<const double*>(b->dptr), static_cast<const double*>(x->dptr), s,
                                   0.0, 1 << 30);
  cudaEventRecord(ev[1], s);
  cudaEventSynchronize(ev[1]);
  cudaEventElapsedTime(&tot[0], ev[0], ev[1]);
  CgCore<float> c = P->core;
  c.max_it = 1 << 30;
  for (int32_t i = 0; i < iters && st == APCG_OK; ++i) {
    cudaEventRecord(ev[1], s);
    st = core_k1(c, P->d32, s, false);
    cudaEventRecord(ev[2], s);
    if (st == APCG_OK) st = core_k2(c, P->d32, s, false, 0.0, 0, 0);
    cudaEventRecord(ev[3], s);
    if (st == APCG_OK) st = core_k3(c, P->d32, s, false, 0.0);
    cudaEventRecord(ev[4], s);
    cudaEventSynchronize(ev[4]);
    for (int k = 1; k < 4; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      tot[k] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  count_kernels(1 + 3 * (int64_t)iters);
  APCG_TRY(st);
  CgState hs;
  APCG_CUDA(cudaMemcpy(&hs, P->core.st, sizeof(hs), cudaMemcpyDeviceToHost));
  if (hs.done == kDoneTimeout) return set_error(APCG_ERR_TIMEOUT, "a bounded device wait ran out (staged float32 SpMV)");
  ms[0] = tot[0];
  for (int k = 1; k < 4; ++k) ms[k] = tot[k] / iters;
  return op.finish();
}

apcg_status apcg_ir_plan_test_stall_copies(apcg_ir_plan P, int32_t on) {
  APCG_CHECK(P, "plan is NULL");
  if (P->A32.stage_cap == 0 || P->S.n > 0)
    return set_error(APCG_ERR_UNSUPPORTED, "the plan's float32 SpMV stages no values");
  P->A32.stage_tx_extra = on ? 16u : 0u;
  P->core.A.stage_tx_extra = P->A32.stage_tx_extra;
  // the captured graph holds the kernels' arguments by value: capture it again
  core_release_graph(P->core);
  APCG_TRY(core_build_graph(P->core, P->d32, P->ctx->stream));
  APCG_CUDA(cudaStreamSynchronize(P->ctx->stream));
  return APCG_OK;
}

apcg_status apcg_ir_plan_layout(apcg_ir_plan P, apcg_plan_layout* out) {
  APCG_CHECK(P && out, "plan or out is NULL");
  // the float32 SpMV's group (the K1 instance choice): 9 for 27-entry rows with per-slice offset lists, else
  // 8 where the rows are long, else one entry at a time
  const int32_t lr = P->A32.long_rows;
  const int32_t group = lr == 0 ? 0 : (P->A32.poff && lr == 9) ? 9 : 8;
  describe_layout(P->A32.sptr != nullptr, dev::col_format(P->A32), group, P->A32.nslices, P->padded, out);
  return APCG_OK;
}

apcg_status apcg_ir_plan_destroy(apcg_ir_plan P) {
  APCG_CHECK(P, "plan is NULL");
  ir_destroy(P);
  return APCG_OK;
}

apcg_status apcg_ir_solve(apcg_ctx ctx, apcg_mat A64, apcg_mat A32, apcg_vec b, apcg_vec x, const apcg_ir_opts* opts,
                          apcg_ir_result* res) {
  apcg_ir_plan P = nullptr;
  APCG_TRY(apcg_ir_plan_create(ctx, A64, A32, opts, &P));
  apcg_status st = apcg_ir_plan_solve(P, b, x, res);
  ir_destroy(P);
  return st;
}

}  // extern "C"
