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
// The outer residual kernel also sets up the inner solve (r32, z = D32^-1 r32,
// p = z, d = 0, rho, (r,r) and the tolerance), so each correction is one
// residual kernel, one inner graph launch (k iterations per body of a
// conditional while node, the float32 instance of the CG core) and one update
// kernel; the host reads two norms once per correction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "apcg_internal.hpp"
#include "cg_core.hpp"
#include "cg_internal.hpp"
#include "kernels_common.cuh"
#include "spmv.cuh"

namespace apcg {
namespace {

constexpr int kThreads = 256;

struct IrState {
  double rnorm2;  // ||b - A x||^2 of the latest outer residual
  double bnorm2;  // ||b||^2
  unsigned int ticket;
  int32_t pad;
};

// val32 = round-to-nearest float32 of val64.
__global__ void to_f32_kernel(const double* __restrict__ v64, float* __restrict__ v32, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v32[i] = (float)v64[i];
}

// dinv32 = 1 / diag(A32) in float32; flags a missing, zero or non-finite entry.
__global__ void jacobi32_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const float* __restrict__ val, int32_t n, float* __restrict__ dinv, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float d = 0.0f;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == (int32_t)i) d += val[e];
    const bool bad = !(d != 0.0f) || !isfinite(d);
    if (bad) atomicOr(err, kDevErrBadDiagonal);
    dinv[i] = bad ? 0.0f : 1.0f / d;
  }
}

struct ResidualArgs {
  const int32_t* rowptr;
  const int32_t* col;
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
};

// r = b - A x in float64 (values TV widened to double), then the inner set-up.
template <int U, class TV>
__global__ void __launch_bounds__(kThreads) residual_kernel(ResidualArgs a, const TV* __restrict__ val) {
  __shared__ dev::SpmvSmem<U, double> sm[kThreads / 32];
  __shared__ double red64[2 * kThreads];
  __shared__ float red32[2 * kThreads];
  double v64[2] = {0.0, 0.0};
  float v32[2] = {0.0f, 0.0f};
  dev::spmv_warp_tiles<U, false, double, TV>(a.rowptr, a.col, val, a.x, a.n, sm[threadIdx.x >> 5].buf,
                                             [&](int32_t i, double ax, double) {
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
    st->hist_len = 0;
    st->body_runs = 0;
    st->alpha = st->beta = st->gamma = st->rho_new = 0.0;
    st->done = (sqrtf(t32[1]) <= tol) ? kDoneConverged : 0;
  }
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

}  // namespace
}  // namespace apcg

struct apcg_ir_plan_s {
  apcg_ctx ctx = nullptr;
  apcg_ir_opts opts{};
  int32_t n = 0;
  int64_t nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val64 = nullptr;  // outer residual values (or nullptr: widen val32)
  const float* val32 = nullptr;   // inner values (the caller's or the plan's copy)
  apcg_id id_a64 = 0, id_a32 = 0, id = 0;
  apcg::CgCore<float> core;       // inner solver; its x is d32
  float* d32 = nullptr;
  apcg::IrState* ost = nullptr;
  double* opartials = nullptr;
  char* ws = nullptr;
  int grid_res = 1, grid_upd = 1, u = 8;
  void* host_state = nullptr;     // pinned: IrState followed by CgState
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

apcg_status launch_residual(apcg_ir_plan P, const double* b, const double* x, cudaStream_t s) {
  ResidualArgs a;
  a.rowptr = P->rowptr;
  a.col = P->col;
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
  a.rtol_inner = P->opts.rtol_inner;
  a.max_inner = P->core.max_it;
  a.inner_k = P->core.k;
  const int g = P->grid_res;
  if (P->val64) {
    switch (P->u) {
      case 4: residual_kernel<4, double><<<g, kThreads, 0, s>>>(a, P->val64); break;
      case 6: residual_kernel<6, double><<<g, kThreads, 0, s>>>(a, P->val64); break;
      default: residual_kernel<8, double><<<g, kThreads, 0, s>>>(a, P->val64); break;
    }
  } else {
    switch (P->u) {
      case 4: residual_kernel<4, float><<<g, kThreads, 0, s>>>(a, P->val32); break;
      case 6: residual_kernel<6, float><<<g, kThreads, 0, s>>>(a, P->val32); break;
      default: residual_kernel<8, float><<<g, kThreads, 0, s>>>(a, P->val32); break;
    }
  }
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
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  const apcg_mat_s& S = A64 ? *A64 : *A32;
  std::unique_ptr<apcg_ir_plan_s, void (*)(apcg_ir_plan)> P(new apcg_ir_plan_s(), ir_destroy);
  P->ctx = ctx;
  P->opts = o;
  P->n = S.nrows;
  P->nnz = S.nnz;
  P->rowptr = S.rowptr;
  P->col = S.col;
  P->val64 = A64 ? static_cast<const double*>(A64->val) : nullptr;
  P->id_a64 = A64 ? A64->id : 0;
  P->id_a32 = A32 ? A32->id : 0;
  CgCore<float>& c = P->core;
  c.n = P->n;
  c.k = o.inner_check_every;
  c.max_it = o.max_inner;
  c.hist_len = 0;
  c.rowptr = S.rowptr;
  c.col = S.col;
  const int sms = ctx_num_sms(ctx);
  core_configure(c, S.nnz, sms);
  P->u = c.u;
  P->grid_res = c.grid_spmv;
  P->grid_upd = std::max(1, std::min(sms * 8, (int)((P->n / 4 + kThreads - 1) / kThreads)));
  // Workspace: val32 copy (if needed), dinv32, r, p, w, z, d (float), partials, states.
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nv = up(sizeof(float) * (size_t)(P->n > 0 ? P->n : 1));
  const size_t nval = A32 ? 0 : up(sizeof(float) * (size_t)(P->nnz > 0 ? P->nnz : 1));
  const size_t nip = up(sizeof(float) * dev::kMaxPartials * 3);
  const size_t nop = up(sizeof(double) * dev::kMaxPartials * 2);
  const size_t nst = up(sizeof(CgState)) + up(sizeof(IrState));
  const size_t total = nval + 6 * nv + nip + nop + nst;
  char* ws = nullptr;
  APCG_CUDA(cudaMallocAsync((void**)&ws, total, ctx->stream));
  P->ws = ws;
  char* q = ws;
  float* v32own = nval ? reinterpret_cast<float*>(q) : nullptr;
  q += nval;
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
  if (v32own) {
    const int g = std::max(1, std::min(sms * 8, (int)((P->nnz + kThreads - 1) / kThreads)));
    to_f32_kernel<<<g, kThreads, 0, ctx->stream>>>(P->val64, v32own, P->nnz);
    APCG_CUDA(cudaGetLastError());
    count_kernels(1);
    P->val32 = v32own;
  } else {
    P->val32 = static_cast<const float*>(A32->val);
  }
  c.val = P->val32;
  if (P->n > 0) {
    const int g = std::max(1, std::min(sms * 8, (int)((P->n + kThreads - 1) / kThreads)));
    jacobi32_kernel<<<g, kThreads, 0, ctx->stream>>>(P->rowptr, P->col, P->val32, P->n, c.dinv,
                                                      ctx->scratch.dev_error);
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
  for (int32_t k = 0;; ++k) {
    st = launch_residual(P, bp, xp, s);
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
    update_kernel<<<g, kThreads, 0, s>>>(xp, P->d32, P->n);
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
    launches += (int64_t)hi->body_runs * 3 * P->core.k;
    res->outer = k + 1;
  }
  res->kernel_launches = launches;
  count_kernels(launches);
  apcg_status st2 = op.finish();
  return st != APCG_OK ? st : st2;
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
