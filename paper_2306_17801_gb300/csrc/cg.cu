// Jacobi-PCG solver plans on one device context (float64).
//
// The iteration kernels live in cg_core.cu; this file owns the plan: the
// Jacobi diagonal (A0, computed and checked once), the workspace, and the
// four ways of running a solve --
//   HOST_SYNC    every reduction goes to the host and is waited for; alpha and
//                beta are computed on the host and passed by value (the
//                host-synchronous form the paper compares against, Sec. 4.1);
//   ASYNC        launches back to back with all scalars on the device; the
//                host reads the 'done' word once every k iterations;
//   ASYNC_GRAPH  k iterations captured once into the body of a conditional
//                while node: one graph launch per solve, no host read until
//                the end (the asynchronous convergence test of Sec. 5);
//   PERSISTENT   the whole solve in one thread-block-cluster launch
//                (cluster_cg.cu), for systems of at most 65536 rows.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "apcg_internal.hpp"
#include "cg_core.hpp"
#include "cg_internal.hpp"
#include "cluster_cg.hpp"
#include "kernels_common.cuh"
#include "sell.hpp"

struct apcg_cg_plan_s {
  apcg_ctx ctx = nullptr;
  apcg_mat_s A;  // copy of the (non-owning) matrix view
  apcg_cg_opts opts{};
  int32_t mode = APCG_MODE_ASYNC_GRAPH;
  apcg::CgCore<double> core;
  char* ws = nullptr;  // workspace block (stream-ordered allocation)
  apcg::CgState* st_host = nullptr;  // pinned mirror of the state block
  apcg_id id = 0;
  bool pending = false;
  int64_t last_launches = 0;
  int64_t padded = 0;  // stored entries of the sliced-ELL copy
  // whole-solve cluster mode
  apcg::ClusterShape shape;
  apcg::SysDesc* sys = nullptr;
  unsigned int* next = nullptr;
  apcg::SysResult* sres = nullptr;
  apcg::SysResult* sres_host = nullptr;
};

namespace apcg {
namespace {

constexpr int kPersistentMaxRows = 65536;  // one cluster of 16 CTAs x 512 threads x 8 rows

apcg_status read_state(apcg_cg_plan P, cudaStream_t s) {
  APCG_CUDA(cudaMemcpyAsync(P->st_host, P->core.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  APCG_CUDA(cudaStreamSynchronize(s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(CgState);
  counters().host_syncs++;
  return APCG_OK;
}

void fill_result(apcg_cg_plan P, apcg_cg_result* res) {
  const CgState* s = P->st_host;
  res->iters = s->iter;
  res->reason = s->done == kDoneBreakdown ? APCG_BREAKDOWN : s->done == kDoneConverged ? APCG_CONVERGED : APCG_NOT_CONVERGED;
  res->rr = s->rr;
  res->bnorm = sqrt(s->bnorm2);
  res->rel_res = res->bnorm > 0.0 ? sqrt(s->rr) / res->bnorm : sqrt(s->rr);
  res->kernel_launches = P->last_launches;
}

// Host-synchronous form: every reduction goes to the host and is waited for;
// alpha and beta are computed on the host and passed by value.
apcg_status solve_host_sync(apcg_cg_plan P, const double* b, double* x) {
  cudaStream_t s = P->ctx->stream;
  CgCore<double>& c = P->core;
  CgState* h = P->st_host;
  APCG_TRY(core_setup_f64(c, b, x, P->opts.rtol, P->opts.atol, s));
  int64_t launches = 1;
  APCG_TRY(read_state(P, s));
  double rho = h->rho;
  const double tol = h->tol;
  int32_t done = h->done, it = 0;
  std::vector<double> ah, bh;
  while (!done) {
    APCG_TRY(core_k1(c, x, s, true));
    APCG_TRY(read_state(P, s));
    const double gamma = h->gamma;
    launches += 1;
    if (!(gamma > 0.0) || !std::isfinite(gamma)) {
      done = kDoneBreakdown;
      break;
    }
    const double alpha = rho / gamma;
    if (it < c.hist_len) ah.push_back(alpha);
    APCG_TRY(core_k2(c, x, s, true, alpha, 0, 0));
    APCG_TRY(read_state(P, s));
    launches += 1;
    ++it;
    const double rr = h->rr, rz = h->rho_new;
    if (rr == 0.0 || ((it % c.k == 0 || it == c.max_it) && std::sqrt(rr) <= tol)) {
      done = kDoneConverged;
    } else if (it >= c.max_it) {
      done = kDoneNotConverged;
    } else if (!std::isfinite(rr)) {
      done = kDoneBreakdown;
    } else {
      const double beta = rz / rho;
      if (it - 1 < c.hist_len) bh.push_back(beta);
      rho = rz;
      APCG_TRY(core_k3(c, x, s, true, beta));
      launches += 1;
    }
  }
  h->iter = it;
  h->done = done;
  P->last_launches = launches;
  if (P->opts.alpha_hist)
    for (size_t i = 0; i < ah.size(); ++i) P->opts.alpha_hist[i] = ah[i];
  if (P->opts.beta_hist)
    for (size_t i = 0; i < bh.size(); ++i) P->opts.beta_hist[i] = bh[i];
  count_kernels(launches);
  return APCG_OK;
}

apcg_status enqueue_async(apcg_cg_plan P, const double* b, double* x, bool graph) {
  cudaStream_t s = P->ctx->stream;
  CgCore<double>& c = P->core;
  APCG_TRY(core_setup_f64(c, b, x, P->opts.rtol, P->opts.atol, s));
  count_kernels(1);
  if (graph) {
    APCG_CUDA(cudaGraphLaunch(c.exec, s));
    counters().graph_launches++;
  } else {
    // Launch k iterations at a time and read 'done' after each block.  Each kernel is a programmatic
    // dependent of the one before it: its launch overlaps its predecessor's last blocks (128^3: 72.2 -> 67.0 us
    // per iteration; the graph form, whose nodes carry no such edge, 65.1).
    const int64_t max_blocks = (int64_t)c.max_it / c.k + 2;
    int64_t launches = 1;
    for (int64_t blk = 0; blk < max_blocks; ++blk) {
      for (int j = 0; j < c.k; ++j) {
        c.pdl = true;
        apcg_status st1 = core_k1(c, x, s, false);
        if (st1 == APCG_OK) st1 = core_k2(c, x, s, false, 0.0, 0, 0);
        if (st1 == APCG_OK) st1 = core_k3(c, x, s, false, 0.0);
        c.pdl = false;
        APCG_TRY(st1);
      }
      launches += 3 * c.k;
      count_kernels(3 * c.k);
      APCG_TRY(read_state(P, s));
      if (P->st_host->done) break;
    }
    P->last_launches = launches;
  }
  APCG_CUDA(cudaMemcpyAsync(P->st_host, c.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(CgState);
  return APCG_OK;
}

// The whole solve in one cluster launch (small systems).
apcg_status enqueue_persistent(apcg_cg_plan P, const double* b, double* x) {
  cudaStream_t s = P->ctx->stream;
  const CgCore<double>& c = P->core;
  ClusterArgs ca{};
  ca.rowptr = P->A.rowptr;
  ca.col = P->A.col;
  ca.val = static_cast<const double*>(P->A.val);
  ca.dinv = c.dinv;
  ca.b = b;
  ca.x = x;
  ca.sys = P->sys;
  ca.order = nullptr;
  ca.nsys = 1;
  ca.check_every = c.k;
  ca.next = P->next;
  ca.res = P->sres;
  ca.rtol = P->opts.rtol;
  ca.atol = P->opts.atol;
  ca.max_it = c.max_it;
  ca.hist_len = c.hist_len;
  ca.alpha_h = c.alpha_h;
  ca.beta_h = c.beta_h;
  APCG_CUDA(cudaMemsetAsync(P->next, 0, sizeof(unsigned int), s));
  APCG_CUDA(launch_cluster_cg(ca, P->shape, 1, s));
  count_kernels(1);
  P->last_launches = 1;
  APCG_CUDA(cudaMemcpyAsync(P->sres_host, P->sres, sizeof(SysResult), cudaMemcpyDeviceToHost, s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(SysResult);
  return APCG_OK;
}

apcg_status finish_async(apcg_cg_plan P) {
  APCG_CUDA(cudaStreamSynchronize(P->ctx->stream));
  counters().host_syncs++;
  const CgCore<double>& c = P->core;
  if (P->mode == APCG_MODE_ASYNC_GRAPH) {
    const int64_t n = (int64_t)P->st_host->body_runs * 3 * c.body;
    count_kernels(n);
    P->last_launches = 1 + n;
  }
  if (c.hist_len > 0) {
    if (P->opts.alpha_hist)
      APCG_CUDA(cudaMemcpy(P->opts.alpha_hist, c.alpha_h, sizeof(double) * c.hist_len, cudaMemcpyDeviceToHost));
    if (P->opts.beta_hist)
      APCG_CUDA(cudaMemcpy(P->opts.beta_hist, c.beta_h, sizeof(double) * c.hist_len, cudaMemcpyDeviceToHost));
    counters().d2h_copies += 2;
  }
  return APCG_OK;
}

apcg_status check_vectors(int32_t n, apcg_vec b, apcg_vec x) {
  APCG_CHECK(b && x, "b or x is NULL");
  APCG_CHECK(b->dtype == APCG_F64 && x->dtype == APCG_F64, "b and x must be float64");
  APCG_CHECK(b->n == n && x->n == n, "b/x length differs from the matrix size %d", n);
  APCG_CHECK(n == 0 || (aligned16(b->dptr) && aligned16(x->dptr)), "b/x must be 16-byte aligned");
  APCG_CHECK(b->dptr != x->dptr || n == 0, "b and x must not alias");
  return APCG_OK;
}

apcg_status check_solve_args(apcg_cg_plan P, apcg_vec b, apcg_vec x) {
  APCG_CHECK(P, "plan is NULL");
  APCG_CHECK(b && x, "b or x is NULL");
  APCG_CHECK(b->dtype == APCG_F64 && x->dtype == APCG_F64, "b and x must be float64");
  const int32_t n = P->core.n;
  APCG_CHECK(b->n == n && x->n == n, "b/x length differs from the matrix size %d", n);
  APCG_CHECK(n == 0 || (aligned16(b->dptr) && aligned16(x->dptr)), "b/x must be 16-byte aligned");
  APCG_CHECK(b->dptr != x->dptr || n == 0, "b and x must not alias");
  return APCG_OK;
}

apcg_status cg_plan_destroy(apcg_cg_plan P) {
  APCG_CHECK(P, "plan is NULL");
  core_release_graph(P->core);
  if (P->core.cap_stream) cudaStreamDestroy(P->core.cap_stream);
  if (P->ws) {
    {
      std::lock_guard<std::mutex> g(global_mutex());
      reg_forget_memory(P->ws);
    }
    cudaFreeAsync(P->ws, P->ctx->stream);  // stream-ordered: released once pending solves finish
  }
  if (P->st_host || P->sres_host) {
    // Pinned memory may still be the target of an enqueued copy.
    cudaStreamSynchronize(P->ctx->stream);
    if (P->st_host) cudaFreeHost(P->st_host);
    if (P->sres_host) cudaFreeHost(P->sres_host);
  }
  delete P;
  return APCG_OK;
}

// A plan on a CSR matrix (A) or on a stencil operator (S); exactly one is given.
apcg_status cg_plan_create(apcg_ctx ctx, apcg_mat A, const apcg_stencil_s* S, const apcg_cg_opts* opts,
                           apcg_cg_plan* out) {
  APCG_CHECK((A || S) && !(A && S) && out, "NULL argument");
  double center = 0.0;
  if (A) {
    APCG_CHECK(A->dtype == APCG_F64, "the CG solver takes a float64 matrix");
    APCG_CHECK(A->nrows == A->ncols, "the matrix must be square");
  } else {
    center = stencil_center(S);
    if (!(center != 0.0) || !std::isfinite(center))
      return set_error(APCG_ERR_BAD_DIAGONAL, "Jacobi: the stencil's centre weight is missing, zero or not finite");
  }
  apcg_cg_opts o;
  if (opts)
    o = *opts;
  else
    apcg_cg_opts_default(&o);
  APCG_CHECK(o.check_every >= 1, "check_every must be >= 1");
  APCG_CHECK(o.rtol >= 0.0 && o.atol >= 0.0, "tolerances must be non-negative");
  APCG_CHECK(o.history_len >= 0, "history_len must be >= 0");
  APCG_CHECK(o.mode >= APCG_MODE_HOST_SYNC && o.mode <= APCG_MODE_AUTO, "bad mode %d", o.mode);
  std::unique_ptr<apcg_cg_plan_s, apcg_status (*)(apcg_cg_plan)> P(new apcg_cg_plan_s(), cg_plan_destroy);
  P->ctx = ctx;
  if (A) {
    P->A = *A;
  } else {
    P->A = apcg_mat_s{};
    P->A.nrows = P->A.ncols = stencil_view(S).n;
    P->A.dtype = APCG_F64;
  }
  P->opts = o;
  CgCore<double>& c = P->core;
  c.n = P->A.nrows;
  if (S) c.S = stencil_view(S);
  c.k = o.check_every;
  c.max_it = o.max_it > 0 ? o.max_it : (c.n > 0 ? 10 * c.n : 10);
  c.hist_len = o.history_len;
  P->mode = o.mode;
  if (S && o.mode == APCG_MODE_PERSISTENT)
    return set_error(APCG_ERR_UNSUPPORTED, "the whole-solve cluster kernel takes a CSR matrix, not a stencil");
  if (S && o.mode == APCG_MODE_AUTO) P->mode = APCG_MODE_ASYNC_GRAPH;
  if (A && (o.mode == APCG_MODE_PERSISTENT || o.mode == APCG_MODE_AUTO)) {
    P->shape = c.n <= kPersistentMaxRows ? default_cluster_shape(c.n) : ClusterShape{};
    if (c.n > kPersistentMaxRows) P->shape.ok = false;
    if (!P->shape.ok) {
      if (o.mode == APCG_MODE_PERSISTENT)
        return set_error(APCG_ERR_UNSUPPORTED, "persistent mode handles at most %d rows (got %d)", kPersistentMaxRows,
                         c.n);
      P->mode = APCG_MODE_ASYNC_GRAPH;
    } else {
      P->mode = APCG_MODE_PERSISTENT;
    }
  }
  core_configure(c, A ? A->nnz : 0, ctx_num_sms(ctx));
  // The iteration kernels read a sliced-ELL copy of A (sell.cuh); the cluster kernel reads the CSR itself.
  SellLayout L;
  const bool need_sell = A && P->mode != APCG_MODE_PERSISTENT;
  if (A) APCG_TRY(csr_layout(ctx, A, need_sell, &L));
  // Workspace: dinv, r, p, w, z, partials, state, histories, cluster bookkeeping (one stream-ordered block).
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nv = up(sizeof(double) * (size_t)(c.n > 0 ? c.n : 1));
  const size_t npart = up(sizeof(double) * dev::kMaxPartials * 3);
  const size_t nst = up(sizeof(CgState));
  const size_t nh = up(sizeof(double) * (size_t)(c.hist_len > 0 ? c.hist_len : 1));
  const size_t nsysb = up(sizeof(SysDesc) + sizeof(SysResult) + 64);
  // columns: one list of offsets per slice where the slices' rows share them (no column stream), else
  // 16-bit offsets from the row where they fit (2 bytes per entry less in every SpMV), else 32-bit indices
  const size_t ncolb = L.pattern ? sizeof(int32_t) * (size_t)(L.padded / 32)
                                 : (L.d16 ? sizeof(int16_t) : sizeof(int32_t)) * (size_t)L.padded;
  const size_t nsell = need_sell ? up(sizeof(int32_t) * ((size_t)L.nslices + 1)) + up(ncolb) +
                                       up(sizeof(double) * (size_t)L.padded)
                                 : 0;
  const size_t total = 5 * nv + npart + nst + 2 * nh + nsysb + nsell;
  char* ws = nullptr;
  APCG_TRY(dev_alloc_async((void**)&ws, total, ctx->stream));
  P->ws = ws;
  c.dinv = reinterpret_cast<double*>(ws);
  c.r = reinterpret_cast<double*>(ws + nv);
  c.p = reinterpret_cast<double*>(ws + 2 * nv);
  c.w = reinterpret_cast<double*>(ws + 3 * nv);
  c.z = reinterpret_cast<double*>(ws + 4 * nv);
  c.partials = reinterpret_cast<double*>(ws + 5 * nv);
  c.st = reinterpret_cast<CgState*>(ws + 5 * nv + npart);
  c.alpha_h = reinterpret_cast<double*>(ws + 5 * nv + npart + nst);
  c.beta_h = reinterpret_cast<double*>(ws + 5 * nv + npart + nst + nh);
  char* tail = ws + 5 * nv + npart + nst + 2 * nh;
  P->sys = reinterpret_cast<SysDesc*>(tail);
  P->sres = reinterpret_cast<SysResult*>(tail + sizeof(SysDesc));
  P->next = reinterpret_cast<unsigned int*>(tail + sizeof(SysDesc) + sizeof(SysResult));
  APCG_CUDA(cudaMemsetAsync(ws + 5 * nv, 0, npart + nst + 2 * nh + nsysb, ctx->stream));
  if (need_sell) {
    char* q = tail + nsysb;
    int32_t* sptr = reinterpret_cast<int32_t*>(q);
    q += up(sizeof(int32_t) * ((size_t)L.nslices + 1));
    int32_t* scol = (L.pattern || L.d16) ? nullptr : reinterpret_cast<int32_t*>(q);
    int16_t* sdcol = L.d16 ? reinterpret_cast<int16_t*>(q) : nullptr;
    int32_t* spat = L.pattern ? reinterpret_cast<int32_t*>(q) : nullptr;
    q += up(ncolb);
    double* sval = reinterpret_cast<double*>(q);
    APCG_CUDA(cudaMemcpyAsync(sptr, L.d_sptr, sizeof(int32_t) * ((size_t)L.nslices + 1), cudaMemcpyDeviceToDevice,
                              ctx->stream));
    APCG_TRY(sell_fill<double, double>(ctx->stream, L, sptr, A->rowptr, A->col, static_cast<const double*>(A->val),
                                       scol, sdcol, spat, sval));
    c.A.n = c.n;
    c.A.nslices = L.nslices;
    c.A.sptr = sptr;
    c.A.col = scol;
    c.A.dcol = sdcol;
    c.A.poff = spat;
    c.A.val = sval;
    c.A.long_rows = L.group;  // the float64 SpMV's group size (K1 and the set-up kernel)
    P->padded = L.padded;
    core_configure(c, A->nnz, ctx_num_sms(ctx));  // the SpMV kernel instance depends on the row length
  }
  SysDesc d0{};
  d0.row0 = 0;
  d0.n = c.n;
  APCG_CUDA(cudaMemcpyAsync(P->sys, &d0, sizeof(d0), cudaMemcpyHostToDevice, ctx->stream));
  APCG_CUDA(cudaMallocHost((void**)&P->sres_host, sizeof(SysResult)));
  APCG_CUDA(cudaMallocHost((void**)&P->st_host, sizeof(CgState)));
  {
    std::lock_guard<std::mutex> g(global_mutex());
    P->id = register_memory(ws, total);
  }
  // A0: the Jacobi diagonal, checked once here (a stencil's is the constant 1 / centre).
  OpScope op(ctx);
  if (A) op.read(A->id);
  op.write(P->id);
  APCG_TRY(op.begin());
  if (c.n > 0 && A) APCG_TRY(launch_jacobi_setup(ctx, A, c.dinv));
  if (c.n > 0 && S) APCG_TRY(launch_fill(ctx, c.dinv, c.n, 1.0 / center));
  APCG_TRY(op.finish());
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));
  counters().host_syncs++;
  APCG_TRY(ctx_check_device_error(ctx));
  *out = P.release();
  return APCG_OK;
}

apcg_status cg_plan_enqueue(apcg_cg_plan P, apcg_vec b, apcg_vec x) {
  APCG_TRY(check_solve_args(P, b, x));
  double* xp = static_cast<double*>(x->dptr);
  const double* bp = static_cast<const double*>(b->dptr);
  if (P->mode == APCG_MODE_ASYNC_GRAPH) APCG_TRY(core_build_graph(P->core, xp, P->ctx->stream));
  OpScope op(P->ctx);
  op.read(P->A.id).read(b->id).rw(x->id).rw(P->id);
  APCG_TRY(op.begin());
  apcg_status st = APCG_OK;
  if (P->mode == APCG_MODE_HOST_SYNC)
    st = solve_host_sync(P, bp, xp);
  else if (P->mode == APCG_MODE_PERSISTENT)
    st = enqueue_persistent(P, bp, xp);
  else
    st = enqueue_async(P, bp, xp, P->mode == APCG_MODE_ASYNC_GRAPH);
  apcg_status st2 = op.finish();
  P->pending = (st == APCG_OK);
  return st != APCG_OK ? st : st2;
}

apcg_status cg_plan_finish(apcg_cg_plan P, apcg_cg_result* res) {
  APCG_CHECK(P && res, "NULL argument");
  APCG_CHECK(P->pending, "no solve is pending on this plan");
  if (P->mode != APCG_MODE_HOST_SYNC) APCG_TRY(finish_async(P));
  P->pending = false;
  if (P->mode == APCG_MODE_PERSISTENT) {
    const SysResult& r = *P->sres_host;
    CgState* h = P->st_host;
    h->iter = r.iters;
    h->done = r.done;
    h->rr = r.rr;
    h->bnorm2 = r.bnorm2;
    if (r.done == kDoneBadDiagonal)
      return set_error(APCG_ERR_BAD_DIAGONAL, "Jacobi: a diagonal entry is missing, zero or not finite");
  }
  fill_result(P, res);
  return APCG_OK;
}

}  // namespace
}  // namespace apcg

using namespace apcg;

extern "C" {

apcg_status apcg_cg_opts_default(apcg_cg_opts* o) {
  APCG_CHECK(o, "opts is NULL");
  memset(o, 0, sizeof(*o));
  o->rtol = 1e-8;
  o->atol = 0.0;
  o->max_it = 0;
  o->check_every = 1;
  o->mode = APCG_MODE_AUTO;
  return APCG_OK;
}

apcg_status apcg_cg_plan_create(apcg_ctx ctx_in, apcg_mat A, const apcg_cg_opts* opts, apcg_cg_plan* out) {
  APCG_CHECK(A && out, "NULL argument");
  APCG_CHECK(A->dtype == APCG_F64 && A->nrows == A->ncols, "the CG solver takes a square float64 matrix");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  return cg_plan_create(ctx, A, nullptr, opts, out);
}

apcg_status apcg_cg_plan_create_stencil(apcg_ctx ctx_in, apcg_stencil S, const apcg_cg_opts* opts,
                                        apcg_cg_plan* out) {
  APCG_CHECK(S && out, "NULL argument");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  return cg_plan_create(ctx, nullptr, S, opts, out);
}

apcg_status apcg_cg_plan_solve(apcg_cg_plan P, apcg_vec b, apcg_vec x, apcg_cg_result* res) {
  APCG_CHECK(res, "res is NULL");
  APCG_TRY(cg_plan_enqueue(P, b, x));
  return cg_plan_finish(P, res);
}

apcg_status apcg_cg_plan_solve_async(apcg_cg_plan P, apcg_vec b, apcg_vec x) { return cg_plan_enqueue(P, b, x); }

apcg_status apcg_cg_plan_result(apcg_cg_plan P, apcg_cg_result* res) { return cg_plan_finish(P, res); }

apcg_status apcg_cg_plan_destroy(apcg_cg_plan P) { return cg_plan_destroy(P); }

apcg_status apcg_cg_plan_layout(apcg_cg_plan P, apcg_plan_layout* out) {
  APCG_CHECK(P && out, "plan or out is NULL");
  const auto& A = P->core.A;
  describe_layout(A.sptr != nullptr, dev::col_format(A), A.long_rows, A.nslices, P->padded, out);
  return APCG_OK;
}

apcg_status apcg_cg_plan_profile(apcg_cg_plan P, apcg_vec b, apcg_vec x, int32_t iters, float* ms) {
  APCG_TRY(check_solve_args(P, b, x));
  APCG_CHECK(iters >= 1 && ms, "iters must be >= 1 and ms non-NULL");
  cudaStream_t s = P->ctx->stream;
  OpScope op(P->ctx);
  op.read(P->A.id).read(b->id).rw(x->id).rw(P->id);
  APCG_TRY(op.begin());
  double* xp = static_cast<double*>(x->dptr);
  // Run past any convergence test: no tolerance and a large cap.
  CgCore<double> c = P->core;
  c.max_it = 1 << 30;
  APCG_TRY(core_setup_f64(c, static_cast<const double*>(b->dptr), xp, 0.0, 0.0, s));
  cudaEvent_t ev[4];
  for (auto& e : ev) APCG_CUDA(cudaEventCreate(&e));
  float tot[3] = {0.f, 0.f, 0.f};
  apcg_status st = APCG_OK;
  for (int32_t i = 0; i < iters && st == APCG_OK; ++i) {
    cudaEventRecord(ev[0], s);
    st = core_k1(c, xp, s, false);
    cudaEventRecord(ev[1], s);
    if (st == APCG_OK) st = core_k2(c, xp, s, false, 0.0, 0, 0);
    cudaEventRecord(ev[2], s);
    if (st == APCG_OK) st = core_k3(c, xp, s, false, 0.0);
    cudaEventRecord(ev[3], s);
    cudaEventSynchronize(ev[3]);
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      tot[k] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  count_kernels(1 + 3 * (int64_t)iters);
  APCG_TRY(st);
  for (int k = 0; k < 3; ++k) ms[k] = tot[k] / iters;
  return op.finish();
}

apcg_status apcg_cg_solve(apcg_ctx ctx_in, apcg_mat A, apcg_vec b, apcg_vec x, const apcg_cg_opts* opts,
                          apcg_cg_result* res) {
  APCG_CHECK(res && A, "NULL argument");
  APCG_TRY(check_vectors(A->nrows, b, x));  // before the plan does any work
  apcg_cg_plan P = nullptr;
  APCG_TRY(apcg_cg_plan_create(ctx_in, A, opts, &P));
  apcg_status st = apcg_cg_plan_solve(P, b, x, res);
  cg_plan_destroy(P);
  return st;
}

apcg_status apcg_cg_solve_host(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col, const double* val,
                               const double* b, double* x, const apcg_cg_opts* opts, apcg_cg_result* res) {
  APCG_CHECK(n >= 0 && nnz >= 0, "negative size");
  APCG_CHECK(rowptr && (nnz == 0 || (col && val)) && (n == 0 || (b && x)) && res, "NULL argument");
  apcg_ctx ctx = host_api_ctx();
  APCG_CHECK(ctx, "could not create the library context: %s", apcg_last_error_string());
  cudaStream_t s = ctx->stream;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t brp = up(sizeof(int32_t) * ((size_t)n + 1)), bcol = up(sizeof(int32_t) * (size_t)nnz),
               bval = up(sizeof(double) * (size_t)nnz), bvec = up(sizeof(double) * (size_t)n);
  char* d = nullptr;
  APCG_TRY(dev_alloc_async((void**)&d, brp + bcol + bval + 2 * bvec + 256, s));
  int32_t* d_rp = reinterpret_cast<int32_t*>(d);
  int32_t* d_col = reinterpret_cast<int32_t*>(d + brp);
  double* d_val = reinterpret_cast<double*>(d + brp + bcol);
  double* d_b = reinterpret_cast<double*>(d + brp + bcol + bval);
  double* d_x = reinterpret_cast<double*>(d + brp + bcol + bval + bvec);
  APCG_CUDA(cudaMemcpyAsync(d_rp, rowptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
  if (nnz) {
    APCG_CUDA(cudaMemcpyAsync(d_col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
    APCG_CUDA(cudaMemcpyAsync(d_val, val, sizeof(double) * (size_t)nnz, cudaMemcpyHostToDevice, s));
  }
  if (n) {
    APCG_CUDA(cudaMemcpyAsync(d_b, b, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s));
    APCG_CUDA(cudaMemcpyAsync(d_x, x, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s));
  }
  counters().h2d_copies += 5;
  counters().h2d_bytes += (int64_t)(sizeof(int32_t) * ((size_t)n + 1 + nnz) + sizeof(double) * (nnz + 2 * (size_t)n));
  apcg_mat A = nullptr;
  apcg_vec vb = nullptr, vx = nullptr;
  apcg_status st = apcg_mat_csr_wrap(d_rp, d_col, d_val, n, n, nnz, APCG_F64, &A);
  if (st == APCG_OK) st = apcg_vec_wrap(d_b, n, APCG_F64, &vb);
  if (st == APCG_OK) st = apcg_vec_wrap(d_x, n, APCG_F64, &vx);
  if (st == APCG_OK) st = apcg_cg_solve(ctx, A, vb, vx, opts, res);
  if (st == APCG_OK && n) {
    cudaError_t e = cudaMemcpyAsync(x, d_x, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "copy of x to the host", __FILE__, __LINE__);
    counters().d2h_copies++;
    counters().d2h_bytes += (int64_t)(sizeof(double) * (size_t)n);
  }
  if (vb) apcg_vec_destroy(vb);
  if (vx) apcg_vec_destroy(vx);
  if (A) apcg_mat_destroy(A);
  {
    std::lock_guard<std::mutex> g(global_mutex());
    reg_forget_memory(d_rp);
    reg_forget_memory(d_b);
    reg_forget_memory(d_x);
  }
  cudaFreeAsync(d, s);
  return st;
}

}  // extern "C"
