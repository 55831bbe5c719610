// Batched Jacobi-PCG: many independent systems, one cluster per system.
//
// Systems are bucketed by size (n in (2^(k-1), 2^k]); each bucket is one
// launch of the whole-solve cluster kernel (cluster_cg.cu) with its own
// launch shape, a persistent grid of clusters that pull systems from a device
// work queue longest first.  All bucket launches of a solve are captured once
// into a CUDA graph as parallel branches, so a batch solve is one graph
// launch and the buckets share the GPU.  The launch shape of each bucket
// (CTAs per cluster; threads per CTA and rows per thread follow from it) comes
// from a rows-per-CTA target, chosen by a built-in default or by the
// autotuner, which times every candidate on the bucket's own systems.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "cluster_cg.hpp"

namespace {

constexpr int kMaxSystemRows = 65536;
constexpr int kDefaultRowsPerCta = 1024;
const int kTuneTargets[] = {256, 512, 1024, 2048, 4096};

struct BatchClass {
  int bucket = 0;
  int n_lo = 0, n_hi = 0;  // smallest and largest n of its systems
  std::vector<int32_t> sys;  // system ids, longest first
  apcg::ClusterShape shape;
  int target = kDefaultRowsPerCta;
  int nclusters = 1;
  int32_t* d_order = nullptr;
  unsigned int* d_next = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float tuned_ms = -1.f;
};

}  // namespace

struct apcg_batch_plan_s {
  apcg_ctx ctx = nullptr;
  int32_t nsys = 0;
  int64_t N = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  const float* val32 = nullptr;  // refinement: float32 values (or nullptr: val rounded in the kernel)
  bool ir = false;               // mixed-precision refinement per system
  apcg_cg_opts opts{};
  apcg_ir_opts iropts{};
  std::vector<int32_t> n;
  std::vector<BatchClass> classes;
  char* ws = nullptr;
  apcg::SysDesc* d_sys = nullptr;
  apcg::SysResult* d_res = nullptr;
  int32_t hist_len = 0;          // float64 CG: alpha/beta of the first hist_len iterations of every system
  double* d_hist = nullptr;      // [2 * nsys * hist_len]: alpha of all systems, then beta
  apcg::SysResult* h_res = nullptr;
  cudaEvent_t start = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double* gb = nullptr;
  double* gx = nullptr;
  apcg_id id = 0;
  bool pending = false;
};

namespace apcg {
namespace {

ClusterShape shape_for_target(int n_hi, int target, bool ir) {
  int C = 1;
  while (C < 16 && cluster_rows_per_cta(n_hi, C) > target) C *= 2;
  return schedulable_shape(n_hi, C, ir);
}

ClusterArgs class_args(apcg_batch_plan P, const BatchClass& c, const double* b, double* x) {
  ClusterArgs a{};
  a.rowptr = P->rowptr;
  a.col = P->col;
  a.val = P->val;
  a.dinv = nullptr;
  a.b = b;
  a.x = x;
  a.sys = P->d_sys;
  a.order = c.d_order;
  a.nsys = (int32_t)c.sys.size();
  a.check_every = P->opts.check_every;
  a.next = c.d_next;
  a.res = P->d_res;
  a.rtol = P->opts.rtol;
  a.atol = P->opts.atol;
  a.max_it = P->opts.max_it;
  a.hist_len = P->hist_len;
  a.alpha_h = P->d_hist;
  a.beta_h = P->d_hist ? P->d_hist + (int64_t)P->nsys * P->hist_len : nullptr;
  if (P->ir) {
    a.val32 = P->val32;
    a.rtol = P->iropts.rtol;
    a.atol = P->iropts.atol;
    a.max_it = P->iropts.max_inner;
    a.check_every = P->iropts.inner_check_every;
    a.rtol_inner = P->iropts.rtol_inner;
    a.max_outer = P->iropts.max_outer;
  }
  return a;
}

void set_shape(BatchClass& c, const ClusterShape& sh) {
  c.shape = sh;
  c.nclusters = std::max(1, std::min((int)c.sys.size(), max_active_clusters(sh)));
}

apcg_status capture_graph(apcg_batch_plan P, const double* b, double* x) {
  if (P->exec && P->gb == b && P->gx == x) return APCG_OK;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->exec = nullptr;
  P->graph = nullptr;
  cudaStream_t s = P->ctx->stream;
  cudaStream_t cap = nullptr;
  APCG_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(P->start, cap);
  for (BatchClass& c : P->classes) {
    if (e != cudaSuccess) break;
    e = cudaStreamWaitEvent(c.stream, P->start, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.d_next, 0, sizeof(unsigned int), c.stream);
    if (e == cudaSuccess) e = launch_cluster_cg(class_args(P, c, b, x), c.shape, c.nclusters, c.stream);
    if (e == cudaSuccess) e = cudaEventRecord(c.done, c.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, c.done, 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_error(e, "batched graph capture", __FILE__, __LINE__);
  }
  if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
  P->graph = g;
  APCG_CUDA(cudaGraphInstantiate(&P->exec, g, 0));
  APCG_CUDA(cudaGraphUpload(P->exec, s));
  P->gb = b;
  P->gx = x;
  (void)s;
  return APCG_OK;
}

void destroy_plan(apcg_batch_plan P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  cudaStream_t s = P->ctx ? P->ctx->stream : nullptr;
  for (BatchClass& c : P->classes) {
    if (c.stream) cudaStreamDestroy(c.stream);
    if (c.done) cudaEventDestroy(c.done);
  }
  if (P->start) cudaEventDestroy(P->start);
  if (P->ws) {
    {
      std::lock_guard<std::mutex> g(global_mutex());
      reg_forget_memory(P->ws);
    }
    cudaFreeAsync(P->ws, s);
  }
  if (P->h_res) {
    cudaStreamSynchronize(s);
    cudaFreeHost(P->h_res);
  }
  delete P;
}

}  // namespace
}  // namespace apcg

using namespace apcg;

extern "C" {

}  // extern "C"

namespace {

apcg_status create_plan(apcg_ctx ctx_in, int32_t nsys, const int32_t* sys_row_off, const int32_t* rowptr,
                        const int32_t* col, const double* val, const float* val32, const apcg_cg_opts* opts,
                        const apcg_ir_opts* iropts, apcg_batch_plan* out) {
  APCG_CHECK(out && sys_row_off && rowptr, "NULL argument");
  APCG_CHECK(nsys >= 1, "nsys must be >= 1");
  APCG_CHECK(sys_row_off[0] == 0, "sys_row_off[0] must be 0");
  for (int32_t s = 0; s < nsys; ++s) {
    const int64_t ns = (int64_t)sys_row_off[s + 1] - sys_row_off[s];
    APCG_CHECK(ns >= 0, "sys_row_off decreases at system %d", s);
    APCG_CHECK(ns <= kMaxSystemRows, "system %d has %lld rows; at most %d are supported", s, (long long)ns,
               kMaxSystemRows);
  }
  apcg_cg_opts o;
  if (opts)
    o = *opts;
  else
    apcg_cg_opts_default(&o);
  APCG_CHECK(o.check_every >= 1 && o.rtol >= 0.0 && o.atol >= 0.0 && o.history_len >= 0, "bad options");
  if (iropts) {
    APCG_CHECK(iropts->rtol >= 0.0 && iropts->atol >= 0.0 && iropts->max_outer >= 0 && iropts->max_inner >= 1 &&
                   iropts->inner_check_every >= 1 && iropts->rtol_inner >= 0.0f && iropts->rtol_inner < 1.0f,
               "bad refinement options");
    APCG_CHECK(val || val32 || sys_row_off[nsys] == 0, "refinement needs float64 or float32 values");
  } else {
    APCG_CHECK(val || sys_row_off[nsys] == 0, "val is NULL");
  }
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  std::unique_ptr<apcg_batch_plan_s, void (*)(apcg_batch_plan)> P(new apcg_batch_plan_s(), destroy_plan);
  P->ctx = ctx;
  P->nsys = nsys;
  P->N = sys_row_off[nsys];
  P->rowptr = rowptr;
  P->col = col;
  P->val = val;
  P->val32 = val32;
  P->ir = iropts != nullptr;
  if (iropts) P->iropts = *iropts;
  P->opts = o;
  P->hist_len = iropts ? 0 : o.history_len;
  P->n.resize(nsys);
  std::vector<SysDesc> desc(nsys);
  for (int32_t s = 0; s < nsys; ++s) {
    P->n[s] = sys_row_off[s + 1] - sys_row_off[s];
    desc[s].row0 = sys_row_off[s];
    desc[s].n = P->n[s];
    desc[s].pad = 0;
  }
  // Buckets by size, systems longest first inside each.
  std::vector<int32_t> ids(nsys);
  for (int32_t s = 0; s < nsys; ++s) ids[s] = s;
  std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t b) { return P->n[a] > P->n[b]; });
  for (int32_t s : ids) {
    const int nn = std::max(1, P->n[s]);
    int bucket = 0;
    while ((1 << bucket) < nn) ++bucket;
    if (P->classes.empty() || P->classes.back().bucket != bucket) {
      BatchClass c;
      c.bucket = bucket;
      c.n_hi = P->n[s];
      P->classes.push_back(c);
    }
    P->classes.back().sys.push_back(s);
    P->classes.back().n_lo = P->n[s];
  }
  // Device block: descriptors, results, per-class orders and counters.
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t b_desc = up(sizeof(SysDesc) * nsys), b_res = up(sizeof(SysResult) * nsys);
  size_t b_cls = 0;
  for (auto& c : P->classes) b_cls += up(sizeof(int32_t) * c.sys.size()) + 256;
  const size_t b_hist = up(sizeof(double) * 2 * (size_t)nsys * (size_t)P->hist_len);
  char* ws = nullptr;
  APCG_TRY(dev_alloc_async((void**)&ws, b_desc + b_res + b_cls + b_hist, ctx->stream));
  P->ws = ws;
  P->d_sys = reinterpret_cast<SysDesc*>(ws);
  P->d_res = reinterpret_cast<SysResult*>(ws + b_desc);
  if (P->hist_len > 0) P->d_hist = reinterpret_cast<double*>(ws + b_desc + b_res + b_cls);
  char* q = ws + b_desc + b_res;
  APCG_CUDA(cudaMemcpyAsync(P->d_sys, desc.data(), sizeof(SysDesc) * nsys, cudaMemcpyHostToDevice, ctx->stream));
  for (auto& c : P->classes) {
    c.d_order = reinterpret_cast<int32_t*>(q);
    q += up(sizeof(int32_t) * c.sys.size());
    c.d_next = reinterpret_cast<unsigned int*>(q);
    q += 256;
    APCG_CUDA(cudaMemcpyAsync(c.d_order, c.sys.data(), sizeof(int32_t) * c.sys.size(), cudaMemcpyHostToDevice,
                              ctx->stream));
    APCG_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    APCG_CUDA(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
    const ClusterShape sh = shape_for_target(c.n_hi, kDefaultRowsPerCta, P->ir);
    if (!sh.ok) return set_error(APCG_ERR_UNSUPPORTED, "no schedulable cluster shape for systems of %d rows", c.n_hi);
    set_shape(c, sh);
  }
  APCG_CUDA(cudaEventCreateWithFlags(&P->start, cudaEventDisableTiming));
  APCG_CUDA(cudaMallocHost((void**)&P->h_res, sizeof(SysResult) * nsys));
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));  // the host arrays above are temporaries
  counters().h2d_copies += 1 + (int64_t)P->classes.size();
  {
    std::lock_guard<std::mutex> g(global_mutex());
    P->id = register_memory(ws, b_desc + b_res + b_cls + b_hist);
  }
  *out = P.release();
  return APCG_OK;
}

}  // namespace

extern "C" {

apcg_status apcg_batch_plan_create(apcg_ctx ctx, int32_t nsys, const int32_t* sys_row_off, const int32_t* rowptr,
                                   const int32_t* col, const double* val, const apcg_cg_opts* opts,
                                   apcg_batch_plan* out) {
  return create_plan(ctx, nsys, sys_row_off, rowptr, col, val, nullptr, opts, nullptr, out);
}

apcg_status apcg_batch_ir_plan_create(apcg_ctx ctx, int32_t nsys, const int32_t* sys_row_off, const int32_t* rowptr,
                                      const int32_t* col, const double* val, const float* val32,
                                      const apcg_ir_opts* opts, apcg_batch_plan* out) {
  apcg_ir_opts o;
  if (opts)
    o = *opts;
  else
    apcg_ir_opts_default(&o);
  return create_plan(ctx, nsys, sys_row_off, rowptr, col, val, val32, nullptr, &o, out);
}

apcg_status apcg_batch_plan_solve(apcg_batch_plan P, const double* b, double* x, apcg_batch_result* results) {
  APCG_CHECK(P, "plan is NULL");
  APCG_CHECK(P->N == 0 || (b && x), "b or x is NULL");
  APCG_TRY(capture_graph(P, b, x));
  apcg_id idb, idx;
  {
    std::lock_guard<std::mutex> g(global_mutex());
    idb = register_memory(b, sizeof(double) * (size_t)P->N);
    idx = register_memory(x, sizeof(double) * (size_t)P->N);
  }
  OpScope op(P->ctx);
  op.read(idb).rw(idx).rw(P->id);
  APCG_TRY(op.begin());
  if (P->d_hist)  // iterations a system does not reach stay NaN (all bits set)
    APCG_CUDA(cudaMemsetAsync(P->d_hist, 0xff, sizeof(double) * 2 * (size_t)P->nsys * P->hist_len, P->ctx->stream));
  APCG_CUDA(cudaGraphLaunch(P->exec, P->ctx->stream));
  counters().graph_launches++;
  count_kernels((int64_t)P->classes.size());
  APCG_TRY(op.finish());
  if (!results) return APCG_OK;
  APCG_CUDA(cudaMemcpyAsync(P->h_res, P->d_res, sizeof(SysResult) * P->nsys, cudaMemcpyDeviceToHost,
                            P->ctx->stream));
  APCG_CUDA(cudaStreamSynchronize(P->ctx->stream));
  counters().d2h_copies++;
  counters().d2h_bytes += (int64_t)(sizeof(SysResult) * P->nsys);
  counters().host_syncs++;
  for (int32_t s = 0; s < P->nsys; ++s) {
    const SysResult& r = P->h_res[s];
    apcg_batch_result& o = results[s];
    o.iters = r.iters;
    o.reason = r.done == kDoneConverged       ? APCG_CONVERGED
               : r.done == kDoneNotConverged  ? APCG_NOT_CONVERGED
               : r.done == kDoneBadDiagonal   ? APCG_BAD_DIAGONAL
                                              : APCG_BREAKDOWN;
    const double bn = std::sqrt(r.bnorm2);
    o.rel_res = bn > 0.0 ? std::sqrt(r.rr) / bn : std::sqrt(r.rr);
    o.outer = r.outer;
    o.pad = 0;
  }
  return APCG_OK;
}

apcg_status apcg_batch_plan_tune(apcg_batch_plan P, const double* b, char* table, size_t cap) {
  APCG_CHECK(P, "plan is NULL");
  APCG_CHECK(P->N == 0 || b, "b is NULL");
  cudaStream_t s = P->ctx->stream;
  double* xs = nullptr;
  APCG_TRY(dev_alloc_async((void**)&xs, sizeof(double) * (size_t)std::max<int64_t>(P->N, 1), s));
  cudaEvent_t e0, e1;
  APCG_CUDA(cudaEventCreate(&e0));
  APCG_CUDA(cudaEventCreate(&e1));
  std::string out;
  apcg_status st = APCG_OK;
  for (BatchClass& c : P->classes) {
    ClusterShape best_shape = c.shape;
    int best_target = c.target;
    float best = -1.f;
    ClusterShape tried[8];
    int ntried = 0;
    for (int target : kTuneTargets) {
      const ClusterShape sh = shape_for_target(c.n_hi, target, P->ir);
      if (!sh.ok) continue;
      bool dup = false;
      for (int i = 0; i < ntried; ++i) dup |= tried[i].C == sh.C;
      if (dup) continue;
      tried[ntried++] = sh;
      set_shape(c, sh);
      float ms_best = 1e30f;
      for (int rep = 0; rep < 2 && st == APCG_OK; ++rep) {  // the first run warms caches
        cudaError_t e = cudaMemsetAsync(xs, 0, sizeof(double) * (size_t)P->N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c.d_next, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_cluster_cg(class_args(P, c, b, xs), c.shape, c.nclusters, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) st = cuda_error(e, "autotune launch", __FILE__, __LINE__);
        count_kernels(1);
        if (rep == 1) ms_best = ms;
      }
      if (st != APCG_OK) break;
      if (best < 0.f || ms_best < best) {
        best = ms_best;
        best_shape = sh;
        best_target = target;
      }
    }
    if (st != APCG_OK) break;
    c.target = best_target;
    c.tuned_ms = best;
    set_shape(c, best_shape);
    char line[160];
    snprintf(line, sizeof(line), "%d %d %d %d %d %.4f\n", c.n_lo, c.n_hi, c.shape.C, c.shape.tpb, c.shape.R, best);
    out += line;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(xs, s);
  if (P->exec) {  // shapes changed: capture again at the next solve
    cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    P->gb = nullptr;
    P->gx = nullptr;
  }
  APCG_TRY(st);
  if (table && cap) {
    const size_t nb = std::min(cap - 1, out.size());
    memcpy(table, out.data(), nb);
    table[nb] = '\0';
  }
  return APCG_OK;
}

apcg_status apcg_batch_plan_history(apcg_batch_plan P, int32_t sys, double* alpha, double* beta) {
  APCG_CHECK(P, "plan is NULL");
  APCG_CHECK(P->hist_len > 0, "the plan records no history (float64 CG plans with opts.history_len > 0 only)");
  APCG_CHECK(sys >= 0 && sys < P->nsys, "system %d outside [0, %d)", sys, P->nsys);
  const size_t H = (size_t)P->hist_len;
  cudaStream_t s = P->ctx->stream;
  OpScope op(P->ctx);
  op.read(P->id);
  APCG_TRY(op.begin());
  if (alpha) APCG_CUDA(cudaMemcpyAsync(alpha, P->d_hist + (size_t)sys * H, sizeof(double) * H, cudaMemcpyDeviceToHost, s));
  if (beta)
    APCG_CUDA(cudaMemcpyAsync(beta, P->d_hist + ((size_t)P->nsys + sys) * H, sizeof(double) * H, cudaMemcpyDeviceToHost,
                              s));
  APCG_TRY(op.finish());
  APCG_CUDA(cudaStreamSynchronize(s));
  counters().d2h_copies += (alpha ? 1 : 0) + (beta ? 1 : 0);
  counters().host_syncs++;
  return APCG_OK;
}

apcg_status apcg_batch_plan_destroy(apcg_batch_plan P) {
  APCG_CHECK(P, "plan is NULL");
  destroy_plan(P);
  return APCG_OK;
}

apcg_status apcg_cg_solve_batched(apcg_ctx ctx, int32_t nsys, const int32_t* sys_row_off, const int32_t* rowptr,
                                  const int32_t* col, const double* val, const double* b, double* x,
                                  const apcg_cg_opts* opts, apcg_batch_result* results) {
  apcg_batch_plan P = nullptr;
  APCG_TRY(apcg_batch_plan_create(ctx, nsys, sys_row_off, rowptr, col, val, opts, &P));
  apcg_status st = apcg_batch_plan_solve(P, b, x, results);
  if (st == APCG_OK && !results) st = apcg_ctx_synchronize(P->ctx);
  destroy_plan(P);
  return st;
}

}  // extern "C"
