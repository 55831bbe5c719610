// Jacobi-preconditioned conjugate gradient on one device context.
//
// The method is textbook Hestenes-Stiefel PCG with diagonal scaling (Sec. 4.1,
// 4.2), its loop body in the order of the mixed-API CG example of Sec. 3.3:
//   w = A p;  gamma = (p,w);  alpha = rho / gamma
//   x += alpha p;  r -= alpha w;  z = D^-1 r;  rho' = (r,z);  rr = (r,r)
//   convergence test every k-th iteration:  sqrt(rr) <= max(rtol ||b||, atol)
//   beta = rho' / rho;  p = z + beta p;  rho = rho'
// with the standard start r = b - A x0, z = D^-1 r, p = z (the paper omits it).
//
// One iteration is three kernels, each fusing the work between two global
// reductions:
//   K1  w = A p and the partial sums of (p,w); the last block forms gamma
//       and alpha = rho / gamma (or flags a breakdown);
//   K2  x += alpha p, r -= alpha w, z = D^-1 r on the fly (never stored), the
//       partial sums of (r,z) and (r,r); the last block counts the
//       iteration, runs the convergence test and forms beta;
//   K3  p = D^-1 r + beta p.
// alpha, beta, rho and the residual norm live in a device state block; every
// kernel starts by reading the 'done' word and returns at once when the solve
// has finished, so work enqueued past convergence costs one launch each (the
// semaphore idea of Sec. 5).  Modes: HOST_SYNC (scalars round-trip through
// the host every iteration), ASYNC (launches back to back, host reads 'done'
// every k iterations), ASYNC_GRAPH (k iterations captured once; a conditional
// while node repeats them on the device until 'done').
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "kernels_common.cuh"
#include "spmv.cuh"

namespace apcg {

namespace {

constexpr int kThreads = 256;
constexpr int kPersistentMaxRows = 65536;  // one cluster of 16 CTAs x 512 threads x 8 rows
constexpr int kUpdV = 2;   // double2 pairs per thread in the update kernel
constexpr int kAypxV = 4;  // double2 pairs per thread in the search-direction kernel

// ------------------------------------------------------------------ kernels

struct CgArgs {
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ col;
  const double* __restrict__ val;
  int32_t n;
  const double* __restrict__ dinv;
  double* x;
  double* r;
  double* p;
  double* w;
  double* z;
  CgState* st;
  double* partials;
  double* alpha_h;
  double* beta_h;
};

__device__ __forceinline__ int32_t read_done(const CgState* st) { return *(volatile const int32_t*)&st->done; }

// r = b - A x0, z = D^-1 r, p = z; rho = (r,z), rr = (r,r), bb = (b,b).
template <int U>
__global__ void __launch_bounds__(kThreads) cg_setup_kernel(CgArgs a, const double* __restrict__ b, double rtol,
                                                            double atol, int32_t max_it, int32_t k,
                                                            int32_t hist_len) {
  __shared__ dev::SpmvSmem<U, double> sm[kThreads / 32];
  __shared__ double red[3 * kThreads];
  double v[3] = {0.0, 0.0, 0.0};
  dev::spmv_warp_tiles<U, false, double>(a.rowptr, a.col, a.val, a.x, a.n, sm[threadIdx.x >> 5].buf,
                                         [&](int32_t i, double ax, double) {
                                    const double bi = __ldg(b + i);
                                    const double ri = bi - ax;
                                    const double zi = __ldg(a.dinv + i) * ri;
                                    a.r[i] = ri;
                                    a.p[i] = zi;
                                    v[0] += ri * zi;
                                    v[1] += ri * ri;
                                    v[2] += bi * bi;
                                  });
  double tot[3];
  if (dev::grid_sum_last<3>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0) {
    CgState* st = a.st;
    st->rho = tot[0];
    st->rr = tot[1];
    st->bnorm2 = tot[2];
    const double tol = fmax(rtol * sqrt(tot[2]), atol);
    st->tol = tol;
    st->iter = 0;
    st->max_it = max_it;
    st->check_every = k;
    st->hist_len = hist_len;
    st->body_runs = 0;
    st->alpha = st->beta = st->gamma = st->rho_new = 0.0;
    st->done = (sqrt(tot[1]) <= tol) ? kDoneConverged : 0;
  }
}

// K1: w = A p; gamma = (p,w); alpha = rho / gamma.
template <int U, bool HOST>
__global__ void __launch_bounds__(kThreads) cg_spmv_dot_kernel(CgArgs a) {
  if (!HOST && read_done(a.st)) return;
  __shared__ dev::SpmvSmem<U, double> sm[kThreads / 32];
  __shared__ double red[kThreads];
  const uint64_t keep = dev::policy_evict_last();
  double v[1] = {0.0};
  dev::spmv_warp_tiles<U, true, double>(a.rowptr, a.col, a.val, a.p, a.n, sm[threadIdx.x >> 5].buf,
                                        [&](int32_t i, double s, double p_i) {
                                          dev::st_hint(a.w + i, s, keep);
                                          v[0] += p_i * s;
                                        });
  double tot[1];
  if (dev::grid_sum_last<1>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0) {
    CgState* st = a.st;
    const double gamma = tot[0];
    st->gamma = gamma;
    if (!HOST) {
      if (!(gamma > 0.0) || !isfinite(gamma)) {
        st->done = kDoneBreakdown;
      } else {
        const double alpha = st->rho / gamma;
        st->alpha = alpha;
        if (st->iter < st->hist_len) a.alpha_h[st->iter] = alpha;
      }
    }
  }
}

// K2: x += alpha p; r -= alpha w; z = D^-1 r (stored for K3); rho' = (r,z);
// on convergence-test iterations also rr = (r,r); then the test and beta.
// The test runs when the iteration count is a multiple of k or reaches max_it,
// decided from the state block at kernel entry, so the same kernel serves
// every position of a captured block.  Without the test the kernel spends
// four float64 operations per row (the float64 pipe is GB300's scarcest
// resource here); (r,r) adds a fifth only when it is needed.
template <bool HOST>
__global__ void __launch_bounds__(kThreads, 4) cg_update_kernel(CgArgs a, double alpha_host,
                                                                cudaGraphConditionalHandle cond, int32_t use_cond) {
  if (!HOST && read_done(a.st)) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      a.st->body_runs += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  const double alpha = HOST ? alpha_host : a.st->alpha;
  bool check = true;
  if (!HOST) {
    const int32_t it = a.st->iter + 1;
    check = (it % a.st->check_every == 0) || it >= a.st->max_it;
  }
  __shared__ double red[2 * kThreads];
  double v[2] = {0.0, 0.0};
  double acc_rz[kUpdV], acc_rr[kUpdV];  // independent chains, combined in a fixed order below
#pragma unroll
  for (int u = 0; u < kUpdV; ++u) acc_rz[u] = acc_rr[u] = 0.0;
  const int64_t n = a.n, np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  double2* x2 = reinterpret_cast<double2*>(a.x);
  double2* r2 = reinterpret_cast<double2*>(a.r);
  double2* z2 = reinterpret_cast<double2*>(a.z);
  const double2* p2 = reinterpret_cast<const double2*>(a.p);
  const double2* w2 = reinterpret_cast<const double2*>(a.w);
  const double2* d2 = reinterpret_cast<const double2*>(a.dinv);
  constexpr int V = kUpdV;  // double2 pairs in flight per thread and array
  const uint64_t keep = dev::policy_evict_last();
  auto sweep = [&](auto with_rr) {
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < np; i0 += V * stride) {
      double2 xx[V], rr[V], pp[V], ww[V], dd[V];
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < np) {
          xx[u] = dev::ld2_hint(x2 + i, keep);
          rr[u] = dev::ld2_hint(r2 + i, keep);
          pp[u] = dev::ld2_nc_hint(p2 + i, keep);
          ww[u] = dev::ld2_nc_hint(w2 + i, keep);
          dd[u] = dev::ld2_nc_hint(d2 + i, keep);
        }
      }
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < np) {
          xx[u].x = fma(alpha, pp[u].x, xx[u].x);
          xx[u].y = fma(alpha, pp[u].y, xx[u].y);
          rr[u].x = fma(-alpha, ww[u].x, rr[u].x);
          rr[u].y = fma(-alpha, ww[u].y, rr[u].y);
          const double2 zz = make_double2(dd[u].x * rr[u].x, dd[u].y * rr[u].y);
          dev::st2_hint(x2 + i, xx[u], keep);
          dev::st2_hint(r2 + i, rr[u], keep);
          dev::st2_hint(z2 + i, zz, keep);
          acc_rz[u] = fma(rr[u].x, zz.x, acc_rz[u]);
          acc_rz[u] = fma(rr[u].y, zz.y, acc_rz[u]);
          if (decltype(with_rr)::value) {
            acc_rr[u] = fma(rr[u].x, rr[u].x, acc_rr[u]);
            acc_rr[u] = fma(rr[u].y, rr[u].y, acc_rr[u]);
          }
        }
      }
    }
  };
  if (check)
    sweep(std::true_type{});
  else
    sweep(std::false_type{});
#pragma unroll
  for (int u = 0; u < kUpdV; ++u) {
    v[0] += acc_rz[u];
    v[1] += acc_rr[u];
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    a.x[i] = fma(alpha, a.p[i], a.x[i]);
    const double ri = fma(-alpha, a.w[i], a.r[i]);
    const double zi = a.dinv[i] * ri;
    a.r[i] = ri;
    a.z[i] = zi;
    v[0] = fma(ri, zi, v[0]);
    if (check) v[1] = fma(ri, ri, v[1]);
  }
  double tot[2];
  if (dev::grid_sum_last<2>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0) {
    CgState* st = a.st;
    const double rz = tot[0], rr = tot[1];
    st->rho_new = rz;
    if (check) st->rr = rr;
    if (!HOST) {
      const int32_t it = st->iter + 1;
      st->iter = it;
      int32_t done = 0;
      // An exactly zero residual ends the solve at any iteration; between
      // tests (r, D^-1 r) = 0 stands for r = 0 (D^-1 is positive).
      if ((check && rr == 0.0) || rz == 0.0)
        done = kDoneConverged;
      else if (check && sqrt(rr) <= st->tol)
        done = kDoneConverged;
      else if (it >= st->max_it)
        done = kDoneNotConverged;
      else if (!isfinite(rz) || (check && !isfinite(rr)))
        done = kDoneBreakdown;
      if (!done) {
        const double beta = rz / st->rho;
        st->beta = beta;
        st->rho = rz;
        if (it - 1 < st->hist_len) a.beta_h[it - 1] = beta;
      }
      st->done = done;
      if (use_cond) {
        st->body_runs += 1;
        cudaGraphSetConditional(cond, done ? 0u : 1u);
      }
    }
  }
}

// K3: p = z + beta p (one fused multiply-add per row).
template <bool HOST>
__global__ void __launch_bounds__(kThreads, 4) cg_aypx_kernel(CgArgs a, double beta_host) {
  if (!HOST && read_done(a.st)) return;
  const double beta = HOST ? beta_host : a.st->beta;
  const int64_t n = a.n, np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  double2* p2 = reinterpret_cast<double2*>(a.p);
  const double2* z2 = reinterpret_cast<const double2*>(a.z);
  constexpr int V = kAypxV;  // double2 pairs in flight per thread and array
  const uint64_t keep = dev::policy_evict_last();
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < np; i0 += V * stride) {
    double2 pp[V], zz[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < np) {
        pp[u] = dev::ld2_hint(p2 + i, keep);
        zz[u] = dev::ld2_nc_hint(z2 + i, keep);
      }
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < np) {
        pp[u].x = fma(beta, pp[u].x, zz[u].x);
        pp[u].y = fma(beta, pp[u].y, zz[u].y);
        dev::st2_hint(p2 + i, pp[u], keep);
      }
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    a.p[i] = fma(beta, a.p[i], a.z[i]);
  }
}

// ------------------------------------------------------------------ launch helpers

int pick_u(const apcg_mat_s* A) {
  const double avg = A->nrows ? (double)A->nnz / A->nrows : 1.0;
  if (avg <= 4.0) return 4;
  if (avg <= 6.0) return 6;
  return 8;
}

template <class K>
int occupancy_grid(K kernel, int sms, int64_t want) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  int64_t g = (int64_t)per_sm * sms;
  if (want < g) g = want;
  if (g > dev::kMaxPartials) g = dev::kMaxPartials;
  return g < 1 ? 1 : (int)g;
}

CgArgs make_args(apcg_cg_plan P, double* x) {
  CgArgs a;
  a.rowptr = P->A.rowptr;
  a.col = P->A.col;
  a.val = static_cast<const double*>(P->A.val);
  a.n = P->n;
  a.dinv = P->dinv;
  a.x = x;
  a.r = P->r;
  a.p = P->p;
  a.w = P->w;
  a.z = P->z;
  a.st = P->st;
  a.partials = P->partials;
  a.alpha_h = P->alpha_h;
  a.beta_h = P->beta_h;
  return a;
}

template <int U>
apcg_status launch_setup_u(apcg_cg_plan P, const CgArgs& a, const double* b, cudaStream_t s) {
  cg_setup_kernel<U><<<P->grid_spmv, kThreads, 0, s>>>(a, b, P->opts.rtol, P->opts.atol, P->max_it, P->k,
                                                        P->hist_len);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

template <int U, bool HOST>
apcg_status launch_k1_u(apcg_cg_plan P, const CgArgs& a, cudaStream_t s) {
  cg_spmv_dot_kernel<U, HOST><<<P->grid_spmv, kThreads, 0, s>>>(a);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

apcg_status launch_setup(apcg_cg_plan P, const CgArgs& a, const double* b, cudaStream_t s) {
  switch (P->u) {
    case 4: return launch_setup_u<4>(P, a, b, s);
    case 6: return launch_setup_u<6>(P, a, b, s);
    default: return launch_setup_u<8>(P, a, b, s);
  }
}

template <bool HOST>
apcg_status launch_k1(apcg_cg_plan P, const CgArgs& a, cudaStream_t s) {
  switch (P->u) {
    case 4: return launch_k1_u<4, HOST>(P, a, s);
    case 6: return launch_k1_u<6, HOST>(P, a, s);
    default: return launch_k1_u<8, HOST>(P, a, s);
  }
}

template <bool HOST>
apcg_status launch_k2(apcg_cg_plan P, const CgArgs& a, cudaStream_t s, double alpha, cudaGraphConditionalHandle h,
                      int use_cond) {
  cg_update_kernel<HOST><<<P->grid_vec, kThreads, 0, s>>>(a, alpha, h, use_cond);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

template <bool HOST>
apcg_status launch_k3(apcg_cg_plan P, const CgArgs& a, cudaStream_t s, double beta) {
  cg_aypx_kernel<HOST><<<P->grid_vec, kThreads, 0, s>>>(a, beta);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

apcg_status read_state(apcg_cg_plan P, cudaStream_t s) {
  APCG_CUDA(cudaMemcpyAsync(P->st_host, P->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  APCG_CUDA(cudaStreamSynchronize(s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(CgState);
  counters().host_syncs++;
  return APCG_OK;
}

// Capture k iterations into the body of a conditional while node.
apcg_status build_graph(apcg_cg_plan P, double* x) {
  if (P->exec && P->graph_x == x) return APCG_OK;
  if (P->exec) {
    cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
  }
  if (P->graph) {
    cudaGraphDestroy(P->graph);
    P->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  APCG_CUDA(cudaGraphCreate(&g, 0));
  P->graph = g;
  cudaGraphConditionalHandle h;
  APCG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  APCG_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const CgArgs a = make_args(P, x);
  APCG_CUDA(cudaStreamBeginCaptureToGraph(P->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  apcg_status st = APCG_OK;
  for (int j = 0; j < P->k && st == APCG_OK; ++j) {
    st = launch_k1<false>(P, a, P->cap_stream);
    if (st == APCG_OK) st = launch_k2<false>(P, a, P->cap_stream, 0.0, h, j == P->k - 1 ? 1 : 0);
    if (st == APCG_OK) st = launch_k3<false>(P, a, P->cap_stream, 0.0);
  }
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(P->cap_stream, &captured);
  if (st != APCG_OK) return st;
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  APCG_CUDA(cudaGraphInstantiate(&P->exec, g, 0));
  APCG_CUDA(cudaGraphUpload(P->exec, P->ctx->stream));
  P->graph_x = x;
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
apcg_status solve_host_sync(apcg_cg_plan P, const CgArgs& a, const double* b) {
  cudaStream_t s = P->ctx->stream;
  CgState* h = P->st_host;
  APCG_TRY(launch_setup(P, a, b, s));
  int64_t launches = 1;
  APCG_TRY(read_state(P, s));
  double rho = h->rho;
  const double tol = h->tol;
  int32_t done = h->done, it = 0;
  std::vector<double> ah, bh;
  while (!done) {
    APCG_TRY(launch_k1<true>(P, a, s));
    APCG_TRY(read_state(P, s));
    const double gamma = h->gamma;
    if (!(gamma > 0.0) || !std::isfinite(gamma)) {
      done = kDoneBreakdown;
      launches += 1;
      break;
    }
    const double alpha = rho / gamma;
    if (it < P->hist_len) ah.push_back(alpha);
    APCG_TRY(launch_k2<true>(P, a, s, alpha, 0, 0));
    APCG_TRY(read_state(P, s));
    launches += 2;
    ++it;
    const double rr = h->rr, rz = h->rho_new;
    if (rr == 0.0 || ((it % P->k == 0 || it == P->max_it) && std::sqrt(rr) <= tol)) {
      done = kDoneConverged;
    } else if (it >= P->max_it) {
      done = kDoneNotConverged;
    } else if (!std::isfinite(rr)) {
      done = kDoneBreakdown;
    } else {
      const double beta = rz / rho;
      if (it - 1 < P->hist_len) bh.push_back(beta);
      rho = rz;
      APCG_TRY(launch_k3<true>(P, a, s, beta));
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

apcg_status enqueue_async(apcg_cg_plan P, const CgArgs& a, const double* b, bool graph) {
  cudaStream_t s = P->ctx->stream;
  APCG_TRY(launch_setup(P, a, b, s));
  count_kernels(1);
  if (graph) {
    APCG_CUDA(cudaGraphLaunch(P->exec, s));
    counters().graph_launches++;
  } else {
    // Launch k iterations at a time and read 'done' after each block.
    const int64_t max_blocks = (int64_t)P->max_it / P->k + 2;
    int64_t launches = 1;
    for (int64_t blk = 0; blk < max_blocks; ++blk) {
      for (int j = 0; j < P->k; ++j) {
        APCG_TRY(launch_k1<false>(P, a, s));
        APCG_TRY(launch_k2<false>(P, a, s, 0.0, 0, 0));
        APCG_TRY(launch_k3<false>(P, a, s, 0.0));
      }
      launches += 3 * P->k;
      count_kernels(3 * P->k);
      APCG_TRY(read_state(P, s));
      if (P->st_host->done) break;
    }
    P->last_launches = launches;
  }
  APCG_CUDA(cudaMemcpyAsync(P->st_host, P->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(CgState);
  return APCG_OK;
}

// The whole solve in one cluster launch (small systems).
apcg_status enqueue_persistent(apcg_cg_plan P, const double* b, double* x) {
  cudaStream_t s = P->ctx->stream;
  ClusterArgs ca{};
  ca.rowptr = P->A.rowptr;
  ca.col = P->A.col;
  ca.val = static_cast<const double*>(P->A.val);
  ca.dinv = P->dinv;
  ca.b = b;
  ca.x = x;
  ca.sys = P->sys;
  ca.order = nullptr;
  ca.nsys = 1;
  ca.check_every = P->k;
  ca.next = P->next;
  ca.res = P->sres;
  ca.rtol = P->opts.rtol;
  ca.atol = P->opts.atol;
  ca.max_it = P->max_it;
  ca.hist_len = P->hist_len;
  ca.alpha_h = P->alpha_h;
  ca.beta_h = P->beta_h;
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
  if (P->mode == APCG_MODE_ASYNC_GRAPH) {
    const int64_t n = (int64_t)P->st_host->body_runs * 3 * P->k;
    count_kernels(n);
    P->last_launches = 1 + n;
  }
  if (P->hist_len > 0) {
    if (P->opts.alpha_hist)
      APCG_CUDA(cudaMemcpy(P->opts.alpha_hist, P->alpha_h, sizeof(double) * P->hist_len, cudaMemcpyDeviceToHost));
    if (P->opts.beta_hist)
      APCG_CUDA(cudaMemcpy(P->opts.beta_hist, P->beta_h, sizeof(double) * P->hist_len, cudaMemcpyDeviceToHost));
    counters().d2h_copies += 2;
  }
  return APCG_OK;
}

apcg_status check_solve_args(apcg_cg_plan P, apcg_vec b, apcg_vec x) {
  APCG_CHECK(P, "plan is NULL");
  APCG_CHECK(b && x, "b or x is NULL");
  APCG_CHECK(b->dtype == APCG_F64 && x->dtype == APCG_F64, "b and x must be float64");
  APCG_CHECK(b->n == P->n && x->n == P->n, "b/x length differs from the matrix size %d", P->n);
  APCG_CHECK(P->n == 0 || (aligned16(b->dptr) && aligned16(x->dptr)), "b/x must be 16-byte aligned");
  APCG_CHECK(b->dptr != x->dptr || P->n == 0, "b and x must not alias");
  return APCG_OK;
}

}  // namespace

apcg_status cg_plan_create(apcg_ctx ctx, apcg_mat A, const apcg_cg_opts* opts, apcg_cg_plan* out) {
  APCG_CHECK(A && out, "NULL argument");
  APCG_CHECK(A->dtype == APCG_F64, "the CG solver takes a float64 matrix");
  APCG_CHECK(A->nrows == A->ncols, "the matrix must be square");
  apcg_cg_opts o;
  if (opts)
    o = *opts;
  else
    apcg_cg_opts_default(&o);
  APCG_CHECK(o.check_every >= 1, "check_every must be >= 1");
  APCG_CHECK(o.rtol >= 0.0 && o.atol >= 0.0, "tolerances must be non-negative");
  APCG_CHECK(o.history_len >= 0, "history_len must be >= 0");
  APCG_CHECK(o.mode >= APCG_MODE_HOST_SYNC && o.mode <= APCG_MODE_AUTO, "bad mode %d", o.mode);
  std::unique_ptr<apcg_cg_plan_s> P(new apcg_cg_plan_s());
  P->ctx = ctx;
  P->A = *A;
  P->opts = o;
  P->n = A->nrows;
  P->k = o.check_every;
  P->max_it = o.max_it > 0 ? o.max_it : (P->n > 0 ? 10 * P->n : 10);
  P->hist_len = o.history_len;
  P->mode = o.mode;
  if (o.mode == APCG_MODE_PERSISTENT || o.mode == APCG_MODE_AUTO) {
    P->shape = default_cluster_shape(P->n);
    if (!P->shape.ok || P->n > kPersistentMaxRows) {
      if (o.mode == APCG_MODE_PERSISTENT)
        return set_error(APCG_ERR_UNSUPPORTED, "persistent mode handles at most %d rows (got %d)", kPersistentMaxRows,
                         P->n);
      P->mode = APCG_MODE_ASYNC_GRAPH;
    } else {
      P->mode = APCG_MODE_PERSISTENT;
    }
  }
  P->u = pick_u(A);
  const int sms = ctx_num_sms(ctx);
  const int64_t tiles = ((int64_t)P->n + 31) / 32;
  const int64_t spmv_blocks = (tiles + kThreads / 32 - 1) / (kThreads / 32);
  const int64_t vec_blocks = (((int64_t)P->n >> 1) + kThreads - 1) / kThreads;
  void* k1 = P->u == 4 ? (void*)cg_spmv_dot_kernel<4, false> : P->u == 6 ? (void*)cg_spmv_dot_kernel<6, false> : (void*)cg_spmv_dot_kernel<8, false>;
  P->grid_spmv = occupancy_grid(k1, sms, spmv_blocks);
  P->grid_vec = occupancy_grid((void*)cg_update_kernel<false>, sms, (vec_blocks + kUpdV - 1) / kUpdV);
  // Workspace: dinv, r, p, w, z, partials, state, histories (one stream-ordered block).
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nv = up(sizeof(double) * (size_t)(P->n > 0 ? P->n : 1));
  const size_t npart = up(sizeof(double) * dev::kMaxPartials * 3);
  const size_t nst = up(sizeof(CgState));
  const size_t nh = up(sizeof(double) * (size_t)(P->hist_len > 0 ? P->hist_len : 1));
  const size_t nsysb = up(sizeof(SysDesc) + sizeof(SysResult) + 64);
  const size_t total = 5 * nv + npart + nst + 2 * nh + nsysb;
  char* ws = nullptr;
  APCG_CUDA(cudaMallocAsync((void**)&ws, total, ctx->stream));
  P->ws = ws;
  P->dinv = reinterpret_cast<double*>(ws);
  P->r = reinterpret_cast<double*>(ws + nv);
  P->p = reinterpret_cast<double*>(ws + 2 * nv);
  P->w = reinterpret_cast<double*>(ws + 3 * nv);
  P->z = reinterpret_cast<double*>(ws + 4 * nv);
  P->partials = reinterpret_cast<double*>(ws + 5 * nv);
  P->st = reinterpret_cast<CgState*>(ws + 5 * nv + npart);
  P->alpha_h = reinterpret_cast<double*>(ws + 5 * nv + npart + nst);
  P->beta_h = reinterpret_cast<double*>(ws + 5 * nv + npart + nst + nh);
  char* tail = ws + 5 * nv + npart + nst + 2 * nh;
  P->sys = reinterpret_cast<SysDesc*>(tail);
  P->sres = reinterpret_cast<SysResult*>(tail + sizeof(SysDesc));
  P->next = reinterpret_cast<unsigned int*>(tail + sizeof(SysDesc) + sizeof(SysResult));
  APCG_CUDA(cudaMemsetAsync(ws + 5 * nv, 0, npart + nst + 2 * nh + nsysb, ctx->stream));
  {
    SysDesc d0{};
    d0.row0 = 0;
    d0.n = P->n;
    APCG_CUDA(cudaMemcpyAsync(P->sys, &d0, sizeof(d0), cudaMemcpyHostToDevice, ctx->stream));
  }
  APCG_CUDA(cudaMallocHost((void**)&P->sres_host, sizeof(SysResult)));
  APCG_CUDA(cudaMallocHost((void**)&P->st_host, sizeof(CgState)));
  APCG_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  {
    std::lock_guard<std::mutex> g(global_mutex());
    P->id = register_memory(ws, total);
  }
  // A0: the Jacobi diagonal, checked once here.
  OpScope op(ctx);
  op.read(A->id).write(P->id);
  APCG_TRY(op.begin());
  if (P->n > 0) APCG_TRY(launch_jacobi_setup(ctx, A, P->dinv));
  APCG_TRY(op.finish());
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));
  counters().host_syncs++;
  apcg_status st = ctx_check_device_error(ctx);
  if (st != APCG_OK) {
    cg_plan_destroy(P.release());
    return st;
  }
  *out = P.release();
  return APCG_OK;
}

apcg_status cg_plan_destroy(apcg_cg_plan P) {
  APCG_CHECK(P, "plan is NULL");
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
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

apcg_status cg_plan_enqueue(apcg_cg_plan P, apcg_vec b, apcg_vec x) {
  APCG_TRY(check_solve_args(P, b, x));
  double* xp = static_cast<double*>(x->dptr);
  if (P->mode == APCG_MODE_ASYNC_GRAPH) APCG_TRY(build_graph(P, xp));
  OpScope op(P->ctx);
  op.read(P->A.id).read(b->id).rw(x->id).rw(P->id);
  APCG_TRY(op.begin());
  const CgArgs a = make_args(P, xp);
  const double* bp = static_cast<const double*>(b->dptr);
  apcg_status st = APCG_OK;
  if (P->mode == APCG_MODE_HOST_SYNC)
    st = solve_host_sync(P, a, bp);
  else if (P->mode == APCG_MODE_PERSISTENT)
    st = enqueue_persistent(P, bp, xp);
  else
    st = enqueue_async(P, a, bp, P->mode == APCG_MODE_ASYNC_GRAPH);
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
  return cg_plan_create(ctx, A, opts, out);
}

apcg_status apcg_cg_plan_solve(apcg_cg_plan P, apcg_vec b, apcg_vec x, apcg_cg_result* res) {
  APCG_CHECK(res, "res is NULL");
  APCG_TRY(cg_plan_enqueue(P, b, x));
  return cg_plan_finish(P, res);
}

apcg_status apcg_cg_plan_solve_async(apcg_cg_plan P, apcg_vec b, apcg_vec x) { return cg_plan_enqueue(P, b, x); }

apcg_status apcg_cg_plan_result(apcg_cg_plan P, apcg_cg_result* res) { return cg_plan_finish(P, res); }

apcg_status apcg_cg_plan_destroy(apcg_cg_plan P) { return cg_plan_destroy(P); }

apcg_status apcg_cg_plan_profile(apcg_cg_plan P, apcg_vec b, apcg_vec x, int32_t iters, float* ms) {
  APCG_TRY(check_solve_args(P, b, x));
  APCG_CHECK(iters >= 1 && ms, "iters must be >= 1 and ms non-NULL");
  cudaStream_t s = P->ctx->stream;
  OpScope op(P->ctx);
  op.read(P->A.id).read(b->id).rw(x->id).rw(P->id);
  APCG_TRY(op.begin());
  double* xp = static_cast<double*>(x->dptr);
  const CgArgs a = make_args(P, xp);
  // Run past any convergence test: a large cap and no tolerance.
  const double rtol = P->opts.rtol, atol = P->opts.atol;
  const int32_t max_it = P->max_it;
  P->opts.rtol = 0.0;
  P->opts.atol = 0.0;
  P->max_it = 1 << 30;
  apcg_status st = launch_setup(P, a, static_cast<const double*>(b->dptr), s);
  P->opts.rtol = rtol;
  P->opts.atol = atol;
  P->max_it = max_it;
  APCG_TRY(st);
  cudaEvent_t ev[4];
  for (auto& e : ev) APCG_CUDA(cudaEventCreate(&e));
  float tot[3] = {0.f, 0.f, 0.f};
  for (int32_t i = 0; i < iters && st == APCG_OK; ++i) {
    cudaEventRecord(ev[0], s);
    st = launch_k1<false>(P, a, s);
    cudaEventRecord(ev[1], s);
    if (st == APCG_OK) st = launch_k2<false>(P, a, s, 0.0, 0, 0);
    cudaEventRecord(ev[2], s);
    if (st == APCG_OK) st = launch_k3<false>(P, a, s, 0.0);
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
  APCG_CHECK(res, "res is NULL");
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
  APCG_CUDA(cudaMallocAsync((void**)&d, brp + bcol + bval + 2 * bvec + 256, s));
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
