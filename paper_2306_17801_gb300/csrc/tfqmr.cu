// Jacobi-preconditioned TFQMR (Sec. 4.3) on one device context (float64).
//
// Freund's transpose-free QMR, two half-steps per iteration, with the Jacobi
// preconditioner on the left: the operator is M = D^-1 A and the right-hand
// side D^-1 b.  Shadow residual r* = r0.  Per iteration (the half-steps of
// the method, grouped into three kernels that end at its three reductions):
//
//   T1 (odd half-step)   x += eta_x d (the previous half-step's update, pending)
//                        u2 = u - alpha v;  w -= alpha p;  d = u + co d;  ||w||^2
//                        last block: theta = ||w|| / tau;  c = (1 + theta^2)^-1/2;
//                                    tau *= theta c;  eta = c^2 alpha;  co = theta^2 eta / alpha
//   T2 (even half-step)  q = M u2 (SpMV);  x += eta_x d;  w -= alpha q;  d = u2 + co d;
//                        ||w||^2, (w, r*)
//                        last block: theta, tau, eta as above; the convergence test
//                                    sqrt(2i + 1) tau <= tol every k iterations;
//                                    beta = (w, r*) / rho;  rho = (w, r*)
//   T3 (directions)      u = w + beta u2;  p = M u = M w + beta q (SpMV of w);
//                        v = p + beta (q + beta v);  (v, r*)
//                        last block: alpha = rho / (v, r*);  co = theta^2 eta / alpha
//
// p = M u is written as M w + beta M u2 (linearity), so that T3 needs the SpMV
// of w, which is complete when T2 ends, instead of that of u, which T3
// itself produces; it saves a kernel and a grid-wide boundary per iteration
// and changes only the rounding.  The update x += eta d of a half-step needs
// eta from that half-step's reduction, so it is applied by the next
// half-step (or, when the solve stops, by a finish kernel).  d lives in two
// buffers that the half-steps alternate (T1 reads d and writes d2, T2 reads d2
// and writes d), so the pending update still finds its d after the sweep has
// written the new one: each half-step applies it once the block's partial sums
// are out, every block but the last on the slice of x of its arrival index,
// while the last block runs the serial tail of the reduction.
//
// An iteration reads the matrix twice (two SpMVs) and reduces four inner
// products at three points, against one SpMV and two or three products for
// CG (Sec. 4.3).  The solve modes are those of the CG plan: HOST_SYNC (every
// reduction read by the host, scalars passed by value), ASYNC (host reads the
// done word every k iterations) and ASYNC_GRAPH (k iterations in the body of
// a conditional while node), and PERSISTENT: the whole solve in one
// thread-block-cluster launch (cluster_tfqmr.cu) for systems of at most
// 16384 rows, with the CSR matrix read in place.  AUTO selects PERSISTENT
// where that kernel fits and ASYNC_GRAPH otherwise.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "cluster_cg.hpp"
#include "kernels_common.cuh"
#include "sell.cuh"
#include "sell.hpp"

namespace apcg {
namespace tq {

constexpr int kThreads = 256;
// 16-byte vectors per thread and array in flight in the x updates that follow a ticket (more spill: T1 at
// 64 registers with 4, the one-entry-at-a-time T2 at 40 registers with more than 2)
constexpr int kXvT1 = 2, kXvT2 = 4, kXvT2Single = 2;
constexpr int kClusterMaxRows = 16384;
// Iterations per body of the graph's conditional while node: k, or the smallest multiple of k of at least this
// many (each K2/T2 still tests at its own iteration count; the while node itself costs about 4 us per body)
constexpr int kMinGraphBody = 8;  // the whole-solve cluster kernel: 16 CTAs x 512 threads x 2 rows

// Device-resident scalars of one TFQMR solve.
struct TqState {
  double rho;      // (r*, w) of the last direction update (rho_1 = (r*, r0))
  double alpha, beta, theta, eta, tau;
  double co;       // coefficient of d in the next half-step: theta^2 eta / alpha
  double eta_x;    // pending update x += eta_x d
  double tol;      // max(rtol ||D^-1 b||, atol)
  double bnorm2;   // ||D^-1 b||^2
  double ww, wr, sigma;  // last reductions (read by the host in the host-synchronous form)
  int32_t iter;    // completed iterations
  int32_t done;    // kDone*
  int32_t max_it, check_every, hist_len;
  int32_t pending;  // eta_x holds an update not yet applied to x: 0 none, 1 along d, 2 along d2
  int32_t body_runs;
  unsigned int ticket;
};

struct TqArgs {
  dev::SellView<double> A;
  int32_t n;
  const double* __restrict__ dinv;
  double* rs;  // r*
  double* x;
  double* u;
  double* u2;
  double* w;
  double* d;   // written by T2 (and zeroed by S1), read by T1
  double* d2;  // written by T1, read by T2
  double* v;
  double* p;
  double* q;
  TqState* st;
  double* partials;
  double* alpha_h;
  double* beta_h;
};

// Scalars passed by value in the host-synchronous form.
struct HostScalars {
  double alpha, beta, co, eta_x;
  int32_t pending;
};

__device__ __forceinline__ int32_t read_done(const TqState* st) { return *(volatile const int32_t*)&st->done; }

// The quasi-residual update after a half-step (last block, device mode); buf:
// the pending code of the d buffer that the half-step wrote (1: d, 2: d2).
// Returns false on a non-finite value.
__device__ __forceinline__ bool quasi_update(TqState* st, double ww, int32_t buf) {
  const double theta = sqrt(ww) / st->tau;
  const double c = 1.0 / sqrt(1.0 + theta * theta);
  const double tau = st->tau * theta * c;
  const double eta = c * c * st->alpha;
  st->theta = theta;
  st->tau = tau;
  st->eta = eta;
  st->eta_x = eta;
  st->pending = buf;
  return isfinite(theta) && isfinite(tau);
}

// x += ex dd over the slice of [0, n) of this block's arrival index, after a grid reduction's ticket: every
// block but the one that arrived last takes one of gridDim.x - 1 slices (a grid of one block takes all), so the
// bytes move while the last block finishes the reduction.  The element left over by the 16-byte vectors of an
// odd n goes to the block that arrived first.
// V: 16-byte vectors per thread and array in flight.
template <int V>
__device__ __forceinline__ void x_update_slice(double* __restrict__ x, const double* __restrict__ dd, double ex,
                                               int64_t n, unsigned arrival, bool last) {
  if (last && gridDim.x > 1) return;
  const int64_t nv = n / 2, parts = gridDim.x > 1 ? (int64_t)gridDim.x - 1 : 1;
  const int64_t lo = nv * (int64_t)arrival / parts, hi = nv * ((int64_t)arrival + 1) / parts;
  double2* xv = reinterpret_cast<double2*>(x);
  const double2* dv = reinterpret_cast<const double2*>(dd);
  for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += V * kThreads) {
    double2 xx[V], de[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = i0 + u * kThreads;
      if (i < hi) {
        xx[u] = xv[i];
        de[u] = __ldg(dv + i);
      }
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = i0 + u * kThreads;
      if (i < hi) {
        xx[u].x = fma(ex, de[u].x, xx[u].x);
        xx[u].y = fma(ex, de[u].y, xx[u].y);
        xv[i] = xx[u];
      }
    }
  }
  if (arrival == 0 && threadIdx.x == 0 && (n & 1)) x[n - 1] = fma(ex, dd[n - 1], x[n - 1]);
}

// S1: r0 = D^-1 (b - A x0);  u = w = r* = r0;  d = 0;  ||r0||^2, ||D^-1 b||^2;
// tau = ||r0||, rho = (r*, r0), the tolerance and the initial test.
template <bool LONG, int CF>
__global__ void __launch_bounds__(kThreads) s1_kernel(TqArgs a, const double* __restrict__ b, double rtol,
                                                      double atol, int32_t max_it, int32_t k, int32_t hist_len) {
  __shared__ double red[2 * kThreads];
  double v[2] = {0.0, 0.0};
  dev::sell_spmv<false, LONG, double, 8, CF>(a.A, a.x, [&](int32_t i, double ax, double) {
                                           const double di = __ldg(a.dinv + i);
                                           const double bi = __ldg(b + i);
                                           const double ri = di * (bi - ax);
                                           const double bh = di * bi;
                                           a.u[i] = ri;
                                           a.w[i] = ri;
                                           a.rs[i] = ri;
                                           a.d[i] = 0.0;
                                           v[0] = fma(ri, ri, v[0]);
                                           v[1] = fma(bh, bh, v[1]);
                                         });
  double tot[2];
  if (dev::grid_sum_last<2>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0) {
    TqState* st = a.st;
    st->rho = tot[0];
    st->ww = tot[0];
    st->bnorm2 = tot[1];
    st->tau = sqrt(tot[0]);
    st->tol = fmax(rtol * sqrt(tot[1]), atol);
    st->theta = st->eta = st->co = st->eta_x = 0.0;
    st->alpha = st->beta = st->sigma = st->wr = 0.0;
    st->pending = 0;
    st->iter = 0;
    st->max_it = max_it;
    st->check_every = k;
    st->hist_len = hist_len;
    st->body_runs = 0;
    st->done = (!isfinite(tot[0]) || !isfinite(tot[1])) ? kDoneBreakdown  // a non-finite b or x0
               : st->tau <= st->tol                          ? kDoneConverged
                                                             : 0;
  }
}

// S2: p = M u;  v = p;  sigma = (v, r*);  alpha = rho / sigma (device mode).
template <bool HOST, bool LONG, int CF>
__global__ void __launch_bounds__(kThreads) s2_kernel(TqArgs a) {
  if (!HOST && read_done(a.st)) return;
  __shared__ double red[kThreads];
  double v[1] = {0.0};
  dev::sell_spmv<false, LONG, double, 8, CF>(a.A, a.u, [&](int32_t i, double au, double) {
                                           const double pi = __ldg(a.dinv + i) * au;
                                           a.p[i] = pi;
                                           a.v[i] = pi;
                                           v[0] = fma(pi, __ldg(a.rs + i), v[0]);
                                         });
  double tot[1];
  if (dev::grid_sum_last<1>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0) {
    TqState* st = a.st;
    st->sigma = tot[0];
    if (!HOST) {
      if (tot[0] == 0.0 || !isfinite(tot[0])) {
        st->done = kDoneBreakdown;
      } else {
        st->alpha = st->rho / tot[0];
        st->co = 0.0;
        if (st->hist_len > 0) a.alpha_h[0] = st->alpha;
      }
    }
  }
}

// T1, the odd half-step (vectors only).
template <bool HOST>
__global__ void __launch_bounds__(kThreads, 4) t1_kernel(TqArgs a, HostScalars h) {
  if (!HOST && read_done(a.st)) return;
  const double alpha = HOST ? h.alpha : a.st->alpha;
  const double co = HOST ? h.co : a.st->co;
  const bool pend = HOST ? h.pending != 0 : a.st->pending != 0;
  const double ex = HOST ? h.eta_x : a.st->eta_x;
  __shared__ double red[kThreads];
  double acc = 0.0;
  const int64_t n = a.n, nv = n / 2, stride = (int64_t)gridDim.x * blockDim.x;
  const double2* uv = reinterpret_cast<const double2*>(a.u);
  const double2* vv = reinterpret_cast<const double2*>(a.v);
  const double2* pv = reinterpret_cast<const double2*>(a.p);
  double2* wv = reinterpret_cast<double2*>(a.w);
  const double2* dv = reinterpret_cast<const double2*>(a.d);
  double2* d2v = reinterpret_cast<double2*>(a.d2);
  double2* u2v = reinterpret_cast<double2*>(a.u2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const double2 uu = dev::ld_stream2(uv + i), vvv = dev::ld_stream2(vv + i), pp = dev::ld_stream2(pv + i);
    double2 ww = wv[i], dd = __ldg(dv + i), u2;
    u2.x = fma(-alpha, vvv.x, uu.x);
    u2.y = fma(-alpha, vvv.y, uu.y);
    ww.x = fma(-alpha, pp.x, ww.x);
    ww.y = fma(-alpha, pp.y, ww.y);
    dd.x = fma(co, dd.x, uu.x);
    dd.y = fma(co, dd.y, uu.y);
    acc = fma(ww.x, ww.x, acc);
    acc = fma(ww.y, ww.y, acc);
    u2v[i] = u2;
    wv[i] = ww;
    d2v[i] = dd;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
    const int64_t i = n - 1;
    a.u2[i] = fma(-alpha, a.v[i], a.u[i]);
    a.w[i] = fma(-alpha, a.p[i], a.w[i]);
    a.d2[i] = fma(co, a.d[i], a.u[i]);
    acc = fma(a.w[i], a.w[i], acc);
  }
  double v[1] = {acc}, tot[1];
  unsigned arrival;
  const bool last = dev::grid_sum_last<1>(v, a.partials, &a.st->ticket, red, tot, &arrival);
  if (pend) x_update_slice<kXvT1>(a.x, a.d, ex, n, arrival, last);
  if (last && threadIdx.x == 0) {
    TqState* st = a.st;
    st->ww = tot[0];
    if (!HOST) {
      if (!quasi_update(st, tot[0], 2)) {
        st->pending = 0;
        st->iter += 1;  // the iteration stopped inside its first half-step
        st->done = kDoneBreakdown;
      } else {
        st->co = st->theta * st->theta * st->eta / st->alpha;
        if (st->tau == 0.0) {  // the quasi-residual vanished: x is exact after this half-step
          st->iter += 1;
          st->done = kDoneConverged;
        }
      }
    }
  }
}

// T2, the even half-step: q = M u2 and the updates, ||w||^2 and (w, r*); the
// test and beta in the last block.  G: the SpMV's group size (0: one entry at
// a time).  The one-at-a-time instance is bounded to 40 registers (six blocks
// per SM, a few bytes of spill): the extra resident warps hide more of the
// gathers' latency (128^3 7-point: 173 against 180 us per iteration at 48
// registers and five blocks).  T3 runs on its own grid at its own occupancy.
template <bool HOST, int G, int CF>
__global__ void __launch_bounds__(kThreads, G == 0 ? 6 : 4) t2_kernel(TqArgs a, HostScalars h,
                                                                   cudaGraphConditionalHandle cond, int32_t use_cond) {
  if (!HOST && read_done(a.st)) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      a.st->body_runs += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  const double alpha = HOST ? h.alpha : a.st->alpha;
  const double co = HOST ? h.co : a.st->co;
  const bool pend = HOST ? h.pending != 0 : a.st->pending != 0;
  const double ex = HOST ? h.eta_x : a.st->eta_x;
  __shared__ double red[2 * kThreads];
  double v[2] = {0.0, 0.0};
  dev::sell_spmv<true, (G > 0), double, (G > 0 ? G : 8), CF>(a.A, a.u2, [&](int32_t i, double au2, double u2i) {
                                          const double qi = __ldg(a.dinv + i) * au2;
                                          const double wi = fma(-alpha, qi, a.w[i]);
                                          a.q[i] = qi;
                                          a.w[i] = wi;
                                          a.d[i] = fma(co, __ldg(a.d2 + i), u2i);
                                          v[0] = fma(wi, wi, v[0]);
                                          v[1] = fma(wi, __ldg(a.rs + i), v[1]);
                                        });
  double tot[2];
  unsigned arrival;
  const bool last = dev::grid_sum_last<2>(v, a.partials, &a.st->ticket, red, tot, &arrival);
  if (pend) x_update_slice<(G == 0 ? kXvT2Single : kXvT2)>(a.x, a.d2, ex, a.n, arrival, last);
  if (last && threadIdx.x == 0) {
    TqState* st = a.st;
    st->ww = tot[0];
    st->wr = tot[1];
    if (!HOST) {
      const int32_t it = st->iter + 1;
      st->iter = it;
      int32_t done = 0;
      if (!quasi_update(st, tot[0], 1)) {
        st->pending = 0;
        done = kDoneBreakdown;
      } else {
        const bool check = (it % st->check_every == 0) || it >= st->max_it;
        if (st->tau == 0.0 || (check && sqrt(2.0 * it + 1.0) * st->tau <= st->tol)) {
          done = kDoneConverged;
        } else if (it >= st->max_it) {
          done = kDoneNotConverged;
        } else if (st->rho == 0.0 || !isfinite(tot[1])) {
          done = kDoneBreakdown;
        } else {
          const double beta = tot[1] / st->rho;
          st->beta = beta;
          st->rho = tot[1];
          if (it - 1 < st->hist_len) a.beta_h[it - 1] = beta;
        }
      }
      st->done = done;
      if (use_cond) {
        st->body_runs += 1;
        cudaGraphSetConditional(cond, done ? 0u : 1u);
      }
    }
  }
}

// T3, the direction update: u = w + beta u2;  p = M w + beta q (= M u);
// v = p + beta (q + beta v);  sigma = (v, r*) and alpha in the last block.
template <bool HOST, int G, int CF>
__global__ void __launch_bounds__(kThreads) t3_kernel(TqArgs a, HostScalars h) {
  if (!HOST && read_done(a.st)) return;
  const double beta = HOST ? h.beta : a.st->beta;
  __shared__ double red[kThreads];
  double v[1] = {0.0};
  dev::sell_spmv<true, (G > 0), double, (G > 0 ? G : 8), CF>(a.A, a.w, [&](int32_t i, double aw, double wi) {
                                          const double mwi = __ldg(a.dinv + i) * aw;
                                          const double qi = a.q[i];
                                          a.u[i] = fma(beta, a.u2[i], wi);
                                          const double pi = fma(beta, qi, mwi);
                                          const double ti = fma(beta, a.v[i], qi);
                                          const double vi = fma(beta, ti, pi);
                                          a.p[i] = pi;
                                          a.v[i] = vi;
                                          v[0] = fma(vi, __ldg(a.rs + i), v[0]);
                                        });
  double tot[1];
  if (dev::grid_sum_last<1>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0) {
    TqState* st = a.st;
    st->sigma = tot[0];
    if (!HOST) {
      if (tot[0] == 0.0 || !isfinite(tot[0])) {
        st->done = kDoneBreakdown;
      } else {
        const double alpha = st->rho / tot[0];
        st->alpha = alpha;
        st->co = st->theta * st->theta * st->eta / alpha;
        if (st->iter < st->hist_len) a.alpha_h[st->iter] = alpha;
      }
    }
  }
}

// The update still pending when the iteration stops: x += eta_x d, along the
// d buffer that the stopping half-step wrote.
__global__ void __launch_bounds__(kThreads) finish_kernel(TqArgs a, HostScalars h, int32_t host) {
  const int32_t pend = host ? h.pending : a.st->pending;
  if (pend != 1 && pend != 2) return;
  const double ex = host ? h.eta_x : a.st->eta_x;
  const double* __restrict__ dd = pend == 2 ? a.d2 : a.d;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
    a.x[i] = fma(ex, dd[i], a.x[i]);
}

template <class K>
int occupancy_grid(K kernel, int sms, int64_t want) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t g = (int64_t)per_sm * sms;
  if (want < g) g = want;
  if (g > dev::kMaxPartials) g = dev::kMaxPartials;
  return g < 1 ? 1 : (int)g;
}

// The host's copy of the quasi-residual update (host-synchronous form); the
// same operations in the same order as quasi_update.
bool host_quasi_update(TqState* h, double ww, int32_t buf) {
  const double theta = std::sqrt(ww) / h->tau;
  const double c = 1.0 / std::sqrt(1.0 + theta * theta);
  h->tau = h->tau * theta * c;
  h->theta = theta;
  h->eta = c * c * h->alpha;
  h->eta_x = h->eta;
  h->pending = buf;
  return std::isfinite(theta) && std::isfinite(h->tau);
}

}  // namespace tq
}  // namespace apcg

struct apcg_tfqmr_plan_s {
  apcg_ctx ctx = nullptr;
  apcg_mat_s A;  // copy of the (non-owning) matrix view
  apcg_cg_opts opts{};
  int32_t mode = APCG_MODE_ASYNC_GRAPH;
  apcg::tq::TqArgs a{};  // x is filled in per solve
  int32_t n = 0, k = 1, max_it = 0, hist_len = 0;
  int32_t body = 1;  // iterations captured in one body of the conditional while node
  int grid_spmv = 1, grid_vec = 1, grid_t3 = 1;  // t3 takes fewer registers than t2: its own persistent grid
  bool long_rows = false;  // the set-up kernels' SpMV path
  int group = 0;           // the iteration kernels' SpMV group size (0: one entry at a time)
  int64_t padded = 0;      // stored entries of the sliced-ELL copy
  char* ws = nullptr;
  apcg::tq::TqState* st_host = nullptr;  // pinned mirror of the state block
  apcg_id id = 0;
  bool pending = false;
  int64_t last_launches = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double* graph_x = nullptr;
  // whole-solve cluster mode (small systems, cluster_tfqmr.cu)
  apcg::ClusterShape shape;
  apcg::SysDesc* sys = nullptr;
  apcg::SysResult* sres = nullptr;
  unsigned int* next = nullptr;
  apcg::SysResult* sres_host = nullptr;
};

namespace apcg {
namespace tq {

using Plan = apcg_tfqmr_plan;

TqArgs args_for(Plan P, double* x) {
  TqArgs a = P->a;
  a.x = x;
  return a;
}

apcg_status launch_s1(Plan P, double* x, const double* b, cudaStream_t s) {
  const TqArgs a = args_for(P, x);
  const double rtol = P->opts.rtol, atol = P->opts.atol;
  const int cf = dev::col_format(P->a.A);
#define APCG_S1(L, F) s1_kernel<L, F><<<P->grid_spmv, kThreads, 0, s>>>(a, b, rtol, atol, P->max_it, P->k, P->hist_len)
#define APCG_S1F(L) \
  (cf == dev::kColPattern ? APCG_S1(L, dev::kColPattern) : cf == dev::kColOff16 ? APCG_S1(L, dev::kColOff16) : APCG_S1(L, dev::kColIndex))
  if (P->long_rows)
    APCG_S1F(true);
  else
    APCG_S1F(false);
#undef APCG_S1F
#undef APCG_S1
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

apcg_status launch_s2(Plan P, double* x, cudaStream_t s, bool host) {
  const TqArgs a = args_for(P, x);
  const int cf = dev::col_format(P->a.A);
#define APCG_S2(H, L, F) s2_kernel<H, L, F><<<P->grid_spmv, kThreads, 0, s>>>(a)
#define APCG_S2F(H, L) \
  (cf == dev::kColPattern ? APCG_S2(H, L, dev::kColPattern) : cf == dev::kColOff16 ? APCG_S2(H, L, dev::kColOff16) : APCG_S2(H, L, dev::kColIndex))
  if (host)
    P->long_rows ? APCG_S2F(true, true) : APCG_S2F(true, false);
  else
    P->long_rows ? APCG_S2F(false, true) : APCG_S2F(false, false);
#undef APCG_S2F
#undef APCG_S2
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

apcg_status launch_t1(Plan P, double* x, cudaStream_t s, bool host, const HostScalars& h) {
  const TqArgs a = args_for(P, x);
  if (host)
    t1_kernel<true><<<P->grid_vec, kThreads, 0, s>>>(a, h);
  else
    t1_kernel<false><<<P->grid_vec, kThreads, 0, s>>>(a, h);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

// The instance of T2 or T3 for the plan's group size and column format.
template <bool HOST, int CF>
void* t2_instance(int g) {
  switch (g) {
    case 5: return (void*)t2_kernel<HOST, 5, CF>;
    case 6: return (void*)t2_kernel<HOST, 6, CF>;
    case 7: return (void*)t2_kernel<HOST, 7, CF>;
    case 8: return (void*)t2_kernel<HOST, 8, CF>;
    case 9: return (void*)t2_kernel<HOST, 9, CF>;
    default: return (void*)t2_kernel<HOST, 0, CF>;
  }
}
template <bool HOST, int CF>
void* t3_instance(int g) {
  switch (g) {
    case 5: return (void*)t3_kernel<HOST, 5, CF>;
    case 6: return (void*)t3_kernel<HOST, 6, CF>;
    case 7: return (void*)t3_kernel<HOST, 7, CF>;
    case 8: return (void*)t3_kernel<HOST, 8, CF>;
    case 9: return (void*)t3_kernel<HOST, 9, CF>;
    default: return (void*)t3_kernel<HOST, 0, CF>;
  }
}
template <bool HOST>
void* t2_for_cf(int cf, int g) {
  return cf == dev::kColPattern ? t2_instance<HOST, dev::kColPattern>(g)
         : cf == dev::kColOff16 ? t2_instance<HOST, dev::kColOff16>(g)
                                : t2_instance<HOST, dev::kColIndex>(g);
}
template <bool HOST>
void* t3_for_cf(int cf, int g) {
  return cf == dev::kColPattern ? t3_instance<HOST, dev::kColPattern>(g)
         : cf == dev::kColOff16 ? t3_instance<HOST, dev::kColOff16>(g)
                                : t3_instance<HOST, dev::kColIndex>(g);
}
void* t2_for(bool host, int cf, int g) { return host ? t2_for_cf<true>(cf, g) : t2_for_cf<false>(cf, g); }
void* t3_for(bool host, int cf, int g) { return host ? t3_for_cf<true>(cf, g) : t3_for_cf<false>(cf, g); }

apcg_status launch_t2(Plan P, double* x, cudaStream_t s, bool host, const HostScalars& h,
                      cudaGraphConditionalHandle cond, int32_t use_cond) {
  TqArgs a = args_for(P, x);
  HostScalars hh = h;
  void* args[] = {&a, &hh, &cond, &use_cond};
  void* k = t2_for(host, dev::col_format(P->a.A), P->group);
  APCG_CUDA(cudaLaunchKernel(k, dim3(P->grid_spmv), dim3(kThreads), args, 0, s));
  return APCG_OK;
}

apcg_status launch_t3(Plan P, double* x, cudaStream_t s, bool host, const HostScalars& h) {
  TqArgs a = args_for(P, x);
  HostScalars hh = h;
  void* args[] = {&a, &hh};
  void* k = t3_for(host, dev::col_format(P->a.A), P->group);
  APCG_CUDA(cudaLaunchKernel(k, dim3(P->grid_t3), dim3(kThreads), args, 0, s));
  return APCG_OK;
}

apcg_status launch_finish(Plan P, double* x, cudaStream_t s, bool host, const HostScalars& h) {
  finish_kernel<<<P->grid_vec, kThreads, 0, s>>>(args_for(P, x), h, host ? 1 : 0);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

apcg_status read_state(Plan P, cudaStream_t s) {
  APCG_CUDA(cudaMemcpyAsync(P->st_host, P->a.st, sizeof(TqState), cudaMemcpyDeviceToHost, s));
  APCG_CUDA(cudaStreamSynchronize(s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(TqState);
  counters().host_syncs++;
  return APCG_OK;
}

// Host-synchronous form: each of the three reductions of an iteration goes to
// the host and is waited for; alpha, beta and the half-step coefficients are
// computed on the host and passed by value.
apcg_status solve_host_sync(Plan P, const double* b, double* x) {
  cudaStream_t s = P->ctx->stream;
  TqState* h = P->st_host;
  int64_t launches = 0;
  APCG_TRY(launch_s1(P, x, b, s));
  launches++;
  APCG_TRY(read_state(P, s));
  TqState m = *h;  // the host's scalars
  std::vector<double> ah, bh;
  HostScalars hs{};
  auto scal = [&]() {
    hs.alpha = m.alpha;
    hs.beta = m.beta;
    hs.co = m.co;
    hs.eta_x = m.eta_x;
    hs.pending = m.pending;
    return hs;
  };
  int32_t done = m.done, it = 0;
  if (!done) {
    APCG_TRY(launch_s2(P, x, s, true));
    launches++;
    APCG_TRY(read_state(P, s));
    if (h->sigma == 0.0 || !std::isfinite(h->sigma)) {
      done = kDoneBreakdown;
    } else {
      m.alpha = m.rho / h->sigma;
      m.co = 0.0;
      ah.push_back(m.alpha);
    }
  }
  while (!done) {
    ++it;
    APCG_TRY(launch_t1(P, x, s, true, scal()));
    launches++;
    APCG_TRY(read_state(P, s));
    if (!host_quasi_update(&m, h->ww, 2)) {
      m.pending = 0;
      done = kDoneBreakdown;
      break;
    }
    m.co = m.theta * m.theta * m.eta / m.alpha;
    if (m.tau == 0.0) {
      done = kDoneConverged;
      break;
    }
    APCG_TRY(launch_t2(P, x, s, true, scal(), 0, 0));
    launches++;
    APCG_TRY(read_state(P, s));
    const double wr = h->wr;
    if (!host_quasi_update(&m, h->ww, 1)) {
      m.pending = 0;
      done = kDoneBreakdown;
      break;
    }
    const bool check = (it % P->k == 0) || it >= P->max_it;
    if (m.tau == 0.0 || (check && std::sqrt(2.0 * it + 1.0) * m.tau <= m.tol)) {
      done = kDoneConverged;
      break;
    }
    if (it >= P->max_it) {
      done = kDoneNotConverged;
      break;
    }
    if (m.rho == 0.0 || !std::isfinite(wr)) {
      done = kDoneBreakdown;
      break;
    }
    m.beta = wr / m.rho;
    m.rho = wr;
    if (it - 1 < P->hist_len) bh.push_back(m.beta);
    APCG_TRY(launch_t3(P, x, s, true, scal()));
    launches++;
    APCG_TRY(read_state(P, s));
    const double sigma = h->sigma;
    if (sigma == 0.0 || !std::isfinite(sigma)) {
      done = kDoneBreakdown;
      break;
    }
    m.alpha = m.rho / sigma;
    m.co = m.theta * m.theta * m.eta / m.alpha;
    if (it < P->hist_len) ah.push_back(m.alpha);
  }
  APCG_TRY(launch_finish(P, x, s, true, scal()));
  launches++;
  APCG_CUDA(cudaStreamSynchronize(s));
  counters().host_syncs++;
  m.iter = it;
  m.done = done;
  *h = m;
  P->last_launches = launches;
  count_kernels(launches);
  if (P->opts.alpha_hist)
    for (size_t i = 0; i < ah.size() && (int)i < P->hist_len; ++i) P->opts.alpha_hist[i] = ah[i];
  if (P->opts.beta_hist)
    for (size_t i = 0; i < bh.size() && (int)i < P->hist_len; ++i) P->opts.beta_hist[i] = bh[i];
  return APCG_OK;
}

void release_graph(Plan P) {
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->exec = nullptr;
  P->graph = nullptr;
  P->graph_x = nullptr;
}

// k iterations (T1, T2, T3 each) in the body of a conditional while node; the
// last T2 of the body decides whether the body runs again.
apcg_status build_graph(Plan P, double* x) {
  if (P->exec && P->graph_x == x) return APCG_OK;
  release_graph(P);
  if (!P->cap_stream) APCG_CUDA(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  APCG_CUDA(cudaGraphCreate(&g, 0));
  P->graph = g;
  cudaGraphConditionalHandle hnd;
  APCG_CUDA(cudaGraphConditionalHandleCreate(&hnd, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  APCG_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  APCG_CUDA(cudaStreamBeginCaptureToGraph(P->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const HostScalars none{};
  apcg_status st = APCG_OK;
  P->body = P->k >= kMinGraphBody ? P->k : P->k * ((kMinGraphBody + P->k - 1) / P->k);
  for (int j = 0; j < P->body && st == APCG_OK; ++j) {
    st = launch_t1(P, x, P->cap_stream, false, none);
    if (st == APCG_OK) st = launch_t2(P, x, P->cap_stream, false, none, hnd, j == P->body - 1 ? 1 : 0);
    if (st == APCG_OK) st = launch_t3(P, x, P->cap_stream, false, none);
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

apcg_status enqueue_async(Plan P, const double* b, double* x, bool graph) {
  cudaStream_t s = P->ctx->stream;
  const HostScalars none{};
  APCG_TRY(launch_s1(P, x, b, s));
  APCG_TRY(launch_s2(P, x, s, false));
  int64_t launches = 2;
  if (graph) {
    APCG_CUDA(cudaGraphLaunch(P->exec, s));
    counters().graph_launches++;
  } else {
    // k iterations at a time, then one read of the state (the done word)
    const int64_t max_blocks = (int64_t)P->max_it / P->k + 2;
    for (int64_t blk = 0; blk < max_blocks; ++blk) {
      for (int j = 0; j < P->k; ++j) {
        APCG_TRY(launch_t1(P, x, s, false, none));
        APCG_TRY(launch_t2(P, x, s, false, none, 0, 0));
        APCG_TRY(launch_t3(P, x, s, false, none));
      }
      launches += 3 * P->k;
      APCG_TRY(read_state(P, s));
      if (P->st_host->done) break;
    }
  }
  APCG_TRY(launch_finish(P, x, s, false, none));
  launches++;
  count_kernels(launches);
  P->last_launches = launches;
  APCG_CUDA(cudaMemcpyAsync(P->st_host, P->a.st, sizeof(TqState), cudaMemcpyDeviceToHost, s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(TqState);
  return APCG_OK;
}

// The whole solve in one cluster launch (small systems).
apcg_status enqueue_persistent(Plan P, const double* b, double* x) {
  cudaStream_t s = P->ctx->stream;
  ClusterArgs ca{};
  ca.rowptr = P->A.rowptr;
  ca.col = P->A.col;
  ca.val = static_cast<const double*>(P->A.val);
  ca.b = b;
  ca.x = x;
  ca.sys = P->sys;
  ca.nsys = 1;
  ca.check_every = P->k;
  ca.next = P->next;
  ca.res = P->sres;
  ca.rtol = P->opts.rtol;
  ca.atol = P->opts.atol;
  ca.max_it = P->max_it;
  ca.hist_len = P->hist_len;
  ca.alpha_h = P->a.alpha_h;
  ca.beta_h = P->a.beta_h;
  APCG_CUDA(cudaMemsetAsync(P->next, 0, sizeof(unsigned int), s));
  APCG_CUDA(launch_cluster_tfqmr(ca, P->shape, 1, s));
  count_kernels(1);
  P->last_launches = 1;
  APCG_CUDA(cudaMemcpyAsync(P->sres_host, P->sres, sizeof(SysResult), cudaMemcpyDeviceToHost, s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(SysResult);
  return APCG_OK;
}

apcg_status finish_async(Plan P) {
  APCG_CUDA(cudaStreamSynchronize(P->ctx->stream));
  counters().host_syncs++;
  if (P->mode == APCG_MODE_ASYNC_GRAPH) {
    const int64_t body = (int64_t)P->st_host->body_runs * 3 * P->body;
    count_kernels(body);
    P->last_launches += body;
  }
  if (P->hist_len > 0) {
    if (P->opts.alpha_hist)
      APCG_CUDA(cudaMemcpy(P->opts.alpha_hist, P->a.alpha_h, sizeof(double) * P->hist_len, cudaMemcpyDeviceToHost));
    if (P->opts.beta_hist)
      APCG_CUDA(cudaMemcpy(P->opts.beta_hist, P->a.beta_h, sizeof(double) * P->hist_len, cudaMemcpyDeviceToHost));
    counters().d2h_copies += 2;
  }
  return APCG_OK;
}

void fill_result(Plan P, apcg_cg_result* res) {
  if (P->mode == APCG_MODE_PERSISTENT) {
    const SysResult& r = *P->sres_host;
    res->iters = r.iters;
    res->reason = r.done == kDoneConverged      ? APCG_CONVERGED
                  : r.done == kDoneBreakdown    ? APCG_BREAKDOWN
                  : r.done == kDoneBadDiagonal ? APCG_BAD_DIAGONAL
                                                : APCG_NOT_CONVERGED;
    res->rr = r.rr;
    res->bnorm = std::sqrt(r.bnorm2);
    res->rel_res = res->bnorm > 0.0 ? std::sqrt(r.rr) / res->bnorm : std::sqrt(r.rr);
    res->kernel_launches = P->last_launches;
    return;
  }
  const TqState* h = P->st_host;
  res->iters = h->iter;
  res->reason = h->done == kDoneConverged ? APCG_CONVERGED
                : h->done == kDoneBreakdown ? APCG_BREAKDOWN
                                            : APCG_NOT_CONVERGED;
  const double bound = std::sqrt(2.0 * h->iter + 1.0) * h->tau;
  res->rr = bound * bound;
  res->bnorm = std::sqrt(h->bnorm2);
  res->rel_res = res->bnorm > 0.0 ? bound / res->bnorm : bound;
  res->kernel_launches = P->last_launches;
}

apcg_status plan_destroy(Plan P) {
  APCG_CHECK(P, "plan is NULL");
  release_graph(P);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  if (P->ws) {
    {
      std::lock_guard<std::mutex> g(global_mutex());
      reg_forget_memory(P->ws);
    }
    cudaFreeAsync(P->ws, P->ctx->stream);
  }
  if (P->st_host || P->sres_host) {
    cudaStreamSynchronize(P->ctx->stream);  // the pinned mirrors may be the target of an enqueued copy
    if (P->st_host) cudaFreeHost(P->st_host);
    if (P->sres_host) cudaFreeHost(P->sres_host);
  }
  delete P;
  return APCG_OK;
}

apcg_status plan_create(apcg_ctx ctx, apcg_mat A, const apcg_cg_opts* opts, Plan* out) {
  apcg_cg_opts o;
  if (opts)
    o = *opts;
  else
    apcg_cg_opts_default(&o);
  APCG_CHECK(o.check_every >= 1, "check_every must be >= 1");
  APCG_CHECK(o.rtol >= 0.0 && o.atol >= 0.0, "negative tolerance");
  APCG_CHECK(o.history_len >= 0, "negative history length");
  std::unique_ptr<apcg_tfqmr_plan_s, apcg_status (*)(Plan)> P(new apcg_tfqmr_plan_s(), plan_destroy);
  P->ctx = ctx;
  P->A = *A;
  P->opts = o;
  P->n = A->nrows;
  P->k = o.check_every;
  P->max_it = o.max_it > 0 ? o.max_it : (P->n > 0 ? 10 * P->n : 10);
  P->hist_len = o.history_len;
  P->mode = (o.mode == APCG_MODE_HOST_SYNC || o.mode == APCG_MODE_ASYNC) ? o.mode : APCG_MODE_ASYNC_GRAPH;
  if (o.mode == APCG_MODE_PERSISTENT || o.mode == APCG_MODE_AUTO) {
    P->shape = P->n <= kClusterMaxRows ? tfqmr_cluster_shape(P->n) : ClusterShape{};
    if (P->n > kClusterMaxRows) P->shape.ok = false;
    if (P->shape.ok)
      P->mode = APCG_MODE_PERSISTENT;
    else if (o.mode == APCG_MODE_PERSISTENT)
      return set_error(APCG_ERR_UNSUPPORTED, "persistent TFQMR handles at most %d rows (got %d)", kClusterMaxRows,
                       P->n);
  }
  SellLayout L;
  APCG_TRY(csr_layout(ctx, A, P->mode != APCG_MODE_PERSISTENT, &L));
  const int sms = ctx_num_sms(ctx);
  P->long_rows = L.long_rows != 0;
  P->group = L.group;
  const int64_t slices = ((int64_t)P->n + 31) / 32;
  const bool sell = P->mode != APCG_MODE_PERSISTENT;
  const bool pat = L.pattern && sell, d16 = L.d16 && sell;
  const int cf = pat ? dev::kColPattern : d16 ? dev::kColOff16 : dev::kColIndex;
  P->grid_spmv = occupancy_grid(t2_for(false, cf, P->group), sms, (slices + 7) / 8);
  P->grid_t3 = occupancy_grid(t3_for(false, cf, P->group), sms, (slices + 7) / 8);
  P->grid_vec = occupancy_grid(t1_kernel<false>, sms, ((int64_t)P->n / 2 + kThreads - 1) / kThreads);
  // Workspace: dinv, r*, u, u2, w, d, d2, v, p, q; partials; state; histories; sliced-ELL copy.
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nv = up(sizeof(double) * (size_t)(P->n > 0 ? P->n : 1));
  const size_t npart = up(sizeof(double) * dev::kMaxPartials * 2);
  const size_t nst = up(sizeof(TqState));
  const size_t nh = up(sizeof(double) * (size_t)(P->hist_len > 0 ? P->hist_len : 1));
  const size_t nsptr = up(sizeof(int32_t) * ((size_t)L.nslices + 1));
  // columns: per-slice offset lists where the slices' rows share them, else 16-bit offsets from the row
  // where they all fit, else 32-bit indices
  const size_t ncol = up(pat ? sizeof(int32_t) * (size_t)std::max<int64_t>(L.padded / 32, 1)
                             : (d16 ? sizeof(int16_t) : sizeof(int32_t)) * (size_t)std::max<int64_t>(L.padded, 1));
  const size_t nval = up(sizeof(double) * (size_t)std::max<int64_t>(L.padded, 1));
  const size_t nsysb = up(sizeof(SysDesc) + sizeof(SysResult) + 64);
  const size_t total = 10 * nv + npart + nst + 2 * nh + nsptr + ncol + nval + nsysb;
  char* ws = nullptr;
  APCG_TRY(dev_alloc_async((void**)&ws, total, ctx->stream));
  P->ws = ws;
  double* vecs[10];
  for (int i = 0; i < 10; ++i) vecs[i] = reinterpret_cast<double*>(ws + i * nv);
  TqArgs& a = P->a;
  a.n = P->n;
  a.dinv = vecs[0];
  a.rs = vecs[1];
  a.u = vecs[2];
  a.u2 = vecs[3];
  a.w = vecs[4];
  a.d = vecs[5];
  a.d2 = vecs[9];
  a.v = vecs[6];
  a.p = vecs[7];
  a.q = vecs[8];
  char* q = ws + 10 * nv;
  a.partials = reinterpret_cast<double*>(q);
  a.st = reinterpret_cast<TqState*>(q + npart);
  a.alpha_h = reinterpret_cast<double*>(q + npart + nst);
  a.beta_h = reinterpret_cast<double*>(q + npart + nst + nh);
  APCG_CUDA(cudaMemsetAsync(q, 0, npart + nst + 2 * nh, ctx->stream));
  q += npart + nst + 2 * nh;
  int32_t* sptr = reinterpret_cast<int32_t*>(q);
  int32_t* scol = (pat || d16) ? nullptr : reinterpret_cast<int32_t*>(q + nsptr);
  int16_t* sdcol = d16 ? reinterpret_cast<int16_t*>(q + nsptr) : nullptr;
  int32_t* spat = pat ? reinterpret_cast<int32_t*>(q + nsptr) : nullptr;
  double* sval = reinterpret_cast<double*>(q + nsptr + ncol);
  if (P->mode != APCG_MODE_PERSISTENT) {
    APCG_CUDA(cudaMemcpyAsync(sptr, L.d_sptr, sizeof(int32_t) * ((size_t)L.nslices + 1), cudaMemcpyDeviceToDevice,
                              ctx->stream));
    APCG_TRY(sell_fill<double, double>(ctx->stream, L, sptr, A->rowptr, A->col, static_cast<const double*>(A->val),
                                       scol, sdcol, spat, sval));
  }
  char* tail = q + nsptr + ncol + nval;
  P->sys = reinterpret_cast<SysDesc*>(tail);
  P->sres = reinterpret_cast<SysResult*>(tail + sizeof(SysDesc));
  P->next = reinterpret_cast<unsigned int*>(tail + sizeof(SysDesc) + sizeof(SysResult));
  SysDesc d0{};
  d0.row0 = 0;
  d0.n = P->n;
  APCG_CUDA(cudaMemcpyAsync(P->sys, &d0, sizeof(d0), cudaMemcpyHostToDevice, ctx->stream));
  APCG_CUDA(cudaMallocHost((void**)&P->sres_host, sizeof(SysResult)));
  P->padded = L.padded;
  a.A.n = P->n;
  a.A.nslices = L.nslices;
  a.A.sptr = sptr;
  a.A.col = scol;
  a.A.dcol = sdcol;
  a.A.poff = spat;
  a.A.val = sval;
  a.A.long_rows = L.long_rows;
  APCG_CUDA(cudaMallocHost((void**)&P->st_host, sizeof(TqState)));
  {
    std::lock_guard<std::mutex> g(global_mutex());
    P->id = register_memory(ws, total);
  }
  // A0: the Jacobi diagonal, checked once here.
  OpScope op(ctx);
  op.read(A->id).write(P->id);
  APCG_TRY(op.begin());
  if (P->n > 0) APCG_TRY(launch_jacobi_setup(ctx, A, vecs[0]));
  APCG_TRY(op.finish());
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));
  counters().host_syncs++;
  APCG_TRY(ctx_check_device_error(ctx));
  *out = P.release();
  return APCG_OK;
}

apcg_status check_solve_args(Plan P, apcg_vec b, apcg_vec x) {
  APCG_CHECK(P, "plan is NULL");
  APCG_CHECK(b && x, "b or x is NULL");
  APCG_CHECK(b->dtype == APCG_F64 && x->dtype == APCG_F64, "b and x must be float64");
  APCG_CHECK(b->n == P->n && x->n == P->n, "b/x length differs from the matrix size %d", P->n);
  APCG_CHECK(P->n == 0 || (aligned16(b->dptr) && aligned16(x->dptr)), "b/x must be 16-byte aligned");
  APCG_CHECK(b->dptr != x->dptr || P->n == 0, "b and x must not alias");
  return APCG_OK;
}

}  // namespace tq
}  // namespace apcg

using namespace apcg;

extern "C" {

apcg_status apcg_tfqmr_plan_create(apcg_ctx ctx_in, apcg_mat A, const apcg_cg_opts* opts, apcg_tfqmr_plan* out) {
  APCG_CHECK(A && out, "NULL argument");
  APCG_CHECK(A->dtype == APCG_F64 && A->nrows == A->ncols, "TFQMR takes a square float64 matrix");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  return tq::plan_create(ctx, A, opts, out);
}

apcg_status apcg_tfqmr_plan_solve(apcg_tfqmr_plan P, apcg_vec b, apcg_vec x, apcg_cg_result* res) {
  APCG_CHECK(res, "res is NULL");
  APCG_TRY(tq::check_solve_args(P, b, x));
  double* xp = static_cast<double*>(x->dptr);
  const double* bp = static_cast<const double*>(b->dptr);
  if (P->mode == APCG_MODE_ASYNC_GRAPH) APCG_TRY(tq::build_graph(P, xp));
  OpScope op(P->ctx);
  op.read(P->A.id).read(b->id).rw(x->id).rw(P->id);
  APCG_TRY(op.begin());
  apcg_status st = P->mode == APCG_MODE_HOST_SYNC    ? tq::solve_host_sync(P, bp, xp)
                   : P->mode == APCG_MODE_PERSISTENT ? tq::enqueue_persistent(P, bp, xp)
                                                     : tq::enqueue_async(P, bp, xp, P->mode == APCG_MODE_ASYNC_GRAPH);
  apcg_status st2 = op.finish();
  APCG_TRY(st);
  APCG_TRY(st2);
  if (P->mode != APCG_MODE_HOST_SYNC) APCG_TRY(tq::finish_async(P));
  tq::fill_result(P, res);
  return APCG_OK;
}

apcg_status apcg_tfqmr_plan_destroy(apcg_tfqmr_plan P) { return tq::plan_destroy(P); }

apcg_status apcg_tfqmr_plan_layout(apcg_tfqmr_plan P, apcg_plan_layout* out) {
  APCG_CHECK(P && out, "plan or out is NULL");
  const bool copy = P->mode != APCG_MODE_PERSISTENT && P->a.A.sptr != nullptr;
  describe_layout(copy, dev::col_format(P->a.A), P->group, P->a.A.nslices, P->padded, out);
  return APCG_OK;
}

apcg_status apcg_tfqmr_solve(apcg_ctx ctx, apcg_mat A, apcg_vec b, apcg_vec x, const apcg_cg_opts* opts,
                             apcg_cg_result* res) {
  APCG_CHECK(res, "res is NULL");
  apcg_tfqmr_plan P = nullptr;
  APCG_TRY(apcg_tfqmr_plan_create(ctx, A, opts, &P));
  apcg_status st = apcg_tfqmr_plan_solve(P, b, x, res);
  tq::plan_destroy(P);
  return st;
}

}  // extern "C"
