// Whole-solve Jacobi-TFQMR (Sec. 4.3) in one thread-block cluster per system,
// for systems of at most 16384 rows (two rows per thread of 16 CTAs x 512).
//
// The arithmetic is that of tfqmr.cu (left Jacobi, r* = r0, the two half-steps,
// M u formed as M w + beta M u2, the pending x update of a half-step applied
// with the next rewrite of d), laid out as the CG cluster kernel lays out CG:
// CTA `rank` owns a power-of-two slice of rows, each thread keeps its rows'
// x, u, u2, w, d, v, p, q, r* and D^-1 in registers, and the CTA's slices of
// u2 and w -- the two vectors an SpMV gathers -- live in shared memory, where
// the other CTAs read them through distributed shared memory.  An iteration
// is four cluster sums ((v, r*) for alpha, ||w|| after each half-step, and
// (w, r*) for beta); every CTA adds the partial sums in the same order, so the
// decisions are uniform across the cluster.  Systems come from the same
// longest-first work queue as the batched CG kernel.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "cluster_cg.hpp"
#include "cluster_loop.cuh"

namespace apcg {
namespace {

using clu::cgx::cluster_group;

// sum over the row's entries of a_ij y_j, y gathered from the CTAs' slices
template <class Rows>
__device__ __forceinline__ double row_gather(const Rows& g, const double* __restrict__ val, int i, const double* s_y,
                                             double* const* peer_y, int rank) {
  double acc = 0.0;
  for (int32_t e = g.rowptr[i]; e < g.rowptr[i + 1]; ++e) {
    const int32_t j = g.col[e];
    const int owner = j >> g.shift;
    const int lj = j & (g.rpc - 1);
    acc = fma(val[e], owner == rank ? s_y[lj] : peer_y[owner][lj], acc);
  }
  return acc;
}

template <int R>
__global__ void __launch_bounds__(kClusterThreads, 1) tfqmr_cluster_kernel(ClusterArgs a, int rpc_max) {
  cluster_group cl = clu::cgx::this_cluster();
  extern __shared__ double dyn[];
  double* s_u2 = dyn;            // this CTA's slice of u2
  double* s_w = dyn + rpc_max;   // this CTA's slice of w (and of u = r0 for the first M u)
  __shared__ clu::Block B;
  const clu::Shared S = clu::setup_block(B, cl, s_u2, s_w);
  double* const* peer_u2 = reinterpret_cast<double* const*>(B.peer_data[0]);
  double* const* peer_w = reinterpret_cast<double* const*>(B.peer_data[1]);
  int parity = 0;
  for (;;) {
    const int idx = clu::next_system(B, a.next, cl, S.rank);
    if (idx >= a.nsys) break;
    const int s = a.order ? a.order[idx] : idx;
    const SysDesc sd = a.sys[s];
    const int64_t row0 = sd.row0;
    const clu::Rows g = clu::make_rows(sd.n, S.C, S.rank, a.rowptr + row0, a.col);
    const int hist = idx == 0 ? a.hist_len : 0;
    double xk[R], uk[R], u2k[R], wk[R], dd[R], vk[R], pk[R], qk[R], rs[R], di[R];
    double v3[3] = {0.0, 0.0, 0.0};
    // set-up: r0 = D^-1 (b - A x0), u = w = r* = r0, d = 0
#pragma unroll
    for (int k = 0; k < R; ++k) {
      xk[k] = uk[k] = u2k[k] = wk[k] = dd[k] = vk[k] = pk[k] = qk[k] = rs[k] = di[k] = 0.0;
      if (clu::owns<R>(g, k)) {
        const int loc = threadIdx.x + k * blockDim.x;
        const int i = g.lbase + loc;
        double ax = 0.0, dg = 0.0;
        for (int32_t e = g.rowptr[i]; e < g.rowptr[i + 1]; ++e) {
          const int32_t j = g.col[e];
          const double aij = a.val[e];
          ax = fma(aij, a.x[row0 + j], ax);
          if (j == i) dg += aij;
        }
        const bool bad = !(dg != 0.0) || !isfinite(dg);
        di[k] = bad ? 0.0 : 1.0 / dg;
        if (bad) v3[2] += 1.0;
        const double bi = a.b[row0 + i];
        const double r0 = di[k] * (bi - ax);
        const double bh = di[k] * bi;
        xk[k] = a.x[row0 + i];
        uk[k] = wk[k] = rs[k] = r0;
        s_w[loc] = r0;
        v3[0] = fma(r0, r0, v3[0]);
        v3[1] = fma(bh, bh, v3[1]);
      }
    }
    clu::cluster_sum<3>(v3, S, parity, cl);  // also publishes u = r0
    double rho = v3[0], tau = sqrt(v3[0]);
    const double bb = v3[1];
    const double tol = fmax(a.rtol * sqrt(bb), a.atol);
    const int max_it = a.max_it > 0 ? a.max_it : (sd.n > 0 ? 10 * sd.n : 10);
    int it = 0, done = 0;
    double alpha = 0.0, beta = 0.0, theta = 0.0, eta = 0.0, co = 0.0, eta_x = 0.0;
    bool pending = false;
    if (v3[2] > 0.0)
      done = kDoneBadDiagonal;
    else if (!isfinite(v3[0]) || !isfinite(bb))  // a non-finite b or x0
      done = kDoneBreakdown;
    else if (tau <= tol)
      done = kDoneConverged;
    if (!done) {
      // p = M u, v = p, sigma = (v, r*)
      double sg[1] = {0.0};
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (clu::owns<R>(g, k)) {
          const int i = g.lbase + threadIdx.x + k * blockDim.x;
          pk[k] = vk[k] = di[k] * row_gather(g, a.val, i, s_w, peer_w, S.rank);
          sg[0] = fma(vk[k], rs[k], sg[0]);
        }
      clu::cluster_sum<1>(sg, S, parity, cl);
      if (sg[0] == 0.0 || !isfinite(sg[0])) {
        done = kDoneBreakdown;
      } else {
        alpha = rho / sg[0];
        if (hist > 0 && S.rank == 0 && threadIdx.x == 0) a.alpha_h[0] = alpha;
      }
    }
    // The scalar recurrences after each cluster sum run in thread 0 and reach every thread with the totals
    // (clu::cluster_sum's scalars hook): computed by every thread, each float64 square root and division would
    // occupy every warp's sub-partition pipe.  Same operations in the same order: the same bits.
    while (!done) {
      // odd half-step: u2 = u - alpha v, w -= alpha p, d = u + co d (after the pending x update)
      double ww[1] = {0.0};
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (clu::owns<R>(g, k)) {
          if (pending) xk[k] = fma(eta_x, dd[k], xk[k]);
          u2k[k] = fma(-alpha, vk[k], uk[k]);
          wk[k] = fma(-alpha, pk[k], wk[k]);
          dd[k] = fma(co, dd[k], uk[k]);
          ww[0] = fma(wk[k], wk[k], ww[0]);
          s_u2[threadIdx.x + k * blockDim.x] = u2k[k];
        }
      // t: [1] theta, [2] tau, [3] eta, [4] co, [5] 1 = breakdown, 2 = quasi-residual zero
      clu::cluster_sum<1>(ww, S, parity, cl, [&](double* t) {  // also publishes u2
        const double th = sqrt(t[0]) / tau;
        const double c = 1.0 / sqrt(1.0 + th * th);
        const double ta = tau * th * c;
        const double et = c * c * alpha;
        t[1] = th;
        t[2] = ta;
        t[3] = et;
        t[4] = th * th * et / alpha;
        t[5] = (!isfinite(th) || !isfinite(ta)) ? 1.0 : ta == 0.0 ? 2.0 : 0.0;
      });
      theta = S.tot[1];
      tau = S.tot[2];
      eta = S.tot[3];
      if (S.tot[5] == 1.0) {
        pending = false;
        ++it;
        done = kDoneBreakdown;
        break;
      }
      eta_x = eta;
      pending = true;
      co = S.tot[4];
      if (S.tot[5] == 2.0) {  // the quasi-residual vanished: x is exact after this half-step
        ++it;
        done = kDoneConverged;
        break;
      }
      // even half-step: q = M u2, w -= alpha q, d = u2 + co d (after the pending x update)
      double s2[2] = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (clu::owns<R>(g, k)) {
          const int loc = threadIdx.x + k * blockDim.x;
          const int i = g.lbase + loc;
          qk[k] = di[k] * row_gather(g, a.val, i, s_u2, peer_u2, S.rank);
          xk[k] = fma(eta_x, dd[k], xk[k]);
          wk[k] = fma(-alpha, qk[k], wk[k]);
          dd[k] = fma(co, dd[k], u2k[k]);
          s_w[loc] = wk[k];
          s2[0] = fma(wk[k], wk[k], s2[0]);
          s2[1] = fma(wk[k], rs[k], s2[1]);
        }
      ++it;
      // t: [2] theta, [3] tau, [4] eta, [5] beta, [6] 1 = breakdown (before the pending update),
      // 2 = converged, 3 = not converged, 4 = breakdown (after it)
      clu::cluster_sum<2>(s2, S, parity, cl, [&](double* t) {  // also publishes w
        const double th = sqrt(t[0]) / tau;
        const double c = 1.0 / sqrt(1.0 + th * th);
        const double ta = tau * th * c;
        const double et = c * c * alpha;
        t[2] = th;
        t[3] = ta;
        t[4] = et;
        t[5] = 0.0;
        const bool check = (it % a.check_every == 0) || it >= max_it;
        double f = 0.0;
        if (!isfinite(th) || !isfinite(ta))
          f = 1.0;
        else if (ta == 0.0 || (check && sqrt(2.0 * it + 1.0) * ta <= tol))
          f = 2.0;
        else if (it >= max_it)
          f = 3.0;
        else if (rho == 0.0 || !isfinite(t[1]))
          f = 4.0;
        else
          t[5] = t[1] / rho;
        t[6] = f;
      });
      theta = S.tot[2];
      tau = S.tot[3];
      eta = S.tot[4];
      const double f = S.tot[6];
      if (f == 1.0) {
        pending = false;
        done = kDoneBreakdown;
        break;
      }
      eta_x = eta;
      pending = true;
      if (f != 0.0) {
        done = f == 2.0 ? kDoneConverged : f == 3.0 ? kDoneNotConverged : kDoneBreakdown;
        break;
      }
      beta = S.tot[5];
      rho = s2[1];
      if (it - 1 < hist && S.rank == 0 && threadIdx.x == 0) a.beta_h[it - 1] = beta;
      // directions: u = w + beta u2, p = M w + beta q, v = p + beta (q + beta v), sigma = (v, r*)
      double sg[1] = {0.0};
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (clu::owns<R>(g, k)) {
          const int i = g.lbase + threadIdx.x + k * blockDim.x;
          const double mw = di[k] * row_gather(g, a.val, i, s_w, peer_w, S.rank);
          uk[k] = fma(beta, u2k[k], wk[k]);
          pk[k] = fma(beta, qk[k], mw);
          const double t = fma(beta, vk[k], qk[k]);
          vk[k] = fma(beta, t, pk[k]);
          sg[0] = fma(vk[k], rs[k], sg[0]);
        }
      // t: [1] alpha, [2] co, [3] 1 = breakdown
      clu::cluster_sum<1>(sg, S, parity, cl, [&](double* t) {
        const bool bad = t[0] == 0.0 || !isfinite(t[0]);
        const double al = bad ? 0.0 : rho / t[0];
        t[1] = al;
        t[2] = bad ? 0.0 : theta * theta * eta / al;
        t[3] = bad ? 1.0 : 0.0;
      });
      if (S.tot[3] != 0.0) {
        done = kDoneBreakdown;
        break;
      }
      alpha = S.tot[1];
      co = S.tot[2];
      if (it < hist && S.rank == 0 && threadIdx.x == 0) a.alpha_h[it] = alpha;
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (clu::owns<R>(g, k)) {
        if (pending) xk[k] = fma(eta_x, dd[k], xk[k]);
        a.x[row0 + g.lbase + threadIdx.x + k * blockDim.x] = xk[k];
      }
    if (S.rank == 0 && threadIdx.x == 0) {
      SysResult* res = a.res + s;
      const double bound = sqrt(2.0 * it + 1.0) * tau;
      res->iters = it;
      res->done = done;
      res->rr = bound * bound;
      res->bnorm2 = bb;
      res->outer = 0;
    }
  }
}

size_t tfqmr_smem(const ClusterShape& sh) { return (size_t)2 * sh.rpc_max * sizeof(double); }

template <int R>
cudaError_t tfqmr_launch_r(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s,
                           int* max_clusters) {
  auto kern = tfqmr_cluster_kernel<R>;
  const size_t smem = tfqmr_smem(sh);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(std::max(1, nclusters) * sh.C), 1, 1);
  cfg.blockDim = dim3((unsigned)sh.tpb, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_clusters) return cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg);
  return cudaLaunchKernelEx(&cfg, kern, args, sh.rpc_max);
}

cudaError_t tfqmr_dispatch(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s,
                           int* max_clusters) {
  return sh.R <= 1 ? tfqmr_launch_r<1>(args, sh, nclusters, s, max_clusters)
                   : tfqmr_launch_r<2>(args, sh, nclusters, s, max_clusters);
}

int tfqmr_max_clusters(const ClusterShape& sh) {
  int n = 0;
  ClusterArgs none{};
  if (tfqmr_dispatch(none, sh, 1, nullptr, &n) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

ClusterShape tfqmr_cluster_shape(int n) {
  int C = 1;
  while (C < clu::kMaxCluster && cluster_rows_per_cta(n, C) > 256) C *= 2;
  ClusterShape sh = cluster_shape_for(n, C);
  // fewer CTAs per cluster until the device can schedule one (each halving doubles the rows per thread)
  while (sh.ok && sh.R <= 2 && sh.C > 1 && tfqmr_max_clusters(sh) < 1) sh = cluster_shape_for(n, sh.C / 2);
  if (!sh.ok || sh.R > 2 || tfqmr_max_clusters(sh) < 1) sh.ok = false;
  return sh;
}

cudaError_t launch_cluster_tfqmr(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s) {
  return tfqmr_dispatch(args, sh, nclusters, s, nullptr);
}

}  // namespace apcg
