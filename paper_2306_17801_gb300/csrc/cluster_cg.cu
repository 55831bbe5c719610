// Whole Jacobi-PCG solves inside one thread-block cluster.
//
// For systems small enough that a kernel launch costs more than an
// iteration's work, the entire solve runs in one launch: a cluster of C CTAs
// (one per SM, C <= 16) owns one system (geometry and iteration loop in
// cluster_loop.cuh).  Two kernels:
//   cg_cluster_kernel     float64 Jacobi-PCG (the paper's method, Sec. 4.2, in
//                         the step order of the mixed-API example of Sec. 3.3);
//   cg_cluster_ir_kernel  float64 iterative refinement around a float32
//                         Jacobi-PCG (the mixed-precision extension): the
//                         outer residual r = b - A x, its norm and x += d in
//                         float64, the inner solve entirely in float32.
// No host round trip, no grid-wide synchronisation and no global-memory
// reduction are needed.  Batched solves run a persistent grid of clusters that
// take systems from an atomic work queue in longest-first order.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "cluster_cg.hpp"
#include "cluster_loop.cuh"

namespace apcg {
namespace {

using clu::cgx::cluster_group;

// Float64 Jacobi-PCG, one cluster per system.  Two CTAs per SM up to R = 4: at 128 registers the R = 4
// instance left one CTA, i.e. one system's cluster, per SM, and every cluster sum and barrier of that system
// idled the SM; at 64 registers (208 bytes of spill) two systems share each SM (1024 shifted 5-point
// systems: the 8281..16384-row class 16.0 -> 10.4 ms, the batch 46.0k -> 68-70k solves/s).
template <int R>
__global__ void __launch_bounds__(kClusterThreads, (R >= 8 ? 1 : 2)) cg_cluster_kernel(ClusterArgs a) {
  cluster_group cl = clu::cgx::this_cluster();
  extern __shared__ double s_p[];  // this CTA's slice of p
  __shared__ clu::Block B;
  const clu::Shared S = clu::setup_block(B, cl, s_p, nullptr);
  double* const* peer_p = reinterpret_cast<double* const*>(B.peer_data[0]);
  int parity = 0;
  for (;;) {
    const int idx = clu::next_system(B, a.next, cl, S.rank);
    if (idx >= a.nsys) break;
    const int s = a.order ? a.order[idx] : idx;
    const SysDesc d = a.sys[s];
    const int64_t row0 = d.row0;
    const clu::Rows g = clu::make_rows(d.n, S.C, S.rank, a.rowptr + row0, a.col);
    double xk[R], rk[R], zk[R], dk[R];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < R; ++k) {
      xk[k] = rk[k] = zk[k] = dk[k] = 0.0;
      if (clu::owns<R>(g, k)) {
        const int loc = threadIdx.x + k * blockDim.x;
        const int i = g.lbase + loc;
        const int32_t e0 = g.rowptr[i], e1 = g.rowptr[i + 1];
        double ax = 0.0, dg = 0.0;
        for (int32_t e = e0; e < e1; ++e) {
          const int32_t j = g.col[e];
          const double aij = a.val[e];
          ax = fma(aij, a.x[row0 + j], ax);
          if (j == i) dg += aij;
        }
        double di;
        if (a.dinv) {
          di = a.dinv[row0 + i];
        } else {
          const bool bad = !(dg != 0.0) || !isfinite(dg);
          di = bad ? 0.0 : 1.0 / dg;
          if (bad) v[3] += 1.0;
        }
        const double bi = a.b[row0 + i];
        dk[k] = di;
        xk[k] = a.x[row0 + i];
        rk[k] = bi - ax;
        zk[k] = di * rk[k];
        s_p[loc] = zk[k];
        v[0] = fma(rk[k], zk[k], v[0]);
        v[1] = fma(rk[k], rk[k], v[1]);
        v[2] = fma(bi, bi, v[2]);
      }
    }
    clu::cluster_sum<4>(v, S, parity, cl);  // also publishes p = z
    double rr = v[1];
    const double bb = v[2];
    const double tol = fmax(a.rtol * sqrt(bb), a.atol);
    const int max_it = a.max_it > 0 ? a.max_it : (d.n > 0 ? 10 * d.n : 10);
    int it = 0, done = 0;
    if (v[3] > 0.0)
      done = kDoneBadDiagonal;
    else if (!isfinite(rr) || !isfinite(bb))  // a non-finite b or x0
      done = kDoneBreakdown;
    else if (sqrt(rr) <= tol)
      done = kDoneConverged;
    else
      done = clu::pcg_loop<R, double, double>(g, a.val, s_p, peer_p, xk, rk, zk, dk, v[0], rr, tol, max_it,
                                              a.check_every, S, parity, cl, a.alpha_h + (int64_t)s * a.hist_len,
                                              a.beta_h + (int64_t)s * a.hist_len, a.hist_len, &it);
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (clu::owns<R>(g, k)) a.x[row0 + g.lbase + threadIdx.x + k * blockDim.x] = xk[k];
    if (S.rank == 0 && threadIdx.x == 0) {
      SysResult* res = a.res + s;
      res->iters = it;
      res->done = done;
      res->rr = rr;
      res->bnorm2 = bb;
      res->outer = 0;
    }
  }
}

// Matrix value as float64 (outer residual) or float32 (inner solve).
__device__ __forceinline__ double val64(const ClusterArgs& a, int64_t e) {
  return a.val ? a.val[e] : (double)a.val32[e];
}
__device__ __forceinline__ float val32(const ClusterArgs& a, int64_t e) {
  return a.val32 ? a.val32[e] : (float)a.val[e];
}

// Float64 refinement around a float32 Jacobi-PCG, one cluster per system.
// Shared memory: the CTA's slice of x (float64, read by the other CTAs in the
// outer residual) followed by its slice of the inner p (float32).
// TI: the type of the values the inner solve reads (float: val32; double: val rounded as read).
template <int R, class TI>
__global__ void __launch_bounds__(kClusterThreads, (R >= 8 ? 1 : 2)) cg_cluster_ir_kernel(ClusterArgs a, int rpc_max) {
  const TI* const vin = std::is_same<TI, float>::value ? (const TI*)a.val32 : (const TI*)a.val;
  cluster_group cl = clu::cgx::this_cluster();
  extern __shared__ double s_dyn[];
  double* s_x = s_dyn;
  float* s_p = reinterpret_cast<float*>(s_dyn + rpc_max);
  __shared__ clu::Block B;
  const clu::Shared S = clu::setup_block(B, cl, s_x, s_p);
  double* const* peer_x = reinterpret_cast<double* const*>(B.peer_data[0]);
  float* const* peer_p = reinterpret_cast<float* const*>(B.peer_data[1]);
  int parity = 0;
  for (;;) {
    const int idx = clu::next_system(B, a.next, cl, S.rank);
    if (idx >= a.nsys) break;
    const int s = a.order ? a.order[idx] : idx;
    const SysDesc d = a.sys[s];
    const int64_t row0 = d.row0;
    const clu::Rows g = clu::make_rows(d.n, S.C, S.rank, a.rowptr + row0, a.col);
    // Float32 Jacobi diagonal and the float64 start.
    double xk[R];
    float dk[R];
    float bad[1] = {0.0f};
#pragma unroll
    for (int k = 0; k < R; ++k) {
      xk[k] = 0.0;
      dk[k] = 0.0f;
      if (clu::owns<R>(g, k)) {
        const int loc = threadIdx.x + k * blockDim.x;
        const int i = g.lbase + loc;
        float dg = 0.0f;
        for (int32_t e = g.rowptr[i]; e < g.rowptr[i + 1]; ++e)
          if (g.col[e] == i) dg += val32(a, e);
        const bool b_ = !(dg != 0.0f) || !isfinite(dg);
        dk[k] = b_ ? 0.0f : 1.0f / dg;
        if (b_) bad[0] += 1.0f;
        xk[k] = a.x[row0 + i];
      }
    }
    clu::cluster_sum<1>(bad, S, parity, cl);
    int done = bad[0] > 0.0f ? kDoneBadDiagonal : 0;
    int outer = 0, inner_total = 0;
    double rr64 = 0.0, bb = 0.0;
    while (!done) {
      // r = b - A x in float64 (x of other CTAs through distributed shared memory)
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (clu::owns<R>(g, k)) s_x[threadIdx.x + k * blockDim.x] = xk[k];
      cl.sync();
      double r64[R];
      double v[2] = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < R; ++k) {
        r64[k] = 0.0;
        if (clu::owns<R>(g, k)) {
          const int i = g.lbase + threadIdx.x + k * blockDim.x;
          double ax = 0.0;
          for (int32_t e = g.rowptr[i]; e < g.rowptr[i + 1]; ++e) {
            const int32_t j = g.col[e];
            const int owner = j >> g.shift;
            const int lj = j & (g.rpc - 1);
            const double xj = owner == S.rank ? s_x[lj] : peer_x[owner][lj];
            ax = fma(val64(a, e), xj, ax);
          }
          const double bi = a.b[row0 + i];
          r64[k] = bi - ax;
          v[0] = fma(r64[k], r64[k], v[0]);
          v[1] = fma(bi, bi, v[1]);
        }
      }
      clu::cluster_sum<2>(v, S, parity, cl);
      rr64 = v[0];
      bb = v[1];
      if (!isfinite(rr64) || !isfinite(bb)) {
        done = kDoneBreakdown;
        break;
      }
      if (sqrt(rr64) <= fmax(a.rtol * sqrt(bb), a.atol)) {
        done = kDoneConverged;
        break;
      }
      if (outer == a.max_outer) {
        done = kDoneNotConverged;
        break;
      }
      // Inner float32 solve of A d = (float) r from d = 0.
      float dd[R], rk[R], zk[R];
      float u[2] = {0.0f, 0.0f};
#pragma unroll
      for (int k = 0; k < R; ++k) {
        dd[k] = rk[k] = zk[k] = 0.0f;
        if (clu::owns<R>(g, k)) {
          rk[k] = (float)r64[k];
          zk[k] = dk[k] * rk[k];
          s_p[threadIdx.x + k * blockDim.x] = zk[k];
          u[0] = fmaf(rk[k], zk[k], u[0]);
          u[1] = fmaf(rk[k], rk[k], u[1]);
        }
      }
      clu::cluster_sum<2>(u, S, parity, cl);  // also publishes p = z
      float rr32 = u[1];
      const float tol32 = a.rtol_inner * sqrtf(rr32);
      if (!(rr32 > 0.0f)) {  // the float32 right-hand side vanished: no further progress possible
        done = kDoneNotConverged;
        break;
      }
      int it = 0;
      const int inner_done = clu::pcg_loop<R, float, TI>(g, vin, s_p, peer_p, dd, rk, zk, dk, u[0], rr32, tol32,
                                                         a.max_it, a.check_every, S, parity, cl, nullptr, nullptr, 0,
                                                         &it);
      (void)inner_done;  // a breakdown or the cap still leaves a usable correction
      inner_total += it;
#pragma unroll
      for (int k = 0; k < R; ++k) xk[k] += (double)dd[k];
      ++outer;
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (clu::owns<R>(g, k)) a.x[row0 + g.lbase + threadIdx.x + k * blockDim.x] = xk[k];
    if (S.rank == 0 && threadIdx.x == 0) {
      SysResult* res = a.res + s;
      res->iters = inner_total;
      res->done = done;
      res->rr = rr64;
      res->bnorm2 = bb;
      res->outer = outer;
    }
  }
}

size_t smem_bytes(const ClusterShape& sh) {
  return (size_t)sh.rpc_max * (sh.ir ? sizeof(double) + sizeof(float) : sizeof(double));
}

template <class K>
cudaError_t prepare(K kern, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

cudaLaunchConfig_t make_cfg(const ClusterShape& sh, int nclusters, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * sh.C), 1, 1);
  cfg.blockDim = dim3((unsigned)sh.tpb, 1, 1);
  cfg.dynamicSmemBytes = smem_bytes(sh);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int R>
cudaError_t launch_r(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = make_cfg(sh, nclusters, s, attr);
  if (sh.ir) {
    auto kern = args.val32 ? cg_cluster_ir_kernel<R, float> : cg_cluster_ir_kernel<R, double>;
    cudaError_t e = prepare(kern, cfg.dynamicSmemBytes);
    return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, kern, args, sh.rpc_max);
  }
  auto kern = cg_cluster_kernel<R>;
  cudaError_t e = prepare(kern, cfg.dynamicSmemBytes);
  return e != cudaSuccess ? e : cudaLaunchKernelEx(&cfg, kern, args);
}

template <int R>
int max_clusters_r(const ClusterShape& sh) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = make_cfg(sh, 1, nullptr, attr);
  int n = 0;
  cudaError_t e;
  if (sh.ir) {
    // both value types have the same footprint class; take the larger
    int n2 = 0;
    auto k1 = cg_cluster_ir_kernel<R, float>;
    auto k2 = cg_cluster_ir_kernel<R, double>;
    e = prepare(k1, cfg.dynamicSmemBytes);
    if (e == cudaSuccess) e = prepare(k2, cfg.dynamicSmemBytes);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k1, &cfg);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n2, k2, &cfg);
    if (e == cudaSuccess) n = std::min(n, n2);
  } else {
    auto kern = cg_cluster_kernel<R>;
    e = prepare(kern, cfg.dynamicSmemBytes);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  return n;  // 0: this shape cannot be scheduled on this device
}

}  // namespace

int cluster_rows_per_cta(int n, int C) {
  int shift = 0;
  while (((n + C - 1) / C) > (1 << shift)) ++shift;
  return 1 << shift;
}

ClusterShape cluster_shape_for(int n_max, int C, bool ir) {
  ClusterShape sh;
  sh.C = C;
  sh.ir = ir;
  const int rpc = cluster_rows_per_cta(n_max, C);
  sh.rpc_max = rpc;
  sh.tpb = rpc >= kClusterThreads ? kClusterThreads : std::max(128, ((rpc + 31) / 32) * 32);
  sh.R = (rpc + sh.tpb - 1) / sh.tpb;
  sh.R = sh.R <= 1 ? 1 : sh.R <= 2 ? 2 : sh.R <= 4 ? 4 : 8;
  sh.ok = rpc <= kClusterThreads * 8;
  return sh;
}

ClusterShape schedulable_shape(int n_max, int C, bool ir) {
  ClusterShape sh = cluster_shape_for(n_max, C, ir);
  while (sh.ok && sh.C > 1 && max_active_clusters(sh) < 1) sh = cluster_shape_for(n_max, sh.C / 2, ir);
  if (sh.ok && max_active_clusters(sh) < 1) sh.ok = false;
  return sh;
}

ClusterShape default_cluster_shape(int n, bool ir) {
  // Spread small systems over as many SMs as a cluster has (the float64 pipe
  // of one SM retires two lanes per cycle), keeping at least 256 rows per CTA.
  int C = 1;
  while (C < clu::kMaxCluster && cluster_rows_per_cta(n, C) > 256) C *= 2;
  return schedulable_shape(n, C, ir);
}

cudaError_t launch_cluster_cg(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s) {
  switch (sh.R) {
    case 1: return launch_r<1>(args, sh, nclusters, s);
    case 2: return launch_r<2>(args, sh, nclusters, s);
    case 4: return launch_r<4>(args, sh, nclusters, s);
    default: return launch_r<8>(args, sh, nclusters, s);
  }
}

int max_active_clusters(const ClusterShape& sh) {
  switch (sh.R) {
    case 1: return max_clusters_r<1>(sh);
    case 2: return max_clusters_r<2>(sh);
    case 4: return max_clusters_r<4>(sh);
    default: return max_clusters_r<8>(sh);
  }
}

}  // namespace apcg
