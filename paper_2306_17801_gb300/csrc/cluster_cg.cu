// Whole Jacobi-PCG solves inside one thread-block cluster.
//
// For systems small enough that a kernel launch costs more than an
// iteration's work, the entire solve runs in one launch: a cluster of C CTAs
// (one per SM, C <= 16) owns one system.  CTA `rank` owns a contiguous slice
// of rpc = 2^shift rows; each thread keeps x, r, z, D^-1 and w of its rows in
// registers, and the CTA keeps its slice of p in shared memory, where the
// other CTAs of the cluster read it through distributed shared memory during
// the SpMV.  The two reductions of an iteration ((p,w); (r,z) with (r,r) on
// test iterations) are block sums published to a shared-memory slot and
// combined after a cluster barrier by every CTA in the same fixed rank order,
// so every CTA holds bit-identical alpha, beta and convergence decisions and
// the control flow stays uniform across the cluster.  A third cluster barrier
// per iteration publishes the updated p.  No host round trip, no grid-wide
// synchronisation and no global-memory reduction are needed.
//
// The arithmetic is the textbook Jacobi-PCG of Sec. 4.1-4.2 in the step order
// of the mixed-API CG example of Sec. 3.3, as in cg.cu.  Batched solves run a
// persistent grid of clusters that take systems from an atomic work queue in
// longest-first order.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "cluster_cg.hpp"
#include "kernels_common.cuh"

namespace cgx = cooperative_groups;

namespace apcg {
namespace {

constexpr int kMaxCluster = 16;

// Sum NV values over the cluster.  Every thread of every CTA returns the same
// totals (ranks combined in order 0..C-1 by the same warp tree everywhere).
template <int NV>
__device__ __forceinline__ void cluster_sum(double (&v)[NV], double* s_red, double (*s_slot)[4],
                                            double* const* s_peer_slot, double* s_tot, int& parity, int C,
                                            cgx::cluster_group& cl) {
  dev::block_sum<NV>(v, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s_slot[parity][k] = v[k];
  }
  cl.sync();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < C ? s_peer_slot[lane][parity * 4 + k] : 0.0;
      t = dev::warp_sum(t);
      if (lane == 0) s_tot[k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = s_tot[k];
  parity ^= 1;
}

template <int R>
__global__ void __launch_bounds__(kClusterThreads) cg_cluster_kernel(ClusterArgs a) {
  cgx::cluster_group cl = cgx::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int tpb = blockDim.x;
  extern __shared__ double s_p[];  // this CTA's slice of p
  __shared__ double s_slot[2][4];
  __shared__ double s_red[4 * kClusterThreads];
  __shared__ double s_tot[4];
  __shared__ double* s_peer[kMaxCluster];
  __shared__ double* s_peer_slot[kMaxCluster];
  __shared__ int s_sys;
  if (threadIdx.x < C) {
    s_peer[threadIdx.x] = cl.map_shared_rank(s_p, (unsigned)threadIdx.x);
    s_peer_slot[threadIdx.x] = cl.map_shared_rank(&s_slot[0][0], (unsigned)threadIdx.x);
  }
  __syncthreads();
  int parity = 0;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_sys = (int)atomicAdd(a.next, 1u);
    cl.sync();
    const int idx = *cl.map_shared_rank(&s_sys, 0u);
    cl.sync();  // every CTA has read the index before rank 0 may overwrite it or exit
    if (idx >= a.nsys) break;
    const int s = a.order ? a.order[idx] : idx;
    const SysDesc d = a.sys[s];
    const int n = d.n;
    const int64_t row0 = d.row0;
    int shift = 0;
    while (((n + C - 1) / C) > (1 << shift)) ++shift;
    const int rpc = 1 << shift;
    const int lbase = rank * rpc;
    const int32_t* __restrict__ rowptr = a.rowptr + row0;
    const int32_t* __restrict__ col = a.col;
    const double* __restrict__ val = a.val;
    double xk[R], rk[R], zk[R], dk[R], wk[R];
    int lk[R];
    bool vk[R];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int loc = threadIdx.x + k * tpb;
      lk[k] = loc;
      vk[k] = loc < rpc && lbase + loc < n;
      xk[k] = rk[k] = zk[k] = dk[k] = wk[k] = 0.0;
      if (vk[k]) {
        const int i = lbase + loc;
        const int32_t e0 = rowptr[i], e1 = rowptr[i + 1];
        double ax = 0.0, dg = 0.0;
        for (int32_t e = e0; e < e1; ++e) {
          const int32_t j = col[e];
          const double aij = val[e];
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
    cluster_sum<4>(v, s_red, s_slot, s_peer_slot, s_tot, parity, C, cl);
    double rho = v[0], rr = v[1];
    const double bb = v[2];
    const double tol = fmax(a.rtol * sqrt(bb), a.atol);
    const int max_it = a.max_it > 0 ? a.max_it : (n > 0 ? 10 * n : 10);
    const int kchk = a.check_every;
    const bool record = (a.hist_len > 0) && (idx == 0) && rank == 0 && threadIdx.x == 0;
    int it = 0;
    int done = 0;
    if (v[3] > 0.0)
      done = kDoneBadDiagonal;
    else if (sqrt(rr) <= tol)
      done = kDoneConverged;
    while (!done) {
      // w = A p (p of other CTAs through distributed shared memory)
      double g[1] = {0.0};
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (vk[k]) {
          const int i = lbase + lk[k];
          const int32_t e0 = rowptr[i], e1 = rowptr[i + 1];
          double w = 0.0;
          for (int32_t e = e0; e < e1; ++e) {
            const int32_t j = col[e];
            const int owner = j >> shift;
            const int lj = j & (rpc - 1);
            const double pj = owner == rank ? s_p[lj] : s_peer[owner][lj];
            w = fma(val[e], pj, w);
          }
          wk[k] = w;
          g[0] = fma(s_p[lk[k]], w, g[0]);
        }
      }
      cluster_sum<1>(g, s_red, s_slot, s_peer_slot, s_tot, parity, C, cl);
      const double gamma = g[0];
      if (!(gamma > 0.0) || !isfinite(gamma)) {
        done = kDoneBreakdown;
        break;
      }
      const double alpha = rho / gamma;
      if (record && it < a.hist_len) a.alpha_h[it] = alpha;
      ++it;
      const bool check = (it % kchk == 0) || it >= max_it;
      double u[2] = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < R; ++k) {
        if (vk[k]) {
          xk[k] = fma(alpha, s_p[lk[k]], xk[k]);
          rk[k] = fma(-alpha, wk[k], rk[k]);
          zk[k] = dk[k] * rk[k];
          u[0] = fma(rk[k], zk[k], u[0]);
          if (check) u[1] = fma(rk[k], rk[k], u[1]);
        }
      }
      cluster_sum<2>(u, s_red, s_slot, s_peer_slot, s_tot, parity, C, cl);
      const double rz = u[0];
      if (check) rr = u[1];
      if ((check && rr == 0.0) || rz == 0.0)
        done = kDoneConverged;
      else if (check && sqrt(rr) <= tol)
        done = kDoneConverged;
      else if (it >= max_it)
        done = kDoneNotConverged;
      else if (!isfinite(rz) || (check && !isfinite(rr)))
        done = kDoneBreakdown;
      if (done) break;
      const double beta = rz / rho;
      rho = rz;
      if (record && it - 1 < a.hist_len) a.beta_h[it - 1] = beta;
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (vk[k]) s_p[lk[k]] = fma(beta, s_p[lk[k]], zk[k]);
      cl.sync();  // the new p is visible to the whole cluster before the next SpMV
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (vk[k]) a.x[row0 + lbase + lk[k]] = xk[k];
    if (rank == 0 && threadIdx.x == 0) {
      SysResult* res = a.res + s;
      res->iters = it;
      res->done = done;
      res->rr = rr;
      res->bnorm2 = bb;
    }
  }
}

template <int R>
cudaError_t launch_r(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s) {
  auto kern = cg_cluster_kernel<R>;
  const size_t smem = sizeof(double) * (size_t)sh.rpc_max;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * sh.C), 1, 1);
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
  return cudaLaunchKernelEx(&cfg, kern, args);
}

template <int R>
int max_clusters_r(const ClusterShape& sh) {
  auto kern = cg_cluster_kernel<R>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  const size_t smem = sizeof(double) * (size_t)sh.rpc_max;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)sh.C, 1, 1);
  cfg.blockDim = dim3((unsigned)sh.tpb, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
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

ClusterShape cluster_shape_for(int n_max, int C) {
  ClusterShape sh;
  sh.C = C;
  const int rpc = cluster_rows_per_cta(n_max, C);
  sh.rpc_max = rpc;
  sh.tpb = rpc >= kClusterThreads ? kClusterThreads : std::max(128, ((rpc + 31) / 32) * 32);
  sh.R = (rpc + sh.tpb - 1) / sh.tpb;
  sh.R = sh.R <= 1 ? 1 : sh.R <= 2 ? 2 : sh.R <= 4 ? 4 : 8;
  sh.ok = rpc <= kClusterThreads * 8;
  return sh;
}

ClusterShape schedulable_shape(int n_max, int C) {
  // Halve the cluster until the device can hold one; larger slices per CTA follow.
  ClusterShape sh = cluster_shape_for(n_max, C);
  while (sh.ok && sh.C > 1 && max_active_clusters(sh) < 1) sh = cluster_shape_for(n_max, sh.C / 2);
  if (sh.ok && max_active_clusters(sh) < 1) sh.ok = false;
  return sh;
}

ClusterShape default_cluster_shape(int n) {
  // Spread small systems over as many SMs as a cluster has (the float64 pipe
  // of one SM retires two lanes per cycle), keeping at least 256 rows per CTA.
  int C = 1;
  while (C < kMaxCluster && cluster_rows_per_cta(n, C) > 256) C *= 2;
  return schedulable_shape(n, C);
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
