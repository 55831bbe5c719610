// Device building blocks of the whole-solve cluster kernels (cluster_cg.cu):
// cluster-wide sums with bit-identical results in every CTA, and the
// Jacobi-PCG iteration loop on the rows a cluster owns, for float64 solves and
// for the float32 inner solves of mixed-precision refinement.
//
// A cluster of C CTAs owns one system.  CTA `rank` owns the slice of rows
// [rank * rpc, (rank + 1) * rpc) (rpc = 2^shift); thread t owns the rows
// rank * rpc + t + k * blockDim.x, k < R, and keeps their vector entries in
// registers.  The CTA's slice of the search direction p lives in shared
// memory, where the SpMV of every CTA reads it through distributed shared
// memory.  All control decisions are taken from cluster sums that every CTA
// forms in the same order, so the control flow is uniform across the cluster
// and every cluster barrier is reached by all of its threads.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "cg_internal.hpp"
#include "cluster_cg.hpp"
#include "kernels_common.cuh"

namespace apcg {
namespace clu {

namespace cgx = cooperative_groups;

constexpr int kMaxCluster = 16;

// Shared-memory bookkeeping of the cluster sums.
struct Shared {
  double* slot;               // the partial sums every CTA pushed to this one, [2][kMaxCluster][4]
  double* const* peer_slot;   // the slot arrays of every CTA of the cluster, [C]
  void* red;                  // block-sum scratch, 4 * blockDim.x values
  double* tot;                // broadcast of the totals and the scalars derived from them, [8]
  int C, rank;
};

// Sum NV values over the block with the adds spread over the SM's four
// sub-partitions (the block sum of the cluster sums below, on the
// latency-critical path of every iteration): each float64 warp instruction
// holds its sub-partition's pipe for about 64 cycles whatever its number of
// active lanes, so a chain of adds in one warp is slow.  Warps 0..3 (one per sub-partition) each add every fourth
// group of 32 values and reduce by shuffles; warp 0 adds their four results.
// The order is fixed, so the result is the same bits on every call.  Not used
// in the grid kernels, where the extra code costs the SpMV a register.  The
// result is valid in threads 0..31; smem must hold NV * blockDim.x values;
// blockDim.x must be a multiple of 32.
template <int NV, class T>
__device__ __forceinline__ void block_sum_quad(T (&v)[NV], T* smem) {
  __shared__ T s_q[NV * 4];
  const int nt = blockDim.x;
  const int nq = nt >= 128 ? 4 : nt >> 5;
  __syncthreads();  // smem and s_q may still be read by a previous call
#pragma unroll
  for (int k = 0; k < NV; ++k) smem[k * nt + threadIdx.x] = v[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  if (q < nq) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T t = smem[k * nt + threadIdx.x];
      for (int i = threadIdx.x + 32 * nq; i < nt; i += 32 * nq) t += smem[k * nt + i];
      t = dev::warp_sum(t);
      if (lane == 0) s_q[k * 4 + q] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T t = lane < nq ? s_q[k * 4 + lane] : T(0);
      t += __shfl_down_sync(dev::kFull, t, 2);
      t += __shfl_down_sync(dev::kFull, t, 1);
      v[k] = t;
    }
  }
}

struct NoScalars {
  __device__ void operator()(double*) const {}
};

// Sum NV values over the cluster.  Each CTA pushes its block sums
// (block_sum_quad) into slot `rank` of every CTA of the cluster (remote stores
// to distributed shared memory, which the cluster barrier's release and
// acquire make visible), and after the barrier every CTA adds its own C slots
// in rank order with the same warp tree of log2(C) levels (C is a power of
// two), so all threads of all CTAs get the same bits without a remote read on
// the critical path (4096 anisotropic systems, batched refinement: 27.0k ->
// 28.5k solves/s; the shorter tree: 64^2 CG 6.46 -> 6.30 us per iteration).
// Slots alternate between two buffers: a buffer is rewritten only two sums
// later, after a barrier that every CTA passes only once done reading it.
// scalars(t) runs in thread 0 once the totals are in t[0 .. NV) and may store
// further scalars derived from them in t[NV .. 8) (a division, a square root,
// a decision), which reach every thread with the totals: computed by every
// thread instead, each float64 operation would occupy every warp's
// sub-partition pipe (about 64 cycles per warp instruction on GB300).
template <int NV, class T, class Scalars = NoScalars>
__device__ __forceinline__ void cluster_sum(T (&v)[NV], const Shared& S, int& parity, cgx::cluster_group& cl,
                                            Scalars scalars = Scalars()) {
  block_sum_quad<NV>(v, reinterpret_cast<T*>(S.red));
  if (threadIdx.x < 32) {  // lane j pushes this CTA's sums into CTA j's slots (remote stores, no round trip)
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double t = __shfl_sync(dev::kFull, (double)v[k], 0);
      if (lane < S.C) S.peer_slot[lane][(parity * kMaxCluster + S.rank) * 4 + k] = t;
    }
  }
  cl.sync();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T t = lane < S.C ? (T)S.slot[(parity * kMaxCluster + lane) * 4 + k] : T(0);
      for (int o = S.C >> 1; o > 0; o >>= 1) t += __shfl_down_sync(dev::kFull, t, o);  // log2(C) steps
      if (lane == 0) S.tot[k] = (double)t;
    }
    if (lane == 0) scalars(S.tot);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = (T)S.tot[k];
  parity ^= 1;
}

// Per-CTA bookkeeping of a whole-solve cluster kernel (static shared memory).
struct Block {
  double slot[2][kMaxCluster][4];
  double red[4 * kClusterThreads];
  double tot[8];
  double* peer_slot[kMaxCluster];
  void* peer_data[2][kMaxCluster];  // the dynamic arrays of every CTA
  int sys;
};

// Map the cluster's shared arrays (slots and up to two dynamic arrays per CTA).
__device__ __forceinline__ Shared setup_block(Block& B, cgx::cluster_group& cl, void* dyn0, void* dyn1) {
  const int C = (int)cl.num_blocks();
  if (threadIdx.x < C) {
    B.peer_slot[threadIdx.x] = cl.map_shared_rank(&B.slot[0][0][0], (unsigned)threadIdx.x);
    B.peer_data[0][threadIdx.x] = cl.map_shared_rank(dyn0, (unsigned)threadIdx.x);
    B.peer_data[1][threadIdx.x] = dyn1 ? cl.map_shared_rank(dyn1, (unsigned)threadIdx.x) : nullptr;
  }
  __syncthreads();
  Shared S;
  S.slot = &B.slot[0][0][0];
  S.peer_slot = B.peer_slot;
  S.red = B.red;
  S.tot = B.tot;
  S.C = C;
  S.rank = (int)cl.block_rank();
  return S;
}

// Next system index of the cluster's work queue (uniform across the cluster).
__device__ __forceinline__ int next_system(Block& B, unsigned int* next, cgx::cluster_group& cl, int rank) {
  if (rank == 0 && threadIdx.x == 0) B.sys = (int)atomicAdd(next, 1u);
  cl.sync();
  const int idx = *cl.map_shared_rank(&B.sys, 0u);
  cl.sync();  // every CTA has read the index before rank 0 may overwrite it or exit
  return idx;
}

// Geometry of the CTA's rows in the current system.
struct Rows {
  int shift, rpc, lbase, n;
  const int32_t* rowptr;  // the system's rows (global nnz positions)
  const int32_t* col;     // system-local column indices
};

__device__ __forceinline__ Rows make_rows(int n, int C, int rank, const int32_t* rowptr_sys, const int32_t* col) {
  Rows g;
  g.shift = 0;
  while (((n + C - 1) / C) > (1 << g.shift)) ++g.shift;
  g.rpc = 1 << g.shift;
  g.lbase = rank * g.rpc;
  g.n = n;
  g.rowptr = rowptr_sys;
  g.col = col;
  return g;
}

template <int R>
__device__ __forceinline__ bool owns(const Rows& g, int k) {
  const int loc = threadIdx.x + k * blockDim.x;
  return loc < g.rpc && g.lbase + loc < g.n;
}

// Jacobi-PCG iterations on the cluster's system until a test stops them.
// On entry: rk = r, zk = D^-1 r, the CTA's slice s_p = z (published by a
// cluster barrier), rho = (r, z); xk is the iterate, updated in place.  The
// test runs when the iteration count is a multiple of kchk or reaches max_it.
// Returns a kDone* code; *iters receives the completed iterations and rr the
// (r,r) of the last test.  Values TV are widened to T.
template <int R, class T, class TV>
__device__ __forceinline__ int pcg_loop(const Rows& g, const TV* __restrict__ val, T* s_p, T* const* s_peer_p, T (&xk)[R],
                        T (&rk)[R], T (&zk)[R], const T (&dk)[R], T rho, T& rr, T tol, int max_it, int kchk,
                        const Shared& S, int& parity, cgx::cluster_group& cl, double* alpha_h, double* beta_h,
                        int hist_len, int* iters) {
  constexpr bool kHoist = std::is_same<T, double>::value;
  T wk[R];
  int it = 0;
  int done = 0;
  while (!done) {
    // w = A p (p of other CTAs through distributed shared memory)
    T gsum[1] = {T(0)};
#pragma unroll
    for (int k = 0; k < R; ++k) {
      wk[k] = T(0);
      if (owns<R>(g, k)) {
        const int loc = threadIdx.x + k * blockDim.x;
        const int i = g.lbase + loc;
        const int32_t e0 = g.rowptr[i], e1 = g.rowptr[i + 1];
        T w = T(0);
        for (int32_t e = e0; e < e1; ++e) {
          const int32_t j = g.col[e];
          const int owner = j >> g.shift;
          const int lj = j & (g.rpc - 1);
          const T pj = owner == S.rank ? s_p[lj] : s_peer_p[owner][lj];
          w = fma((T)val[e], pj, w);
        }
        wk[k] = w;
        gsum[0] = fma(s_p[loc], w, gsum[0]);
      }
    }
    // gamma = (p, w).  float64: thread 0 forms alpha = rho / gamma (t[1]) or flags a breakdown (t[2]) once
    // for the CTA; float32 operations are cheap, every thread forms them (measured faster for the float32
    // inner solves of the refinement kernel)
    T alpha;
    if constexpr (kHoist) {
      cluster_sum<1>(gsum, S, parity, cl, [&](double* t) {
        const T gamma = (T)t[0];
        const bool bad = !(gamma > T(0)) || !isfinite(gamma);
        t[1] = bad ? 0.0 : (double)(rho / gamma);
        t[2] = bad ? 1.0 : 0.0;
      });
      if (S.tot[2] != 0.0) {
        done = kDoneBreakdown;
        break;
      }
      alpha = (T)S.tot[1];
    } else {
      cluster_sum<1>(gsum, S, parity, cl);
      const T gamma = gsum[0];
      if (!(gamma > T(0)) || !isfinite(gamma)) {
        done = kDoneBreakdown;
        break;
      }
      alpha = rho / gamma;
    }
    if (hist_len > 0 && it < hist_len && S.rank == 0 && threadIdx.x == 0) alpha_h[it] = alpha;
    ++it;
    const bool check = (it % kchk == 0) || it >= max_it;
    T u[2] = {T(0), T(0)};
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (owns<R>(g, k)) {
        const int loc = threadIdx.x + k * blockDim.x;
        xk[k] = fma(alpha, s_p[loc], xk[k]);
        rk[k] = fma(-alpha, wk[k], rk[k]);
        zk[k] = dk[k] * rk[k];
        u[0] = fma(rk[k], zk[k], u[0]);
        if (check) u[1] = fma(rk[k], rk[k], u[1]);
      }
    }
    // (r, z) and, on test iterations, (r, r); thread 0 takes the decision (t[3]) and forms beta (t[2])
    const T rr_prev = rr;
    T beta;
    if constexpr (!kHoist) {
      cluster_sum<2>(u, S, parity, cl);
      const T rz = u[0];
      if (check) rr = u[1];
      if ((check && rr == T(0)) || rz == T(0))
        done = kDoneConverged;
      else if (check && sqrt(rr) <= tol)
        done = kDoneConverged;
      else if (it >= max_it)
        done = kDoneNotConverged;
      else if (!isfinite(rz) || (check && !isfinite(rr)))
        done = kDoneBreakdown;
      if (done) break;
      beta = rz / rho;
      rho = rz;
    } else {
      cluster_sum<2>(u, S, parity, cl, [&](double* t) {
        const T rz = (T)t[0];
        const T rrn = check ? (T)t[1] : rr_prev;
        int d = 0;
        if ((check && rrn == T(0)) || rz == T(0))
          d = kDoneConverged;
        else if (check && sqrt(rrn) <= tol)
          d = kDoneConverged;
        else if (it >= max_it)
          d = kDoneNotConverged;
        else if (!isfinite(rz) || (check && !isfinite(rrn)))
          d = kDoneBreakdown;
        t[2] = d ? 0.0 : (double)(rz / rho);
        t[3] = (double)d;
      });
      const T rz = u[0];
      if (check) rr = u[1];
      done = (int)S.tot[3];
      if (done) break;
      beta = (T)S.tot[2];
      rho = rz;
    }
    if (hist_len > 0 && it - 1 < hist_len && S.rank == 0 && threadIdx.x == 0) beta_h[it - 1] = beta;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (owns<R>(g, k)) {
        const int loc = threadIdx.x + k * blockDim.x;
        s_p[loc] = fma(beta, s_p[loc], zk[k]);
      }
    }
    cl.sync();  // the new p is visible to the whole cluster before the next SpMV
  }
  *iters = it;
  return done;
}

}  // namespace clu
}  // namespace apcg
