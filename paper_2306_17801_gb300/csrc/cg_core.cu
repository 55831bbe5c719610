// The three iteration kernels of Jacobi-PCG, for float64 and float32.
//
// The method is textbook Hestenes-Stiefel PCG with diagonal scaling (Sec. 4.1,
// 4.2), its loop body in the order of the mixed-API CG example of Sec. 3.3:
//   w = A p;  gamma = (p,w);  alpha = rho / gamma
//   x += alpha p;  r -= alpha w;  z = D^-1 r;  rho' = (r,z);  rr = (r,r)
//   convergence test every k-th iteration:  sqrt(rr) <= tol
//   beta = rho' / rho;  p = z + beta p;  rho = rho'
// One iteration is three kernels, each fusing the work between two global
// reductions:
//   K1  w = A p and the partial sums of (p,w); the last block forms gamma and
//       alpha = rho / gamma (or flags a breakdown);
//   K2  r -= alpha w, z = D^-1 r (stored for K3), the partial sums of (r,z)
//       and, on test iterations, (r,r); the last block counts the iteration,
//       runs the test and forms beta while the other blocks apply x += alpha p,
//       each to the slice of x of its arrival index;
//   K3  p = z + beta p.
// alpha, beta, rho and the residual norm live in the device state block;
// every kernel starts by reading the 'done' word and returns at once when the
// solve has finished (the semaphore idea of Sec. 5).  Arithmetic and
// accumulation are in T: float64 for the CG solver, float32 for the inner
// solver of mixed-precision refinement; scalars are stored in the state block
// as double (exact for float).  On GB300 the float64 pipe (two lanes per SM
// per cycle) is as scarce as HBM bandwidth, so the float64 kernels spend
// one FMA per nonzero in K1, four float64 operations per row in K2 (five on
// test iterations) and one in K3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "cg_core.hpp"
#include "kernels_common.cuh"
#include "sell.cuh"
#include "stencil.cuh"

namespace apcg {
namespace {

constexpr int kThreads = 256;
constexpr int kUpdV = 1;   // 16-byte vectors per thread and array in K2's sweep (1 measured fastest)
constexpr int kXupdV = 4;  // 16-byte vectors per thread and array in K2's x update (2: +3%, 8: +16% per iteration)
constexpr int kAypxV = 4;  // 16-byte vectors per thread and array in K3
constexpr int kMinGraphBody = 8;  // iterations per body of the captured conditional while node, at least

// 16-byte vector of T: double2 or float4.
template <class T>
struct V16;
template <>
struct V16<double> {
  using type = double2;
  static constexpr int E = 2;
};
template <>
struct V16<float> {
  using type = float4;
  static constexpr int E = 4;
};

template <class T>
struct Args {
  dev::SellView<T> A;  // the plan's sliced-ELL copy of the matrix (CSR plans)
  int32_t n;
  const T* __restrict__ dinv;
  T* x;
  T* r;
  T* p;
  T* w;
  T* z;
  CgState* st;
  T* partials;
  double* alpha_h;
  double* beta_h;
};

template <class T>
Args<T> make_args(const CgCore<T>& c, T* x) {
  Args<T> a;
  a.A = c.A;
  a.n = c.n;
  a.dinv = c.dinv;
  a.x = x;
  a.r = c.r;
  a.p = c.p;
  a.w = c.w;
  a.z = c.z;
  a.st = c.st;
  a.partials = c.partials;
  a.alpha_h = c.alpha_h;
  a.beta_h = c.beta_h;
  return a;
}

__device__ __forceinline__ int32_t read_done(const CgState* st) { return *(volatile const int32_t*)&st->done; }

// Entry of a device-scalar iteration kernel: when it was launched as a programmatic dependent of the previous
// kernel (the launches one by one of the ASYNC mode), wait until that kernel has finished and its writes are
// visible, then let the next kernel's launch begin while this one runs (its blocks start as this kernel's
// blocks leave the SMs).  Without a programmatic edge (graph nodes, other launches) both are no-ops.
__device__ __forceinline__ void dependent_launch_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch configuration of a programmatic dependent launch on stream s.
struct DependentLaunch {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  DependentLaunch(int grid, size_t dyn_smem, cudaStream_t s) {
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = dyn_smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
};

// The state block copied into shared memory at kernel entry by asynchronous 16-byte copies (cp.async, one
// per thread of the first warp; the threads do not wait for them), so that the block completing a grid
// reduction reads the scalars of its epilogue without a round trip to L2 in its serial tail.  The copy is
// taken at entry; only that last block writes the state during the kernel.
constexpr int kStateChunks = (int)(sizeof(CgState) / 16);
static_assert(sizeof(CgState) % 16 == 0, "state block copied in 16-byte pieces");

__device__ __forceinline__ void state_prefetch(const CgState* st, CgState* s) {
  if (threadIdx.x < kStateChunks) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char*>(s) + 16 * threadIdx.x);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                 "l"(__cvta_generic_to_global(reinterpret_cast<const char*>(st) + 16 * threadIdx.x))
                 : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
}

// Completes the copy; the barriers of the grid reduction that follows make it visible to the whole block.
__device__ __forceinline__ void state_prefetch_wait() {
  if (threadIdx.x < kStateChunks) asm volatile("cp.async.wait_all;" ::: "memory");
}

// r = b - A x0, z = D^-1 r, p = z; rho = (r,z), rr = (r,r), bb = (b,b) (float64 solve).
// spmv(epi) applies the operator to x with the given row epilogue.
template <class Spmv>
__device__ __forceinline__ void setup_body(const Args<double>& a, const double* __restrict__ b, double rtol,
                                           double atol, int32_t max_it, int32_t k, int32_t hist_len, Spmv spmv) {
  __shared__ double red[3 * kThreads];
  double v[3] = {0.0, 0.0, 0.0};
  spmv([&](int32_t i, double ax, double) {
    const double bi = __ldg(b + i);
    const double ri = bi - ax;
    const double zi = __ldg(a.dinv + i) * ri;
    a.r[i] = ri;
    a.p[i] = zi;
    v[0] = fma(ri, zi, v[0]);
    v[1] = fma(ri, ri, v[1]);
    v[2] = fma(bi, bi, v[2]);
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
    // a non-finite b or x0 is a breakdown, not convergence against an infinite tolerance
    st->done = (!isfinite(tot[1]) || !isfinite(tot[2])) ? kDoneBreakdown : (sqrt(tot[1]) <= tol) ? kDoneConverged : 0;
  }
}

template <bool LONG, int CF>
__global__ void __launch_bounds__(kThreads) setup_kernel(Args<double> a, const double* __restrict__ b, double rtol,
                                                         double atol, int32_t max_it, int32_t k, int32_t hist_len) {
  setup_body(a, b, rtol, atol, max_it, k, hist_len,
             [&](auto epi) { dev::sell_spmv<false, LONG, double, 8, CF>(a.A, a.x, epi); });
}

// The stencil operator travels as its own parameter (not in Args, which every
// kernel takes: a larger Args costs the CSR kernels registers).
template <int NP>
__global__ void __launch_bounds__(kThreads) setup_stencil_kernel(Args<double> a, dev::StencilView S,
                                                                 const double* __restrict__ b, double rtol,
                                                                 double atol, int32_t max_it, int32_t k,
                                                                 int32_t hist_len) {
  setup_body(a, b, rtol, atol, max_it, k, hist_len,
             [&](auto epi) { dev::stencil_spmv<NP, false, double>(S, a.x, epi); });
}

// The last block of K1: gamma, and alpha = rho / gamma (device mode) or a breakdown flag.  pre: the state
// as the kernel found it (done was 0: the kernel returns at entry otherwise).  RECHECK: the kernel's own warps
// may have set done meanwhile (a bounded wait of the staged SpMV that ran out); then gamma is incomplete and
// done keeps that code.
template <bool HOST, bool RECHECK, class T>
__device__ __forceinline__ void k1_finish(const Args<T>& a, T gamma, const CgState& pre) {
  CgState* st = a.st;
  st->gamma = gamma;
  if (!HOST && !(RECHECK && read_done(st))) {
    if (!(gamma > T(0)) || !isfinite(gamma)) {
      st->done = kDoneBreakdown;
    } else {
      const T alpha = (T)pre.rho / gamma;
      st->alpha = alpha;
      if (pre.iter < pre.hist_len) a.alpha_h[pre.iter] = alpha;
    }
  }
}

// K1 (G: group size of the long-row path; CF: column format, dev::ColFormat; STAGED: float32 values staged
// in shared memory by bulk copies, dev::sell_spmv_staged, with stage_smem_bytes of dynamic shared memory)
template <bool HOST, bool LONG, class T, int G = 8, int CF = dev::kColIndex, bool STAGED = false>
__global__ void __launch_bounds__(kThreads) k1_kernel(Args<T> a) {
  if (!HOST) dependent_launch_entry();
  if (!HOST && read_done(a.st)) return;
  // the staged float32 instance keeps no copy: with it the compiler schedules the staged SpMV on 40 instead of
  // 48 registers and the kernel runs about 40% slower (160^3 refinement, inner K1 100.6 -> 142.5 us)
  __shared__ __align__(16) CgState pre;
  if (!HOST && !STAGED) state_prefetch(a.st, &pre);
  __shared__ T red[kThreads];
  T v[1] = {T(0)};
  auto epi = [&](int32_t i, T s, T p_i) {
    a.w[i] = s;
    v[0] = fma(p_i, s, v[0]);
  };
  if constexpr (STAGED) {
    static_assert(std::is_same<T, float>::value && CF == dev::kColPattern && LONG, "staged K1: float32 offset lists");
    extern __shared__ __align__(128) unsigned char stage_smem[];
    const int w = threadIdx.x >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(stage_smem) + 2 * w;
    float* stage = reinterpret_cast<float*>(stage_smem + dev::kStageBarrierBytes) + (size_t)w * 2 * a.A.stage_cap * 32;
    dev::sell_spmv_staged<true, G>(a.A, a.p, stage, bars, &a.st->done, kDoneTimeout, epi);
  } else {
    dev::sell_spmv<true, LONG, T, G, CF>(a.A, a.p, epi);
  }
  if (!HOST) state_prefetch_wait();
  T tot[1];
  if (dev::grid_sum_last<1>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0)
    k1_finish<HOST, STAGED>(a, tot[0], STAGED ? *a.st : pre);
}

// K1 on a stencil operator (stencil.cuh): the same per-row arithmetic.  Resident blocks per SM by term
// count: the 7-term instance at one (the compiler then keeps more gathers in flight on 78 registers, three
// blocks per SM: 128^3 K1 44.0 -> 42.4 us against 48 registers and five), the 27-term one at three (80
// registers; 128 and two blocks 1% slower, 64 and four 2% slower), the others where their register counts
// were before these bounds.
template <int NP>
constexpr int stencil_min_blocks() {
  return NP == 7 ? 1 : NP == 27 ? 3 : NP == 9 ? 5 : NP == 0 ? 2 : 6;
}
template <bool HOST, int NP, class T>
__global__ void __launch_bounds__(kThreads, stencil_min_blocks<NP>()) k1_stencil_kernel(Args<T> a,
                                                                                       dev::StencilView S) {
  if (!HOST && read_done(a.st)) return;
  __shared__ __align__(16) CgState pre;
  if (!HOST) state_prefetch(a.st, &pre);
  __shared__ T red[kThreads];
  T v[1] = {T(0)};
  dev::stencil_spmv<NP, true, T>(S, a.p, [&](int32_t i, T s, T p_i) {
    a.w[i] = s;
    v[0] = fma(p_i, s, v[0]);
  });
  if (!HOST) state_prefetch_wait();
  T tot[1];
  if (dev::grid_sum_last<1>(v, a.partials, &a.st->ticket, red, tot) && threadIdx.x == 0)
    k1_finish<HOST, false>(a, tot[0], pre);
}

// K2.  The test runs when the iteration count is a multiple of k or reaches
// max_it, decided from the state block at kernel entry, so one kernel serves
// every position of a captured block.
template <bool HOST, class T>
__global__ void __launch_bounds__(kThreads, 4) k2_kernel(Args<T> a, double alpha_host, cudaGraphConditionalHandle cond,
                                                         int32_t use_cond) {
  using VT = typename V16<T>::type;
  constexpr int E = V16<T>::E;
  if (!HOST) dependent_launch_entry();
  if (!HOST && read_done(a.st)) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      a.st->body_runs += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  __shared__ __align__(16) CgState pre;
  if (!HOST) state_prefetch(a.st, &pre);
  const T alpha = HOST ? (T)alpha_host : (T)a.st->alpha;
  bool check = true;
  if (!HOST) {
    const int32_t it = a.st->iter + 1;
    check = (it % a.st->check_every == 0) || it >= a.st->max_it;
  }
  __shared__ T red[2 * kThreads];
  T v[2] = {T(0), T(0)};
  T acc_rz[kUpdV], acc_rr[kUpdV];  // independent chains, combined in a fixed order below
#pragma unroll
  for (int u = 0; u < kUpdV; ++u) acc_rz[u] = acc_rr[u] = T(0);
  const int64_t n = a.n, nv = n / E, stride = (int64_t)gridDim.x * blockDim.x;
  VT* rv = reinterpret_cast<VT*>(a.r);
  VT* zv = reinterpret_cast<VT*>(a.z);
  const VT* wv = reinterpret_cast<const VT*>(a.w);
  const VT* dv = reinterpret_cast<const VT*>(a.dinv);
  auto sweep = [&](auto with_rr) {
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nv; i0 += kUpdV * stride) {
      VT rr[kUpdV], ww[kUpdV], dd[kUpdV];
#pragma unroll
      for (int u = 0; u < kUpdV; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < nv) {
          rr[u] = rv[i];
          ww[u] = dev::ld_stream2(wv + i);
          dd[u] = __ldg(dv + i);
        }
      }
#pragma unroll
      for (int u = 0; u < kUpdV; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < nv) {
          T* re = reinterpret_cast<T*>(&rr[u]);
          const T* we = reinterpret_cast<const T*>(&ww[u]);
          const T* de = reinterpret_cast<const T*>(&dd[u]);
          VT zz;
          T* ze = reinterpret_cast<T*>(&zz);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            re[e] = fma(-alpha, we[e], re[e]);
            ze[e] = de[e] * re[e];
            acc_rz[u] = fma(re[e], ze[e], acc_rz[u]);
            if (decltype(with_rr)::value) acc_rr[u] = fma(re[e], re[e], acc_rr[u]);
          }
          rv[i] = rr[u];
          zv[i] = zz;
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
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int64_t i = nv * E; i < n; ++i) {
      a.x[i] = fma(alpha, a.p[i], a.x[i]);
      const T ri = fma(-alpha, a.w[i], a.r[i]);
      const T zi = a.dinv[i] * ri;
      a.r[i] = ri;
      a.z[i] = zi;
      v[0] = fma(ri, zi, v[0]);
      if (check) v[1] = fma(ri, ri, v[1]);
    }
  }
  if (!HOST) state_prefetch_wait();
  T tot[2];
  unsigned arrival;
  const bool last = dev::grid_sum_last<2>(v, a.partials, &a.st->ticket, red, tot, &arrival);
  // x += alpha p once the block's partial sums are out: every block but the one that arrives last takes the
  // slice of x of its arrival index, so these bytes move while the last block runs the serial tail of the
  // reduction (a single block takes all of x)
  {
    const int64_t parts = gridDim.x > 1 ? (int64_t)gridDim.x - 1 : 1;
    if (!last || gridDim.x == 1) {
      const int64_t lo = nv * (int64_t)arrival / parts, hi = nv * ((int64_t)arrival + 1) / parts;
      VT* xv = reinterpret_cast<VT*>(a.x);
      const VT* pv = reinterpret_cast<const VT*>(a.p);
      for (int64_t i0 = lo + threadIdx.x; i0 < hi; i0 += kXupdV * kThreads) {
        VT xx[kXupdV], pp[kXupdV];
#pragma unroll
        for (int u = 0; u < kXupdV; ++u) {
          const int64_t i = i0 + u * kThreads;
          if (i < hi) {
            xx[u] = xv[i];
            pp[u] = __ldg(pv + i);
          }
        }
#pragma unroll
        for (int u = 0; u < kXupdV; ++u) {
          const int64_t i = i0 + u * kThreads;
          if (i < hi) {
            T* xe = reinterpret_cast<T*>(&xx[u]);
            const T* pe = reinterpret_cast<const T*>(&pp[u]);
#pragma unroll
            for (int e = 0; e < E; ++e) xe[e] = fma(alpha, pe[e], xe[e]);
            xv[i] = xx[u];
          }
        }
      }
    }
  }
  if (last && threadIdx.x == 0) {
    CgState* st = a.st;
    const T rz = tot[0], rr = tot[1];
    st->rho_new = rz;
    if (check) st->rr = rr;
    if (!HOST) {
      const int32_t it = pre.iter + 1;
      st->iter = it;
      int32_t done = 0;
      // An exactly zero residual ends the solve at any iteration; between
      // tests (r, D^-1 r) = 0 stands for r = 0 (D^-1 is positive).
      if ((check && rr == T(0)) || rz == T(0))
        done = kDoneConverged;
      else if (check && sqrt(rr) <= (T)pre.tol)
        done = kDoneConverged;
      else if (it >= pre.max_it)
        done = kDoneNotConverged;
      else if (!isfinite(rz) || (check && !isfinite(rr)))
        done = kDoneBreakdown;
      if (!done) {
        const T beta = rz / (T)pre.rho;
        st->beta = beta;
        st->rho = rz;
        if (it - 1 < pre.hist_len) a.beta_h[it - 1] = beta;
      }
      st->done = done;
      if (use_cond) {
        st->body_runs = pre.body_runs + 1;
        cudaGraphSetConditional(cond, done ? 0u : 1u);
      }
    }
  }
}

// K3: p = z + beta p (one FMA per row).
template <bool HOST, class T>
__global__ void __launch_bounds__(kThreads, 4) k3_kernel(Args<T> a, double beta_host) {
  using VT = typename V16<T>::type;
  constexpr int E = V16<T>::E;
  if (!HOST) dependent_launch_entry();
  if (!HOST && read_done(a.st)) return;
  const T beta = HOST ? (T)beta_host : (T)a.st->beta;
  const int64_t n = a.n, nv = n / E, stride = (int64_t)gridDim.x * blockDim.x;
  VT* pv = reinterpret_cast<VT*>(a.p);
  const VT* zv = reinterpret_cast<const VT*>(a.z);
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nv; i0 += kAypxV * stride) {
    VT pp[kAypxV], zz[kAypxV];
#pragma unroll
    for (int u = 0; u < kAypxV; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < nv) {
        pp[u] = pv[i];
        zz[u] = dev::ld_stream2(zv + i);
      }
    }
#pragma unroll
    for (int u = 0; u < kAypxV; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < nv) {
        T* pe = reinterpret_cast<T*>(&pp[u]);
        const T* ze = reinterpret_cast<const T*>(&zz[u]);
#pragma unroll
        for (int e = 0; e < E; ++e) pe[e] = fma(beta, pe[e], ze[e]);
        pv[i] = pp[u];
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int64_t i = nv * E; i < n; ++i) a.p[i] = fma(beta, a.p[i], a.z[i]);
}

template <class K>
int occupancy_grid(K kernel, int sms, int64_t want, size_t dyn_smem = 0) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, dyn_smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t g = (int64_t)per_sm * sms;
  if (want < g) g = want;
  if (g > dev::kMaxPartials) g = dev::kMaxPartials;
  return g < 1 ? 1 : (int)g;
}

template <bool HOST, class T>
apcg_status k1_stencil_dispatch(const CgCore<T>& c, const Args<T>& a, cudaStream_t s) {
  switch (c.S.npts) {
    case 5: k1_stencil_kernel<HOST, 5, T><<<c.grid_spmv, kThreads, 0, s>>>(a, c.S); break;
    case 7: k1_stencil_kernel<HOST, 7, T><<<c.grid_spmv, kThreads, 0, s>>>(a, c.S); break;
    case 9: k1_stencil_kernel<HOST, 9, T><<<c.grid_spmv, kThreads, 0, s>>>(a, c.S); break;
    case 27: k1_stencil_kernel<HOST, 27, T><<<c.grid_spmv, kThreads, 0, s>>>(a, c.S); break;
    default: k1_stencil_kernel<HOST, 0, T><<<c.grid_spmv, kThreads, 0, s>>>(a, c.S); break;
  }
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

// The K1 instance for the plan's layout: one entry at a time, or groups of G.  The float64 plans choose G in
// 5..9 (csr_layout); the float32 inner solves of the refinement keep 0 or 8 with per-entry column indices:
// they are bound by HBM, not by wasted FMA slots, and larger groups cost them occupancy (refinement at 160^3
// with groups of 9: 110.2 against 107.3 ms).
template <bool HOST, class T, int CF>
void* k1_instance_d(const CgCore<T>& c) {
  if constexpr (std::is_same<T, double>::value) {
    switch (c.A.long_rows) {
      case 5: return (void*)k1_kernel<HOST, true, T, 5, CF>;
      case 6: return (void*)k1_kernel<HOST, true, T, 6, CF>;
      case 7: return (void*)k1_kernel<HOST, true, T, 7, CF>;
      case 9: return (void*)k1_kernel<HOST, true, T, 9, CF>;
      default: break;
    }
  }
  // float32 with per-slice offset lists: 27-entry rows in three whole groups of 9 (no column loads, so the
  // larger group costs no occupancy; 160^3 refinement 86.2 -> 81.6 ms)
  if constexpr (CF == dev::kColPattern && std::is_same<T, float>::value) {
    if (c.A.long_rows && c.A.stage_cap > 0)
      return c.A.long_rows == 9 ? (void*)k1_kernel<HOST, true, T, 9, CF, true>
                                : (void*)k1_kernel<HOST, true, T, 8, CF, true>;
    if (c.A.long_rows == 9) return (void*)k1_kernel<HOST, true, T, 9, CF>;
  }
  return c.A.long_rows ? (void*)k1_kernel<HOST, true, T, 8, CF> : (void*)k1_kernel<HOST, false, T, 8, CF>;
}

// Dynamic shared memory of the plan's K1 instance (the staged float32 form only).
template <class T>
int k1_dyn_smem(const CgCore<T>& c) {
  if constexpr (std::is_same<T, float>::value)
    if (c.S.n == 0 && c.A.poff && c.A.long_rows && c.A.stage_cap > 0)
      return dev::stage_smem_bytes(c.A.stage_cap, kThreads / 32);
  return 0;
}

template <bool HOST, class T>
void* k1_instance(const CgCore<T>& c) {
  if (c.A.poff) return k1_instance_d<HOST, T, dev::kColPattern>(c);
  if (c.A.dcol) return k1_instance_d<HOST, T, dev::kColOff16>(c);
  return k1_instance_d<HOST, T, dev::kColIndex>(c);
}

template <bool HOST, class T>
apcg_status k1_dispatch(const CgCore<T>& c, const Args<T>& a, cudaStream_t s) {
  if (c.S.n > 0) return k1_stencil_dispatch<HOST>(c, a, s);
  void* args[] = {const_cast<Args<T>*>(&a)};
  if (!HOST && c.pdl) {
    DependentLaunch L(c.grid_spmv, (size_t)k1_dyn_smem(c), s);
    APCG_CUDA(cudaLaunchKernelExC(&L.cfg, k1_instance<HOST>(c), args));
    return APCG_OK;
  }
  APCG_CUDA(cudaLaunchKernel(k1_instance<HOST>(c), dim3(c.grid_spmv), dim3(kThreads), args, (size_t)k1_dyn_smem(c),
                             s));
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

}  // namespace

template <class T>
void core_configure(CgCore<T>& c, int64_t nnz, int sms) {
  (void)nnz;
  const int64_t slices = ((int64_t)c.n + 31) / 32;
  const int64_t spmv_blocks = (slices + kThreads / 32 - 1) / (kThreads / 32);
  const int64_t vec_blocks = (((int64_t)c.n / V16<T>::E) + (int64_t)kThreads * kUpdV - 1) / ((int64_t)kThreads * kUpdV);
  if (c.S.n > 0) {  // the grid of the instance that runs (one resident wave)
    void* ks = c.S.npts == 5 ? (void*)k1_stencil_kernel<false, 5, T> : c.S.npts == 7 ? (void*)k1_stencil_kernel<false, 7, T>
             : c.S.npts == 9 ? (void*)k1_stencil_kernel<false, 9, T> : c.S.npts == 27 ? (void*)k1_stencil_kernel<false, 27, T>
             : (void*)k1_stencil_kernel<false, 0, T>;
    c.grid_spmv = occupancy_grid(ks, sms, ((int64_t)c.n + kThreads - 1) / kThreads);
  }
  else {
    const int dyn = k1_dyn_smem(c);
    if (dyn > 48 * 1024) {  // above the default limit: opt in (both instances, once per plan)
      cudaFuncSetAttribute(k1_instance<false>(c), cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
      cudaFuncSetAttribute(k1_instance<true>(c), cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
      cudaGetLastError();
    }
    c.grid_spmv = occupancy_grid(k1_instance<false>(c), sms, spmv_blocks, (size_t)dyn);
  }
  c.grid_vec = occupancy_grid((void*)k2_kernel<false, T>, sms, vec_blocks);
}

template <class T>
apcg_status core_k1(const CgCore<T>& c, T* x, cudaStream_t s, bool host) {
  const Args<T> a = make_args(c, x);
  return host ? k1_dispatch<true>(c, a, s) : k1_dispatch<false>(c, a, s);
}

template <class T>
apcg_status core_k2(const CgCore<T>& c, T* x, cudaStream_t s, bool host, double alpha,
                    cudaGraphConditionalHandle cond, int use_cond) {
  const Args<T> a = make_args(c, x);
  if (host)
    k2_kernel<true, T><<<c.grid_vec, kThreads, 0, s>>>(a, alpha, cond, use_cond);
  else if (c.pdl) {
    DependentLaunch L(c.grid_vec, 0, s);
    APCG_CUDA(cudaLaunchKernelEx(&L.cfg, k2_kernel<false, T>, a, alpha, cond, use_cond));
  } else
    k2_kernel<false, T><<<c.grid_vec, kThreads, 0, s>>>(a, alpha, cond, use_cond);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

template <class T>
apcg_status core_k3(const CgCore<T>& c, T* x, cudaStream_t s, bool host, double beta) {
  const Args<T> a = make_args(c, x);
  if (host)
    k3_kernel<true, T><<<c.grid_vec, kThreads, 0, s>>>(a, beta);
  else if (c.pdl) {
    DependentLaunch L(c.grid_vec, 0, s);
    APCG_CUDA(cudaLaunchKernelEx(&L.cfg, k3_kernel<false, T>, a, beta));
  } else
    k3_kernel<false, T><<<c.grid_vec, kThreads, 0, s>>>(a, beta);
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

template <class T>
void core_release_graph(CgCore<T>& c) {
  if (c.exec) cudaGraphExecDestroy(c.exec);
  if (c.graph) cudaGraphDestroy(c.graph);
  c.exec = nullptr;
  c.graph = nullptr;
  c.graph_x = nullptr;
}

template <class T>
apcg_status core_build_graph(CgCore<T>& c, T* x, cudaStream_t upload) {
  if (c.exec && c.graph_x == x) return APCG_OK;
  core_release_graph(c);
  if (!c.cap_stream) APCG_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  APCG_CUDA(cudaGraphCreate(&g, 0));
  c.graph = g;
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
  APCG_CUDA(cudaStreamBeginCaptureToGraph(c.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  apcg_status st = APCG_OK;
  // k iterations per body, or the smallest multiple of k of at least kMinGraphBody: every K2 still tests at its
  // own iteration count and kernels after a finished test return at entry, while the while node itself costs
  // about 4 us per body (64^2 at k = 1: 18.0 -> 14.1 us per iteration)
  c.body = c.k >= kMinGraphBody ? c.k : c.k * ((kMinGraphBody + c.k - 1) / c.k);
  for (int j = 0; j < c.body && st == APCG_OK; ++j) {
    st = core_k1(c, x, c.cap_stream, false);
    if (st == APCG_OK) st = core_k2(c, x, c.cap_stream, false, 0.0, h, j == c.body - 1 ? 1 : 0);
    if (st == APCG_OK) st = core_k3(c, x, c.cap_stream, false, 0.0);
  }
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(c.cap_stream, &captured);
  if (st != APCG_OK) return st;
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  APCG_CUDA(cudaGraphInstantiate(&c.exec, g, 0));
  APCG_CUDA(cudaGraphUpload(c.exec, upload));
  c.graph_x = x;
  return APCG_OK;
}

apcg_status core_setup_f64(const CgCore<double>& c, const double* b, double* x, double rtol, double atol,
                           cudaStream_t s) {
  const Args<double> a = make_args(c, x);
  if (c.S.n > 0) {
    const int g = c.grid_spmv;
    switch (c.S.npts) {
      case 5: setup_stencil_kernel<5><<<g, kThreads, 0, s>>>(a, c.S, b, rtol, atol, c.max_it, c.k, c.hist_len); break;
      case 7: setup_stencil_kernel<7><<<g, kThreads, 0, s>>>(a, c.S, b, rtol, atol, c.max_it, c.k, c.hist_len); break;
      case 9: setup_stencil_kernel<9><<<g, kThreads, 0, s>>>(a, c.S, b, rtol, atol, c.max_it, c.k, c.hist_len); break;
      case 27: setup_stencil_kernel<27><<<g, kThreads, 0, s>>>(a, c.S, b, rtol, atol, c.max_it, c.k, c.hist_len); break;
      default: setup_stencil_kernel<0><<<g, kThreads, 0, s>>>(a, c.S, b, rtol, atol, c.max_it, c.k, c.hist_len); break;
    }
  } else {
    const int g = c.grid_spmv;
    const bool lr = c.A.long_rows != 0;
#define APCG_SETUP(L, F) setup_kernel<L, F><<<g, kThreads, 0, s>>>(a, b, rtol, atol, c.max_it, c.k, c.hist_len)
    if (c.A.poff)
      lr ? APCG_SETUP(true, dev::kColPattern) : APCG_SETUP(false, dev::kColPattern);
    else if (c.A.dcol)
      lr ? APCG_SETUP(true, dev::kColOff16) : APCG_SETUP(false, dev::kColOff16);
    else
      lr ? APCG_SETUP(true, dev::kColIndex) : APCG_SETUP(false, dev::kColIndex);
#undef APCG_SETUP
  }
  APCG_CUDA(cudaGetLastError());
  return APCG_OK;
}

template void core_configure<double>(CgCore<double>&, int64_t, int);
template void core_configure<float>(CgCore<float>&, int64_t, int);
template apcg_status core_k1<double>(const CgCore<double>&, double*, cudaStream_t, bool);
template apcg_status core_k1<float>(const CgCore<float>&, float*, cudaStream_t, bool);
template apcg_status core_k2<double>(const CgCore<double>&, double*, cudaStream_t, bool, double,
                                     cudaGraphConditionalHandle, int);
template apcg_status core_k2<float>(const CgCore<float>&, float*, cudaStream_t, bool, double,
                                    cudaGraphConditionalHandle, int);
template apcg_status core_k3<double>(const CgCore<double>&, double*, cudaStream_t, bool, double);
template apcg_status core_k3<float>(const CgCore<float>&, float*, cudaStream_t, bool, double);
template apcg_status core_build_graph<double>(CgCore<double>&, double*, cudaStream_t);
template apcg_status core_build_graph<float>(CgCore<float>&, float*, cudaStream_t);
template void core_release_graph<double>(CgCore<double>&);
template void core_release_graph<float>(CgCore<float>&);

}  // namespace apcg
