// Device helpers shared by the library's kernels: cache-hinted loads, warp and
// block sums, and the deterministic grid reduction that writes a result
// straight into a device scalar.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace apcg {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxPartials = 4096;  // upper bound on the grid of any reducing kernel

// Streaming loads (evict-first): matrix values and column indices are read
// once per sweep and should not displace the vectors from L2.
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ int16_t ld_stream(const int16_t* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream2(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream2(const float4* p) { return __ldcs(p); }
// Read-only path for gathered vector entries (L1-allocating).
template <class T>
__device__ __forceinline__ T ld_ro(const T* p) {
  return __ldg(p);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;  // valid in lane 0
}

// Sum NV values over the block in a fixed order.  On GB300 every float64
// add is scarce (the float64 pipe retires two lanes per SM per cycle), so the
// tree is not built from shuffles in every warp: each thread parks its values
// in shared memory, lane l of warp 0 adds the values of threads l, l+32, ...
// in order, and one shuffle tree in warp 0 finishes.  smem must hold
// NV * blockDim.x values.  Thread 0 receives the totals in v[].
template <int NV, class T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* smem) {
  const int nt = blockDim.x;
  __syncthreads();  // smem may still be read by a previous call
#pragma unroll
  for (int k = 0; k < NV; ++k) smem[k * nt + threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      T t = T(0);
      for (int i = threadIdx.x; i < nt; i += 32) t += smem[k * nt + i];
      v[k] = warp_sum(t);
    }
  }
}

// Deterministic grid-wide sum of NV values per thread.  Each block writes its
// NV block sums to partials[k * gridDim.x + blockIdx.x]; the block that
// arrives last (atomic ticket) sums the partials in block order and returns
// true; only its thread 0 holds valid totals in tot[].  The ticket is reset
// to zero for the next kernel.  partials must hold NV * gridDim.x values and
// smem NV * blockDim.x values.
template <int NV, class T>
__device__ __forceinline__ bool grid_sum_last(T (&v)[NV], T* partials, unsigned int* ticket, T* smem, T (&tot)[NV]) {
  __shared__ bool s_last;
  block_sum<NV>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  T s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    s[k] = T(0);
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s[k] += __ldcg(partials + k * gridDim.x + i);
  }
  block_sum<NV>(s, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = s[k];
    *ticket = 0u;
  }
  return true;
}

}  // namespace dev
}  // namespace apcg
