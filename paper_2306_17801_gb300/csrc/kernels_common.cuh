// Device helpers shared by the library's kernels: cache-hinted loads, warp and
// block sums, and the deterministic grid reduction that writes a result
// straight into a device scalar.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

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

// ---------------------------------------------------------------- exact sums of float64 values
//
// A float64 add holds its SM sub-partition's float64 pipe for about 64 cycles
// on GB300, so a tree of float64 adds is a long serial chain: at the end of
// every block, and -- in the block that completes a grid reduction -- a tail
// during which every other SM idles.  These sums run on the integer pipes:
// each value is converted exactly to a 128-bit two's-complement fixed-point
// number aligned to the largest exponent among the values summed (bits more
// than kShift + 52 below the largest value's leading bit are dropped, a
// relative 2^-112 of the largest term), the numbers are added exactly as
// 24-bit limbs by warp reductions, and the total is rounded to float64 once
// (round to nearest even).  The result does not depend on the order of the
// values, so it is deterministic, and it is at least as accurate as any
// float64 summation order.  An infinity or NaN among the values makes the
// total NaN.
namespace fx {

constexpr int kShift = 60;          // the largest value's significand (< 2^53) lands below bit 113
constexpr unsigned kNonFinite = 2047;

// Biased exponent field of v, with zeros and subnormals counted as 1 (their scale).
__device__ __forceinline__ unsigned exp_field(double v) {
  const unsigned e = (unsigned)(__double_as_longlong(v) >> 52) & 0x7ffu;
  return e ? e : 1u;
}

__device__ __forceinline__ void add128(uint64_t& h, uint64_t& l, uint64_t bh, uint64_t bl) {
  const uint64_t t = l + bl;
  h += bh + (t < l ? 1ull : 0ull);
  l = t;
}

__device__ __forceinline__ void neg128(uint64_t& h, uint64_t& l) {
  l = ~l + 1ull;
  h = ~h + (l == 0ull ? 1ull : 0ull);
}

// 64-bit shifts with PTX semantics: a shift amount of 64 or more yields 0 (no undefined behaviour, no branch).
__device__ __forceinline__ uint64_t shl64(uint64_t x, unsigned s) {
  uint64_t r;
  asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}
__device__ __forceinline__ uint64_t shr64(uint64_t x, unsigned s) {
  uint64_t r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}

// v * 2^(1075 - E + kShift) truncated toward zero, as a 128-bit two's-complement number (E >= exp_field(v),
// E < kNonFinite).  Branch-free: lanes holding values of different scales do not diverge.
__device__ __forceinline__ void to_fixed(double v, unsigned E, uint64_t& h, uint64_t& l) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const unsigned ef = (unsigned)(bits >> 52) & 0x7ffu;
  const uint64_t m = (bits & ((1ull << 52) - 1ull)) | (ef ? (1ull << 52) : 0ull);
  const int sh = (int)(ef ? ef : 1u) - (int)E + kShift;  // <= kShift < 64
  h = shr64(m, (unsigned)(64 - sh));                      // 0 unless sh > 0
  l = sh >= 0 ? shl64(m, (unsigned)sh) : shr64(m, (unsigned)(-sh));
  const uint64_t nl = ~l + 1ull, nh = ~h + (l == 0ull ? 1ull : 0ull);
  const bool neg = (bits >> 63) != 0ull;
  l = neg ? nl : l;
  h = neg ? nh : h;
}

// Bits [24j, 24j + 24) of the 128-bit pattern (h, l).
template <int J>
__device__ __forceinline__ unsigned limb(uint64_t h, uint64_t l) {
  constexpr int s = 24 * J;
  uint64_t v;
  if constexpr (s == 0)
    v = l;
  else if constexpr (s < 64)
    v = (l >> s) | (s > 40 ? (h << (64 - s)) : 0ull);
  else
    v = h >> (s - 64);
  return (unsigned)(v & 0xffffffull);
}

// X * 2^(E - 1075 - kShift) rounded to float64 (X = (h, l), two's complement).  The result is assembled
// from its bits on the integer pipes; only a subnormal result goes through scalbn.
__device__ __forceinline__ double from_fixed(uint64_t h, uint64_t l, unsigned E) {
  const bool neg = (int64_t)h < 0;
  if (neg) neg128(h, l);
  if (h == 0ull && l == 0ull) return 0.0;
  const int p = h ? 127 - __clzll((long long)h) : 63 - __clzll((long long)l);  // leading bit
  uint64_t mant;  // 2^52 <= mant < 2^53 after normalisation; value = mant * 2^(r + E - 1075 - kShift)
  int r = p - 52;
  if (p <= 52) {
    mant = l << (52 - p);
  } else {
    mant = r < 64 ? ((l >> r) | (h << (64 - r))) : (h >> (r - 64));
    mant &= (1ull << 53) - 1ull;
    const int g = r - 1;  // guard bit; sticky = any bit below it
    const unsigned guard = (unsigned)((g < 64 ? (l >> g) : (h >> (g - 64))) & 1ull);
    const bool sticky = g < 64 ? (g > 0 && (l << (64 - g)) != 0ull)
                               : (l != 0ull || (g > 64 && (h << (128 - g)) != 0ull));
    if (guard && (sticky || (mant & 1ull))) {
      if (++mant == (1ull << 53)) {
        mant >>= 1;
        ++r;
      }
    }
  }
  const int be = r + (int)E - kShift;  // biased exponent of the result
  uint64_t bits;
  if (be >= 2047)
    bits = 0x7ff0000000000000ull;
  else if (be >= 1)
    bits = ((uint64_t)be << 52) | (mant & ((1ull << 52) - 1ull));
  else
    bits = (uint64_t)__double_as_longlong(scalbn((double)mant, be - 1075));
  return __longlong_as_double((long long)(bits | (neg ? 0x8000000000000000ull : 0ull)));
}

// Block-wide maximum of NV exponents; every thread receives them.  s: NV * 32 words of shared memory.
template <int NV>
__device__ __forceinline__ void block_max(unsigned (&e)[NV], unsigned* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const unsigned m = __reduce_max_sync(kFull, e[k]);
    if (lane == 0) s[k * 32 + wid] = m;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) e[k] = __reduce_max_sync(kFull, lane < nw ? s[k * 32 + lane] : 0u);
}

// Block-wide exact sum of NV fixed-point numbers aligned to E[k]; thread 0 receives the totals rounded to
// float64 (NaN where E[k] marks a non-finite value).  s: NV * 6 * 32 words of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum_fixed(const uint64_t (&h)[NV], const uint64_t (&l)[NV],
                                                const unsigned (&E)[NV], unsigned* s, double (&out)[NV]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    unsigned L[6];
    L[0] = __reduce_add_sync(kFull, limb<0>(h[k], l[k]));
    L[1] = __reduce_add_sync(kFull, limb<1>(h[k], l[k]));
    L[2] = __reduce_add_sync(kFull, limb<2>(h[k], l[k]));
    L[3] = __reduce_add_sync(kFull, limb<3>(h[k], l[k]));
    L[4] = __reduce_add_sync(kFull, limb<4>(h[k], l[k]));
    L[5] = __reduce_add_sync(kFull, limb<5>(h[k], l[k]));
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < 6; ++j) s[(k * 6 + j) * 32 + wid] = L[j];
    }
  }
  __syncthreads();
  if (wid == 0) {
    uint64_t S = 0ull;  // lane t < 6 NV: limb t % 6 of value t / 6 summed over the warps (< 2^34)
    if (lane < 6 * NV)
      for (int w = 0; w < nw; ++w) S += s[lane * 32 + w];
    // lane k < NV assembles value k from its six limb sums and rounds it
    const int kk = lane < NV ? lane : 0;
    uint64_t th = 0ull, tl = 0ull;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const uint64_t Sj = __shfl_sync(kFull, S, kk * 6 + j);
      const int sh = 24 * j;
      if (sh == 0)
        add128(th, tl, 0ull, Sj);
      else if (sh < 64)
        add128(th, tl, Sj >> (64 - sh), Sj << sh);
      else
        add128(th, tl, Sj << (sh - 64), 0ull);
    }
    unsigned Ek = E[0];
#pragma unroll
    for (int k = 1; k < NV; ++k) Ek = kk == k ? E[k] : Ek;
    const double r = Ek >= kNonFinite ? __longlong_as_double(0x7ff8000000000000ll) : from_fixed(th, tl, Ek);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double rk = __shfl_sync(kFull, r, k);
      if (lane == 0) out[k] = rk;
    }
  }
}

}  // namespace fx

// Exact block sum of NV float64 values per thread (fx above); thread 0 receives the totals.  smem must hold
// NV * 224 32-bit words (NV * blockDim.x doubles for blocks of at least 112 threads).
template <int NV>
__device__ __forceinline__ void block_sum_exact(double (&v)[NV], double* smem) {
  unsigned* s = reinterpret_cast<unsigned*>(smem);
  __syncthreads();  // smem may still be read by a previous call
  unsigned E[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) E[k] = fx::exp_field(v[k]);
  fx::block_max<NV>(E, s);
  uint64_t h[NV], l[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    h[k] = l[k] = 0ull;
    if (E[k] < fx::kNonFinite) fx::to_fixed(v[k], E[k], h[k], l[k]);
  }
  fx::block_sum_fixed<NV>(h, l, E, s + NV * 32, v);
}

// The last block's exact sum of the float64 partials of a grid reduction (fx above): partials[k * gridDim.x
// + i], gridDim.x <= 16 * blockDim.x; thread 0 receives the totals.  smem: NV * blockDim.x doubles.
template <int NV>
__device__ __forceinline__ void grid_partials_exact(const double* partials, double* smem, double (&tot)[NV]) {
  // this thread's partials i = threadIdx.x + j * blockDim.x: the first kKeep kept in registers between the
  // pass that finds the largest exponent and the pass that converts them
  constexpr int kKeep = 4;
  const int G = (int)gridDim.x, bd = (int)blockDim.x;
  double keep[NV][kKeep];
  unsigned E[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    E[k] = 1u;
#pragma unroll
    for (int j = 0; j < kKeep; ++j) {
      const int i = (int)threadIdx.x + j * bd;
      keep[k][j] = i < G ? __ldcg(partials + k * G + i) : 0.0;
      E[k] = max(E[k], fx::exp_field(keep[k][j]));
    }
    for (int i = (int)threadIdx.x + kKeep * bd; i < G; i += bd) E[k] = max(E[k], fx::exp_field(__ldcg(partials + k * G + i)));
  }
  unsigned* s = reinterpret_cast<unsigned*>(smem);
  fx::block_max<NV>(E, s);
  uint64_t h[NV], l[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    h[k] = l[k] = 0ull;
    if (E[k] >= fx::kNonFinite) continue;
#pragma unroll
    for (int j = 0; j < kKeep; ++j) {
      uint64_t a, b;
      fx::to_fixed(keep[k][j], E[k], a, b);
      fx::add128(h[k], l[k], a, b);
    }
    for (int i = (int)threadIdx.x + kKeep * bd; i < G; i += bd) {
      uint64_t a, b;
      fx::to_fixed(__ldcg(partials + k * G + i), E[k], a, b);
      fx::add128(h[k], l[k], a, b);
    }
  }
  fx::block_sum_fixed<NV>(h, l, E, s + NV * 32, tot);
}

// Deterministic grid-wide sum of NV values per thread.  Each block writes its
// NV block sums to partials[k * gridDim.x + blockIdx.x]; the block that
// arrives last (one acquire-release ticket increment) sums the partials and
// returns true; only its thread 0 holds valid totals in tot[].  arrival, when
// given, receives the block's arrival index (0 .. gridDim.x - 1, the last block
// gridDim.x - 1) in every thread.  The ticket is reset to zero for the next
// kernel.  partials must hold NV * gridDim.x values
// and smem NV * blockDim.x values.  float64 block sums take the exact integer
// path above when kBlockExact; the last block's sum of the partials takes it
// when kGridExact, and otherwise is a float64 tree in block order.  float32
// values always take float32 trees.
#ifndef APCG_BLOCK_EXACT
#define APCG_BLOCK_EXACT 1
#endif
#ifndef APCG_GRID_EXACT
#define APCG_GRID_EXACT 1
#endif
constexpr bool kBlockExact = APCG_BLOCK_EXACT != 0;
constexpr bool kGridExact = APCG_GRID_EXACT != 0;

template <int NV, class T>
__device__ __forceinline__ bool grid_sum_last(T (&v)[NV], T* partials, unsigned int* ticket, T* smem, T (&tot)[NV],
                                              unsigned* arrival = nullptr) {
  constexpr bool f64 = std::is_same<T, double>::value;
  __shared__ bool s_last;
  __shared__ unsigned s_arrival;
  if constexpr (f64 && kBlockExact)
    block_sum_exact<NV>(v, smem);
  else
    block_sum<NV>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
    // one acquire-release increment: its release orders this block's partials before it, its acquire
    // (in the block that arrives last) orders every block's partials before the loads below, which the
    // barrier then extends to the block's other threads
    unsigned t;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(t) : "l"(ticket) : "memory");
    s_last = (t == gridDim.x - 1);
    if (arrival) s_arrival = t;
  }
  __syncthreads();
  if (arrival) *arrival = s_arrival;
  if (!s_last) return false;
  if constexpr (f64 && kGridExact) {
    grid_partials_exact<NV>(reinterpret_cast<const double*>(partials), reinterpret_cast<double*>(smem),
                            reinterpret_cast<double(&)[NV]>(tot));
  } else {
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
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

}  // namespace dev
}  // namespace apcg
