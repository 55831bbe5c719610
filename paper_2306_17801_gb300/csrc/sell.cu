// Conversion of a CSR matrix into the sliced-ELL layout of sell.cuh (once per plan).
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels_common.cuh"
#include "sell.hpp"

namespace apcg {
namespace {

// One thread per (slice, lane): writes the row's entries k = 0..width-1 of its
// slice, padding with value 0 and a harmless column (the row itself, or row
// n - 1 for the lanes past the last row), as an index (scol) or as the
// 16-bit offset from the row (sdcol; the plan has checked that it fits).
template <class TI, class TO>
__global__ void sell_fill_kernel(int32_t n, int32_t nslices, const int32_t* __restrict__ sptr,
                                 const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const TI* __restrict__ val, int32_t* __restrict__ scol, int16_t* __restrict__ sdcol,
                                 TO* __restrict__ sval) {
  const int64_t total = (int64_t)nslices * 32;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += stride) {
    const int64_t s = r >> 5;
    const int lane = (int)(r & 31);
    const int32_t base = sptr[s];
    const int32_t width = (sptr[s + 1] - base) >> 5;
    int32_t e0 = 0, len = 0;
    if (r < n) {
      e0 = rowptr[r];
      len = rowptr[r + 1] - e0;
    }
    const int32_t pad_col = r < n ? (int32_t)r : (n > 0 ? n - 1 : 0);
    for (int32_t k = 0; k < width; ++k) {
      const int64_t dst = (int64_t)base + 32 * (int64_t)k + lane;
      const bool real = k < len;
      const int32_t c = real ? col[e0 + k] : pad_col;
      if (scol) scol[dst] = c;
      if (sdcol) sdcol[dst] = (int16_t)(c - (int32_t)r);
      if (sval) sval[dst] = real ? (TO)val[e0 + k] : TO(0);
    }
  }
}

constexpr int kScanThreads = 1024, kScanPer = 4, kScanChunk = kScanThreads * kScanPer;
enum : int32_t { kBadRowptr = 1, kBadColumn = 2 };

constexpr int kGroupMin = 5, kGroupMax = 9, kGroups = kGroupMax - kGroupMin + 1;

// Totals over the slices for one choice of slice widths.
struct WidthStats {
  unsigned long long padded;          // sum over slices of 32 * width
  unsigned long long slots[kGroups];  // FMA slots per lane with groups of G = kGroupMin.. (whole groups per slice)
  int32_t max_width;
  int32_t pad0;
};

struct LayoutStats {
  WidthStats rows;     // width = the slice's longest row (index formats)
  WidthStats pat;      // width = the size of the union of the slice's column offsets (pattern format)
  int32_t max_offset;  // largest |col - row| over the entries (checked structures only)
  int32_t bad;         // kBadRowptr | kBadColumn
  int32_t unsorted;    // some row's columns do not strictly increase
  int32_t pad1;
};

// A warp's running totals (lane 0 holds them).
struct WidthAcc {
  unsigned long long pad = 0, sl[kGroups] = {};
  int32_t mw = 0;
  __device__ void add(int32_t w) {
    pad += 32ull * (unsigned)w;
#pragma unroll
    for (int gi = 0; gi < kGroups; ++gi) {
      const int G = kGroupMin + gi;
      sl[gi] += (unsigned long long)((w + G - 1) / G) * (unsigned long long)G;
    }
    mw = max(mw, w);
  }
};

// Adds the warps' totals into *out with one set of atomics per block (the
// counters are integers, so the order of the adds does not matter).  Every
// thread of the block calls it once.
__device__ void flush_widths(const WidthAcc& a, WidthStats* out) {
  __shared__ unsigned long long s_pad, s_sl[kGroups];
  __shared__ int32_t s_mw;
  if (threadIdx.x == 0) {
    s_pad = 0ull;
    for (int gi = 0; gi < kGroups; ++gi) s_sl[gi] = 0ull;
    s_mw = 0;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    if (a.pad) atomicAdd(&s_pad, a.pad);
    for (int gi = 0; gi < kGroups; ++gi)
      if (a.sl[gi]) atomicAdd(&s_sl[gi], a.sl[gi]);
    if (a.mw) atomicMax(&s_mw, a.mw);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_pad) atomicAdd(&out->padded, s_pad);
    for (int gi = 0; gi < kGroups; ++gi)
      if (s_sl[gi]) atomicAdd(&out->slots[gi], s_sl[gi]);
    if (s_mw) atomicMax(&out->max_width, s_mw);
  }
}

// One warp per slice (grid-stride): lane l reads rowptr[32 s + l] and the
// next entry, checks that they do not decrease and stay in [0, nnz], and the
// warp's maximum row length is the slice width.  Reads rowptr[0, n] only.
__global__ void slice_width_kernel(int32_t n, int64_t nnz, int32_t nslices, const int32_t* __restrict__ rowptr,
                                   int32_t* __restrict__ width, LayoutStats* __restrict__ st) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  WidthAcc acc;
  bool bad = false;
  if (blockIdx.x == 0 && threadIdx.x == 0) bad = rowptr[0] != 0 || (int64_t)rowptr[n] != nnz;
  for (int64_t s = w0; s < nslices; s += nw) {
    const int64_t r = s * 32 + lane;
    int32_t len = 0;
    if (r < n) {
      const int32_t a = rowptr[r], b = rowptr[r + 1];
      bad |= a < 0 || b < a || (int64_t)b > nnz;
      len = b > a ? b - a : 0;
    }
    const int32_t w = (int32_t)__reduce_max_sync(dev::kFull, (unsigned)len);
    if (lane == 0) {
      width[s] = w;
      acc.add(w);
    }
  }
  if (__any_sync(dev::kFull, bad) && lane == 0) atomicOr(&st->bad, kBadRowptr);
  flush_widths(acc, &st->rows);
}

// Merges the column offsets (col - row) of the 32 rows of slice s, held one
// row per lane, into their increasing union: each step takes the smallest
// offset any lane has next and advances the lanes that hold it, calling
// step(offset, lane_has_it, entry) in union order.  Every step consumes at
// least one entry, so a slice takes at most its entry count of steps, also
// where a row's columns do not increase (*unsorted is then set in that lane).
template <class Step>
__device__ __forceinline__ int32_t slice_union(int32_t n, int64_t s, const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col, bool* unsorted, Step step) {
  const int lane = threadIdx.x & 31;
  const int64_t r = s * 32 + lane;
  int32_t e = 0, e1 = 0;
  if (r < n) {
    e = rowptr[r];
    e1 = rowptr[r + 1];
  }
  // offsets lie in (-n, n), so INT32_MAX marks an exhausted row
  int32_t cur = e < e1 ? __ldg(col + e) - (int32_t)r : INT32_MAX;
  int32_t u = 0;
  for (;;) {
    const int32_t m = __reduce_min_sync(dev::kFull, cur);
    if (m == INT32_MAX) break;
    const bool has = cur == m;
    step(m, has, e);
    if (has) {
      ++e;
      const int32_t nx = e < e1 ? __ldg(col + e) - (int32_t)r : INT32_MAX;
      *unsorted |= nx <= cur;
      cur = nx;
    }
    ++u;
  }
  return u;
}

// On a structure that passed the checks: the size of each slice's union of
// column offsets (its width in the pattern format), whether every row's
// columns strictly increase, and the largest |col - row|.
__global__ void slice_pattern_kernel(int32_t n, int32_t nslices, const int32_t* __restrict__ rowptr,
                                     const int32_t* __restrict__ col, int32_t* __restrict__ uwidth,
                                     LayoutStats* __restrict__ st) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  WidthAcc acc;
  bool unsorted = false;
  int32_t m = 0;
  for (int64_t s = w0; s < nslices; s += nw) {
    const int32_t u = slice_union(n, s, rowptr, col, &unsorted, [&](int32_t off, bool has, int32_t) {
      if (has) m = max(m, off < 0 ? -off : off);
    });
    if (lane == 0) {
      uwidth[s] = u;
      acc.add(u);
    }
  }
  m = (int32_t)__reduce_max_sync(dev::kFull, (unsigned)m);
  const bool any_unsorted = __any_sync(dev::kFull, unsorted);
  if (lane == 0) {
    if (m) atomicMax(&st->max_offset, m);
    if (any_unsorted) atomicOr(&st->unsorted, 1);
  }
  flush_widths(acc, &st->pat);
}

// Pattern format fill, one warp per slice: walks the slice's union of
// offsets as slice_pattern_kernel did (so the widths agree), writing at union
// position k the value of each row's entry with that offset, or 0, and (if
// spat) the offset itself.
template <class TI, class TO>
__global__ void sell_fill_pattern_kernel(int32_t n, int32_t nslices, const int32_t* __restrict__ sptr,
                                         const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                         const TI* __restrict__ val, int32_t* __restrict__ spat,
                                         TO* __restrict__ sval) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = w0; s < nslices; s += nw) {
    const int32_t base = sptr[s];
    const int32_t width = (sptr[s + 1] - base) >> 5;
    bool unsorted = false;
    int32_t k = 0;
    slice_union(n, s, rowptr, col, &unsorted, [&](int32_t off, bool has, int32_t e) {
      if (k < width) {
        if (sval) sval[(int64_t)base + 32 * (int64_t)k + lane] = has ? (TO)val[e] : TO(0);
        if (spat && lane == 0) spat[(base >> 5) + k] = off;
      }
      ++k;
    });
  }
}

// Flags kBadColumn when an entry of col[0, nnz) lies outside [0, ncols).
__global__ void col_range_kernel(const int32_t* __restrict__ col, int64_t nnz, int32_t ncols,
                                 LayoutStats* __restrict__ st) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int32_t c = __ldg(col + e);
    bad |= (c < 0) | (c >= ncols);
  }
  if (__any_sync(dev::kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->bad, kBadColumn);
}

// Exclusive scan of 32 * width into sptr, in three steps: each block scans a
// chunk of kScanChunk slices (kScanPer per thread) and writes the chunk's
// total; one block scans the chunk totals (their grand total goes to
// csum[nchunks]); every slice then adds its chunk's offset.  Sums are
// formed in 64 bits; the host rejects a total beyond the int32 range before
// the offsets are used.
__device__ __forceinline__ long long block_exclusive_scan(long long t, long long* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(dev::kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nwarps = blockDim.x >> 5;
    const long long y = lane < nwarps ? warp_tot[lane] : 0;
    long long inc = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long z = __shfl_up_sync(dev::kFull, inc, o);
      if (lane >= o) inc += z;
    }
    if (lane < nwarps) warp_tot[lane] = inc - y;
  }
  __syncthreads();
  return warp_tot[wid] + incl - t;
}

__global__ void __launch_bounds__(kScanThreads) scan_chunks_kernel(const int32_t* __restrict__ width, int32_t nslices,
                                                                  int32_t* __restrict__ sptr,
                                                                  long long* __restrict__ csum) {
  __shared__ long long warp_tot[32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
  long long v[kScanPer];
  long long t = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = base + k < nslices ? 32LL * width[base + k] : 0;
    t += v[k];
  }
  long long run = block_exclusive_scan(t, warp_tot);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < nslices) sptr[base + k] = (int32_t)run;
    run += v[k];
  }
  if (threadIdx.x == blockDim.x - 1) csum[blockIdx.x] = run;
}

__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(long long* __restrict__ csum, int nchunks) {
  __shared__ long long warp_tot[32];
  const int per = (nchunks + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = threadIdx.x * per;
  long long t = 0;
  for (int i = b0; i < b0 + per && i < nchunks; ++i) t += csum[i];
  long long run = block_exclusive_scan(t, warp_tot);
  for (int i = b0; i < b0 + per && i < nchunks; ++i) {
    const long long x = csum[i];
    csum[i] = run;
    run += x;
  }
  if (threadIdx.x == blockDim.x - 1) csum[nchunks] = run;
}

__global__ void scan_add_kernel(int32_t* __restrict__ sptr, int32_t nslices, const long long* __restrict__ csum,
                                int nchunks) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nslices; i += stride)
    sptr[i] = i < nslices ? sptr[i] + (int32_t)csum[i / kScanChunk] : (int32_t)csum[nchunks];
}

}  // namespace

apcg_status csr_layout(apcg_ctx ctx, const apcg_mat_s* A, bool want_sptr, SellLayout* out) {
  APCG_CHECK(A->nrows == A->ncols, "the matrix must be square (%d x %d)", A->nrows, A->ncols);
  const int32_t n = A->nrows;
  out->n = n;
  out->nslices = (n + 31) / 32;
  out->stream = ctx->stream;
  const int nchunks = (int)(((int64_t)out->nslices + kScanChunk - 1) / kScanChunk);
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t b_st = up(sizeof(LayoutStats)), b_w = up(sizeof(int32_t) * ((size_t)out->nslices + 1)),
               b_c = up(sizeof(long long) * ((size_t)nchunks + 1)),
               b_s = want_sptr ? up(sizeof(int32_t) * ((size_t)out->nslices + 1)) : 0;
  char* blk = nullptr;
  APCG_TRY(dev_alloc_async((void**)&blk, b_st + 2 * b_w + b_c + b_s, ctx->stream));
  out->d_block = blk;
  LayoutStats* st = reinterpret_cast<LayoutStats*>(blk);
  int32_t* width = reinterpret_cast<int32_t*>(blk + b_st);
  int32_t* uwidth = reinterpret_cast<int32_t*>(blk + b_st + b_w);
  long long* csum = reinterpret_cast<long long*>(blk + b_st + 2 * b_w);
  if (want_sptr) out->d_sptr = reinterpret_cast<int32_t*>(blk + b_st + 2 * b_w + b_c);
  APCG_CUDA(cudaMemsetAsync(st, 0, sizeof(LayoutStats), ctx->stream));
  const int sms = ctx_num_sms(ctx);
  const int gw = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)out->nslices + 7) / 8, 8LL * sms));
  auto read_stats = [&](LayoutStats* h) -> apcg_status {
    APCG_CUDA(cudaMemcpyAsync(h, st, sizeof(*h), cudaMemcpyDeviceToHost, ctx->stream));
    APCG_CUDA(cudaStreamSynchronize(ctx->stream));
    counters().d2h_copies++;
    counters().d2h_bytes += (int64_t)sizeof(*h);
    return APCG_OK;
  };
  // ordered after every pending writer of the matrix on other contexts
  OpScope op(ctx);
  op.read(A->id);
  APCG_TRY(op.begin());
  slice_width_kernel<<<gw, 256, 0, ctx->stream>>>(n, A->nnz, out->nslices, A->rowptr, width, st);
  int launches = 1;
  if (A->nnz > 0) {
    const int gc = (int)std::min<int64_t>((A->nnz + 255) / 256, 8LL * sms);
    col_range_kernel<<<gc, 256, 0, ctx->stream>>>(A->col, A->nnz, A->ncols, st);
    ++launches;
  }
  APCG_CUDA(cudaGetLastError());
  LayoutStats h;
  APCG_TRY(read_stats(&h));
  if (h.bad) APCG_TRY(op.finish());
  APCG_CHECK(!(h.bad & kBadRowptr), "CSR: rowptr must start at 0, never decrease and end at nnz = %lld",
             (long long)A->nnz);
  APCG_CHECK(!(h.bad & kBadColumn), "CSR: a column index is outside [0, ncols = %d)", A->ncols);
  if (!want_sptr) {  // structure check only: no slices are built
    count_kernels(launches);
    APCG_TRY(op.finish());
    out->nslices = 0;
    return APCG_OK;
  }
  // The structure is valid by now, so the next pass may follow rowptr: the union of each slice's column
  // offsets, the rows' column order and the largest offset.
  if (A->nnz > 0) {
    slice_pattern_kernel<<<gw, 256, 0, ctx->stream>>>(n, out->nslices, A->rowptr, A->col, uwidth, st);
    APCG_CUDA(cudaGetLastError());
    ++launches;
    APCG_TRY(read_stats(&h));
  }
  // The pattern format where every row's columns increase and the unions pad the slices by at most 1/16
  // more than their longest rows do (rows * 2 <= padded keeps row + offset inside the int32 range).
  out->pattern = A->nnz > 0 && !h.unsorted && h.pat.padded <= h.rows.padded + h.rows.padded / 16 &&
                 (int64_t)n * 2 <= (int64_t)INT32_MAX - 64;
  const WidthStats& W = out->pattern ? h.pat : h.rows;
  out->padded = (int64_t)W.padded;
  out->max_width = W.max_width;
  if (out->padded > (int64_t)INT32_MAX - 64) {
    APCG_TRY(op.finish());
    return set_error(APCG_ERR_UNSUPPORTED, "the sliced-ELL copy would exceed the int32 index range");
  }
  if (out->nslices > 0) {
    const int32_t* w = out->pattern ? uwidth : width;
    scan_chunks_kernel<<<nchunks, kScanThreads, 0, ctx->stream>>>(w, out->nslices, out->d_sptr, csum);
    scan_top_kernel<<<1, kScanThreads, 0, ctx->stream>>>(csum, nchunks);
    const int ga = (int)std::min<int64_t>(((int64_t)out->nslices + 256) / 256, 8LL * sms);
    scan_add_kernel<<<ga, 256, 0, ctx->stream>>>(out->d_sptr, out->nslices, csum, nchunks);
    launches += 3;
  } else {
    APCG_CUDA(cudaMemsetAsync(out->d_sptr, 0, sizeof(int32_t), ctx->stream));
  }
  APCG_CUDA(cudaGetLastError());
  count_kernels(launches);
  APCG_TRY(op.finish());
  // The grouped path for mean widths of 8 or more, groups of 9 where they issue fewer FMA slots per lane
  // than groups of 8 (8 on a tie).
  const unsigned long long s8 = W.slots[8 - kGroupMin], s9 = W.slots[9 - kGroupMin];
  out->long_rows = 0;
  if (out->nslices > 0 && out->padded >= 8LL * 32 * out->nslices) out->long_rows = s9 < s8 ? 9 : 8;
  // The float64 CG SpMV also groups mean widths from 4.5 to 8, with the group size of 5..9 that issues the fewest
  // FMA slots (the larger on a tie): whole groups of 7 on 7-point rows load a slice's entries together, where
  // one entry at a time hides less latency (128^3: 46.4 against 50.6 us per launch).
  out->group = 0;
  if (out->nslices > 0 && 2 * out->padded >= 9LL * 32 * out->nslices) {  // mean width >= 4.5
    int best = kGroupMax;
    for (int G = kGroupMax - 1; G >= kGroupMin; --G)
      if (W.slots[G - kGroupMin] < W.slots[best - kGroupMin]) best = G;
    out->group = best;
  }
  // 16-bit column offsets where every entry lies within 32767 of its row (index formats only)
  out->d16 = !out->pattern && A->nnz > 0 && h.max_offset <= 32767;
  return APCG_OK;
}

template <class TI, class TO>
apcg_status sell_fill(cudaStream_t s, const SellLayout& L, const int32_t* d_sptr, const int32_t* rowptr,
                      const int32_t* col, const TI* val, int32_t* scol, int16_t* sdcol, int32_t* spat, TO* sval) {
  if (L.nslices == 0) return APCG_OK;
  const int64_t total = (int64_t)L.nslices * 32;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 65536);
  if (L.pattern) {
    if (scol || sdcol) return set_error(APCG_ERR_INVALID_ARG, "pattern layout with per-entry columns");
    sell_fill_pattern_kernel<TI, TO><<<grid, 256, 0, s>>>(L.n, L.nslices, d_sptr, rowptr, col, val, spat, sval);
  } else {
    if (spat) return set_error(APCG_ERR_INVALID_ARG, "per-slice offsets without the pattern layout");
    sell_fill_kernel<TI, TO><<<grid, 256, 0, s>>>(L.n, L.nslices, d_sptr, rowptr, col, val, scol, sdcol, sval);
  }
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return APCG_OK;
}

template apcg_status sell_fill<double, double>(cudaStream_t, const SellLayout&, const int32_t*, const int32_t*,
                                               const int32_t*, const double*, int32_t*, int16_t*, int32_t*, double*);
template apcg_status sell_fill<double, float>(cudaStream_t, const SellLayout&, const int32_t*, const int32_t*,
                                              const int32_t*, const double*, int32_t*, int16_t*, int32_t*, float*);
template apcg_status sell_fill<float, float>(cudaStream_t, const SellLayout&, const int32_t*, const int32_t*,
                                             const int32_t*, const float*, int32_t*, int16_t*, int32_t*, float*);

}  // namespace apcg
