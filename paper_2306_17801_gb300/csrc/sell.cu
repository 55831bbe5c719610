// Conversion of a CSR matrix into the sliced-ELL layout of sell.cuh (once per plan).
#include <cuda_runtime.h>

#include <algorithm>

#include "sell.hpp"

namespace apcg {
namespace {

// One thread per (slice, lane): writes the row's entries k = 0..width-1 of its
// slice, padding with value 0 and a harmless column (the row itself, or 0).
template <class TI, class TO>
__global__ void sell_fill_kernel(int32_t n, int32_t nslices, const int32_t* __restrict__ sptr,
                                 const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const TI* __restrict__ val, int32_t* __restrict__ scol, TO* __restrict__ sval) {
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
    const int32_t pad_col = r < n ? (int32_t)r : 0;
    for (int32_t k = 0; k < width; ++k) {
      const int64_t dst = (int64_t)base + 32 * (int64_t)k + lane;
      const bool real = k < len;
      if (scol) scol[dst] = real ? col[e0 + k] : pad_col;
      if (sval) sval[dst] = real ? (TO)val[e0 + k] : TO(0);
    }
  }
}

}  // namespace

apcg_status sell_layout(cudaStream_t s, int32_t n, const int32_t* rowptr_dev, SellLayout* out) {
  std::vector<int32_t> rp((size_t)n + 1);
  APCG_CUDA(cudaMemcpyAsync(rp.data(), rowptr_dev, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s));
  APCG_CUDA(cudaStreamSynchronize(s));
  counters().d2h_copies++;
  counters().d2h_bytes += (int64_t)(sizeof(int32_t) * rp.size());
  return sell_layout_host(n, rp, out);
}

apcg_status sell_layout_host(int32_t n, const std::vector<int32_t>& rp, SellLayout* out) {
  out->n = n;
  out->nslices = (n + 31) / 32;
  out->sptr.assign((size_t)out->nslices + 1, 0);
  out->max_width = 0;
  int64_t acc = 0;
  for (int32_t sl = 0; sl < out->nslices; ++sl) {
    int32_t w = 0;
    const int32_t r1 = std::min(n, (sl + 1) * 32);
    for (int32_t r = sl * 32; r < r1; ++r) w = std::max(w, rp[r + 1] - rp[r]);
    out->max_width = std::max(out->max_width, w);
    out->sptr[sl] = (int32_t)acc;
    acc += 32 * (int64_t)w;
    if (acc > (int64_t)INT32_MAX - 64)
      return set_error(APCG_ERR_UNSUPPORTED, "the sliced-ELL copy would exceed the int32 index range");
  }
  out->sptr[out->nslices] = (int32_t)acc;
  out->padded = acc;
  out->long_rows = 0;
  if (out->nslices > 0 && acc >= 8LL * 32 * out->nslices) {
    // FMA slots issued per lane with groups of 8 and of 9 (whole groups per slice); fewer wins, 8 on a tie
    int64_t slots8 = 0, slots9 = 0;
    for (int32_t sl = 0; sl < out->nslices; ++sl) {
      const int64_t w = (out->sptr[sl + 1] - out->sptr[sl]) / 32;
      slots8 += (w + 7) / 8 * 8;
      slots9 += (w + 8) / 9 * 9;
    }
    out->long_rows = slots9 < slots8 ? 9 : 8;
  }
  return APCG_OK;
}

template <class TI, class TO>
apcg_status sell_fill(cudaStream_t s, const SellLayout& L, const int32_t* d_sptr, const int32_t* rowptr,
                      const int32_t* col, const TI* val, int32_t* scol, TO* sval) {
  if (L.nslices == 0) return APCG_OK;
  const int64_t total = (int64_t)L.nslices * 32;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 65536);
  sell_fill_kernel<TI, TO><<<grid, 256, 0, s>>>(L.n, L.nslices, d_sptr, rowptr, col, val, scol, sval);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return APCG_OK;
}

template apcg_status sell_fill<double, double>(cudaStream_t, const SellLayout&, const int32_t*, const int32_t*,
                                               const int32_t*, const double*, int32_t*, double*);
template apcg_status sell_fill<double, float>(cudaStream_t, const SellLayout&, const int32_t*, const int32_t*,
                                              const int32_t*, const double*, int32_t*, float*);
template apcg_status sell_fill<float, float>(cudaStream_t, const SellLayout&, const int32_t*, const int32_t*,
                                             const int32_t*, const float*, int32_t*, float*);

}  // namespace apcg
