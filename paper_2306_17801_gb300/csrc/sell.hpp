// Host side of the sliced-ELL conversion (see sell.cuh for the layout).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "apcg_internal.hpp"

namespace apcg {

// Slice geometry of a CSR matrix, computed on the device by csr_layout (all
// zero when only the structure was checked).  The slice offsets stay on the
// device in a stream-ordered temporary that the layout frees (in stream
// order) when it goes out of scope.
struct SellLayout {
  int32_t n = 0;
  int32_t nslices = 0;
  int64_t padded = 0;          // entries including padding (multiple of 32)
  int32_t long_rows = 0;       // 0: mean slice width < 8; else the group size of the grouped SpMV (8 or 9)
  int32_t group = 0;           // float64 CG SpMV: 0 (one entry at a time) or its group size, 5..9
  bool d16 = false;            // every entry lies within 32767 of its row: 16-bit column offsets fit
  bool pattern = false;        // slices share their rows' column offsets (dev::kColPattern); widths and
                               // padded then count each slice's union of offsets
  int32_t max_width = 0;       // entries per row of the widest slice
  int32_t* d_sptr = nullptr;   // [nslices + 1] slice offsets on the device (inside d_block), or null
  void* d_block = nullptr;
  cudaStream_t stream = nullptr;

  SellLayout() = default;
  SellLayout(const SellLayout&) = delete;
  SellLayout& operator=(const SellLayout&) = delete;
  ~SellLayout() {
    if (d_block) cudaFreeAsync(d_block, stream);
  }
};

// The layout report of apcg_*_plan_layout for a plan whose SpMV view has the
// given column format (dev::ColFormat, numerically APCG_COLS_*; a view without
// slice offsets is reported as APCG_COLS_NONE).
inline void describe_layout(bool has_copy, int col_format, int group, int64_t nslices, int64_t padded,
                            apcg_plan_layout* out) {
  out->col_format = has_copy ? col_format : APCG_COLS_NONE;
  out->group = has_copy ? group : 0;
  out->nslices = has_copy ? nslices : 0;
  out->padded = has_copy ? padded : 0;
}

// Structure check of a CSR matrix at plan creation, on the device: rowptr
// starts at 0, never decreases and ends at nnz; every column index lies in
// [0, ncols).  With want_sptr, the same pass measures the slice widths and a
// scan writes the sliced-ELL offsets to out->d_sptr.  Blocks once on the
// context's stream to read a few counters back; returns APCG_ERR_INVALID_ARG
// before any kernel reads through a bad structure (the checking kernels read
// rowptr[0, n] and col[0, nnz) only).
apcg_status csr_layout(apcg_ctx ctx, const apcg_mat_s* A, bool want_sptr, SellLayout* out);

// Scatter CSR rows into the slices: column indices (if scol != nullptr), column
// offsets from the row (if sdcol != nullptr; only where L.d16) and values
// converted from TI to TO (if sval != nullptr).  Where L.pattern, the slices
// take their union layout instead: the per-slice offsets go to spat (if not
// null; sptr[nslices] / 32 entries) and scol, sdcol must be null.  d_sptr is
// the layout's sptr on the device.
template <class TI, class TO>
apcg_status sell_fill(cudaStream_t s, const SellLayout& L, const int32_t* d_sptr, const int32_t* rowptr,
                      const int32_t* col, const TI* val, int32_t* scol, int16_t* sdcol, int32_t* spat, TO* sval);

}  // namespace apcg
