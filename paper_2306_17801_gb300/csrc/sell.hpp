// Host side of the sliced-ELL conversion (see sell.cuh for the layout).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "apcg_internal.hpp"

namespace apcg {

struct SellLayout {
  int32_t n = 0;
  int32_t nslices = 0;
  int64_t padded = 0;          // entries including padding (multiple of 32)
  int32_t long_rows = 0;       // 0: mean slice width < 8; else the group size of the grouped SpMV (8 or 9)
  int32_t max_width = 0;       // entries per row of the widest slice
  std::vector<int32_t> sptr;   // [nslices + 1]
};

// Structure check of a CSR matrix at plan creation (blocks on the context's stream): rowptr copied back and
// checked on the host, column indices checked by a device pass.  Returns APCG_ERR_INVALID_ARG before any
// kernel reads through the structure.  rp_out, if given, receives the host copy of rowptr.
apcg_status csr_check(apcg_ctx ctx, const apcg_mat_s* A, std::vector<int32_t>* rp_out);

// Slice offsets of a CSR matrix whose rowptr lives on the device (copied back once, blocks on s).
apcg_status sell_layout(cudaStream_t s, int32_t n, const int32_t* rowptr_dev, SellLayout* out);
// The same from a host copy of rowptr ([n + 1], already checked by csr_check).
apcg_status sell_layout_host(int32_t n, const std::vector<int32_t>& rp, SellLayout* out);

// Scatter CSR rows into the slices: column indices (if scol != nullptr) and
// values converted from TI to TO (if sval != nullptr).  d_sptr is the layout's
// sptr on the device.
template <class TI, class TO>
apcg_status sell_fill(cudaStream_t s, const SellLayout& L, const int32_t* d_sptr, const int32_t* rowptr,
                      const int32_t* col, const TI* val, int32_t* scol, TO* sval);

}  // namespace apcg
