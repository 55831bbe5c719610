// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "apcg.h"
#include "dep_tracker.hpp"

namespace apcg {

// ------------------------------------------------------------------ errors

apcg_status set_error(apcg_status st, const char* fmt, ...);
apcg_status cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define APCG_CUDA(...)                                                   \
  do {                                                                   \
    cudaError_t e_ = (__VA_ARGS__);                                      \
    if (e_ != cudaSuccess) return ::apcg::cuda_error(e_, #__VA_ARGS__, __FILE__, __LINE__); \
  } while (0)

#define APCG_CHECK(cond, ...)                                           \
  do {                                                                  \
    if (!(cond)) return ::apcg::set_error(APCG_ERR_INVALID_ARG, __VA_ARGS__); \
  } while (0)

#define APCG_TRY(...)                \
  do {                               \
    apcg_status s_ = (__VA_ARGS__);  \
    if (s_ != APCG_OK) return s_;    \
  } while (0)

// ------------------------------------------------------------------ counters

struct Counters {
  std::atomic<int64_t> kernel_launches{0}, graph_launches{0}, waits_inserted{0}, waits_elided{0},
      events_recorded{0}, host_syncs{0}, d2h_copies{0}, d2h_bytes{0}, h2d_copies{0}, h2d_bytes{0};
};
Counters& counters();

// ------------------------------------------------------------------ contexts

constexpr int kEventRing = 128;

// Device-side error word of a context: kernels OR flags into it.
enum : int32_t { kDevErrBadDiagonal = 1, kDevErrNonFinite = 2, kDevErrTimeout = 4 };

struct ReduceScratch {
  double* partials = nullptr;  // [kMaxPartials * 3]
  unsigned int* ticket = nullptr;
  int32_t* dev_error = nullptr;
};

}  // namespace apcg

struct apcg_ctx_s {
  uint64_t id = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  apcg_stream_type type = APCG_STREAM_DEFAULT_BLOCKING;
  cudaEvent_t ring[apcg::kEventRing] = {};
  uint64_t seq = 0;             // sequence number of the last recorded launch
  bool pending = false;         // a marked launch is between begin and end
  bool zombie = false;          // destroyed by the user, kept until idle
  apcg::ReduceScratch scratch;  // per-context reduction scratch (lazily allocated)
  int num_sms = 0;
};

struct apcg_scalar_s {
  double* dptr = nullptr;
  apcg_id id = 0;
  int slot = -1;
};

struct apcg_vec_s {
  void* dptr = nullptr;
  int64_t n = 0;
  apcg_dtype dtype = APCG_F64;
  apcg_id id = 0;
};

struct apcg_mat_s {
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;
  int32_t nrows = 0, ncols = 0;
  int64_t nnz = 0;
  apcg_dtype dtype = APCG_F64;
  apcg_id id = 0;
};

namespace apcg {

// Serialises the tracker, the registry and context bookkeeping.
std::mutex& global_mutex();

// The hidden global-blocking context used when a call passes ctx == NULL.
apcg_status resolve_ctx(apcg_ctx in, apcg_ctx* out);

// One marked launch: begin() for each operand, the caller enqueues its
// kernel(s) on ctx->stream, finish() ends the marks (records one event) and,
// for a global-blocking context, waits for completion.
class OpScope {
 public:
  explicit OpScope(apcg_ctx ctx) : ctx_(ctx) {}
  OpScope& read(apcg_id id) { return add(id, kRead); }
  OpScope& write(apcg_id id) { return add(id, kWrite); }
  OpScope& rw(apcg_id id) { return add(id, kReadWrite); }
  // The launch may raise a device-side error flag (checked by a global-blocking finish).
  OpScope& may_flag_errors() {
    flags_errors_ = true;
    return *this;
  }
  apcg_status begin();
  apcg_status finish();

 private:
  OpScope& add(apcg_id id, int mode) {
    if (id) ids_.push_back({id, mode});
    return *this;
  }
  struct Item {
    apcg_id id;
    int mode;
  };
  apcg_ctx ctx_;
  std::vector<Item> ids_;
  bool flags_errors_ = false;
};

apcg_status ensure_scratch(apcg_ctx ctx);
apcg_status ctx_check_device_error(apcg_ctx ctx);
int ctx_num_sms(apcg_ctx ctx);
// Stream-ordered device allocation from the library's memory pool (one per device, created on first use).
// The pool keeps freed memory for reuse instead of handing it back to the driver at every synchronisation,
// so plans created and destroyed per call (the host-buffer solve) do not map fresh pages each time.
// Free with cudaFreeAsync.
apcg_status dev_alloc_async(void** p, size_t bytes, cudaStream_t s);

// Registry of memory IDs (creates on first registration).
apcg_id register_memory(const void* p, size_t bytes);

// Counted helpers.
inline void count_kernels(int64_t n) { counters().kernel_launches += n; }

bool aligned16(const void* p);

}  // namespace apcg
