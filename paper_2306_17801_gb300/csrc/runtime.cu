// Runtime of the library: errors, counters, device contexts (Sec. 3.1), memory
// IDs and intent marking (Sec. 3.1.2), managed device scalars (Sec. 3.2) and
// the host-only simulator of the marking rules.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <unordered_map>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "kernels_common.cuh"

namespace apcg {

// ------------------------------------------------------------------ errors

static thread_local std::string t_last_error = "no error";

apcg_status set_error(apcg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return st;
}

apcg_status cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  const char* base = strrchr(file, '/');
  return set_error(e == cudaErrorMemoryAllocation ? APCG_ERR_NO_MEMORY : APCG_ERR_CUDA, "%s failed: %s (%s:%d)", what,
                   cudaGetErrorString(e), base ? base + 1 : file, line);
}

Counters& counters() {
  static Counters c;
  return c;
}

std::mutex& global_mutex() {
  static std::mutex m;
  return m;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ------------------------------------------------------------------ registry

namespace {

struct Registry {
  uint64_t next_id = 1;
  uint64_t next_ctx = 1;
  std::map<uintptr_t, std::pair<apcg_id, size_t>> mem;
  std::unordered_map<uint64_t, apcg_ctx> ctxs;  // live and zombie contexts
  DepTracker tracker;
  apcg_ctx global_ctx = nullptr;
};

Registry& reg() {
  static Registry r;
  return r;
}

apcg_ctx lookup_ctx(uint64_t id) {
  auto it = reg().ctxs.find(id);
  return it == reg().ctxs.end() ? nullptr : it->second;
}

// Tracker backend on CUDA events: launch `seq` of a context is the event in
// ring slot seq % kEventRing.  A slot re-recorded by a later launch of the
// same stream stands for a later point, so waiting on it is conservative.
struct CudaBackend {
  bool complete(uint64_t c, uint64_t s) {
    apcg_ctx x = lookup_ctx(c);
    if (!x) return true;  // collected only once idle
    if (s > x->seq) return false;
    return cudaEventQuery(x->ring[s % kEventRing]) == cudaSuccess;
  }
  void wait(uint64_t w, uint64_t c, uint64_t s) {
    apcg_ctx wx = lookup_ctx(w), x = lookup_ctx(c);
    if (!wx || !x) return;
    cudaStreamWaitEvent(wx->stream, x->ring[s % kEventRing], 0);
    counters().waits_inserted++;
  }
  void elided(uint64_t, uint64_t, uint64_t) { counters().waits_elided++; }
};

// Record a fresh event at the current tail of ctx (caller holds the mutex).
apcg_status record_tail(apcg_ctx ctx) {
  ctx->seq++;
  APCG_CUDA(cudaEventRecord(ctx->ring[ctx->seq % kEventRing], ctx->stream));
  counters().events_recorded++;
  return APCG_OK;
}

// Make `waiter` wait for everything enqueued on `waitee` so far (mutex held).
apcg_status wait_tail(apcg_ctx waiter, apcg_ctx waitee) {
  APCG_TRY(record_tail(waitee));
  APCG_CUDA(cudaStreamWaitEvent(waiter->stream, waitee->ring[waitee->seq % kEventRing], 0));
  counters().waits_inserted++;
  reg().tracker.note_known(waiter->id, waitee->id, waitee->seq);
  return APCG_OK;
}

void release_ctx_resources(apcg_ctx c) {
  for (int i = 0; i < kEventRing; ++i)
    if (c->ring[i]) cudaEventDestroy(c->ring[i]);
  delete c;
}

// Drop zombie contexts whose work has finished (mutex held).
void collect_zombies() {
  std::vector<uint64_t> dead;
  for (auto& kv : reg().ctxs) {
    apcg_ctx c = kv.second;
    if (c->zombie && cudaEventQuery(c->ring[c->seq % kEventRing]) == cudaSuccess) dead.push_back(kv.first);
  }
  for (uint64_t id : dead) {
    apcg_ctx c = reg().ctxs[id];
    reg().ctxs.erase(id);
    reg().tracker.forget_context(id);
    release_ctx_resources(c);
  }
}

apcg_status new_ctx(cudaStream_t borrowed, apcg_stream_type type, apcg_ctx* out) {
  std::unique_ptr<apcg_ctx_s> c(new apcg_ctx_s());
  APCG_CUDA(cudaGetDevice(&c->device));
  APCG_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  if (borrowed) {
    c->stream = borrowed;
    c->owns_stream = false;
  } else {
    APCG_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->owns_stream = true;
  }
  for (int i = 0; i < kEventRing; ++i) {
    cudaError_t e = cudaEventCreateWithFlags(&c->ring[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(c->ring[j]);
      if (c->owns_stream) cudaStreamDestroy(c->stream);
      return cuda_error(e, "cudaEventCreateWithFlags", __FILE__, __LINE__);
    }
  }
  c->type = type;
  // Slot 0 stands for "nothing enqueued yet": record it so queries succeed.
  cudaEventRecord(c->ring[0], c->stream);
  std::lock_guard<std::mutex> g(global_mutex());
  c->id = reg().next_ctx++;
  reg().ctxs[c->id] = c.get();
  collect_zombies();
  *out = c.release();
  return APCG_OK;
}

}  // namespace

apcg_id register_memory(const void* p, size_t bytes) {
  auto& m = reg().mem;
  auto it = m.find(reinterpret_cast<uintptr_t>(p));
  if (it != m.end()) {
    if (bytes > it->second.second) it->second.second = bytes;
    return it->second.first;
  }
  apcg_id id = reg().next_id++;
  m[reinterpret_cast<uintptr_t>(p)] = {id, bytes};
  return id;
}

void reg_forget_memory(const void* p) {
  auto it = reg().mem.find(reinterpret_cast<uintptr_t>(p));
  if (it == reg().mem.end()) return;
  reg().tracker.forget(it->second.first);
  reg().mem.erase(it);
}

apcg_ctx host_api_ctx() {
  static std::once_flag once;
  static apcg_ctx ctx = nullptr;
  std::call_once(once, [] {
    apcg_ctx c = nullptr;
    if (new_ctx(nullptr, APCG_STREAM_DEFAULT_BLOCKING, &c) == APCG_OK) ctx = c;
  });
  return ctx;
}

apcg_status resolve_ctx(apcg_ctx in, apcg_ctx* out) {
  if (in) {
    *out = in;
    return APCG_OK;
  }
  {
    std::lock_guard<std::mutex> g(global_mutex());
    if (reg().global_ctx) {
      *out = reg().global_ctx;
      return APCG_OK;
    }
  }
  apcg_ctx c = nullptr;
  APCG_TRY(new_ctx(nullptr, APCG_STREAM_GLOBAL_BLOCKING, &c));
  std::lock_guard<std::mutex> g(global_mutex());
  if (reg().global_ctx) {  // another thread won the race
    reg().ctxs.erase(c->id);
    if (c->owns_stream) cudaStreamDestroy(c->stream);
    release_ctx_resources(c);
  } else {
    reg().global_ctx = c;
  }
  *out = reg().global_ctx;
  return APCG_OK;
}

apcg_status OpScope::begin() {
  std::lock_guard<std::mutex> g(global_mutex());
  if (ctx_->type == APCG_STREAM_GLOBAL_BLOCKING) {
    for (auto& kv : reg().ctxs) {
      apcg_ctx o = kv.second;
      if (o != ctx_ && !o->zombie) APCG_TRY(wait_tail(ctx_, o));
    }
  }
  CudaBackend be;
  for (const Item& it : ids_) reg().tracker.begin(be, ctx_->id, it.id, it.mode);
  ctx_->pending = true;
  return APCG_OK;
}

apcg_status OpScope::finish() {
  {
    std::lock_guard<std::mutex> g(global_mutex());
    APCG_TRY(record_tail(ctx_));
    for (const Item& it : ids_) reg().tracker.end(ctx_->id, it.id, it.mode, ctx_->seq);
    ctx_->pending = false;
  }
  if (ctx_->type == APCG_STREAM_GLOBAL_BLOCKING) {
    APCG_CUDA(cudaStreamSynchronize(ctx_->stream));
    counters().host_syncs++;
    if (flags_errors_) return ctx_check_device_error(ctx_);
  }
  return APCG_OK;
}

apcg_status ensure_scratch(apcg_ctx ctx) {
  if (ctx->scratch.partials) return APCG_OK;
  const size_t bytes = sizeof(double) * dev::kMaxPartials * 3 + 256;
  void* p = nullptr;
  APCG_TRY(dev_alloc_async(&p, bytes, ctx->stream));
  APCG_CUDA(cudaMemsetAsync(p, 0, bytes, ctx->stream));
  ctx->scratch.partials = static_cast<double*>(p);
  char* tail = static_cast<char*>(p) + sizeof(double) * dev::kMaxPartials * 3;
  ctx->scratch.ticket = reinterpret_cast<unsigned int*>(tail);
  ctx->scratch.dev_error = reinterpret_cast<int32_t*>(tail + 128);
  return APCG_OK;
}

apcg_status ctx_check_device_error(apcg_ctx ctx) {
  if (!ctx->scratch.dev_error) return APCG_OK;
  int32_t flag = 0;
  APCG_CUDA(cudaMemcpyAsync(&flag, ctx->scratch.dev_error, sizeof(flag), cudaMemcpyDeviceToHost, ctx->stream));
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(flag);
  if (!flag) return APCG_OK;
  APCG_CUDA(cudaMemsetAsync(ctx->scratch.dev_error, 0, sizeof(int32_t), ctx->stream));
  if (flag & kDevErrBadDiagonal)
    return set_error(APCG_ERR_BAD_DIAGONAL, "Jacobi: a diagonal entry is missing, zero or not finite");
  if (flag & kDevErrTimeout) return set_error(APCG_ERR_TIMEOUT, "a bounded device wait ran out");
  return set_error(APCG_ERR_BREAKDOWN, "a non-finite value was produced on the device");
}

int ctx_num_sms(apcg_ctx ctx) { return ctx->num_sms > 0 ? ctx->num_sms : 1; }

apcg_status dev_alloc_async(void** p, size_t bytes, cudaStream_t s) {
  constexpr int kMaxDevices = 64;
  static cudaMemPool_t pools[kMaxDevices] = {};
  static std::mutex m;
  int dev = 0;
  APCG_CUDA(cudaGetDevice(&dev));
  APCG_CHECK(dev >= 0 && dev < kMaxDevices, "device ordinal %d out of range", dev);
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> g(m);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t created;
      APCG_CUDA(cudaMemPoolCreate(&created, &props));
      uint64_t keep = UINT64_MAX;
      APCG_CUDA(cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep));
      pools[dev] = created;
    }
    pool = pools[dev];
  }
  APCG_CUDA(cudaMallocFromPoolAsync(p, bytes, pool, s));
  return APCG_OK;
}

// ------------------------------------------------------------------ scalar pool

namespace {

constexpr int kSlotsPerChunk = 1024;

struct ScalarPool {
  std::vector<double*> chunks;
  std::vector<int> free_slots;
  struct Pending {
    int slot;
    std::vector<Access> fence;
  };
  std::vector<Pending> pending;
  double* slot_ptr(int s) { return chunks[s / kSlotsPerChunk] + (s % kSlotsPerChunk); }
};

ScalarPool& pool() {
  static ScalarPool p;
  return p;
}

bool fence_done(const std::vector<Access>& f) {
  CudaBackend be;
  for (const Access& a : f)
    if (!be.complete(a.ctx, a.seq)) return false;
  return true;
}

apcg_status pool_acquire(int* slot) {
  ScalarPool& P = pool();
  for (size_t i = 0; i < P.pending.size();) {
    if (fence_done(P.pending[i].fence)) {
      P.free_slots.push_back(P.pending[i].slot);
      P.pending[i] = P.pending.back();
      P.pending.pop_back();
    } else {
      ++i;
    }
  }
  if (P.free_slots.empty()) {
    double* chunk = nullptr;
    APCG_CUDA(cudaMalloc(&chunk, sizeof(double) * kSlotsPerChunk));
    const int base = (int)P.chunks.size() * kSlotsPerChunk;
    P.chunks.push_back(chunk);
    for (int i = kSlotsPerChunk - 1; i >= 0; --i) P.free_slots.push_back(base + i);
  }
  *slot = P.free_slots.back();
  P.free_slots.pop_back();
  return APCG_OK;
}

enum ScalarOp : int { kOpSet = 0, kOpDiv, kOpRecip, kOpNeg, kOpCopy, kOpMul, kOpSqrt };

__global__ void scalar_op_kernel(int op, double* out, const double* a, const double* b, double v) {
  double r = 0.0;
  switch (op) {
    case kOpSet: r = v; break;
    case kOpDiv: r = *a / *b; break;
    case kOpRecip: r = 1.0 / *a; break;
    case kOpNeg: r = -*a; break;
    case kOpCopy: r = *a; break;
    case kOpMul: r = *a * *b; break;
    case kOpSqrt: r = sqrt(*a); break;
  }
  *out = r;
}

apcg_status scalar_op(apcg_ctx ctx_in, int op, apcg_scalar out, apcg_scalar a, apcg_scalar b, double v) {
  APCG_CHECK(out, "output scalar is NULL");
  const bool needs_a = op != kOpSet, needs_b = op == kOpDiv || op == kOpMul;
  APCG_CHECK(!needs_a || a, "input scalar is NULL");
  APCG_CHECK(!needs_b || b, "second input scalar is NULL");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op_scope(ctx);
  if (needs_a) op_scope.read(a->id);
  if (needs_b) op_scope.read(b->id);
  op_scope.write(out->id);
  APCG_TRY(op_scope.begin());
  scalar_op_kernel<<<1, 1, 0, ctx->stream>>>(op, out->dptr, needs_a ? a->dptr : nullptr, needs_b ? b->dptr : nullptr, v);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op_scope.finish();
}

}  // namespace

// ------------------------------------------------------------------ simulator

}  // namespace apcg

struct apcg_sim_s {
  int32_t nctx = 0;
  std::vector<uint64_t> seq, done_upto;
  apcg::DepTracker tracker;
  std::string log;
};

namespace apcg {
namespace {
struct SimBackend {
  apcg_sim_s* s;
  bool complete(uint64_t c, uint64_t q) { return s->done_upto[c] >= q; }
  void wait(uint64_t w, uint64_t c, uint64_t q) {
    s->log += std::to_string(w) + "<-" + std::to_string(c) + "@" + std::to_string(q) + "\n";
  }
  void elided(uint64_t w, uint64_t c, uint64_t q) {
    s->log += std::to_string(w) + ".." + std::to_string(c) + "@" + std::to_string(q) + "\n";
  }
};
}  // namespace
}  // namespace apcg

using namespace apcg;

// ================================================================== C ABI

extern "C" {

const char* apcg_last_error_string(void) { return t_last_error.c_str(); }

int32_t apcg_version(void) { return 10000; }

apcg_status apcg_get_counters(apcg_counters* out) {
  APCG_CHECK(out, "out is NULL");
  Counters& c = counters();
  out->kernel_launches = c.kernel_launches;
  out->graph_launches = c.graph_launches;
  out->waits_inserted = c.waits_inserted;
  out->waits_elided = c.waits_elided;
  out->events_recorded = c.events_recorded;
  out->host_syncs = c.host_syncs;
  out->d2h_copies = c.d2h_copies;
  out->d2h_bytes = c.d2h_bytes;
  out->h2d_copies = c.h2d_copies;
  out->h2d_bytes = c.h2d_bytes;
  return APCG_OK;
}

apcg_status apcg_reset_counters(void) {
  Counters& c = counters();
  c.kernel_launches = 0;
  c.graph_launches = 0;
  c.waits_inserted = 0;
  c.waits_elided = 0;
  c.events_recorded = 0;
  c.host_syncs = 0;
  c.d2h_copies = 0;
  c.d2h_bytes = 0;
  c.h2d_copies = 0;
  c.h2d_bytes = 0;
  return APCG_OK;
}

// ------------------------------------------------------------------ contexts

apcg_status apcg_ctx_create(apcg_ctx* out) {
  APCG_CHECK(out, "out is NULL");
  return new_ctx(nullptr, APCG_STREAM_DEFAULT_BLOCKING, out);
}

apcg_status apcg_ctx_create_from_stream(void* cuda_stream, apcg_ctx* out) {
  APCG_CHECK(out, "out is NULL");
  APCG_CHECK(cuda_stream, "stream is NULL (the legacy default stream cannot be borrowed)");
  return new_ctx(static_cast<cudaStream_t>(cuda_stream), APCG_STREAM_DEFAULT_BLOCKING, out);
}

apcg_status apcg_ctx_set_stream_type(apcg_ctx ctx, apcg_stream_type type) {
  APCG_CHECK(ctx, "ctx is NULL");
  APCG_CHECK(type == APCG_STREAM_DEFAULT_BLOCKING || type == APCG_STREAM_GLOBAL_BLOCKING, "bad stream type %d",
             (int)type);
  std::lock_guard<std::mutex> g(global_mutex());
  ctx->type = type;
  return APCG_OK;
}

apcg_status apcg_ctx_get_stream_type(apcg_ctx ctx, apcg_stream_type* type) {
  APCG_CHECK(ctx && type, "NULL argument");
  *type = ctx->type;
  return APCG_OK;
}

apcg_status apcg_ctx_get_stream(apcg_ctx ctx, void** s) {
  APCG_CHECK(ctx && s, "NULL argument");
  *s = ctx->stream;
  return APCG_OK;
}

apcg_status apcg_ctx_wait_for_context(apcg_ctx waiter, apcg_ctx waitee) {
  APCG_CHECK(waiter && waitee, "NULL context");
  if (waiter == waitee) return APCG_OK;
  std::lock_guard<std::mutex> g(global_mutex());
  return wait_tail(waiter, waitee);
}

apcg_status apcg_ctx_query_idle(apcg_ctx ctx, int32_t* idle) {
  APCG_CHECK(ctx && idle, "NULL argument");
  cudaError_t e = cudaStreamQuery(ctx->stream);
  if (e == cudaSuccess) {
    *idle = 1;
    return APCG_OK;
  }
  if (e == cudaErrorNotReady) {
    *idle = 0;
    return APCG_OK;
  }
  return cuda_error(e, "cudaStreamQuery", __FILE__, __LINE__);
}

apcg_status apcg_ctx_synchronize(apcg_ctx ctx) {
  APCG_CHECK(ctx, "ctx is NULL");
  APCG_CUDA(cudaStreamSynchronize(ctx->stream));
  counters().host_syncs++;
  return ctx_check_device_error(ctx);
}

apcg_status apcg_ctx_fork(apcg_ctx parent, int32_t n, apcg_ctx* children) {
  APCG_CHECK(parent && (n == 0 || children) && n >= 0, "bad fork arguments");
  for (int32_t i = 0; i < n; ++i) {
    apcg_ctx c = nullptr;
    apcg_status st = new_ctx(nullptr, parent->type, &c);
    if (st != APCG_OK) {
      for (int32_t j = 0; j < i; ++j) apcg_ctx_destroy(children[j]);
      return st;
    }
    children[i] = c;
    std::lock_guard<std::mutex> g(global_mutex());
    APCG_TRY(wait_tail(c, parent));
  }
  return APCG_OK;
}

apcg_status apcg_ctx_join(apcg_ctx parent, int32_t n, apcg_ctx* children, apcg_join_mode mode) {
  APCG_CHECK(parent && (n == 0 || children) && n >= 0, "bad join arguments");
  APCG_CHECK(mode == APCG_JOIN_DESTROY || mode == APCG_JOIN_SYNC || mode == APCG_JOIN_NO_SYNC, "bad join mode");
  {
    std::lock_guard<std::mutex> g(global_mutex());
    for (int32_t i = 0; i < n; ++i) {
      APCG_CHECK(children[i] && children[i] != parent, "bad child context %d", i);
      APCG_TRY(wait_tail(parent, children[i]));
    }
    if (mode == APCG_JOIN_SYNC)
      for (int32_t i = 0; i < n; ++i) APCG_TRY(wait_tail(children[i], parent));
  }
  if (mode == APCG_JOIN_DESTROY)
    for (int32_t i = 0; i < n; ++i) {
      APCG_TRY(apcg_ctx_destroy(children[i]));
      children[i] = nullptr;
    }
  return APCG_OK;
}

apcg_status apcg_ctx_destroy(apcg_ctx ctx) {
  APCG_CHECK(ctx, "ctx is NULL");
  std::lock_guard<std::mutex> g(global_mutex());
  APCG_CHECK(!ctx->zombie, "context already destroyed");
  if (ctx->scratch.partials) {
    cudaFreeAsync(ctx->scratch.partials, ctx->stream);
    ctx->scratch = ReduceScratch{};
  }
  APCG_TRY(record_tail(ctx));
  ctx->zombie = true;
  if (ctx->owns_stream) cudaStreamDestroy(ctx->stream);  // returns at once; released when idle
  ctx->stream = nullptr;
  if (reg().global_ctx == ctx) reg().global_ctx = nullptr;
  collect_zombies();
  return APCG_OK;
}

// ------------------------------------------------------------------ memory IDs and marking

apcg_status apcg_register_memory(const void* ptr, size_t bytes, apcg_id* id) {
  APCG_CHECK(ptr && id, "NULL argument");
  std::lock_guard<std::mutex> g(global_mutex());
  *id = register_memory(ptr, bytes);
  return APCG_OK;
}

apcg_status apcg_get_pointer_attributes(const void* ptr, apcg_id* id, size_t* bytes) {
  APCG_CHECK(ptr, "ptr is NULL");
  std::lock_guard<std::mutex> g(global_mutex());
  auto it = reg().mem.find(reinterpret_cast<uintptr_t>(ptr));
  APCG_CHECK(it != reg().mem.end(), "pointer %p is not registered", ptr);
  if (id) *id = it->second.first;
  if (bytes) *bytes = it->second.second;
  return APCG_OK;
}

apcg_status apcg_unregister_memory(const void* ptr) {
  APCG_CHECK(ptr, "ptr is NULL");
  std::lock_guard<std::mutex> g(global_mutex());
  auto it = reg().mem.find(reinterpret_cast<uintptr_t>(ptr));
  APCG_CHECK(it != reg().mem.end(), "pointer %p is not registered", ptr);
  reg().tracker.forget(it->second.first);
  reg().mem.erase(it);
  return APCG_OK;
}

apcg_status apcg_mark_intent_begin(apcg_ctx ctx, apcg_id id, apcg_access mode, const char* desc) {
  (void)desc;
  APCG_CHECK(ctx && !ctx->zombie, "bad context");
  APCG_CHECK(id != 0, "object id 0 is not valid");
  APCG_CHECK(mode == APCG_ACCESS_READ || mode == APCG_ACCESS_WRITE || mode == APCG_ACCESS_READ_WRITE, "bad mode");
  std::lock_guard<std::mutex> g(global_mutex());
  CudaBackend be;
  reg().tracker.begin(be, ctx->id, id, (int)mode);
  ctx->pending = true;
  return APCG_OK;
}

apcg_status apcg_mark_intent_end(apcg_ctx ctx, apcg_id id, apcg_access mode, const char* desc) {
  (void)desc;
  APCG_CHECK(ctx && !ctx->zombie, "bad context");
  APCG_CHECK(id != 0, "object id 0 is not valid");
  APCG_CHECK(mode == APCG_ACCESS_READ || mode == APCG_ACCESS_WRITE || mode == APCG_ACCESS_READ_WRITE, "bad mode");
  std::lock_guard<std::mutex> g(global_mutex());
  // One event per launch: the first end after a begin records it, later ends reuse it.
  if (ctx->pending) {
    APCG_TRY(record_tail(ctx));
    ctx->pending = false;
  }
  reg().tracker.end(ctx->id, id, (int)mode, ctx->seq);
  return APCG_OK;
}

apcg_status apcg_host_access(apcg_id id, apcg_access mode) {
  APCG_CHECK(id != 0, "object id 0 is not valid");
  std::vector<cudaEvent_t> evs;
  {
    std::lock_guard<std::mutex> g(global_mutex());
    CudaBackend be;
    for (const Access& a : reg().tracker.conflicts(id, (int)mode)) {
      if (be.complete(a.ctx, a.seq)) continue;
      apcg_ctx c = lookup_ctx(a.ctx);
      if (c) evs.push_back(c->ring[a.seq % kEventRing]);
    }
  }
  for (cudaEvent_t e : evs) APCG_CUDA(cudaEventSynchronize(e));
  if (!evs.empty()) counters().host_syncs++;
  return APCG_OK;
}

// ------------------------------------------------------------------ scalars

apcg_status apcg_scalar_create(apcg_dtype dtype, apcg_scalar* out) {
  APCG_CHECK(out, "out is NULL");
  if (dtype != APCG_F64) return set_error(APCG_ERR_UNSUPPORTED, "managed scalars are float64 only");
  std::lock_guard<std::mutex> g(global_mutex());
  int slot = -1;
  APCG_TRY(pool_acquire(&slot));
  apcg_scalar s = new apcg_scalar_s();
  s->slot = slot;
  s->dptr = pool().slot_ptr(slot);
  s->id = reg().next_id++;
  *out = s;
  return APCG_OK;
}

apcg_status apcg_scalar_set_async(apcg_ctx ctx, apcg_scalar s, double v) {
  return scalar_op(ctx, kOpSet, s, nullptr, nullptr, v);
}

apcg_status apcg_scalar_get(apcg_scalar s, double* v) {
  APCG_CHECK(s && v, "NULL argument");
  APCG_TRY(apcg_host_access(s->id, APCG_ACCESS_READ));
  APCG_CUDA(cudaMemcpy(v, s->dptr, sizeof(double), cudaMemcpyDeviceToHost));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(double);
  return APCG_OK;
}

apcg_status apcg_scalar_device_ptr(apcg_scalar s, double** dptr) {
  APCG_CHECK(s && dptr, "NULL argument");
  *dptr = s->dptr;
  return APCG_OK;
}

apcg_status apcg_scalar_id(apcg_scalar s, apcg_id* id) {
  APCG_CHECK(s && id, "NULL argument");
  *id = s->id;
  return APCG_OK;
}

apcg_status apcg_scalar_div_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar num, apcg_scalar den) {
  return scalar_op(ctx, kOpDiv, out, num, den, 0.0);
}
apcg_status apcg_scalar_recip_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a) {
  return scalar_op(ctx, kOpRecip, out, a, nullptr, 0.0);
}
apcg_status apcg_scalar_neg_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a) {
  return scalar_op(ctx, kOpNeg, out, a, nullptr, 0.0);
}
apcg_status apcg_scalar_copy_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a) {
  return scalar_op(ctx, kOpCopy, out, a, nullptr, 0.0);
}
apcg_status apcg_scalar_mul_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a, apcg_scalar b) {
  return scalar_op(ctx, kOpMul, out, a, b, 0.0);
}
apcg_status apcg_scalar_sqrt_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a) {
  return scalar_op(ctx, kOpSqrt, out, a, nullptr, 0.0);
}

apcg_status apcg_scalar_destroy(apcg_scalar s) {
  APCG_CHECK(s, "scalar is NULL");
  std::lock_guard<std::mutex> g(global_mutex());
  // The slot returns to the pool only after every recorded access has finished.
  pool().pending.push_back({s->slot, reg().tracker.conflicts(s->id, kReadWrite)});
  reg().tracker.forget(s->id);
  delete s;
  return APCG_OK;
}

// ------------------------------------------------------------------ simulator

apcg_status apcg_sim_create(int32_t nctx, apcg_sim* out) {
  APCG_CHECK(out && nctx > 0 && nctx < 1024, "bad simulator arguments");
  apcg_sim s = new apcg_sim_s();
  s->nctx = nctx;
  s->seq.assign(nctx, 0);
  s->done_upto.assign(nctx, 0);
  *out = s;
  return APCG_OK;
}

apcg_status apcg_sim_op(apcg_sim sim, int32_t ctx, int32_t nids, const apcg_id* ids, const int32_t* modes) {
  APCG_CHECK(sim && ctx >= 0 && ctx < sim->nctx && nids >= 0 && (nids == 0 || (ids && modes)), "bad arguments");
  for (int32_t i = 0; i < nids; ++i)
    APCG_CHECK(modes[i] >= 1 && modes[i] <= 3 && ids[i] != 0, "bad id or mode at %d", i);
  SimBackend be{sim};
  for (int32_t i = 0; i < nids; ++i) sim->tracker.begin(be, (uint64_t)ctx, ids[i], modes[i]);
  const uint64_t q = ++sim->seq[ctx];
  for (int32_t i = 0; i < nids; ++i) sim->tracker.end((uint64_t)ctx, ids[i], modes[i], q);
  return APCG_OK;
}

apcg_status apcg_sim_complete(apcg_sim sim, int32_t ctx, uint64_t seq) {
  APCG_CHECK(sim && ctx >= 0 && ctx < sim->nctx, "bad arguments");
  if (seq > sim->done_upto[ctx]) sim->done_upto[ctx] = seq;
  return APCG_OK;
}

apcg_status apcg_sim_log(apcg_sim sim, char* buf, size_t len) {
  APCG_CHECK(sim && buf && len > 0, "bad arguments");
  const size_t n = std::min(len - 1, sim->log.size());
  memcpy(buf, sim->log.data(), n);
  buf[n] = '\0';
  APCG_CHECK(sim->log.size() < len, "log truncated: %zu bytes needed", sim->log.size() + 1);
  return APCG_OK;
}

apcg_status apcg_sim_destroy(apcg_sim sim) {
  APCG_CHECK(sim, "sim is NULL");
  delete sim;
  return APCG_OK;
}

}  // extern "C"
