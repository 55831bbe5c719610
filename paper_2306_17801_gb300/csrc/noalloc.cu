// Jacobi-PCG for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at solve time: a host framework that has
// reserved nearly all device memory for its own pool (so a library allocation
// would fail), or a real-time loop that must not allocate after start-up
// (device allocation can synchronise the device and its cost is unbounded).
// apcg_cg_solve_noalloc serves them: it runs the whole-solve cluster kernel
// (cluster_cg.cu) for one system, with the Jacobi diagonal and the solve's
// bookkeeping in the file-scope array below instead of an allocated
// workspace.  Every GPU that loads the library holds this array until the
// process exits, so it is kept modest: 65536 rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "cluster_cg.hpp"

namespace {

constexpr int kNoAllocMaxRows = 65536;
constexpr int kNoAllocTail = 32;  // doubles after dinv: descriptor, result, counter, error word
// dinv[0 .. kNoAllocMaxRows) followed by the bookkeeping block.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxRows + kNoAllocTail];

// Error word of the bookkeeping block.
enum : int32_t { kErrBadDiagonal = 1, kErrStructure = 2 };

struct Tail {
  apcg::SysDesc sys;
  apcg::SysResult res;
  unsigned int next;  // the cluster kernel's work counter: 1 (= nsys) leaves it nothing to solve
  int32_t error;
};
static_assert(sizeof(Tail) <= sizeof(double) * kNoAllocTail, "bookkeeping block too large");

// Device address of the scratch array on the current device.  Looked up on every call
// (cudaGetSymbolAddress allocates nothing), so a cudaDeviceReset between calls cannot leave a stale address.
apcg_status scratch_address(double** out) {
  void* p = nullptr;
  APCG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = static_cast<double*>(p);
  return APCG_OK;
}

// Reset the bookkeeping block: one system of n rows, work counter and error word zero.
__global__ void noalloc_init_kernel(Tail* t, int32_t n) {
  t->sys.row0 = 0;
  t->sys.n = n;
  t->sys.pad = 0;
  t->res = apcg::SysResult{};
  t->next = 0u;
  t->error = 0;
}

// The CSR structure, read only within its declared sizes (rowptr[0..n], col[0..nnz)): rowptr starts at 0,
// never decreases and ends at nnz; every column lies in [0, n).  A violation sets the error word and takes
// the solve's work away, so that no later kernel reads through the structure.
__global__ void noalloc_check_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int32_t n,
                                     int64_t nnz, Tail* t) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (tid == 0) bad = rowptr[0] != 0 || (int64_t)rowptr[n] != nnz;
  for (int64_t i = tid; i < n; i += stride) bad |= rowptr[i + 1] < rowptr[i];
  for (int64_t e = tid; e < nnz; e += stride) bad |= col[e] < 0 || col[e] >= n;
  if (bad) {
    atomicOr(&t->error, kErrStructure);
    t->next = 1u;
  }
}

// dinv := 1 / diag(A) after a clean structure check; a missing, zero or non-finite diagonal sets the error
// word and takes the solve's work away (x is then left as it was).
__global__ void noalloc_jacobi_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                      const double* __restrict__ val, int32_t n, double* __restrict__ dinv, Tail* t) {
  if (*(volatile int32_t*)&t->error) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = 0.0;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == (int32_t)i) d += val[e];
    const bool bad = !(d != 0.0) || !isfinite(d);
    if (bad) {
      atomicOr(&t->error, kErrBadDiagonal);
      t->next = 1u;
    }
    dinv[i] = bad ? 0.0 : 1.0 / d;
  }
}

}  // namespace

using namespace apcg;

extern "C" apcg_status apcg_cg_solve_noalloc(void* cuda_stream, int32_t n, int64_t nnz, const int32_t* rowptr,
                                             const int32_t* col, const double* val, const double* b, double* x,
                                             const apcg_cg_opts* opts, apcg_cg_result* res) {
  APCG_CHECK(res, "res is NULL");
  APCG_CHECK(n >= 0 && nnz >= 0, "negative size");
  APCG_CHECK(n <= kNoAllocMaxRows, "n = %d exceeds the %d rows that the static scratch of apcg_cg_solve_noalloc holds",
             n, kNoAllocMaxRows);
  APCG_CHECK(nnz <= (int64_t)INT32_MAX - 4096, "nnz %lld exceeds the int32 index range", (long long)nnz);
  APCG_CHECK(rowptr && (nnz == 0 || (col && val)) && (n == 0 || (b && x)), "NULL argument");
  APCG_CHECK(n == 0 || (aligned16(b) && aligned16(x)), "b/x must be 16-byte aligned");
  apcg_cg_opts o;
  if (opts)
    o = *opts;
  else
    apcg_cg_opts_default(&o);
  APCG_CHECK(o.check_every >= 1 && o.rtol >= 0.0 && o.atol >= 0.0, "bad options");
  const ClusterShape sh = default_cluster_shape(n);
  if (!sh.ok) return set_error(APCG_ERR_UNSUPPORTED, "no schedulable cluster shape for %d rows", n);
  double* scratch = nullptr;
  APCG_TRY(scratch_address(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  Tail* tail = reinterpret_cast<Tail*>(scratch + kNoAllocMaxRows);
  noalloc_init_kernel<<<1, 1, 0, s>>>(tail, n);
  APCG_CUDA(cudaGetLastError());
  int launches = 1;
  if (n > 0) {
    const int64_t work = std::max<int64_t>(n, nnz);
    const int cblocks = (int)std::min<int64_t>((work + 255) / 256, 1024);
    noalloc_check_kernel<<<cblocks, 256, 0, s>>>(rowptr, col, n, nnz, tail);
    APCG_CUDA(cudaGetLastError());
    noalloc_jacobi_kernel<<<(n + 255) / 256, 256, 0, s>>>(rowptr, col, val, n, scratch, tail);
    APCG_CUDA(cudaGetLastError());
    launches += 2;
  }
  ClusterArgs ca{};
  ca.rowptr = rowptr;
  ca.col = col;
  ca.val = val;
  ca.dinv = scratch;
  ca.b = b;
  ca.x = x;
  ca.sys = &tail->sys;
  ca.order = nullptr;
  ca.nsys = 1;
  ca.check_every = o.check_every;
  ca.next = &tail->next;
  ca.res = &tail->res;
  ca.rtol = o.rtol;
  ca.atol = o.atol;
  ca.max_it = o.max_it;
  ca.hist_len = 0;
  APCG_CUDA(launch_cluster_cg(ca, sh, 1, s));
  launches += 1;
  count_kernels(launches);
  Tail h;
  APCG_CUDA(cudaMemcpyAsync(&h, tail, sizeof(Tail), cudaMemcpyDeviceToHost, s));
  APCG_CUDA(cudaStreamSynchronize(s));
  counters().d2h_copies++;
  counters().d2h_bytes += sizeof(Tail);
  counters().host_syncs++;
  memset(res, 0, sizeof(*res));
  res->kernel_launches = launches;
  if (h.error & kErrStructure)
    return set_error(APCG_ERR_INVALID_ARG,
                     "malformed CSR structure (rowptr must start at 0, not decrease and end at nnz; columns in [0, n))");
  if ((h.error & kErrBadDiagonal) || h.res.done == kDoneBadDiagonal)
    return set_error(APCG_ERR_BAD_DIAGONAL, "Jacobi: a diagonal entry is missing, zero or not finite");
  res->iters = h.res.iters;
  res->reason = h.res.done == kDoneConverged      ? APCG_CONVERGED
                : h.res.done == kDoneNotConverged ? APCG_NOT_CONVERGED
                                                  : APCG_BREAKDOWN;
  res->rr = h.res.rr;
  res->bnorm = std::sqrt(h.res.bnorm2);
  res->rel_res = res->bnorm > 0.0 ? std::sqrt(h.res.rr) / res->bnorm : std::sqrt(h.res.rr);
  return APCG_OK;
}
