// Launch-floor measurements: the fixed costs that bound the per-iteration
// time of a latency-bound solve (a 64^2 system moves 0.7 MB per iteration,
// 0.1 us at HBM speed, so its iterations cost what launches and host round
// trips cost).  Used by the benchmark's small-system report.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>

#include "apcg_internal.hpp"

namespace apcg {
namespace {

__global__ void empty_kernel() {}

// Float64 FMA throughput: kChains independent chains a = fma(a, m, c) per thread, iterated `iters` times
// (m and c are kernel arguments, so nothing folds; |m| < 1 keeps the values finite and normal).  Each
// thread's sum goes to sink so that no chain is dead code.
constexpr int kFmaChains = 8;
constexpr int kFmaThreads = 256;

__global__ void __launch_bounds__(kFmaThreads) fma64_kernel(int32_t iters, double m, double c, double* sink) {
  double a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = 1e-3 * threadIdx.x + k;
  for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace apcg

using namespace apcg;

extern "C" {

apcg_status apcg_launch_floor(apcg_ctx ctx_in, int32_t reps, double* us) {
  APCG_CHECK(us && reps >= 1, "us must be non-NULL and reps >= 1");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  cudaStream_t s = ctx->stream;
  APCG_CUDA(cudaStreamSynchronize(s));
  // one empty kernel, launched and waited for
  double t0 = now_us();
  for (int32_t i = 0; i < reps; ++i) {
    empty_kernel<<<1, 32, 0, s>>>();
    APCG_CUDA(cudaStreamSynchronize(s));
  }
  us[0] = (now_us() - t0) / reps;
  // a graph of three dependent empty kernels, launched and waited for
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t cap = nullptr;
  APCG_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    empty_kernel<<<1, 32, 0, cap>>>();
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  cudaStreamDestroy(cap);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (e == cudaSuccess) e = cudaGraphUpload(ge, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    t0 = now_us();
    for (int32_t i = 0; i < reps && e == cudaSuccess; ++i) {
      e = cudaGraphLaunch(ge, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    us[1] = (now_us() - t0) / reps;
  }
  // the same graph launched back to back: device time per three-kernel graph
  if (e == cudaSuccess) {
    t0 = now_us();
    for (int32_t i = 0; i < reps && e == cudaSuccess; ++i) e = cudaGraphLaunch(ge, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    us[3] = (now_us() - t0) / reps;
  }
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_error(e, "launch-floor graph", __FILE__, __LINE__);
  // an 8-byte device-to-host copy and wait (what a host-synchronous iteration pays per reduction)
  double* d = nullptr;
  double* h = nullptr;
  APCG_TRY(dev_alloc_async((void**)&d, sizeof(double), s));
  e = cudaMallocHost((void**)&h, sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    t0 = now_us();
    for (int32_t i = 0; i < reps && e == cudaSuccess; ++i) {
      e = cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    us[2] = (now_us() - t0) / reps;
  }
  cudaFreeAsync(d, s);
  cudaStreamSynchronize(s);
  if (h) cudaFreeHost(h);
  if (e != cudaSuccess) return cuda_error(e, "launch-floor copy", __FILE__, __LINE__);
  count_kernels((int64_t)reps * 7);
  return APCG_OK;
}

apcg_status apcg_fp64_fma_peak(apcg_ctx ctx_in, int32_t reps, double* gflops) {
  APCG_CHECK(gflops && reps >= 1, "gflops must be non-NULL and reps >= 1");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  cudaStream_t s = ctx->stream;
  int per_sm = 0;
  APCG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma64_kernel, kFmaThreads, 0));
  const int grid = std::max(1, per_sm) * ctx_num_sms(ctx);
  const int32_t iters = 1024;
  double* sink = nullptr;
  APCG_TRY(dev_alloc_async((void**)&sink, sizeof(double) * (size_t)grid * kFmaThreads, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = -1.f;
  for (int32_t r = 0; r <= reps && e == cudaSuccess; ++r) {  // launch 0 warms up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      fma64_kernel<<<grid, kFmaThreads, 0, s>>>(iters, 0.99999999, 1e-8, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best < 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  count_kernels((int64_t)reps + 1);
  if (e != cudaSuccess) return cuda_error(e, "float64 FMA peak", __FILE__, __LINE__);
  const double flops = 2.0 * kFmaChains * (double)iters * (double)grid * kFmaThreads;
  *gflops = flops / (best * 1e-3) / 1e9;
  return APCG_OK;
}

}  // extern "C"
