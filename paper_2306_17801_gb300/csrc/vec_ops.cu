// The asynchronous vector and matrix operations of Sec. 3.3 (VecDotAsync,
// VecNormAsync, VecAXPYAsync, VecAYPX, VecScaleAsync, VecCopy,
// KSP_MatMultAsync, KSP_PCApplyAsync) on float64 views, each one marked
// kernel on the caller's context.  Managed scalars are read and written on
// the device; reductions finish in the last block and write the scalar slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "kernels_common.cuh"
#include "spmv.cuh"

namespace apcg {
namespace {

constexpr int kVecThreads = 256;
constexpr int kSpmvThreads = 256;
constexpr int kSpmvU = 8;

int vec_grid(apcg_ctx ctx, int64_t n_pairs, int cap) {
  int64_t g = (n_pairs + kVecThreads - 1) / kVecThreads;
  const int64_t lim = (int64_t)ctx_num_sms(ctx) * 8;
  if (g > lim) g = lim;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

// ------------------------------------------------------------------ kernels

__global__ void __launch_bounds__(kVecThreads) dot_kernel(int64_t n, const double* __restrict__ x,
                                                          const double* __restrict__ y, double* out, int take_sqrt,
                                                          double* partials, unsigned int* ticket) {
  __shared__ double smem[kVecThreads];
  double v[1] = {0.0};
  const int64_t np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  const double2* x2 = reinterpret_cast<const double2*>(x);
  const double2* y2 = reinterpret_cast<const double2*>(y);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
    const double2 a = __ldg(x2 + i), b = __ldg(y2 + i);
    v[0] += a.x * b.x;
    v[0] += a.y * b.y;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) v[0] += x[n - 1] * y[n - 1];
  double tot[1];
  if (dev::grid_sum_last<1>(v, partials, ticket, smem, tot) && threadIdx.x == 0) *out = take_sqrt ? sqrt(tot[0]) : tot[0];
}

// y := y + s * a * x  (s = +1 or -1)
__global__ void __launch_bounds__(kVecThreads) axpy_kernel(int64_t n, double* __restrict__ y, const double* a_ptr,
                                                           double s, const double* __restrict__ x) {
  const double a = s * *a_ptr;
  const int64_t np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  double2* y2 = reinterpret_cast<double2*>(y);
  const double2* x2 = reinterpret_cast<const double2*>(x);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
    double2 t = y2[i];
    const double2 u = __ldg(x2 + i);
    t.x += a * u.x;
    t.y += a * u.y;
    y2[i] = t;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) y[n - 1] += a * x[n - 1];
}

// y := x + b * y
__global__ void __launch_bounds__(kVecThreads) aypx_kernel(int64_t n, double* __restrict__ y, const double* b_ptr,
                                                           const double* __restrict__ x) {
  const double b = *b_ptr;
  const int64_t np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  double2* y2 = reinterpret_cast<double2*>(y);
  const double2* x2 = reinterpret_cast<const double2*>(x);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
    double2 t = y2[i];
    const double2 u = __ldg(x2 + i);
    t.x = u.x + b * t.x;
    t.y = u.y + b * t.y;
    y2[i] = t;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) y[n - 1] = x[n - 1] + b * y[n - 1];
}

// y := a * y
__global__ void __launch_bounds__(kVecThreads) scale_kernel(int64_t n, double* __restrict__ y, const double* a_ptr) {
  const double a = *a_ptr;
  const int64_t np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  double2* y2 = reinterpret_cast<double2*>(y);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
    double2 t = y2[i];
    t.x *= a;
    t.y *= a;
    y2[i] = t;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) y[n - 1] *= a;
}

// y := src (copy) or y := v (set, src == nullptr)
__global__ void __launch_bounds__(kVecThreads) copy_set_kernel(int64_t n, double* __restrict__ y,
                                                               const double* __restrict__ src, double v) {
  const int64_t np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  double2* y2 = reinterpret_cast<double2*>(y);
  const double2* s2 = reinterpret_cast<const double2*>(src);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride)
    y2[i] = src ? __ldg(s2 + i) : make_double2(v, v);
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) y[n - 1] = src ? src[n - 1] : v;
}

// w := x .* y
__global__ void __launch_bounds__(kVecThreads) pmult_kernel(int64_t n, double* __restrict__ w,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ y) {
  const int64_t np = n >> 1, stride = (int64_t)gridDim.x * blockDim.x;
  double2* w2 = reinterpret_cast<double2*>(w);
  const double2* x2 = reinterpret_cast<const double2*>(x);
  const double2* y2 = reinterpret_cast<const double2*>(y);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
    const double2 a = __ldg(x2 + i), b = __ldg(y2 + i);
    w2[i] = make_double2(a.x * b.x, a.y * b.y);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) w[n - 1] = x[n - 1] * y[n - 1];
}

// y := A x; with DOT, also out := x'y (A square).
template <int U, bool DOT>
__global__ void __launch_bounds__(kSpmvThreads) spmv_kernel(const int32_t* __restrict__ rowptr,
                                                            const int32_t* __restrict__ col,
                                                            const double* __restrict__ val, int32_t nrows,
                                                            const double* __restrict__ x, double* __restrict__ y,
                                                            double* out, double* partials, unsigned int* ticket) {
  __shared__ dev::SpmvSmem<U, double> sm[kSpmvThreads / 32];
  __shared__ double red[kSpmvThreads];
  double v[1] = {0.0};
  dev::spmv_warp_tiles<U, DOT, double>(rowptr, col, val, x, nrows, sm[threadIdx.x >> 5].buf,
                                       [&](int32_t row, double s, double x_row) {
                                         y[row] = s;
                                         if (DOT) v[0] += x_row * s;
                                       });
  if (!DOT) return;
  double tot[1];
  if (dev::grid_sum_last<1>(v, partials, ticket, red, tot) && threadIdx.x == 0) *out = tot[0];
}

// dinv := 1 / diag(A); flags a missing, zero or non-finite diagonal entry.
__global__ void jacobi_setup_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, int32_t n, double* __restrict__ dinv,
                                    int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double d = 0.0;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == (int32_t)i) d += val[e];
    if (!(d != 0.0) || !isfinite(d)) {
      atomicOr(err, kDevErrBadDiagonal);
      dinv[i] = 0.0;
    } else {
      dinv[i] = 1.0 / d;
    }
  }
}

// ------------------------------------------------------------------ host helpers

apcg_status check_vec(apcg_vec v, const char* name) {
  APCG_CHECK(v, "%s is NULL", name);
  APCG_CHECK(v->dtype == APCG_F64, "%s: only float64 vectors are supported by this operation", name);
  APCG_CHECK(v->n == 0 || aligned16(v->dptr), "%s: pointer %p is not 16-byte aligned", name, v->dptr);
  return APCG_OK;
}

apcg_status same_len(apcg_vec a, apcg_vec b) {
  APCG_CHECK(a->n == b->n, "vector lengths differ (%lld vs %lld)", (long long)a->n, (long long)b->n);
  return APCG_OK;
}

}  // namespace

apcg_status launch_fill(apcg_ctx ctx, double* y, int64_t n, double v) {
  copy_set_kernel<<<vec_grid(ctx, n >> 1, 1 << 20), kVecThreads, 0, ctx->stream>>>(n, y, nullptr, v);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return APCG_OK;
}

apcg_status launch_jacobi_setup(apcg_ctx ctx, apcg_mat A, double* dinv) {
  APCG_TRY(ensure_scratch(ctx));
  const int g = vec_grid(ctx, A->nrows, 1 << 20);
  jacobi_setup_kernel<<<g, kVecThreads, 0, ctx->stream>>>(A->rowptr, A->col, static_cast<const double*>(A->val),
                                                          A->nrows, dinv, ctx->scratch.dev_error);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return APCG_OK;
}

}  // namespace apcg

using namespace apcg;

extern "C" {

// ------------------------------------------------------------------ objects

apcg_status apcg_vec_wrap(void* dptr, int64_t n, apcg_dtype dtype, apcg_vec* out) {
  APCG_CHECK(out, "out is NULL");
  APCG_CHECK(n >= 0, "negative length");
  APCG_CHECK(n == 0 || dptr, "NULL data pointer");
  APCG_CHECK(dtype == APCG_F64 || dtype == APCG_F32, "bad dtype");
  APCG_CHECK(n == 0 || aligned16(dptr), "pointer %p is not 16-byte aligned", dptr);
  apcg_vec v = new apcg_vec_s();
  v->dptr = dptr;
  v->n = n;
  v->dtype = dtype;
  {
    std::lock_guard<std::mutex> g(global_mutex());
    v->id = register_memory(dptr ? dptr : static_cast<void*>(v), (size_t)n * (dtype == APCG_F64 ? 8 : 4));
  }
  *out = v;
  return APCG_OK;
}

apcg_status apcg_vec_id(apcg_vec v, apcg_id* id) {
  APCG_CHECK(v && id, "NULL argument");
  *id = v->id;
  return APCG_OK;
}

apcg_status apcg_vec_destroy(apcg_vec v) {
  APCG_CHECK(v, "vector is NULL");
  delete v;  // the registration (and its marks) stays with the memory
  return APCG_OK;
}

apcg_status apcg_mat_csr_wrap(const int32_t* rowptr, const int32_t* col, const void* val, int32_t nrows,
                              int32_t ncols, int64_t nnz, apcg_dtype dtype, apcg_mat* out) {
  APCG_CHECK(out, "out is NULL");
  APCG_CHECK(nrows >= 0 && ncols >= 0 && nnz >= 0, "negative size");
  APCG_CHECK(nnz <= (int64_t)INT32_MAX - 4096, "nnz %lld exceeds the int32 index range", (long long)nnz);
  APCG_CHECK(rowptr, "rowptr is NULL");
  APCG_CHECK(nnz == 0 || (col && val), "col/val is NULL");
  APCG_CHECK(dtype == APCG_F64 || dtype == APCG_F32, "bad dtype");
  APCG_CHECK(nnz == 0 || aligned16(val), "val pointer is not 16-byte aligned");
  apcg_mat A = new apcg_mat_s();
  A->rowptr = rowptr;
  A->col = col;
  A->val = val;
  A->nrows = nrows;
  A->ncols = ncols;
  A->nnz = nnz;
  A->dtype = dtype;
  {
    std::lock_guard<std::mutex> g(global_mutex());
    A->id = register_memory(rowptr, sizeof(int32_t) * ((size_t)nrows + 1));
  }
  *out = A;
  return APCG_OK;
}

apcg_status apcg_mat_validate(apcg_mat A) {
  APCG_CHECK(A, "matrix is NULL");
  APCG_TRY(apcg_host_access(A->id, APCG_ACCESS_READ));
  std::vector<int32_t> rp((size_t)A->nrows + 1), col((size_t)A->nnz);
  APCG_CUDA(cudaMemcpy(rp.data(), A->rowptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost));
  if (A->nnz) APCG_CUDA(cudaMemcpy(col.data(), A->col, sizeof(int32_t) * col.size(), cudaMemcpyDeviceToHost));
  counters().d2h_copies += 2;
  counters().d2h_bytes += (int64_t)(sizeof(int32_t) * (rp.size() + col.size()));
  APCG_CHECK(rp[0] == 0, "rowptr[0] = %d, expected 0", rp[0]);
  APCG_CHECK(rp[A->nrows] == A->nnz, "rowptr[nrows] = %d, expected nnz = %lld", rp[A->nrows], (long long)A->nnz);
  for (int32_t i = 0; i < A->nrows; ++i) APCG_CHECK(rp[i] <= rp[i + 1], "rowptr decreases at row %d", i);
  for (int64_t e = 0; e < A->nnz; ++e)
    APCG_CHECK(col[e] >= 0 && col[e] < A->ncols, "column index %d out of range at entry %lld", col[e], (long long)e);
  return APCG_OK;
}

apcg_status apcg_mat_id(apcg_mat A, apcg_id* id) {
  APCG_CHECK(A && id, "NULL argument");
  *id = A->id;
  return APCG_OK;
}

apcg_status apcg_mat_destroy(apcg_mat A) {
  APCG_CHECK(A, "matrix is NULL");
  delete A;
  return APCG_OK;
}

// ------------------------------------------------------------------ vector operations

apcg_status apcg_vec_dot_async(apcg_ctx ctx_in, apcg_vec x, apcg_vec y, apcg_scalar out) {
  APCG_TRY(check_vec(x, "x"));
  APCG_TRY(check_vec(y, "y"));
  APCG_TRY(same_len(x, y));
  APCG_CHECK(out, "out scalar is NULL");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  APCG_TRY(ensure_scratch(ctx));
  OpScope op(ctx);
  op.read(x->id).read(y->id).write(out->id);
  APCG_TRY(op.begin());
  const int g = vec_grid(ctx, x->n >> 1, dev::kMaxPartials);
  dot_kernel<<<g, kVecThreads, 0, ctx->stream>>>(x->n, static_cast<const double*>(x->dptr),
                                                 static_cast<const double*>(y->dptr), out->dptr, 0,
                                                 ctx->scratch.partials, ctx->scratch.ticket);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_vec_norm2_async(apcg_ctx ctx_in, apcg_vec x, apcg_scalar out) {
  APCG_TRY(check_vec(x, "x"));
  APCG_CHECK(out, "out scalar is NULL");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  APCG_TRY(ensure_scratch(ctx));
  OpScope op(ctx);
  op.read(x->id).write(out->id);
  APCG_TRY(op.begin());
  const int g = vec_grid(ctx, x->n >> 1, dev::kMaxPartials);
  const double* p = static_cast<const double*>(x->dptr);
  dot_kernel<<<g, kVecThreads, 0, ctx->stream>>>(x->n, p, p, out->dptr, 1, ctx->scratch.partials,
                                                 ctx->scratch.ticket);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_vec_axpy_async(apcg_ctx ctx_in, apcg_vec y, apcg_scalar a, int32_t negate, apcg_vec x) {
  APCG_TRY(check_vec(x, "x"));
  APCG_TRY(check_vec(y, "y"));
  APCG_TRY(same_len(x, y));
  APCG_CHECK(a, "scalar is NULL");
  APCG_CHECK(x->dptr != y->dptr || x->n == 0, "x and y must not alias");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.read(x->id).read(a->id).rw(y->id);
  APCG_TRY(op.begin());
  axpy_kernel<<<vec_grid(ctx, y->n >> 1, 1 << 20), kVecThreads, 0, ctx->stream>>>(
      y->n, static_cast<double*>(y->dptr), a->dptr, negate ? -1.0 : 1.0, static_cast<const double*>(x->dptr));
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_vec_aypx_async(apcg_ctx ctx_in, apcg_vec y, apcg_scalar b, apcg_vec x) {
  APCG_TRY(check_vec(x, "x"));
  APCG_TRY(check_vec(y, "y"));
  APCG_TRY(same_len(x, y));
  APCG_CHECK(b, "scalar is NULL");
  APCG_CHECK(x->dptr != y->dptr || x->n == 0, "x and y must not alias");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.read(x->id).read(b->id).rw(y->id);
  APCG_TRY(op.begin());
  aypx_kernel<<<vec_grid(ctx, y->n >> 1, 1 << 20), kVecThreads, 0, ctx->stream>>>(
      y->n, static_cast<double*>(y->dptr), b->dptr, static_cast<const double*>(x->dptr));
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_vec_scale_async(apcg_ctx ctx_in, apcg_vec y, apcg_scalar a) {
  APCG_TRY(check_vec(y, "y"));
  APCG_CHECK(a, "scalar is NULL");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.read(a->id).rw(y->id);
  APCG_TRY(op.begin());
  scale_kernel<<<vec_grid(ctx, y->n >> 1, 1 << 20), kVecThreads, 0, ctx->stream>>>(
      y->n, static_cast<double*>(y->dptr), a->dptr);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_vec_copy_async(apcg_ctx ctx_in, apcg_vec dst, apcg_vec src) {
  APCG_TRY(check_vec(dst, "dst"));
  APCG_TRY(check_vec(src, "src"));
  APCG_TRY(same_len(dst, src));
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.read(src->id).write(dst->id);
  APCG_TRY(op.begin());
  if (dst->dptr != src->dptr) {
    copy_set_kernel<<<vec_grid(ctx, dst->n >> 1, 1 << 20), kVecThreads, 0, ctx->stream>>>(
        dst->n, static_cast<double*>(dst->dptr), static_cast<const double*>(src->dptr), 0.0);
    APCG_CUDA(cudaGetLastError());
    count_kernels(1);
  }
  return op.finish();
}

apcg_status apcg_vec_set_async(apcg_ctx ctx_in, apcg_vec y, double v) {
  APCG_TRY(check_vec(y, "y"));
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.write(y->id);
  APCG_TRY(op.begin());
  copy_set_kernel<<<vec_grid(ctx, y->n >> 1, 1 << 20), kVecThreads, 0, ctx->stream>>>(
      y->n, static_cast<double*>(y->dptr), nullptr, v);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_vec_pointwise_mult_async(apcg_ctx ctx_in, apcg_vec w, apcg_vec x, apcg_vec y) {
  APCG_TRY(check_vec(w, "w"));
  APCG_TRY(check_vec(x, "x"));
  APCG_TRY(check_vec(y, "y"));
  APCG_TRY(same_len(w, x));
  APCG_TRY(same_len(w, y));
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.read(x->id).read(y->id).write(w->id);
  APCG_TRY(op.begin());
  pmult_kernel<<<vec_grid(ctx, w->n >> 1, 1 << 20), kVecThreads, 0, ctx->stream>>>(
      w->n, static_cast<double*>(w->dptr), static_cast<const double*>(x->dptr), static_cast<const double*>(y->dptr));
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

// ------------------------------------------------------------------ matrix operations

static apcg_status mat_mult_impl(apcg_ctx ctx_in, apcg_mat A, apcg_vec x, apcg_vec y, apcg_scalar out) {
  APCG_CHECK(A, "matrix is NULL");
  APCG_CHECK(A->dtype == APCG_F64, "only float64 matrices are supported by this operation");
  APCG_TRY(check_vec(x, "x"));
  APCG_TRY(check_vec(y, "y"));
  APCG_CHECK(x->n == A->ncols, "x has %lld elements, A has %d columns", (long long)x->n, A->ncols);
  APCG_CHECK(y->n == A->nrows, "y has %lld elements, A has %d rows", (long long)y->n, A->nrows);
  APCG_CHECK(x->dptr != y->dptr || A->nrows == 0, "x and y must not alias");
  APCG_CHECK(!out || A->nrows == A->ncols, "the fused dot needs a square matrix");
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  if (out) APCG_TRY(ensure_scratch(ctx));
  OpScope op(ctx);
  op.read(A->id).read(x->id).write(y->id);
  if (out) op.write(out->id);
  APCG_TRY(op.begin());
  const int64_t tiles = ((int64_t)A->nrows + 31) / 32;
  int64_t g = (tiles + (kSpmvThreads / 32) - 1) / (kSpmvThreads / 32);
  const int64_t lim = (int64_t)ctx_num_sms(ctx) * 8;
  if (g > lim) g = lim;
  if (g < 1) g = 1;
  auto kern = out ? spmv_kernel<kSpmvU, true> : spmv_kernel<kSpmvU, false>;
  kern<<<(int)g, kSpmvThreads, 0, ctx->stream>>>(A->rowptr, A->col, static_cast<const double*>(A->val), A->nrows,
                                                 static_cast<const double*>(x->dptr), static_cast<double*>(y->dptr),
                                                 out ? out->dptr : nullptr, ctx->scratch.partials,
                                                 ctx->scratch.ticket);
  APCG_CUDA(cudaGetLastError());
  count_kernels(1);
  return op.finish();
}

apcg_status apcg_mat_mult_async(apcg_ctx ctx, apcg_mat A, apcg_vec x, apcg_vec y) {
  return mat_mult_impl(ctx, A, x, y, nullptr);
}

apcg_status apcg_mat_mult_dot_async(apcg_ctx ctx, apcg_mat A, apcg_vec x, apcg_vec y, apcg_scalar out) {
  APCG_CHECK(out, "out scalar is NULL");
  return mat_mult_impl(ctx, A, x, y, out);
}

apcg_status apcg_pc_jacobi_setup_async(apcg_ctx ctx_in, apcg_mat A, apcg_vec dinv) {
  APCG_CHECK(A, "matrix is NULL");
  APCG_CHECK(A->dtype == APCG_F64, "only float64 matrices are supported by this operation");
  APCG_CHECK(A->nrows == A->ncols, "Jacobi needs a square matrix");
  APCG_TRY(check_vec(dinv, "dinv"));
  APCG_CHECK(dinv->n == A->nrows, "dinv length %lld != %d rows", (long long)dinv->n, A->nrows);
  apcg_ctx ctx;
  APCG_TRY(resolve_ctx(ctx_in, &ctx));
  OpScope op(ctx);
  op.read(A->id).write(dinv->id).may_flag_errors();
  APCG_TRY(op.begin());
  APCG_TRY(launch_jacobi_setup(ctx, A, static_cast<double*>(dinv->dptr)));
  return op.finish();
}

apcg_status apcg_pc_jacobi_apply_async(apcg_ctx ctx, apcg_vec dinv, apcg_vec r, apcg_vec z) {
  return apcg_vec_pointwise_mult_async(ctx, z, dinv, r);
}

}  // extern "C"
