/*
 * Multi-threaded timing variant of the float64 Jacobi-PCG oracle.
 *
 * TEST INFRASTRUCTURE ONLY, and for timing only: the checker is the
 * single-threaded oracle in pcg_oracle.c; this file exists so that the CPU
 * baseline can be measured on all of a host's cores, standing in for a
 * multi-core CPU solver run beside the GPU (the paper's CPU variant of
 * Sec. 4.1-4.2).  It shares nothing with the CUDA library.
 *
 * It runs the same steps as oracle_pcg, in the same order (Sec. 3.3's loop:
 * w = A p, gamma = (p,w), alpha = rho/gamma, x += alpha p, r -= alpha w,
 * rr = (r,r), test every k-th iteration, z = r ./ d, rho' = (r,z),
 * beta = rho'/rho, p = z + beta p), with every vector loop and the SpMV split
 * over OpenMP threads by a static schedule.  Each inner product is a
 * Neumaier-compensated partial sum per thread over its static block of
 * indices, the partials then added in thread order: for a fixed thread
 * count the result is deterministic, and it differs from the sequential
 * oracle only in summation order.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t iters;
  int32_t reason; /* 0 converged, 1 not converged, 2 breakdown, 3 bad diagonal, 4 no memory */
  double rr;
  double bnorm;
} oracle_omp_result;

typedef struct {
  double s, c;
  char pad[48]; /* one cache line per thread */
} partial;

static double dot_omp(int64_t n, const double* x, const double* y, partial* part, int nt) {
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num(), T = omp_get_num_threads();
    const int64_t lo = n * t / T, hi = n * (t + 1) / T;
    double s = 0.0, c = 0.0;
    for (int64_t i = lo; i < hi; ++i) {
      const double v = x[i] * y[i];
      const double u = s + v;
      if (fabs(s) >= fabs(v))
        c += (s - u) + v;
      else
        c += (v - u) + s;
      s = u;
    }
    part[t].s = s;
    part[t].c = c;
    if (t == 0)
      for (int k = T; k < nt; ++k) part[k].s = part[k].c = 0.0;
  }
  double s = 0.0, c = 0.0;
  for (int k = 0; k < nt; ++k) {
    const double v = part[k].s;
    const double u = s + v;
    if (fabs(s) >= fabs(v))
      c += (s - u) + v;
    else
      c += (v - u) + s;
    s = u;
    c += part[k].c;
  }
  return s + c;
}

static void spmv_omp(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                     double* y, int nt) {
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

int oracle_pcg_omp(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* b, double* x,
                   double rtol, double atol, int32_t max_it, int32_t check_every, int32_t nthreads,
                   oracle_omp_result* res) {
  memset(res, 0, sizeof(*res));
  if (check_every < 1) check_every = 1;
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
  const size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double *d = (double*)malloc(sz), *r = (double*)malloc(sz), *z = (double*)malloc(sz), *p = (double*)malloc(sz),
         *w = (double*)malloc(sz);
  partial* part = (partial*)calloc((size_t)nt, sizeof(partial));
  if (!d || !r || !z || !p || !w || !part) {
    free(d); free(r); free(z); free(p); free(w); free(part);
    res->reason = 4;
    return 4;
  }
  int status = 1, bad = 0;
#pragma omp parallel for num_threads(nt) schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < n; ++i) {
    double di = 0.0;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == i) di += val[e];
    d[i] = di;
    if (!(di != 0.0) || !isfinite(di)) bad = 1;
  }
  if (bad) {
    status = 3;
    goto done;
  }
  spmv_omp(n, rowptr, col, val, x, w, nt);
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    r[i] = b[i] - w[i];
    z[i] = r[i] / d[i];
    p[i] = z[i];
  }
  double rho = dot_omp(n, r, z, part, nt);
  const double bn = sqrt(dot_omp(n, b, b, part, nt));
  double rr = dot_omp(n, r, r, part, nt);
  double tol = rtol * bn;
  if (atol > tol) tol = atol;
  res->bnorm = bn;
  res->rr = rr;
  if (!isfinite(rr) || !isfinite(bn)) {
    status = 2;
    goto done;
  }
  if (sqrt(rr) <= tol) {
    status = 0;
    goto done;
  }
  for (int32_t it = 1; it <= max_it; ++it) {
    spmv_omp(n, rowptr, col, val, p, w, nt);
    const double gamma = dot_omp(n, p, w, part, nt);
    if (!(gamma > 0.0) || !isfinite(gamma)) {
      status = 2;
      break;
    }
    const double alpha = rho / gamma;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * w[i];
    rr = dot_omp(n, r, r, part, nt);
    res->iters = it;
    res->rr = rr;
    if (rr == 0.0) {
      status = 0;
      break;
    }
    if ((it % check_every == 0 || it == max_it) && sqrt(rr) <= tol) {
      status = 0;
      break;
    }
    if (it == max_it) {
      status = 1;
      break;
    }
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i) z[i] = r[i] / d[i];
    const double rho_new = dot_omp(n, r, z, part, nt);
    const double beta = rho_new / rho;
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
done:
  res->reason = status;
  free(d); free(r); free(z); free(p); free(w); free(part);
  return status;
}
