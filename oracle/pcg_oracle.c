/*
 * Plain CPU oracle for the Jacobi-preconditioned conjugate-gradient path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA library (no header, no helper, no table) and is deliberately slow and
 * sequential so that a reader can check it against the paper by eye.
 *
 * What it computes
 * ----------------
 * Sec. 4.2 runs textbook Hestenes-Stiefel CG with Jacobi (diagonal scaling)
 * preconditioning (Sec. 4.1).  The loop body follows the order of the mixed
 * sync/async main-loop example of Sec. 3.3 (w = Ap, a = p'w, a = beta/a,
 * x += a p, r -= a w, z = B r, convergence test, beta = z'r, p = z + b p);
 * the initialisation, which the paper omits, is the standard one:
 *
 *   r = b - A x0;  z = r ./ d;  rho = (r,z);  p = z;  bn = ||b||
 *   iteration i = 1, 2, ...:
 *     w = A p;  gamma = (p,w);  gamma <= 0 or not finite -> breakdown
 *     alpha = rho / gamma
 *     x += alpha p;  r -= alpha w;  rr = (r,r)
 *     stop (converged) if rr == 0, or if i % k == 0 (or i == max_it)
 *       and sqrt(rr) <= max(rtol * bn, atol)
 *     stop (not converged) if i == max_it
 *     z = r ./ d;  rho_new = (r,z);  beta = rho_new / rho
 *     p = z + beta p;  rho = rho_new
 *
 * The test "sqrt(rr) <= tol" is also applied once before the loop (i = 0),
 * after a check that rr and bn are finite (a NaN or infinity in b or x0 is a
 * breakdown, not convergence against an infinite tolerance).
 * Every inner product uses Neumaier-compensated summation in the working
 * precision, so the oracle is at least as accurate as any GPU reduction tree.
 *
 * The float variant runs the same steps entirely in float (float matrix
 * values, float vectors, float compensated sums).  The iterative-refinement
 * driver wraps it: r = b - A x in double, ||r|| test, inner float PCG on
 * A32 d = r, x += d (double).
 *
 * The ``mutation`` argument plants one deliberate mistake (0 = none); the
 * pin tests use it to show that each pin catches the error it targets.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  OR_CONVERGED = 0,
  OR_NOT_CONVERGED = 1,
  OR_BREAKDOWN = 2,
  OR_BAD_DIAGONAL = 3,
  OR_NO_MEMORY = 4
};

/* Neumaier-compensated inner product in double. */
double oracle_dot(int64_t n, const double* x, const double* y) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = x[i] * y[i];
    double u = s + t;
    if (fabs(s) >= fabs(t))
      c += (s - u) + t;
    else
      c += (t - u) + s;
    s = u;
  }
  return s + c;
}

/* Neumaier-compensated sum of a vector in double. */
double oracle_sum(int64_t n, const double* x) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = x[i];
    double u = s + t;
    if (fabs(s) >= fabs(t))
      c += (s - u) + t;
    else
      c += (t - u) + s;
    s = u;
  }
  return s + c;
}

static float dot_f32(int64_t n, const float* x, const float* y) {
  float s = 0.0f, c = 0.0f;
  for (int64_t i = 0; i < n; ++i) {
    float t = x[i] * y[i];
    float u = s + t;
    if (fabsf(s) >= fabsf(t))
      c += (s - u) + t;
    else
      c += (t - u) + s;
    s = u;
  }
  return s + c;
}

/* y = A x, row by row, terms in column order. */
void oracle_spmv(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                 double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

/* y = A x with float values and vectors, float accumulation. */
void oracle_spmv_f32(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val, const float* x,
                     float* y) {
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

/* d[i] = A(i,i); returns 0 if every diagonal entry is present and nonzero. */
int oracle_diagonal(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, double* d) {
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == i) d[i] += val[e];
    if (!(d[i] != 0.0) || !isfinite(d[i])) bad = 1;
  }
  return bad;
}

typedef struct {
  int32_t iters;      /* completed iterations (x updates) */
  int32_t reason;     /* OR_* */
  double rr;          /* final (r,r) of the recursively updated residual */
  double bnorm;       /* ||b|| */
} oracle_result;

/*
 * Jacobi-PCG in double.  x holds x0 on entry and the iterate on exit.
 * Histories (length hist_len, entry i-1 for iteration i; may be NULL):
 * alpha, beta (computed at the end of iteration i), gamma = (p,Ap), rho = (r,z)
 * before iteration i, rr = (r,r) after iteration i.
 */
int oracle_pcg(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* b, double* x,
               double rtol, double atol, int32_t max_it, int32_t check_every, int32_t hist_len, double* alpha_h,
               double* beta_h, double* gamma_h, double* rho_h, double* rr_h, int32_t mutation, oracle_result* res) {
  memset(res, 0, sizeof(*res));
  if (check_every < 1) check_every = 1;
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!d || !r || !z || !p || !w) {
    free(d); free(r); free(z); free(p); free(w);
    res->reason = OR_NO_MEMORY;
    return OR_NO_MEMORY;
  }
  int status = OR_NOT_CONVERGED;
  if (oracle_diagonal(n, rowptr, col, val, d)) {
    status = OR_BAD_DIAGONAL;
    goto done;
  }
  /* r = b - A x0 */
  oracle_spmv(n, rowptr, col, val, x, w);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
  for (int64_t i = 0; i < n; ++i) z[i] = (mutation == 3) ? r[i] : r[i] / d[i];
  double rho = oracle_dot(n, r, z);
  for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  double bn = sqrt(oracle_dot(n, b, b));
  double rr = oracle_dot(n, r, r);
  double tol = rtol * bn;
  if (atol > tol) tol = atol;
  res->bnorm = bn;
  res->rr = rr;
  if (!isfinite(rr) || !isfinite(bn)) { /* a non-finite b or x0: the tolerance would be meaningless */
    status = OR_BREAKDOWN;
    goto done;
  }
  if (sqrt(rr) <= tol) {
    status = OR_CONVERGED;
    goto done;
  }
  for (int32_t it = 1; it <= max_it; ++it) {
    if (mutation == 5)
      oracle_spmv(n, rowptr, col, val, z, w); /* wrong operand */
    else
      oracle_spmv(n, rowptr, col, val, p, w);
    double gamma = oracle_dot(n, p, w);
    if (it <= hist_len) {
      if (gamma_h) gamma_h[it - 1] = gamma;
      if (rho_h) rho_h[it - 1] = rho;
    }
    if (!(gamma > 0.0) || !isfinite(gamma)) {
      status = OR_BREAKDOWN;
      break;
    }
    double alpha = rho / gamma;
    if (mutation == 4) alpha = gamma / rho;
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
    if (mutation == 1)
      for (int64_t i = 0; i < n; ++i) r[i] += alpha * w[i];
    else
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * w[i];
    rr = oracle_dot(n, r, r);
    res->iters = it;
    res->rr = rr;
    if (it <= hist_len) {
      if (alpha_h) alpha_h[it - 1] = alpha;
      if (rr_h) rr_h[it - 1] = rr;
    }
    if (rr == 0.0) {
      status = OR_CONVERGED;
      break;
    }
    if ((it % check_every == 0 || it == max_it) && sqrt(rr) <= tol) {
      status = OR_CONVERGED;
      break;
    }
    if (it == max_it) {
      status = OR_NOT_CONVERGED;
      break;
    }
    for (int64_t i = 0; i < n; ++i) z[i] = (mutation == 3) ? r[i] : r[i] / d[i];
    double rho_new = oracle_dot(n, r, z);
    double beta = (mutation == 2) ? rho / rho_new : rho_new / rho;
    if (it <= hist_len && beta_h) beta_h[it - 1] = beta;
    if (mutation == 6)
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] - beta * p[i];
    else
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
done:
  res->reason = status;
  free(d); free(r); free(z); free(p); free(w);
  return status;
}

/* Inner product of float vectors with the products and the sum in double,
 * rounded to float once at the end: a planted mistake (mutation 1 of the float
 * solver), never the method. */
static float dot_f32_in_double(int64_t n, const float* x, const float* y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += (double)x[i] * (double)y[i];
  return (float)s;
}

/*
 * Jacobi-PCG entirely in float: float values val32, float vectors, float
 * compensated sums.  Solves A32 xf = bf; xf holds the start on entry.
 * The stop test is sqrt(rr) <= rtol * ||bf|| (every check_every iterations).
 * Histories as in oracle_pcg (length hist_len, may be NULL; the float values
 * widened to double): alpha and beta of iteration i, rho = (r,z) before
 * iteration i (rho_h[0] is the initial (r0, z0)).
 * Planted mistakes (mutation): 1 dots accumulated in double, 2 Jacobi step
 * dropped (z = r), 3 beta inverted, 4 wrong sign in p = z + beta p.
 */
int oracle_pcg_f32(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val, const float* bf, float* xf,
                   float rtol, int32_t max_it, int32_t check_every, int32_t hist_len, double* alpha_h, double* beta_h,
                   double* rho_h, int32_t mutation, oracle_result* res) {
  memset(res, 0, sizeof(*res));
  if (check_every < 1) check_every = 1;
  size_t sz = sizeof(float) * (size_t)(n > 0 ? n : 1);
  float *d = (float*)malloc(sz), *r = (float*)malloc(sz), *z = (float*)malloc(sz), *p = (float*)malloc(sz),
        *w = (float*)malloc(sz);
  if (!d || !r || !z || !p || !w) {
    free(d); free(r); free(z); free(p); free(w);
    res->reason = OR_NO_MEMORY;
    return OR_NO_MEMORY;
  }
  int status = OR_NOT_CONVERGED;
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0f;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == i) d[i] += val[e];
    if (!(d[i] != 0.0f)) status = OR_BAD_DIAGONAL;
  }
  if (status == OR_BAD_DIAGONAL) goto done;
  float (*dotf)(int64_t, const float*, const float*) = (mutation == 1) ? dot_f32_in_double : dot_f32;
  oracle_spmv_f32(n, rowptr, col, val, xf, w);
  for (int64_t i = 0; i < n; ++i) r[i] = bf[i] - w[i];
  for (int64_t i = 0; i < n; ++i) z[i] = (mutation == 2) ? r[i] : r[i] / d[i];
  float rho = dotf(n, r, z);
  for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  float bn = sqrtf(dotf(n, bf, bf));
  float rr = dotf(n, r, r);
  float tol = rtol * bn;
  res->bnorm = bn;
  res->rr = rr;
  if (sqrtf(rr) <= tol) {
    status = OR_CONVERGED;
    goto done;
  }
  for (int32_t it = 1; it <= max_it; ++it) {
    oracle_spmv_f32(n, rowptr, col, val, p, w);
    float gamma = dotf(n, p, w);
    if (it <= hist_len && rho_h) rho_h[it - 1] = (double)rho;
    if (!(gamma > 0.0f) || !isfinite(gamma)) {
      status = OR_BREAKDOWN;
      break;
    }
    float alpha = rho / gamma;
    if (it <= hist_len && alpha_h) alpha_h[it - 1] = (double)alpha;
    for (int64_t i = 0; i < n; ++i) xf[i] += alpha * p[i];
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * w[i];
    rr = dotf(n, r, r);
    res->iters = it;
    res->rr = rr;
    if (rr == 0.0f) {
      status = OR_CONVERGED;
      break;
    }
    if ((it % check_every == 0 || it == max_it) && sqrtf(rr) <= tol) {
      status = OR_CONVERGED;
      break;
    }
    if (it == max_it) {
      status = OR_NOT_CONVERGED;
      break;
    }
    for (int64_t i = 0; i < n; ++i) z[i] = (mutation == 2) ? r[i] : r[i] / d[i];
    float rho_new = dotf(n, r, z);
    float beta = (mutation == 3) ? rho / rho_new : rho_new / rho;
    if (it <= hist_len && beta_h) beta_h[it - 1] = (double)beta;
    if (mutation == 4)
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] - beta * p[i];
    else
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
done:
  res->reason = status;
  free(d); free(r); free(z); free(p); free(w);
  return status;
}

typedef struct {
  int32_t outer;        /* corrections applied */
  int32_t inner_total;  /* inner iterations summed over corrections */
  int32_t reason;       /* OR_* */
  int32_t pad;
  double rel_res;       /* ||b - A x|| / ||b|| at exit, true residual in double */
} oracle_ir_result;

/*
 * Mixed-precision iterative refinement: outer loop in double on A64, inner
 * Jacobi-PCG in float on A32 (same pattern) with relative tolerance
 * rtol_inner on the inner right-hand side and at most max_inner iterations.
 */
int oracle_ir(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val64, const float* val32,
              const double* b, double* x, double rtol, int32_t max_outer, float rtol_inner, int32_t max_inner,
              int32_t inner_check_every, oracle_ir_result* res) {
  memset(res, 0, sizeof(*res));
  size_t sz = (size_t)(n > 0 ? n : 1);
  double* r = (double*)malloc(sizeof(double) * sz);
  float* rf = (float*)malloc(sizeof(float) * sz);
  float* df = (float*)malloc(sizeof(float) * sz);
  if (!r || !rf || !df) {
    free(r); free(rf); free(df);
    res->reason = OR_NO_MEMORY;
    return OR_NO_MEMORY;
  }
  double bn = sqrt(oracle_dot(n, b, b));
  int status = OR_NOT_CONVERGED;
  for (int32_t k = 0;; ++k) {
    oracle_spmv(n, rowptr, col, val64, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double rn = sqrt(oracle_dot(n, r, r));
    res->rel_res = bn > 0.0 ? rn / bn : rn;
    if (!isfinite(rn) || !isfinite(bn)) {
      status = OR_BREAKDOWN;
      break;
    }
    if (rn <= rtol * bn) {
      status = OR_CONVERGED;
      break;
    }
    if (k == max_outer) break;
    for (int64_t i = 0; i < n; ++i) {
      rf[i] = (float)r[i];
      df[i] = 0.0f;
    }
    oracle_result ir;
    int st = oracle_pcg_f32(n, rowptr, col, val32, rf, df, rtol_inner, max_inner, inner_check_every, 0, NULL, NULL,
                            NULL, 0, &ir);
    res->inner_total += ir.iters;
    if (st == OR_BAD_DIAGONAL || st == OR_NO_MEMORY) {
      status = st;
      break;
    }
    if (st == OR_BREAKDOWN && ir.iters == 0) {
      status = OR_BREAKDOWN;
      break;
    }
    for (int64_t i = 0; i < n; ++i) x[i] += (double)df[i];
    res->outer = k + 1;
  }
  res->reason = status;
  free(r); free(rf); free(df);
  return status;
}
