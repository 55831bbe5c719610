/*
 * Plain CPU oracle for Jacobi-preconditioned TFQMR.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA library and is deliberately slow and sequential.
 *
 * What it computes
 * ----------------
 * Sec. 4.3 solves the Laplace problems of Sec. 4.1 with the transpose-free
 * quasi-minimal residual method of Freund (1993), Jacobi preconditioned, and
 * notes that an iteration costs two matrix-vector products and about twice
 * the inner products of a CG iteration.  The paper prints no listing; this is
 * Freund's method as usually stated (two half-steps per iteration), applied
 * with the Jacobi preconditioner on the left: the operator is M = D^-1 A and
 * the right-hand side D^-1 b, D = diag(A).  Shadow residual r* = r0.
 *
 *   r0 = D^-1 (b - A x0);  u = w = r* = r0;  v = p = M u;  d = 0
 *   tau = ||r0||;  theta = eta = 0;  rho = (r*, r0);  bn = ||D^-1 b||
 *   breakdown if tau or bn is not finite; stop (converged) if tau <= tol = max(rtol * bn, atol)
 *   iteration i = 1, 2, ...:
 *     sigma = (v, r*);  sigma == 0 or not finite -> breakdown
 *     alpha = rho / sigma
 *     half-step m = 2i-1 ("odd"):      u2 = u - alpha v;  w -= alpha p
 *                                      d = u + (theta^2 eta / alpha) d
 *     half-step m = 2i   ("even"):     q = M u2;  w -= alpha q
 *                                      d = u2 + (theta^2 eta / alpha) d
 *       after each half-step:  theta = ||w|| / tau;  c = 1 / sqrt(1 + theta^2)
 *                              tau = tau theta c;  eta = c^2 alpha;  x += eta d
 *       a quasi-residual of exactly zero (tau = 0) stops at once: x is exact
 *     test (when i % k == 0 or i == max_it): converged if sqrt(2i + 1) tau <= tol
 *       (Freund's bound ||r_m|| <= sqrt(m + 1) tau_m on the true residual of
 *       the preconditioned system after m half-steps)
 *     stop (not converged) if i == max_it
 *     rho' = (w, r*);  rho == 0 or rho' not finite -> breakdown
 *     beta = rho' / rho;  rho = rho'
 *     u = w + beta u2;  p = M u;  v = p + beta (q + beta v)
 *
 * (p = M u is kept for the next odd half-step; v is the direction that
 * defines alpha and is not M u.)
 *
 * Inner products and norms use the compensated dot of pcg_oracle.c.  The
 * ``mutation`` argument plants one mistake (0 = none) for the pin tests:
 * 1 drops the eta d update of the even half-step, 2 flips the sign of beta,
 * 3 uses theta instead of theta^2 in the d recurrence, 4 omits the Jacobi
 * scaling of q.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

double oracle_dot(int64_t n, const double* x, const double* y);
void oracle_spmv(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* x,
                 double* y);
int oracle_diagonal(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, double* d);

enum { TQ_CONVERGED = 0, TQ_NOT_CONVERGED = 1, TQ_BREAKDOWN = 2, TQ_BAD_DIAGONAL = 3, TQ_NO_MEMORY = 4 };

typedef struct {
  int32_t iters;   /* completed iterations (two half-steps each) */
  int32_t reason;  /* TQ_* */
  double tau;      /* quasi-residual norm at exit */
  double bound;    /* sqrt(2 iters + 1) tau: bound on ||D^-1 (b - A x)|| */
  double bnorm;    /* ||D^-1 b|| */
} oracle_tfqmr_result;

/* y = D^-1 (A x) with D given as its diagonal d. */
static void apply_m(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* d,
                    const double* x, double* y) {
  oracle_spmv(n, rowptr, col, val, x, y);
  for (int64_t i = 0; i < n; ++i) y[i] = y[i] / d[i];
}

/* Quasi-residual update after a half-step; returns 0 if theta is not finite. */
static int half_step_end(int64_t n, const double* w, double alpha, double* theta, double* tau, double* eta,
                         double* x, const double* dv, int skip_x) {
  const double wn = sqrt(oracle_dot(n, w, w));
  *theta = wn / *tau;
  const double c = 1.0 / sqrt(1.0 + (*theta) * (*theta));
  *tau = (*tau) * (*theta) * c;
  *eta = c * c * alpha;
  if (!isfinite(*theta) || !isfinite(*tau)) return 0; /* breakdown: x keeps the last finite iterate */
  if (!skip_x)
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + (*eta) * dv[i];
  return 1;
}

/*
 * Solve A x = b (x holds x0 on entry).  Histories (may be NULL) receive alpha,
 * beta and tau (after the even half-step) of the first hist_len iterations.
 */
int oracle_tfqmr(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* b, double* x,
                 double rtol, double atol, int32_t max_it, int32_t check_every, int32_t hist_len, double* alpha_h,
                 double* beta_h, double* tau_h, int32_t mutation, oracle_tfqmr_result* res) {
  memset(res, 0, sizeof(*res));
  if (check_every < 1) check_every = 1;
  if (max_it <= 0) max_it = n > 0 ? (int32_t)(10 * n) : 10;
  double* buf = (double*)calloc((size_t)(n > 0 ? n : 1) * 11, sizeof(double));
  if (!buf) {
    res->reason = TQ_NO_MEMORY;
    return TQ_NO_MEMORY;
  }
  const int64_t N = n > 0 ? n : 1;
  double *dg = buf, *r = buf + N, *u = buf + 2 * N, *u2 = buf + 3 * N, *w = buf + 4 * N, *rs = buf + 5 * N;
  double *v = buf + 6 * N, *q = buf + 7 * N, *dv = buf + 8 * N, *bh = buf + 9 * N, *pu = buf + 10 * N;
  if (oracle_diagonal(n, rowptr, col, val, dg) != 0) {
    free(buf);
    res->reason = TQ_BAD_DIAGONAL;
    return TQ_BAD_DIAGONAL;
  }
  /* r0 = D^-1 (b - A x0) */
  oracle_spmv(n, rowptr, col, val, x, r);
  for (int64_t i = 0; i < n; ++i) {
    r[i] = (b[i] - r[i]) / dg[i];
    bh[i] = b[i] / dg[i];
    u[i] = w[i] = rs[i] = r[i];
    dv[i] = 0.0;
  }
  apply_m(n, rowptr, col, val, dg, u, pu);
  for (int64_t i = 0; i < n; ++i) v[i] = pu[i];
  double tau = sqrt(oracle_dot(n, r, r));
  double theta = 0.0, eta = 0.0;
  double rho = oracle_dot(n, rs, r);
  const double bn = sqrt(oracle_dot(n, bh, bh));
  const double tol = fmax(rtol * bn, atol);
  res->bnorm = bn;
  int reason = TQ_NOT_CONVERGED;
  int32_t it = 0;
  if (!isfinite(tau) || !isfinite(bn)) { /* a non-finite b or x0 */
    reason = TQ_BREAKDOWN;
  } else if (tau <= tol) {
    reason = TQ_CONVERGED;
  } else {
    for (it = 1;; ++it) {
      const double sigma = oracle_dot(n, v, rs);
      if (sigma == 0.0 || !isfinite(sigma)) {
        reason = TQ_BREAKDOWN;
        it -= 1;
        break;
      }
      const double alpha = rho / sigma;
      if (it <= hist_len && alpha_h) alpha_h[it - 1] = alpha;
      /* odd half-step */
      const double co = (mutation == 3 ? theta : theta * theta) * eta / alpha;
      for (int64_t i = 0; i < n; ++i) {
        u2[i] = u[i] - alpha * v[i];
        w[i] = w[i] - alpha * pu[i];
        dv[i] = u[i] + co * dv[i];
      }
      if (!half_step_end(n, w, alpha, &theta, &tau, &eta, x, dv, 0)) {
        reason = TQ_BREAKDOWN;
        break;
      }
      if (tau == 0.0) {
        reason = TQ_CONVERGED;
        break;
      }
      /* even half-step */
      if (mutation == 4)
        oracle_spmv(n, rowptr, col, val, u2, q);
      else
        apply_m(n, rowptr, col, val, dg, u2, q);
      const double ce = (mutation == 3 ? theta : theta * theta) * eta / alpha;
      for (int64_t i = 0; i < n; ++i) {
        w[i] = w[i] - alpha * q[i];
        dv[i] = u2[i] + ce * dv[i];
      }
      if (!half_step_end(n, w, alpha, &theta, &tau, &eta, x, dv, mutation == 1)) {
        reason = TQ_BREAKDOWN;
        break;
      }
      if (it <= hist_len && tau_h) tau_h[it - 1] = tau;
      if (tau == 0.0 || ((it % check_every == 0 || it == max_it) && sqrt(2.0 * it + 1.0) * tau <= tol)) {
        reason = TQ_CONVERGED;
        break;
      }
      if (it == max_it) {
        reason = TQ_NOT_CONVERGED;
        break;
      }
      const double rho_new = oracle_dot(n, w, rs);
      if (rho == 0.0 || !isfinite(rho_new)) {
        reason = TQ_BREAKDOWN;
        break;
      }
      double beta = rho_new / rho;
      if (mutation == 2) beta = -beta;
      if (it <= hist_len && beta_h) beta_h[it - 1] = beta;
      rho = rho_new;
      for (int64_t i = 0; i < n; ++i) {
        u[i] = w[i] + beta * u2[i];
        q[i] = q[i] + beta * v[i]; /* q + beta v, reusing q */
      }
      apply_m(n, rowptr, col, val, dg, u, pu);
      for (int64_t i = 0; i < n; ++i) v[i] = pu[i] + beta * q[i];
    }
  }
  res->iters = it;
  res->reason = reason;
  res->tau = tau;
  res->bound = sqrt(2.0 * it + 1.0) * tau;
  free(buf);
  return reason;
}
