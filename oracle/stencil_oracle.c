/*
 * Plain CPU oracle for the matrix-free stencil operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA library.
 *
 * What it computes
 * ----------------
 * The Laplace problems of Sec. 4.1 are finite-difference stencils on a
 * structured grid; the paper's JAX comparison (Sec. 4.4) applies the operator
 * as a convolution instead of an assembled matrix.  A constant-coefficient
 * stencil on an nx x ny x nz grid (x fastest, then y, then z) with terms
 * (dx_k, dy_k, dz_k, w_k) maps x to
 *
 *   y[i] = sum over k of w_k * x[i + dx_k + nx (dy_k + ny dz_k)]
 *
 * where a term whose neighbour (ix + dx_k, iy + dy_k, iz + dz_k) lies outside
 * the grid is dropped (Dirichlet boundary by elimination, as in the assembled
 * stencil matrices).  Terms are added in the order given, each product
 * rounded before the sum (gcc -ffp-contract=off).
 *
 * ``mutation`` plants one mistake for the pin tests: 1 wraps neighbours
 * around the x boundary (periodic) instead of dropping them, 2 swaps the
 * roles of dx and dy.
 */
#include <stdint.h>

void oracle_stencil_apply(int32_t nx, int32_t ny, int32_t nz, int32_t npts, const int32_t* offsets,
                          const double* weights, const double* x, double* y, int32_t mutation) {
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / ((int64_t)nx * ny);
    double s = 0.0;
    for (int32_t k = 0; k < npts; ++k) {
      int64_t dx = offsets[3 * k], dy = offsets[3 * k + 1];
      const int64_t dz = offsets[3 * k + 2];
      if (mutation == 2) {
        const int64_t t = dx;
        dx = dy;
        dy = t;
      }
      int64_t jx = ix + dx;
      const int64_t jy = iy + dy, jz = iz + dz;
      if (mutation == 1) jx = (jx + nx) % nx;
      if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
      const int64_t j = jx + (int64_t)nx * (jy + (int64_t)ny * jz);
      s = s + weights[k] * x[j];
    }
    y[i] = s;
  }
}
