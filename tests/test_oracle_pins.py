"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every check here uses something independent of the oracle's code: a textbook
library routine (dense Cholesky, symmetric eigensolver, exactly rounded
summation, scipy's sparse product), a closed form (Laplacian spectra, the CG
condition-number bound), or an invariant that Jacobi-PCG must satisfy
(D^-1-orthogonal residuals, A-conjugate steps, the Lanczos connection between
the CG coefficients and the spectrum of D^-1 A).  The last test plants a
mistake in the oracle (its ``mutation`` switch) and shows that at least one
pin fails for each; the float32 solver has its own pins (IEEE float32 rounding of a
worked example, the float32 summation bound of the product, the refinement's
contraction bound) and planted mistakes.
"""

import math

import numpy as np
import pytest
import scipy.linalg as sla

from synthetic import (
    diagonal_csr,
    laplace_2d_5pt,
    laplace_3d_7pt,
    random_spd_csr,
    rhs_from_solution,
    sine_mode_2d,
    sine_mode_3d,
    single_problem,
    aniso_3d_7pt_fp32exact,
    diffusion_3d_27pt,
)
from synthetic.stencils import CSR


# --------------------------------------------------------------------------- helpers


def lap_eig_1d(N, j):
    """Eigenvalue of the 1-D Dirichlet second difference [-1 2 -1] for sine mode j."""
    return 4.0 * math.sin(j * math.pi / (2 * (N + 1))) ** 2


def cg_bound(kappa, rtol):
    """Iterations after which ||r_k||/||r_0|| <= rtol is guaranteed (exact arithmetic).

    From ||e_k||_A <= 2 q^k ||e_0||_A, q = (sqrt k - 1)/(sqrt k + 1), and
    ||r||_2 / ||r_0||_2 <= sqrt(kappa) ||e||_A / ||e_0||_A, with
    ln(1/q) >= 2/sqrt(kappa).
    """
    s = math.sqrt(kappa)
    return math.ceil(0.5 * s * math.log(2.0 * s / rtol))


def _nonsym_csr(n, density, rng):
    import scipy.sparse as sp

    m = sp.random(n, n, density=density, random_state=rng, format="csr")
    m.data = rng.uniform(-2, 2, m.data.shape[0])
    m.sort_indices()
    return CSR(m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64))


# --------------------------------------------------------------------------- building blocks


def test_spmv_matches_scipy_on_nonsymmetric(orc):
    rng = np.random.default_rng(11)
    for n in (1, 7, 130):
        A = _nonsym_csr(n, 0.2, rng)
        x = rng.standard_normal(n)
        y = orc.spmv(A, x)
        ref = A.to_scipy() @ x
        assert np.allclose(y, ref, rtol=1e-14, atol=1e-14)


def test_dot_is_compensated(orc):
    # exactly rounded reference: math.fsum of exactly representable products
    rng = np.random.default_rng(3)
    x = np.concatenate([[1e16, 1.0, -1e16], rng.standard_normal(1000) * 1e8, [3.0, -rng.standard_normal(1000).sum()]])
    y = np.ones_like(x)
    exact = math.fsum(x.tolist())
    got = orc.dot(x, y)
    assert abs(got - exact) <= 4 * np.finfo(float).eps * max(abs(exact), 1.0)
    # the naive left-to-right sum loses the +1
    assert orc.dot(np.array([1e16, 1.0, -1e16]), np.ones(3)) == 1.0


def test_diagonal_detects_missing_entry(orc):
    A = CSR(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([2.0, 1.0]))
    d, bad = orc.diagonal(A)
    assert bad and d[0] == 2.0 and d[1] == 0.0
    res = orc.pcg(A, np.ones(2))
    assert res["reason"] == "bad_diagonal"


# --------------------------------------------------------------------------- solution pins


@pytest.mark.parametrize("seed,n", [(0, 5), (1, 40), (2, 150), (3, 200)])
def test_pcg_matches_dense_cholesky_random_spd(orc, seed, n):
    rng = np.random.default_rng(seed)
    A = random_spd_csr(n, 0.08, rng, dominance=0.3)
    b = rng.standard_normal(n)
    Ad = A.to_dense()
    xc = sla.cho_solve(sla.cho_factor(Ad), b)
    kappa = np.linalg.cond(Ad)
    res = orc.pcg(A, b, rtol=1e-14, max_it=10 * n)
    assert res["reason"] == "converged"
    err = np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc)
    assert err <= max(kappa, 10.0) * 1e-13
    assert res["iters"] <= n + 5  # finite termination, up to rounding


@pytest.mark.parametrize("N", [3, 8, 14])
def test_pcg_matches_dense_cholesky_laplacians(orc, N):
    rng = np.random.default_rng(N)
    for A in (laplace_2d_5pt(N), laplace_3d_7pt(min(N, 8)), laplace_2d_5pt(N, shift=0.37)):
        xt = rng.uniform(-1, 1, A.n)
        b = rhs_from_solution(A, xt)
        xc = sla.cho_solve(sla.cho_factor(A.to_dense()), b)
        res = orc.pcg(A, b, rtol=1e-13)
        assert res["reason"] == "converged"
        assert np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc) < 1e-10


def test_closed_form_laplacian_spectrum_matches_eigensolver():
    for N in (4, 9):
        A = laplace_2d_5pt(N).to_dense()
        ev = np.sort(np.linalg.eigvalsh(A))
        cf = np.sort([lap_eig_1d(N, i) + lap_eig_1d(N, j) for i in range(1, N + 1) for j in range(1, N + 1)])
        assert np.allclose(ev, cf, atol=1e-12)
        A3 = laplace_3d_7pt(N).to_dense()
        ev3 = np.sort(np.linalg.eigvalsh(A3))
        cf3 = np.sort(
            [lap_eig_1d(N, i) + lap_eig_1d(N, j) + lap_eig_1d(N, k) for i in range(1, N + 1) for j in range(1, N + 1) for k in range(1, N + 1)]
        )
        assert np.allclose(ev3, cf3, atol=1e-12)
    # kappa = cot^2(pi / (2(N+1))) for both the 2-D and 3-D operators
    assert abs(1.0 / math.tan(math.pi / 130) ** 2 - 1711.66) < 0.01
    assert abs(1.0 / math.tan(math.pi / 258) ** 2 - 6743.68) < 0.01


@pytest.mark.parametrize("dim,N", [(2, 64), (3, 24)])
def test_iterations_within_condition_number_bound(orc, dim, N):
    p = single_problem("c1" if dim == 2 else "c2", seed=0, size=N)
    kappa = 1.0 / math.tan(math.pi / (2 * (N + 1))) ** 2
    bound = cg_bound(kappa, 1e-8)
    res = orc.pcg(p.A, p.b, rtol=1e-8)
    assert res["reason"] == "converged"
    assert res["iters"] <= bound
    if dim == 2 and N == 64:
        assert bound == 473
        assert np.linalg.norm(res["x"] - p.x_true) / np.linalg.norm(p.x_true) < 1e-6


@pytest.mark.parametrize("dim,N,modes", [(2, 64, [(1, 1)]), (2, 64, [(3, 7)]), (3, 20, [(2, 5, 9)])])
def test_eigenvector_rhs_converges_in_one_iteration(orc, dim, N, modes):
    A = laplace_2d_5pt(N) if dim == 2 else laplace_3d_7pt(N)
    d = 4.0 if dim == 2 else 6.0
    (j,) = modes
    v = sine_mode_2d(N, *j) if dim == 2 else sine_mode_3d(N, *j)
    lam = sum(lap_eig_1d(N, jj) for jj in j)
    res = orc.pcg(A, v, rtol=1e-10, hist_len=2)
    assert res["iters"] == 1 and res["reason"] == "converged"
    assert abs(res["alpha"][0] - d / lam) <= 1e-12 * (d / lam)
    assert np.allclose(res["x"], v / lam, rtol=0, atol=1e-12 * np.abs(v / lam).max())


def test_sum_of_m_modes_collapses_at_iteration_m(orc):
    N = 32
    A = laplace_2d_5pt(N)
    modes = [(1, 1), (2, 3), (5, 5), (9, 2), (14, 20)]
    lams = [lap_eig_1d(N, a) + lap_eig_1d(N, b) for a, b in modes]
    assert len(set(np.round(lams, 12))) == len(modes)
    b = sum((k + 1) * sine_mode_2d(N, *m) for k, m in enumerate(modes))
    res = orc.pcg(A, b, rtol=0.0, max_it=len(modes), hist_len=len(modes))
    rr0 = float(b @ b)
    assert res["rr"] / rr0 < 1e-16  # rounding, amplified by the spread of the 5 eigenvalues
    hist = res["rr_hist"]
    assert hist[len(modes) - 2] / rr0 > 1e-4  # not collapsed one step early
    x_exact = sum((k + 1) * sine_mode_2d(N, *m) / lam for k, (m, lam) in enumerate(zip(modes, lams)))
    assert np.allclose(res["x"], x_exact, atol=1e-8)


def test_diagonal_matrix_is_exact_in_one_iteration(orc):
    rng = np.random.default_rng(5)
    d = rng.uniform(0.5, 50.0, 300)
    b = rng.standard_normal(300)
    res = orc.pcg(diagonal_csr(d), b, rtol=1e-12)
    assert res["iters"] == 1 and res["reason"] == "converged"
    assert np.allclose(res["x"], b / d, rtol=1e-15, atol=0)


def test_zero_rhs_converges_at_iteration_zero(orc):
    A = laplace_2d_5pt(6)
    res = orc.pcg(A, np.zeros(A.n), rtol=1e-8)
    assert res["iters"] == 0 and res["reason"] == "converged" and not res["x"].any()


def test_nonzero_initial_guess(orc):
    rng = np.random.default_rng(8)
    A = random_spd_csr(60, 0.1, rng)
    b = rng.standard_normal(60)
    x0 = rng.standard_normal(60)
    xc = sla.cho_solve(sla.cho_factor(A.to_dense()), b)
    res = orc.pcg(A, b, x0=x0, rtol=1e-13)
    assert np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc) < 1e-10


def test_indefinite_matrix_breaks_down(orc):
    A = CSR(np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 3.0, 3.0, 1.0]))
    res = orc.pcg(A, np.array([1.0, 0.0]), rtol=1e-12)
    assert res["reason"] == "breakdown"


def test_max_it_and_check_cadence(orc):
    p = single_problem("c1", seed=0, size=32)
    r1 = orc.pcg(p.A, p.b, rtol=1e-8, check_every=1)
    r10 = orc.pcg(p.A, p.b, rtol=1e-8, check_every=10)
    assert r10["iters"] % 10 == 0 and r1["iters"] <= r10["iters"] < r1["iters"] + 10
    r20 = orc.pcg(p.A, p.b, rtol=0.0, max_it=20)
    assert r20["iters"] == 20 and r20["reason"] == "not_converged"


# --------------------------------------------------------------------------- invariants of the iterates


def _iterates(orc, A, b, m):
    """x_1..x_m from the oracle by re-running with max_it = j (rtol = 0)."""
    return [orc.pcg(A, b, rtol=0.0, max_it=j)["x"] for j in range(0, m + 1)]


@pytest.mark.parametrize("seed", [0, 1])
def test_residuals_d_orthogonal_and_steps_a_conjugate(orc, seed):
    rng = np.random.default_rng(100 + seed)
    n = 40
    A = random_spd_csr(n, 0.15, rng, dominance=0.5)
    Ad = A.to_dense()
    dinv = 1.0 / np.diag(Ad)
    b = rng.standard_normal(n)
    xs = _iterates(orc, A, b, 6)
    rs = [b - Ad @ x for x in xs]
    steps = [xs[j + 1] - xs[j] for j in range(6)]
    for i in range(6):
        for j in range(i + 1, 6):
            num = rs[i] @ (dinv * rs[j])
            den = math.sqrt((rs[i] @ (dinv * rs[i])) * (rs[j] @ (dinv * rs[j])))
            assert abs(num) / den < 1e-10
            num = steps[i] @ Ad @ steps[j]
            den = math.sqrt((steps[i] @ Ad @ steps[i]) * (steps[j] @ Ad @ steps[j]))
            assert abs(num) / den < 1e-10


def _lanczos_T(alpha, beta):
    k = len(alpha)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alpha[j] + (beta[j - 1] / alpha[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(beta[j]) / alpha[j]
    return T


def test_cg_coefficients_reproduce_preconditioned_spectrum(orc):
    """After n steps the Lanczos matrix built from (alpha, beta) has the spectrum of D^-1 A."""
    rng = np.random.default_rng(7)
    n = 8
    A = random_spd_csr(n, 0.5, rng, dominance=0.2)
    Ad = A.to_dense()
    s = 1.0 / np.sqrt(np.diag(Ad))
    ev = np.sort(np.linalg.eigvalsh(s[:, None] * Ad * s[None, :]))
    b = rng.standard_normal(n)
    res = orc.pcg(A, b, rtol=0.0, max_it=n, hist_len=n)
    T = _lanczos_T(res["alpha"], res["beta"][: n - 1])
    rv = np.sort(np.linalg.eigvalsh(T))
    assert np.allclose(rv, ev, rtol=1e-9, atol=1e-12)


def test_ritz_values_inside_laplacian_spectrum(orc):
    N = 64
    p = single_problem("c1", seed=0)
    res = orc.pcg(p.A, p.b, rtol=0.0, max_it=60, hist_len=60)
    T = _lanczos_T(res["alpha"], res["beta"][:59])
    rv = np.linalg.eigvalsh(T)
    # D = 4 I: spectrum of D^-1 A is lambda/4
    lo = 2 * lap_eig_1d(N, 1) / 4.0
    hi = 2 * lap_eig_1d(N, N) / 4.0
    assert rv.min() >= lo * (1 - 1e-9) and rv.max() <= hi * (1 + 1e-9)
    assert abs(rv.max() - hi) / hi < 1e-3  # extreme Ritz value converges first


# --------------------------------------------------------------------------- float32 inner solver and refinement


def test_f32_pcg_matches_cholesky_to_float_accuracy(orc):
    rng = np.random.default_rng(21)
    A = aniso_3d_7pt_fp32exact(6, 7, 5, 1.0, 30.0, 2.5)
    xt = rng.uniform(-1, 1, A.n)
    b = rhs_from_solution(A, xt).astype(np.float32)
    res = orc.pcg_f32(A, b, rtol=1e-5, max_it=2000)
    xc = sla.cho_solve(sla.cho_factor(A.to_dense()), b.astype(np.float64))
    kappa = np.linalg.cond(A.to_dense())
    assert res["reason"] == "converged"
    assert np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc) < kappa * 2e-5


@pytest.mark.parametrize("kind", ["aniso", "diffusion"])
def test_iterative_refinement_reaches_double_accuracy(orc, kind):
    rng = np.random.default_rng(31)
    if kind == "aniso":
        A = aniso_3d_7pt_fp32exact(10, 9, 11, 1.0, 250.0, 7.0)
    else:
        A = diffusion_3d_27pt(9, 10.0 ** rng.uniform(-2, 2, 9**3))
    xt = rng.uniform(-1, 1, A.n)
    b = rhs_from_solution(A, xt)
    res = orc.ir(A, b, rtol=1e-10)
    assert res["reason"] == "converged"
    true_rel = np.linalg.norm(b - A.to_scipy() @ res["x"]) / np.linalg.norm(b)
    assert true_rel <= 1e-10 and abs(true_rel - res["rel_res"]) <= 1e-12
    xc = sla.cho_solve(sla.cho_factor(A.to_dense()), b)
    kappa = np.linalg.cond(A.to_dense())
    assert np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc) <= kappa * 1e-10
    assert res["outer"] >= 2  # float32 alone cannot reach 1e-10


U32 = 2.0**-24  # unit roundoff of float32


def test_spmv_f32_matches_scipy_within_float_bound(orc):
    """The float32 product agrees with scipy's float64 product of the same float32 operands within the
    float32 summation bound (m+1) 2u32 sum|a x| per row (m entries in the row)."""
    rng = np.random.default_rng(5)
    for A in (random_spd_csr(200, 0.05, rng), _nonsym_csr(300, 0.03, rng), diffusion_3d_27pt(6, 10.0 ** rng.uniform(-2, 2, 216))):
        v32 = A.val.astype(np.float32)
        x32 = rng.uniform(-1, 1, A.n).astype(np.float32)
        y = orc.spmv_f32(A, x32)
        assert y.dtype == np.float32
        S = CSR(A.rowptr, A.col, v32.astype(np.float64)).to_scipy()
        y64 = S @ x32.astype(np.float64)
        Sabs = CSR(A.rowptr, A.col, np.abs(v32.astype(np.float64))).to_scipy()
        m = np.diff(A.rowptr)
        bound = (m + 1) * 2 * U32 * (Sabs @ np.abs(x32.astype(np.float64)))
        assert np.all(np.abs(y.astype(np.float64) - y64) <= bound)


def test_spmv_f32_rounds_every_partial_sum_to_float32(orc):
    """Row [1, 1, 1] times x = [1, 2^-24, 2^-24]: each float32 partial sum 1 + 2^-24 is a tie and rounds
    to 1 (ties to even), so the float32 result is exactly 1; accumulated in float64 the sum is 1 + 2^-23,
    which float32 represents.  Terms are added in the row's stored order: [2^-24, 2^-24, 1] gives 1 + 2^-23."""
    A3 = CSR(np.array([0, 3, 6, 7], np.int32), np.array([0, 1, 2, 2, 1, 0, 2], np.int32), np.ones(7))
    x = np.array([1.0, 2.0**-24, 2.0**-24], np.float32)
    y = orc.spmv_f32(A3, x)
    assert y[0] == np.float32(1.0)
    assert y[1] == np.float32(1.0 + 2.0**-23)
    assert float((A3.to_scipy() @ x.astype(np.float64))[0]) == 1.0 + 2.0**-23


def _f32_tridiag_rho0_case():
    """3x3 tridiagonal SPD matrix with unit diagonal (D = I, so z0 = r0 = b) and b = (1 + 2^-12) (1,1,1)."""
    e = 2.0**-4
    A = CSR(np.array([0, 2, 5, 7], np.int32), np.array([0, 1, 0, 1, 2, 1, 2], np.int32), np.array([1, e, e, 1, e, e, 1.0]))
    return A, np.full(3, 1 + 2.0**-12, np.float32)


def test_f32_pcg_initial_rho_is_the_float32_value(orc):
    """rho0 = (r0, z0) = 3 (1 + 2^-12)^2 under float32 arithmetic: each product (1 + 2^-12)^2 =
    1 + 2^-11 + 2^-24 lies halfway between float32 neighbours and rounds to 1 + 2^-11 (ties to even); the
    three products then add exactly to 3 + 3 2^-11.  Products or sums carried in float64 would give
    3 + 3 2^-11 + 3 2^-24, which rounds to 3 + 3 2^-11 + 2^-22."""
    A, b = _f32_tridiag_rho0_case()
    res = orc.pcg_f32(A, b, rtol=0.0, max_it=1, hist_len=1)
    assert res["rho"][0] == 3 + 3 * 2.0**-11


def test_f32_pcg_eigenvector_rhs_alpha(orc):
    """b = a sine mode of the 5-point Laplacian (D = 4I): one iteration with alpha1 = d / lambda, to float32
    accuracy."""
    N = 16
    v = sine_mode_2d(N, 2, 3).astype(np.float32)
    lam = lap_eig_1d(N, 2) + lap_eig_1d(N, 3)
    res = orc.pcg_f32(laplace_2d_5pt(N), v, rtol=1e-5, max_it=50, hist_len=1)
    assert res["iters"] == 1 and abs(res["alpha"][0] - 4.0 / lam) <= 8 * U32 * 4.0 / lam


def test_f32_pcg_residuals_d_orthogonal(orc):
    """The float32 iterates' true residuals are D^-1-orthogonal to float32 accuracy."""
    rng = np.random.default_rng(42)
    A = random_spd_csr(30, 0.2, rng, dominance=0.5)
    A = CSR(A.rowptr, A.col, A.val.astype(np.float32).astype(np.float64))
    Ad = A.to_dense()
    b = rng.standard_normal(30).astype(np.float32)
    dinv = 1.0 / np.diag(Ad)
    rs = [b - Ad @ orc.pcg_f32(A, b, rtol=0.0, max_it=j)["x"].astype(np.float64) for j in range(4)]
    for i in range(4):
        for j in range(i + 1, 4):
            den = math.sqrt(abs(rs[i] @ (dinv * rs[i])) * abs(rs[j] @ (dinv * rs[j])))
            assert abs(rs[i] @ (dinv * rs[j])) / den < 1e-4


@pytest.mark.parametrize("kind", ["aniso", "diffusion"])
def test_refinement_contraction_per_correction(orc, kind):
    """Each correction of the refinement scales the float64 true residual by at most 2 eta + 4 kappa u32
    (eta = inner relative tolerance): the float32 rounding of r, the inner residual eta ||r|| and the
    rounding of A's values to float32 (the standard analysis of iterative refinement, e.g. Higham,
    Accuracy and Stability of Numerical Algorithms, Ch. 12).  So the number of corrections to reach rtol
    is at most ceil(log(rtol) / log(2 eta + 4 kappa u32)) and, float32 alone stopping near u32 kappa, at
    least 2 for rtol 1e-10."""
    rng = np.random.default_rng(31)
    if kind == "aniso":
        A = aniso_3d_7pt_fp32exact(10, 9, 11, 1.0, 250.0, 7.0)
    else:
        A = diffusion_3d_27pt(9, 10.0 ** rng.uniform(-2, 2, 9**3))
    b = rhs_from_solution(A, rng.uniform(-1, 1, A.n))
    eta = 1e-4
    kappa = np.linalg.cond(A.to_dense())
    q = 2 * eta + 4 * kappa * U32
    full = orc.ir(A, b, rtol=1e-10, rtol_inner=eta)
    assert full["reason"] == "converged"
    assert 2 <= full["outer"] <= math.ceil(math.log(1e-10) / math.log(q))
    rel = [1.0] + [orc.ir(A, b, rtol=1e-10, rtol_inner=eta, max_outer=j)["rel_res"] for j in range(1, full["outer"] + 1)]
    for k in range(full["outer"]):
        assert rel[k + 1] <= q * rel[k]


# --------------------------------------------------------------------------- planted mistakes


def _pins_pass(orc, mutation):
    """Run a fast subset of the pins against the oracle with a planted mistake."""
    out = {}
    rng = np.random.default_rng(42)
    n = 30
    A = random_spd_csr(n, 0.2, rng, dominance=0.5)
    Ad = A.to_dense()
    b = rng.standard_normal(n)
    xc = sla.cho_solve(sla.cho_factor(Ad), b)
    res = orc.pcg(A, b, rtol=1e-12, max_it=300, mutation=mutation)
    out["cholesky"] = res["reason"] == "converged" and np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc) < 1e-8
    dinv = 1.0 / np.diag(Ad)
    xs = [orc.pcg(A, b, rtol=0.0, max_it=j, mutation=mutation)["x"] for j in range(4)]
    rs = [b - Ad @ x for x in xs]
    ok = True
    for i in range(4):
        for j in range(i + 1, 4):
            den = math.sqrt(abs(rs[i] @ (dinv * rs[i])) * abs(rs[j] @ (dinv * rs[j]))) + 1e-300
            ok &= abs(rs[i] @ (dinv * rs[j])) / den < 1e-8
    out["d_orthogonal"] = bool(ok)
    N = 16
    v = sine_mode_2d(N, 2, 3)
    lam = lap_eig_1d(N, 2) + lap_eig_1d(N, 3)
    r1 = orc.pcg(laplace_2d_5pt(N), v, rtol=1e-10, max_it=50, hist_len=1, mutation=mutation)
    out["eigen_rhs"] = r1["iters"] == 1 and abs(r1["alpha"][0] - 4.0 / lam) < 1e-12 * 4.0 / lam
    return out


def test_pins_catch_planted_mistakes(orc):
    clean = _pins_pass(orc, 0)
    assert all(clean.values()), clean
    for m in (1, 2, 3, 4, 5, 6):
        got = _pins_pass(orc, m)
        assert not all(got.values()), f"mutation {m} went unnoticed: {got}"


def _pins_pass_f32(orc, mutation):
    """The float32 pins above, run against the float32 solver with a planted mistake."""
    out = {}
    rng = np.random.default_rng(42)
    A = random_spd_csr(30, 0.2, rng, dominance=0.5)
    A = CSR(A.rowptr, A.col, A.val.astype(np.float32).astype(np.float64))
    Ad = A.to_dense()
    b = rng.standard_normal(30).astype(np.float32)
    xc = sla.cho_solve(sla.cho_factor(Ad), b.astype(np.float64))
    res = orc.pcg_f32(A, b, rtol=1e-6, max_it=300, mutation=mutation)
    err = np.linalg.norm(res["x"] - xc) / np.linalg.norm(xc)
    out["cholesky"] = res["reason"] == "converged" and err < np.linalg.cond(Ad) * 2e-5
    dinv = 1.0 / np.diag(Ad)
    rs = [b - Ad @ orc.pcg_f32(A, b, rtol=0.0, max_it=j, mutation=mutation)["x"].astype(np.float64) for j in range(4)]
    ok = True
    for i in range(4):
        for j in range(i + 1, 4):
            den = math.sqrt(abs(rs[i] @ (dinv * rs[i])) * abs(rs[j] @ (dinv * rs[j]))) + 1e-300
            ok &= abs(rs[i] @ (dinv * rs[j])) / den < 1e-4
    out["d_orthogonal"] = bool(ok)
    N = 16
    v = sine_mode_2d(N, 2, 3).astype(np.float32)
    lam = lap_eig_1d(N, 2) + lap_eig_1d(N, 3)
    r1 = orc.pcg_f32(laplace_2d_5pt(N), v, rtol=1e-5, max_it=50, hist_len=1, mutation=mutation)
    out["eigen_rhs"] = r1["iters"] == 1 and abs(r1["alpha"][0] - 4.0 / lam) <= 8 * U32 * 4.0 / lam
    A3, b3 = _f32_tridiag_rho0_case()
    out["rho0_float32"] = orc.pcg_f32(A3, b3, rtol=0.0, max_it=1, hist_len=1, mutation=mutation)["rho"][0] == 3 + 3 * 2.0**-11
    return out


def test_f32_pins_catch_planted_mistakes(orc):
    """Float32 solver mistakes: dots carried in float64, the Jacobi step dropped, beta inverted, the sign of
    the search-direction update flipped; each fails at least one float32 pin."""
    clean = _pins_pass_f32(orc, 0)
    assert all(clean.values()), clean
    for m in (1, 2, 3, 4):
        got = _pins_pass_f32(orc, m)
        assert not all(got.values()), f"float32 mutation {m} went unnoticed: {got}"


def test_non_finite_inputs_are_breakdowns(orc):
    """A NaN or infinity in b or x0 ends every oracle solver with a breakdown (reading 10), never with
    convergence against an infinite tolerance."""
    from synthetic import laplace_2d_5pt

    A = laplace_2d_5pt(8)
    for bad in (np.nan, np.inf, -np.inf):
        b = np.ones(A.n)
        b[5] = bad
        assert orc.pcg(A, b)["reason"] == "breakdown"
        assert orc.tfqmr(A, b)["reason"] == "breakdown"
        assert orc.ir(A, b)["reason"] == "breakdown"
        x0 = np.zeros(A.n)
        x0[2] = bad
        assert orc.pcg(A, np.ones(A.n), x0=x0)["reason"] == "breakdown"
