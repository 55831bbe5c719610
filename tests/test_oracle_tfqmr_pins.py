"""Pins of the TFQMR oracle against facts other than itself.

* scipy's own TFQMR (an independent implementation of Freund's method) run on
  the Jacobi-scaled system D^-1 A x = D^-1 b gives the same iterate after every
  full iteration (two of its half-step callbacks);
* Freund's bound: the true residual of the scaled system after i iterations is
  at most sqrt(2i + 1) tau_i;
* the converged x equals a dense LU solve within the conditioning bound, on
  symmetric and nonsymmetric matrices;
* special cases: a diagonal matrix and an eigenvector right-hand side are
  solved exactly by the first half-step (alpha = 1 / lambda of D^-1 A);
* every planted mistake (the oracle's mutation argument) fails one of the pins.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import oracle
from synthetic import (
    convection_diffusion_2d,
    diagonal_csr,
    laplace_2d_5pt,
    rhs_from_solution,
    sine_mode_2d,
)


def _scaled(A, b):
    M = A.to_scipy()
    d = M.diagonal()
    return (sp.diags(1.0 / d) @ M).tocsr(), b / d


def _scipy_iterates(A, b, n_half):
    Mh, bh = _scaled(A, b)
    xs = []
    sla.tfqmr(Mh, bh, rtol=1e-300, atol=0.0, maxiter=n_half, callback=lambda xk: xs.append(xk.copy()))
    return xs


def _problems():
    rng = np.random.default_rng(7)
    A1 = laplace_2d_5pt(17, shift=0.2)
    A2 = convection_diffusion_2d(19, 0.45, -0.3, shift=0.1)
    out = []
    for A in (A1, A2):
        b = rhs_from_solution(A, rng.uniform(-1, 1, A.n))
        out.append((A, b))
    return out


@pytest.mark.parametrize("k", [0, 1])
def test_tfqmr_matches_scipy_iterates(k):
    A, b = _problems()[k]
    xs = _scipy_iterates(A, b, 24)
    for i in range(1, 12):
        r = oracle.tfqmr(A, b, rtol=0.0, max_it=i)
        xi = xs[2 * i - 1]
        assert np.linalg.norm(r["x"] - xi) / np.linalg.norm(xi) <= 1e-12, i


@pytest.mark.parametrize("k", [0, 1])
def test_tfqmr_quasi_residual_bound(k):
    A, b = _problems()[k]
    Mh, bh = _scaled(A, b)
    for i in range(1, 25):
        r = oracle.tfqmr(A, b, rtol=0.0, max_it=i)
        true = np.linalg.norm(bh - Mh @ r["x"])
        assert true <= r["bound"] * (1 + 1e-10), (i, true, r["bound"])
        assert abs(r["bound"] - np.sqrt(2 * i + 1) * r["tau"]) <= 1e-15 * r["bound"]


@pytest.mark.parametrize("k", [0, 1])
def test_tfqmr_converges_to_dense_solution(k):
    A, b = _problems()[k]
    r = oracle.tfqmr(A, b, rtol=1e-12)
    assert r["reason"] == "converged"
    D = A.to_dense()
    xd = np.linalg.solve(D, b)
    Mh, _ = _scaled(A, b)
    kappa = np.linalg.cond(Mh.toarray())
    assert np.linalg.norm(r["x"] - xd) / np.linalg.norm(xd) <= 2 * kappa * 1e-12


def test_tfqmr_diagonal_is_exact_in_one_half_step():
    d = np.array([2.0, 3.0, 5.0, 7.0, 11.0])
    b = np.array([1.0, -2.0, 3.0, 0.5, 4.0])
    r = oracle.tfqmr(diagonal_csr(d), b, rtol=1e-14, hist_len=1)
    assert r["reason"] == "converged" and r["iters"] == 1
    assert np.array_equal(r["x"], b / d) or np.max(np.abs(r["x"] - b / d)) <= 1e-16
    assert r["alpha"][0] == 1.0 and r["tau"] == 0.0


def test_tfqmr_eigenvector_rhs_one_half_step():
    N, j1, j2 = 15, 2, 3
    A = laplace_2d_5pt(N)
    v = sine_mode_2d(N, j1, j2)
    lam = 4 * np.sin(j1 * np.pi / (2 * (N + 1))) ** 2 + 4 * np.sin(j2 * np.pi / (2 * (N + 1))) ** 2
    r = oracle.tfqmr(A, v, rtol=1e-12, hist_len=1)
    assert r["reason"] == "converged" and r["iters"] == 1
    # D = 4 I: the scaled operator has eigenvalue lam / 4 on v, so alpha = 4 / lam and x = v / lam
    assert abs(r["alpha"][0] - 4.0 / lam) <= 1e-14 * (4.0 / lam)
    assert np.max(np.abs(r["x"] - v / lam)) <= 1e-13 * np.max(np.abs(v / lam))


def test_tfqmr_zero_rhs_and_bad_diagonal():
    A = laplace_2d_5pt(6)
    r = oracle.tfqmr(A, np.zeros(A.n))
    assert r["reason"] == "converged" and r["iters"] == 0 and not r["x"].any()
    from synthetic.stencils import CSR

    B = CSR(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([2.0, 1.0]))
    assert oracle.tfqmr(B, np.ones(2))["reason"] == "bad_diagonal"


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_tfqmr_pins_catch_planted_mistakes(mutation):
    caught = False
    for A, b in _problems():
        xs = _scipy_iterates(A, b, 12)
        Mh, bh = _scaled(A, b)
        for i in range(1, 6):
            r = oracle.tfqmr(A, b, rtol=0.0, max_it=i, mutation=mutation)
            xi = xs[2 * i - 1]
            if np.linalg.norm(r["x"] - xi) / np.linalg.norm(xi) > 1e-8:
                caught = True
            if np.linalg.norm(bh - Mh @ r["x"]) > r["bound"] * (1 + 1e-10):
                caught = True
    assert caught, mutation


def test_tfqmr_rounding_sensitivity():
    """One-ulp perturbations of b move TFQMR's alpha/beta far more on a nonsymmetric system than on a
    symmetric one, where both TFQMR's and CG's stay at rounding level (the reason the GPU parity bar for
    TFQMR is scaled by the measured sensitivity)."""

    def sens(solver, A, b):
        ref = solver(A, b, rtol=1e-8, hist_len=10)
        sign = np.random.default_rng(3).choice([-1.0, 1.0], b.size)
        o = solver(A, b * (1.0 + sign * 2.0**-53), rtol=1e-8, hist_len=10)
        return max(float(np.max(np.abs(o[k] - ref[k]) / np.abs(ref[k]))) for k in ("alpha", "beta"))

    (A1, b1), (A2, b2) = _problems()
    assert sens(oracle.tfqmr, A1, b1) <= 1e-13
    assert sens(oracle.pcg, A1, b1) <= 1e-13
    assert sens(oracle.tfqmr, A2, b2) >= 1e-14
