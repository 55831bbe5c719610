"""Pins of the matrix-free stencil oracle: it is the product with the assembled
stencil matrix, computed by scipy (an independent implementation), on square
and oblong grids, with random and integer inputs; planted mistakes (periodic
wrap at the x boundary, swapped axes) are caught.  It also pins the synthetic
stencil descriptions to the assembled Laplace matrices the CSR path solves.
"""

import numpy as np
import pytest

import oracle
from synthetic import laplace_2d_5pt, laplace_3d_7pt, laplace_3d_27pt, stencil_matrix, stencil_terms
from synthetic.stencils import laplace_2d_9pt

CASES = [("5pt", (17, 11, 1)), ("9pt", (13, 19, 1)), ("7pt", (9, 7, 11)), ("27pt", (6, 8, 5)), ("7pt", (1, 5, 4))]


@pytest.mark.parametrize("kind,dims", CASES)
def test_stencil_apply_is_the_assembled_product(kind, dims):
    offs, w = stencil_terms(kind, dims, shift=0.25)
    A = stencil_matrix(kind, dims, shift=0.25).to_scipy()
    rng = np.random.default_rng(3)
    n = int(np.prod(dims))
    x = rng.uniform(-1, 1, n)
    y = oracle.stencil_apply(dims, offs, w, x)
    ref = A @ x
    assert np.max(np.abs(y - ref)) <= 1e-15 * np.max(np.abs(A) @ np.abs(x))
    xi = rng.integers(-1000, 1000, n).astype(np.float64)
    assert np.array_equal(oracle.stencil_apply(dims, offs, w, xi), A @ xi)


def test_stencil_matrices_are_the_laplace_generators():
    for kind, make, N, dims in (
        ("5pt", laplace_2d_5pt, 12, (12, 12, 1)),
        ("9pt", laplace_2d_9pt, 10, (10, 10, 1)),
        ("7pt", laplace_3d_7pt, 7, (7, 7, 7)),
        ("27pt", laplace_3d_27pt, 5, (5, 5, 5)),
    ):
        A, B = make(N), stencil_matrix(kind, dims)
        assert np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)
        offs, w = stencil_terms(kind, dims)
        lin = offs[:, 0] + dims[0] * (offs[:, 1] + dims[1] * offs[:, 2])
        assert np.all(np.diff(lin) > 0)  # terms in the column order of the assembled rows


def _aniso_2d(nx, ny, wx, wy, c):
    """c I + wx (x-neighbours) + wy (y-neighbours) on an nx x ny grid, assembled with Kronecker products."""
    import scipy.sparse as sp

    Tx = sp.diags([np.ones(nx - 1), np.ones(nx - 1)], [-1, 1])
    Ty = sp.diags([np.ones(ny - 1), np.ones(ny - 1)], [-1, 1])
    A = c * sp.identity(nx * ny) + wx * sp.kron(sp.identity(ny), Tx) + wy * sp.kron(Ty, sp.identity(nx))
    offs = np.array([(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)], dtype=np.int32)
    w = np.array([wy, wx, c, wx, wy])
    return A.tocsr(), offs, w


def test_stencil_apply_anisotropic_terms():
    A, offs, w = _aniso_2d(13, 9, -0.5, -2.25, 5.5)
    x = np.random.default_rng(8).uniform(-1, 1, 13 * 9)
    y = oracle.stencil_apply((13, 9, 1), offs, w, x)
    assert np.max(np.abs(y - A @ x)) <= 1e-15 * np.max(np.abs(A) @ np.abs(x))


@pytest.mark.parametrize("mutation", [1, 2])
def test_stencil_pins_catch_planted_mistakes(mutation):
    caught = False
    for kind, dims in CASES:
        offs, w = stencil_terms(kind, dims)
        A = stencil_matrix(kind, dims).to_scipy()
        x = np.random.default_rng(5).uniform(-1, 1, int(np.prod(dims)))
        y = oracle.stencil_apply(dims, offs, w, x, mutation=mutation)
        caught |= not np.allclose(y, A @ x, rtol=0, atol=1e-12)
    A, offs, w = _aniso_2d(13, 9, -0.5, -2.25, 5.5)
    x = np.random.default_rng(8).uniform(-1, 1, 13 * 9)
    caught |= not np.allclose(oracle.stencil_apply((13, 9, 1), offs, w, x, mutation=mutation), A @ x, rtol=0, atol=1e-12)
    assert caught
