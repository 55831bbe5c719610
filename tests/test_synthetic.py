"""Input generators: sizes, structure and the float32-exact construction."""

import numpy as np

from synthetic import (
    aniso_3d_7pt_fp32exact,
    batch_aniso_7pt,
    batch_shifted_5pt,
    diffusion_3d_27pt,
    laplace_2d_5pt,
    laplace_3d_7pt,
    laplace_3d_27pt,
    single_problem,
)


def _check_structure(A):
    rp, col = A.rowptr, A.col
    assert rp[0] == 0 and rp[-1] == A.nnz and np.all(np.diff(rp) >= 1)
    for i in range(A.n):
        c = col[rp[i] : rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c
    S = A.to_scipy()
    assert abs(S - S.T).max() == 0.0


def test_stencil_sizes_match_closed_forms():
    for N in (3, 5, 9):
        assert laplace_2d_5pt(N).nnz == 5 * N * N - 4 * N
        assert laplace_3d_7pt(N).nnz == 7 * N**3 - 6 * N * N
        assert laplace_3d_27pt(N).nnz == (3 * N - 2) ** 3
    p = single_problem("c1")
    assert (p.n, p.nnz) == (4096, 20224)


def test_structure_symmetric_sorted():
    rng = np.random.default_rng(0)
    for A in (laplace_2d_5pt(5), laplace_3d_7pt(4), laplace_3d_27pt(4), diffusion_3d_27pt(4, 10 ** rng.uniform(-2, 2, 64))):
        _check_structure(A)
        assert np.linalg.eigvalsh(A.to_dense()).min() > 0


def test_diffusion_rows_weakly_dominant():
    rng = np.random.default_rng(1)
    A = diffusion_3d_27pt(5, 10 ** rng.uniform(-2, 2, 125)).to_dense()
    d = np.diag(A)
    off = np.abs(A).sum(axis=1) - np.abs(d)
    assert np.all(d >= off * (1 - 1e-14))
    assert np.all(d[0] > off[0])


def test_aniso_values_are_float32_exact_and_dominant():
    A = aniso_3d_7pt_fp32exact(4, 5, 6, 1.0, 123.456, 7.89)
    assert np.array_equal(A.val.astype(np.float32).astype(np.float64), A.val)
    D = A.to_dense()
    assert np.all(np.diag(D) >= np.abs(D).sum(axis=1) - np.abs(np.diag(D)))


def test_batches_concatenate_consistently():
    for B in (batch_shifted_5pt(6, seed=2), batch_aniso_7pt(5, seed=3)):
        assert B.rowptr[-1] == B.nnz and B.sys_row_off[-1] == B.n_total
        for s in range(B.nsys):
            A, b, xt = B.system(s)
            _check_structure(A)
            assert np.allclose(A.to_scipy() @ xt, b, rtol=0, atol=1e-12)
            assert A.col.max() < A.n


def test_generators_are_deterministic():
    a = single_problem("c1", seed=4)
    b = single_problem("c1", seed=4)
    assert np.array_equal(a.b, b.b) and np.array_equal(a.x_true, b.x_true)
    B1 = batch_shifted_5pt(4, seed=9)
    B2 = batch_shifted_5pt(4, seed=9)
    assert np.array_equal(B1.val, B2.val) and np.array_equal(B1.b, B2.b)


def test_graph_laplacian_rows_and_definiteness():
    from synthetic import graph_laplacian_csr

    rng = np.random.default_rng(3)
    A = graph_laplacian_csr(3000, rng, hub_degrees=(127, 20))
    _check_structure(A)
    lens = np.diff(A.rowptr)
    hubs = [3000 // 3, 2 * 3000 // 3]
    assert lens[hubs[0]] == 128 and lens[hubs[1]] == 21 and (lens == 1).any()
    D = A.to_dense()
    assert np.allclose(D, D.T)
    # diagonally dominant by the shift: every row sum is exactly the shift
    assert np.allclose(D.sum(axis=1), 1.0)
    assert np.linalg.eigvalsh(D).min() > 0.999
