"""The matrix-free stencil operator and Jacobi-PCG on it, against the oracle.

* y = S x against the oracle's stencil apply (the assembled product, pinned to
  scipy): within the summation bound (m + 1) 2u sum|w x| (the GPU fuses each
  product into the row sum), exactly on integer inputs, and bit for bit equal
  to the GPU's CSR SpMV of the assembled matrix (the same FMA chain per row);
* CG on the stencil against the oracle's CG on the assembled matrix: alpha and
  beta of the first 10 iterations within 1e-12, the same iteration count, x
  within 1e-7 at rtol 1e-8, in every mode, on ragged grids and at 128^3.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import rhs_from_solution, single_problem, stencil_matrix, stencil_terms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402

V = C.c_void_p


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    apcg.load()
    c = apcg.ctx_create()
    yield c
    apcg.call("apcg_ctx_destroy", V(c))


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _apply(ctx, dims, offs, w, x):
    S = apcg.stencil_create(dims, offs, w)
    xt = _t(x)
    y = torch.empty_like(xt)
    vx, vy = apcg.vec_wrap(xt), apcg.vec_wrap(y)
    apcg.call("apcg_stencil_apply_async", V(ctx), V(S), V(vx), V(vy))
    apcg.call("apcg_ctx_synchronize", V(ctx))
    for h in (vx, vy):
        apcg.call("apcg_vec_destroy", V(h))
    apcg.call("apcg_stencil_destroy", V(S))
    return y.cpu().numpy()


def _csr_apply(ctx, A, x):
    rowptr, col, val, xt = _t(A.rowptr), _t(A.col), _t(A.val), _t(x)
    y = torch.empty_like(xt)
    M = apcg.mat_wrap(rowptr, col, val)
    vx, vy = apcg.vec_wrap(xt), apcg.vec_wrap(y)
    apcg.call("apcg_mat_mult_async", V(ctx), V(M), V(vx), V(vy))
    apcg.call("apcg_ctx_synchronize", V(ctx))
    for h, fn in ((vx, "apcg_vec_destroy"), (vy, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
        apcg.call(fn, V(h))
    return y.cpu().numpy()


APPLY_CASES = [
    ("5pt", (33, 17, 1)),
    ("9pt", (21, 30, 1)),
    ("7pt", (13, 9, 11)),
    ("27pt", (10, 7, 9)),
    ("7pt", (1, 40, 3)),
]


@pytest.mark.parametrize("kind,dims", APPLY_CASES)
def test_stencil_apply(ctx, kind, dims):
    offs, w = stencil_terms(kind, dims, shift=0.125)
    n = int(np.prod(dims))
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, n)
    y = _apply(ctx, dims, offs, w, x)
    ref = oracle.stencil_apply(dims, offs, w, x)
    bound = (len(w) + 1) * 2 * 2.0**-53 * (oracle.stencil_apply(dims, offs, np.abs(w), np.abs(x)))
    assert np.all(np.abs(y - ref) <= bound)
    xi = rng.integers(-1000, 1000, n).astype(np.float64)
    assert np.array_equal(_apply(ctx, dims, offs, w, xi), oracle.stencil_apply(dims, offs, w, xi))
    # the same FMA chain as the CSR SpMV of the assembled rows (columns ascending)
    A = stencil_matrix(kind, dims, shift=0.125)
    assert np.array_equal(y, _csr_apply(ctx, A, x))


def test_stencil_apply_generic_terms(ctx):
    """A term count without a specialised kernel (4 terms, offsets of 2) and unsorted input order."""
    dims = (19, 14, 6)
    offs = np.array([(2, 0, 0), (0, 0, 0), (0, -2, 1), (-1, 1, 0)], dtype=np.int32)
    w = np.array([0.5, 3.0, -1.25, 0.75])
    x = np.random.default_rng(4).uniform(-1, 1, int(np.prod(dims)))
    lin = offs[:, 0] + dims[0] * (offs[:, 1] + dims[1] * offs[:, 2])
    order = np.argsort(lin, kind="stable")
    ref = oracle.stencil_apply(dims, offs[order], w[order], x)
    y = _apply(ctx, dims, offs, w, x)
    bound = 5 * 2 * 2.0**-53 * oracle.stencil_apply(dims, offs, np.abs(w), np.abs(x))
    assert np.all(np.abs(y - ref) <= bound)


def test_stencil_argument_errors(ctx):
    offs = np.array([(1, 0, 0), (1, 0, 0)], dtype=np.int32)
    with pytest.raises(apcg.ApcgError):
        apcg.stencil_create((4, 4, 1), offs, [1.0, 2.0])  # duplicate offset
    with pytest.raises(apcg.ApcgError):
        apcg.stencil_create((0, 4, 1), offs[:1], [1.0])  # empty grid
    S = apcg.stencil_create((8, 8, 1), np.array([(1, 0, 0), (-1, 0, 0)], np.int32), [-1.0, -1.0])
    with pytest.raises(apcg.ApcgError):  # no centre term: no Jacobi diagonal
        apcg.cg_plan_create_stencil(ctx, S, apcg.cg_opts(mode="async_graph"))
    apcg.call("apcg_stencil_destroy", V(S))
    offs, w = stencil_terms("5pt", (8, 8, 1))
    S = apcg.stencil_create((8, 8, 1), offs, w)
    with pytest.raises(apcg.ApcgError):  # the cluster kernel reads a CSR matrix
        apcg.cg_plan_create_stencil(ctx, S, apcg.cg_opts(mode="persistent"))
    apcg.call("apcg_stencil_destroy", V(S))


def _stencil_cg(ctx, kind, dims, b, shift=0.0, **kw):
    offs, w = stencil_terms(kind, dims, shift=shift)
    S = apcg.stencil_create(dims, offs, w)
    opts = apcg.cg_opts(history_len=10, **kw)
    plan = apcg.cg_plan_create_stencil(ctx, S, opts)
    apcg.call("apcg_stencil_destroy", V(S))  # the plan keeps its own copy
    bt = _t(b)
    x = torch.zeros_like(bt)
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    res = apcg.cg_plan_solve(plan, vb, vx)
    res["alpha"], res["beta"] = list(opts._hist[0]), list(opts._hist[1])
    apcg.call("apcg_cg_plan_destroy", V(plan))
    for h in (vb, vx):
        apcg.call("apcg_vec_destroy", V(h))
    return res, x.cpu().numpy()


def _check(res, x, ref, k):
    assert res["reason"] == ref["reason"] == "converged"
    assert abs(res["iters"] - ref["iters"]) <= max(k - 1, 0) or res["iters"] == ref["iters"]
    h = min(10, ref["iters"] - 1)
    assert np.max(np.abs(np.array(res["alpha"][:h]) - ref["alpha"][:h]) / np.abs(ref["alpha"][:h])) <= 1e-12
    assert np.max(np.abs(np.array(res["beta"][:h]) - ref["beta"][:h]) / np.abs(ref["beta"][:h])) <= 1e-12
    if res["iters"] == ref["iters"]:
        assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-7
    assert res["rel_res"] <= 1e-8


@pytest.mark.parametrize("kind,dims,shift", [("5pt", (37, 29, 1), 0.0), ("9pt", (31, 31, 1), 0.0),
                                             ("7pt", (17, 23, 19), 0.0), ("27pt", (15, 13, 11), 0.5)])
@pytest.mark.parametrize("mode", ["host_sync", "async", "async_graph"])
def test_stencil_cg_parity(ctx, kind, dims, shift, mode):
    A = stencil_matrix(kind, dims, shift=shift)
    b = rhs_from_solution(A, np.random.default_rng(6).uniform(-1, 1, A.n))
    k = 3 if mode == "async" else 1
    ref = oracle.pcg(A, b, rtol=1e-8, check_every=k, hist_len=10)
    res, x = _stencil_cg(ctx, kind, dims, b, shift=shift, rtol=1e-8, check_every=k, mode=mode)
    _check(res, x, ref, k)


def test_stencil_cg_full_size_128cube(ctx):
    """The benchmark system (128^3 7-point, the same b) solved matrix-free."""
    p = single_problem("c2", seed=0)
    ref = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=10, hist_len=10)
    res, x = _stencil_cg(ctx, "7pt", (128, 128, 128), p.b, rtol=1e-8, check_every=10, mode="async_graph",
                         max_it=5000)
    _check(res, x, ref, 10)


def _stencil_ir(ctx, kind, dims, b, shift=0.0, **kw):
    offs, w = stencil_terms(kind, dims, shift=shift)
    S = apcg.stencil_create(dims, offs, w)
    plan = apcg.ir_plan_create_stencil(ctx, S, apcg.ir_opts(**kw))
    apcg.call("apcg_stencil_destroy", V(S))
    bt = _t(b)
    x = torch.zeros_like(bt)
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    res = apcg.ir_plan_solve(plan, vb, vx)
    apcg.call("apcg_ir_plan_destroy", V(plan))
    for h in (vb, vx):
        apcg.call("apcg_vec_destroy", V(h))
    return res, x.cpu().numpy()


@pytest.mark.parametrize("kind,dims,shift", [("5pt", (41, 37, 1), 0.0), ("9pt", (31, 31, 1), 0.0),
                                             ("7pt", (17, 19, 13), 0.0), ("27pt", (11, 11, 11), 0.5)])
def test_stencil_refinement_reaches_double_accuracy(ctx, kind, dims, shift):
    import scipy.linalg as sla

    A = stencil_matrix(kind, dims, shift=shift)
    b = rhs_from_solution(A, np.random.default_rng(8).uniform(-1, 1, A.n))
    res, x = _stencil_ir(ctx, kind, dims, b, shift=shift, rtol=1e-10, rtol_inner=1e-4, inner_check_every=1)
    assert res["reason"] == "converged" and res["outer"] >= 1
    true_rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert true_rel <= 1.05e-10 and abs(true_rel - res["rel_res"]) <= 1e-12
    D = A.to_dense()
    xc = sla.cho_solve(sla.cho_factor(D), b)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(x - xc) / np.linalg.norm(xc) <= kappa * 2e-10
    ref = oracle.ir(A, b, rtol=1e-10)
    assert ref["reason"] == "converged" and abs(ref["outer"] - res["outer"]) <= 1


def test_stencil_refinement_full_size_128cube(ctx):
    """128^3 7-point refined to 1e-10 against the float64 stencil CG to 1e-10."""
    p = single_problem("c2", seed=0)
    res, x_ir = _stencil_ir(ctx, "7pt", (128, 128, 128), p.b, rtol=1e-10, inner_check_every=10)
    assert res["reason"] == "converged"
    rel_ir = np.linalg.norm(p.b - oracle.spmv(p.A, x_ir)) / np.linalg.norm(p.b)
    assert rel_ir <= 1.05e-10
    r64, x64 = _stencil_cg(ctx, "7pt", (128, 128, 128), p.b, rtol=1e-10, check_every=10, mode="async_graph",
                           max_it=10000)
    assert r64["reason"] == "converged"
    assert np.linalg.norm(x_ir - x64) / np.linalg.norm(x64) <= 1e-6
