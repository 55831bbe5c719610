"""Large systems with irregular rows against the oracle.

The benchmark-size tests use stencils, whose slices of 32 rows are almost
uniform.  These systems stress the sliced-ELL SpMV where they are not: a
7-point Laplacian whose size is ragged against every slice and grid boundary,
and weighted graph Laplacians whose rows range from the diagonal alone to 128
or 129 entries (hub rows far longer than their slice neighbours, so slices
carry heavy padding).  Parity bars as for the other CG tests: alpha/beta of the
first 10 iterations within 1e-12 relative, the same iteration count, x within
1e-7 of the oracle's at rtol 1e-8.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import graph_laplacian_csr, laplace_3d_7pt, rhs_from_solution

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    apcg.load()
    c = apcg.ctx_create()
    yield c
    apcg.call("apcg_ctx_destroy", C.c_void_p(c))


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _solve(ctx, A, b, mode, k=1):
    rowptr, col, val, bt = _t(A.rowptr), _t(A.col), _t(A.val), _t(b)
    x = torch.zeros_like(bt)
    M = apcg.mat_wrap(rowptr, col, val)
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    res = apcg.cg_solve(ctx, M, vb, vx, apcg.cg_opts(rtol=1e-8, check_every=k, mode=mode, history_len=10))
    for h, fn in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
        apcg.call(fn, C.c_void_p(h))
    return res, x.cpu().numpy()


def _check(res, x, ref, k):
    assert res["reason"] == ref["reason"] == "converged"
    assert abs(res["iters"] - ref["iters"]) <= k - 1 if k > 1 else res["iters"] == ref["iters"]
    h = min(10, ref["iters"] - 1)
    a, b = np.array(res["alpha"][:h]), np.array(res["beta"][:h])
    assert np.max(np.abs(a - ref["alpha"][:h]) / np.abs(ref["alpha"][:h])) <= 1e-12
    assert np.max(np.abs(b - ref["beta"][:h]) / np.abs(ref["beta"][:h])) <= 1e-12
    if res["iters"] == ref["iters"]:
        assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-7
    assert res["rel_res"] <= 1e-8


@pytest.mark.parametrize("mode", ["host_sync", "async_graph"])
def test_7pt_ragged_size(ctx, mode):
    A = laplace_3d_7pt(71)  # 357,911 rows: the last slice and the last stage are partial
    rng = np.random.default_rng(5)
    b = rhs_from_solution(A, rng.uniform(-1, 1, A.n))
    ref = oracle.pcg(A, b, rtol=1e-8, check_every=1, hist_len=10)
    res, x = _solve(ctx, A, b, mode)
    _check(res, x, ref, 1)


@pytest.mark.parametrize("hub_degree", [127, 128])
@pytest.mark.parametrize("mode", ["host_sync", "async_graph"])
def test_graph_laplacian_hub_rows(ctx, hub_degree, mode):
    rng = np.random.default_rng(hub_degree)
    A = graph_laplacian_csr(330_000, rng, hub_degrees=(hub_degree, 40, hub_degree))
    lens = np.diff(A.rowptr)
    assert lens.max() == hub_degree + 1 and (lens == 1).any()
    b = rhs_from_solution(A, rng.uniform(-1, 1, A.n))
    ref = oracle.pcg(A, b, rtol=1e-8, check_every=1, hist_len=10)
    res, x = _solve(ctx, A, b, mode)
    _check(res, x, ref, 1)


def test_graph_laplacian_check_interval(ctx):
    rng = np.random.default_rng(9)
    A = graph_laplacian_csr(400_000, rng, mean_degree=3.0, hub_degrees=(64,))
    b = rhs_from_solution(A, rng.uniform(-1, 1, A.n))
    ref = oracle.pcg(A, b, rtol=1e-8, check_every=5, hist_len=10)
    res, x = _solve(ctx, A, b, "async", k=5)
    _check(res, x, ref, 5)
