"""Jacobi-preconditioned TFQMR on the GPU against the oracle, through the C ABI.

Bars: the same iteration count (up to one check interval when the test lands
within rounding of the threshold, and one more iteration where the oracle's
own path moves under one-ulp perturbations), x within 1e-7 relative of the
oracle's x at rtol 1e-8, Freund's bound on the GPU iterate's own true
residual, and alpha/beta of the first 10 iterations within
max(1e-12, 10 S) relative, where S is the oracle's own sensitivity: the
largest relative change of those alpha/beta when b is perturbed by one unit
in the last place (three random sign patterns).  TFQMR's short recurrences
amplify rounding differences far more than CG's on nonsymmetric or
high-contrast systems (S reaches 1e-10 within 10 iterations on the 27-point
variable-coefficient system, against 1e-15 for CG), so a fixed 1e-12 bar
would test the conditioning of the method rather than the implementation.
The GPU also forms M u as M w + beta M u2 (linearity) where the oracle
applies M to u; the two differ only in rounding.  The persistent mode (the
whole solve in one thread-block-cluster launch, systems of at most 16384
rows) is held to the same bars as the three multi-kernel modes.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import (
    convection_diffusion_2d,
    diagonal_csr,
    laplace_2d_5pt,
    rhs_from_solution,
    sine_mode_2d,
    single_problem,
)
from synthetic.stencils import CSR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402

MODES = ["host_sync", "async", "async_graph", "persistent"]


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


def _solve(ctx, A: CSR, b, hist=10, **kw):
    rowptr, col, val, bt = _t(A.rowptr), _t(A.col), _t(A.val), _t(b)
    x = torch.zeros_like(bt)
    M = apcg.mat_wrap(rowptr, col, val)
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    try:
        res = apcg.tfqmr_solve(ctx, M, vb, vx, apcg.cg_opts(history_len=hist, **kw))
    finally:
        for h, fn in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
            apcg.call(fn, C.c_void_p(h))
    return res, x.cpu().numpy()


def _sensitivity(A, b, k, h):
    """Largest relative change of the oracle's first h alpha/beta under one-ulp perturbations of b."""
    ref = oracle.tfqmr(A, b, rtol=1e-8, check_every=k, hist_len=h)
    worst = 0.0
    for t in range(3):
        sign = np.random.default_rng(1000 + t).choice([-1.0, 1.0], b.size)
        o = oracle.tfqmr(A, b * (1.0 + sign * 2.0**-53), rtol=1e-8, check_every=k, hist_len=h)
        for key in ("alpha", "beta"):
            worst = max(worst, float(np.max(np.abs(o[key] - ref[key]) / np.abs(ref[key]))))
    return worst


def _check(res, x, ref, k, rtol=1e-8, sens=0.0, A=None, b=None):
    assert res["reason"] == ref["reason"] == "converged", (res, ref["reason"])
    sensitive = sens > 1e-13  # where one-ulp perturbations already move the oracle's own path
    slack = max(k - 1, 0) + (1 if sensitive else 0)
    assert abs(res["iters"] - ref["iters"]) <= slack, (res["iters"], ref["iters"])
    h = min(10, ref["iters"] - 1)
    bar = max(1e-12, 10.0 * sens)
    if h > 0:
        a, bb = np.array(res["alpha"][:h]), np.array(res["beta"][:h])
        assert np.max(np.abs(a - ref["alpha"][:h]) / np.abs(ref["alpha"][:h])) <= bar, (bar, sens)
        assert np.max(np.abs(bb - ref["beta"][:h]) / np.abs(ref["beta"][:h])) <= bar, (bar, sens)
    if res["iters"] == ref["iters"]:
        assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-7
        if not sensitive:
            assert abs(res["rel_res"] - ref["bound"] / ref["bnorm"]) <= 1e-6 * ref["bound"] / ref["bnorm"]
    assert res["rel_res"] <= rtol
    if A is not None:
        # Freund's bound holds for the GPU iterate itself: ||D^-1 (b - A x)|| <= sqrt(2i + 1) tau
        d = A.to_scipy().diagonal()
        true = np.linalg.norm((b - oracle.spmv(A, x)) / d)
        assert true <= res["rel_res"] * res["bnorm"] * (1 + 1e-6) + 1e-15 * res["bnorm"], (true, res)


def _systems():
    rng = np.random.default_rng(11)
    out = {}
    for name, A in (
        ("lap5_shift", laplace_2d_5pt(37, shift=0.05)),
        ("convdiff", convection_diffusion_2d(45, 0.6, -0.35, shift=0.02)),
        ("diff27", single_problem("c3", seed=2, size=13).A),
        ("lap7", single_problem("c2", seed=2, size=19).A),
    ):
        out[name] = (A, rhs_from_solution(A, rng.uniform(-1, 1, A.n)))
    return out


SYSTEMS = _systems()
_SENS = {}


def _sens(name, k):
    if (name, k) not in _SENS:
        A, b = SYSTEMS[name]
        _SENS[(name, k)] = _sensitivity(A, b, k, 10)
    return _SENS[(name, k)]


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k", [1, 3])
def test_tfqmr_parity(ctx, name, mode, k):
    A, b = SYSTEMS[name]
    ref = oracle.tfqmr(A, b, rtol=1e-8, check_every=k, hist_len=10)
    res, x = _solve(ctx, A, b, rtol=1e-8, check_every=k, mode=mode)
    _check(res, x, ref, k, sens=_sens(name, k), A=A, b=b)


@pytest.mark.parametrize("mode", MODES)
def test_tfqmr_edge_cases(ctx, mode):
    # zero right-hand side: converged before the first iteration, x untouched
    A = laplace_2d_5pt(9)
    res, x = _solve(ctx, A, np.zeros(A.n), mode=mode)
    assert res["reason"] == "converged" and res["iters"] == 0 and not x.any()
    # diagonal matrix and an eigenvector right-hand side: exact after the first half-step
    d = np.array([2.0, 3.0, 5.0, 7.0, 11.0, 13.0, 17.0])
    b = np.arange(1.0, 8.0)
    res, x = _solve(ctx, diagonal_csr(d), b, mode=mode, rtol=1e-14)
    assert res["reason"] == "converged" and res["iters"] == 1
    assert np.max(np.abs(x - b / d) / np.abs(b / d)) <= 1e-15
    N = 31
    v = sine_mode_2d(N, 3, 5)
    lam = 4 * np.sin(3 * np.pi / (2 * (N + 1))) ** 2 + 4 * np.sin(5 * np.pi / (2 * (N + 1))) ** 2
    res, x = _solve(ctx, laplace_2d_5pt(N), v, mode=mode, rtol=1e-12)
    assert res["reason"] == "converged" and res["iters"] == 1
    assert abs(res["alpha"][0] - 4.0 / lam) <= 1e-14 * 4.0 / lam
    assert np.max(np.abs(x - v / lam)) <= 1e-12 * np.max(np.abs(v / lam))
    # n = 1
    res, x = _solve(ctx, diagonal_csr(np.array([4.0])), np.array([3.0]), mode=mode)
    assert res["reason"] == "converged" and abs(x[0] - 0.75) < 1e-16
    # iteration cap: the same iterate as the oracle after max_it iterations
    A, b = SYSTEMS["convdiff"]
    ref = oracle.tfqmr(A, b, rtol=0.0, max_it=7, hist_len=7)
    res, x = _solve(ctx, A, b, mode=mode, rtol=0.0, max_it=7, hist=7)
    assert res["reason"] == "not_converged" and res["iters"] == 7
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-10


def test_tfqmr_bad_diagonal_is_an_error(ctx):
    A = CSR(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([2.0, 1.0]))
    with pytest.raises(apcg.ApcgError):
        _solve(ctx, A, np.ones(2))


def test_tfqmr_plan_reuse_and_async_graph_syncs(ctx):
    A, b = SYSTEMS["lap5_shift"]
    rowptr, col, val, bt = _t(A.rowptr), _t(A.col), _t(A.val), _t(b)
    M = apcg.mat_wrap(rowptr, col, val)
    x = torch.zeros_like(bt)
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    plan = apcg.tfqmr_plan_create(ctx, M, apcg.cg_opts(rtol=1e-8, check_every=5, mode="async_graph"))
    r1 = apcg.tfqmr_plan_solve(plan, vb, vx)
    x1 = x.cpu().numpy().copy()
    x.zero_()
    apcg.reset_counters()
    r2 = apcg.tfqmr_plan_solve(plan, vb, vx)
    c = apcg.get_counters()
    assert r1["iters"] == r2["iters"] and np.array_equal(x1, x.cpu().numpy())
    assert c["host_syncs"] <= 3 and c["graph_launches"] == 1
    apcg.call("apcg_tfqmr_plan_destroy", C.c_void_p(plan))
    for h, fn in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
        apcg.call(fn, C.c_void_p(h))


def test_tfqmr_persistent_selection(ctx):
    # AUTO runs a small system in one launch, and the result equals that of an explicit PERSISTENT plan
    A, b = SYSTEMS["convdiff"]
    ra, xa = _solve(ctx, A, b, rtol=1e-8, check_every=3, mode="auto")
    rp, xp = _solve(ctx, A, b, rtol=1e-8, check_every=3, mode="persistent")
    assert ra["kernel_launches"] == rp["kernel_launches"] == 1
    assert ra["iters"] == rp["iters"] and np.array_equal(xa, xp)
    # above 16384 rows AUTO falls back to the graph form and PERSISTENT is refused
    big = laplace_2d_5pt(130, shift=0.1)
    bb = rhs_from_solution(big, np.random.default_rng(5).uniform(-1, 1, big.n))
    r, _ = _solve(ctx, big, bb, rtol=1e-6, check_every=10, mode="auto")
    assert r["reason"] == "converged" and r["kernel_launches"] > 1
    with pytest.raises(apcg.ApcgError):
        _solve(ctx, big, bb, mode="persistent")


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_tfqmr_full_size(ctx, cfg):
    """The benchmark systems (64^2 5-point, 128^3 7-point) at rtol 1e-8."""
    p = single_problem(cfg, seed=0)
    k = 1 if cfg == "c1" else 10
    ref = oracle.tfqmr(p.A, p.b, rtol=1e-8, check_every=k, hist_len=10)
    for mode in ("async_graph", "persistent") if p.n <= 16384 else ("async_graph",):
        res, x = _solve(ctx, p.A, p.b, rtol=1e-8, check_every=k, mode=mode, max_it=20000)
        _check(res, x, ref, k, A=p.A, b=p.b)
