"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances (floating point): alpha/beta of the first 10 iterations within
1e-12 relative and the final x within 1e-7 relative of the oracle's x at rtol
1e-8 (the targets of the FP64 path); the iteration count equal up to one
check interval k (a convergence test that lands within rounding of the
threshold may flip).  The SpMV fuses each product into its row sum (one FMA
per nonzero) while the oracle rounds product and sum separately, so a row of
m terms may differ by the standard summation bound (m + 1) * 2u * sum|a_ij x_j|.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import (
    diagonal_csr,
    laplace_2d_5pt,
    random_spd_csr,
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
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    apcg.load()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx(dev):
    c = apcg.ctx_create()
    yield c
    apcg.call("apcg_ctx_destroy", C.c_void_p(c))


class Dev:
    """A CSR system resident on the GPU with its apcg views."""

    def __init__(self, A: CSR, b=None, x0=None, device="cuda:0"):
        self.A = A
        self.rowptr = torch.from_numpy(np.ascontiguousarray(A.rowptr)).to(device)
        self.col = torch.from_numpy(np.ascontiguousarray(A.col)).to(device)
        self.val = torch.from_numpy(np.ascontiguousarray(A.val)).to(device)
        self.mat = apcg.mat_wrap(self.rowptr, self.col, self.val)
        n = A.n
        self.b = torch.from_numpy(np.ascontiguousarray(b if b is not None else np.zeros(n))).to(device)
        self.x = torch.from_numpy(np.ascontiguousarray(x0 if x0 is not None else np.zeros(n))).to(device)
        self.vb = apcg.vec_wrap(self.b)
        self.vx = apcg.vec_wrap(self.x)

    def solve(self, ctx, **kw):
        opts = apcg.cg_opts(**kw)
        return apcg.cg_solve(ctx, self.mat, self.vb, self.vx, opts)

    def close(self):
        apcg.call("apcg_vec_destroy", C.c_void_p(self.vb))
        apcg.call("apcg_vec_destroy", C.c_void_p(self.vx))
        apcg.call("apcg_mat_destroy", C.c_void_p(self.mat))


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _oracle_x_at(A, b, ref, iters):
    """The oracle's iterate after exactly `iters` iterations: its converged x when it stopped there too,
    else a rerun without a tolerance and capped at that count (near the threshold rounding may move the
    stop by one test block, so the solutions are compared at the GPU's count)."""
    if ref["iters"] == iters:
        return ref["x"]
    return oracle.pcg(A, b, rtol=0.0, max_it=iters)["x"]


def _ragged_nonsym(n, rng):
    """Rows of very different lengths: empty rows, short rows, one long row."""
    lens = rng.integers(0, 12, n)
    lens[rng.integers(0, n, 3)] = 0
    lens[n // 3] = min(n, 900)  # spans several 256-entry chunks of a warp tile
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    col = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    val = rng.uniform(-2, 2, col.shape[0])
    return CSR(rowptr.astype(np.int32), col, val)


# ---------------------------------------------------------------- building blocks


@pytest.mark.parametrize("kind", ["lap5", "lap7", "diff27", "ragged", "ragged_tail"])
def test_spmv_bit_exact(dev, ctx, kind):
    rng = np.random.default_rng(1)
    if kind == "lap5":
        A = laplace_2d_5pt(45)
    elif kind == "lap7":
        A = single_problem("c2", size=21).A
    elif kind == "diff27":
        A = single_problem("c3", size=13).A
    elif kind == "ragged":
        A = _ragged_nonsym(2000, rng)
    else:
        A = _ragged_nonsym(33, rng)
    x = rng.standard_normal(A.n)
    d = Dev(A, x0=x)
    y = torch.empty(A.n, dtype=torch.float64, device=dev)
    vy = apcg.vec_wrap(y)
    apcg.call("apcg_mat_mult_async", C.c_void_p(ctx), C.c_void_p(d.mat), C.c_void_p(d.vx), C.c_void_p(vy))
    apcg.call("apcg_ctx_synchronize", C.c_void_p(ctx))
    m = np.diff(A.rowptr).astype(np.float64)
    bound = (m + 1) * 2 * np.finfo(float).eps * (abs(A.to_scipy()) @ np.abs(x))
    assert np.all(np.abs(y.cpu().numpy() - oracle.spmv(A, x)) <= bound)
    s = apcg.scalar_create()
    apcg.call("apcg_mat_mult_dot_async", C.c_void_p(ctx), C.c_void_p(d.mat), C.c_void_p(d.vx), C.c_void_p(vy), C.c_void_p(s))
    ref = oracle.dot(x, oracle.spmv(A, x))
    assert abs(apcg.scalar_get(s) - ref) <= 1e-13 * max(abs(ref), np.abs(x).sum())
    apcg.call("apcg_scalar_destroy", C.c_void_p(s))
    apcg.call("apcg_vec_destroy", C.c_void_p(vy))
    d.close()


@pytest.mark.parametrize("n", [0, 1, 2, 3, 257, 100_003, 3_000_001])
def test_dot_and_norm(dev, ctx, n):
    rng = np.random.default_rng(n)
    xh, yh = rng.standard_normal(n), rng.standard_normal(n)
    x = torch.from_numpy(xh).to(dev)
    y = torch.from_numpy(yh).to(dev)
    vx, vy = apcg.vec_wrap(x), apcg.vec_wrap(y)
    s = apcg.scalar_create()
    apcg.call("apcg_vec_dot_async", C.c_void_p(ctx), C.c_void_p(vx), C.c_void_p(vy), C.c_void_p(s))
    ref = oracle.dot(xh, yh)
    assert abs(apcg.scalar_get(s) - ref) <= 1e-14 * max(np.abs(xh * yh).sum(), 1e-300)
    apcg.call("apcg_vec_norm2_async", C.c_void_p(ctx), C.c_void_p(vx), C.c_void_p(s))
    ref = np.sqrt(oracle.dot(xh, xh))
    assert abs(apcg.scalar_get(s) - ref) <= 1e-14 * max(ref, 1e-300)
    # repeated launches are deterministic (fixed reduction order)
    vals = []
    for _ in range(3):
        apcg.call("apcg_vec_dot_async", C.c_void_p(ctx), C.c_void_p(vx), C.c_void_p(vy), C.c_void_p(s))
        vals.append(apcg.scalar_get(s))
    assert len(set(vals)) == 1
    for h in (vx, vy):
        apcg.call("apcg_vec_destroy", C.c_void_p(h))
    apcg.call("apcg_scalar_destroy", C.c_void_p(s))


def test_vector_updates(dev, ctx):
    rng = np.random.default_rng(4)
    n = 10_001
    xh, yh = rng.standard_normal(n), rng.standard_normal(n)
    x, y = torch.from_numpy(xh).to(dev), torch.from_numpy(yh.copy()).to(dev)
    vx, vy = apcg.vec_wrap(x), apcg.vec_wrap(y)
    a = apcg.scalar_create()
    apcg.call("apcg_scalar_set_async", C.c_void_p(ctx), C.c_void_p(a), 0.75)
    apcg.call("apcg_vec_axpy_async", C.c_void_p(ctx), C.c_void_p(vy), C.c_void_p(a), 1, C.c_void_p(vx))
    ref = yh - 0.75 * xh
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-15, atol=1e-15)
    apcg.call("apcg_vec_aypx_async", C.c_void_p(ctx), C.c_void_p(vy), C.c_void_p(a), C.c_void_p(vx))
    ref = xh + 0.75 * ref
    assert np.allclose(y.cpu().numpy(), ref, rtol=1e-15, atol=1e-15)
    before = y.cpu().numpy()  # the updates above may fuse a multiply-add: scale from the device values
    apcg.call("apcg_vec_scale_async", C.c_void_p(ctx), C.c_void_p(vy), C.c_void_p(a))
    assert np.array_equal(y.cpu().numpy(), before * 0.75)
    apcg.call("apcg_vec_pointwise_mult_async", C.c_void_p(ctx), C.c_void_p(vy), C.c_void_p(vx), C.c_void_p(vx))
    assert np.array_equal(y.cpu().numpy(), xh * xh)
    apcg.call("apcg_vec_copy_async", C.c_void_p(ctx), C.c_void_p(vy), C.c_void_p(vx))
    assert np.array_equal(y.cpu().numpy(), xh)
    apcg.call("apcg_vec_set_async", C.c_void_p(ctx), C.c_void_p(vy), C.c_double(-2.5))
    assert np.all(y.cpu().numpy() == -2.5)
    for h in (vx, vy):
        apcg.call("apcg_vec_destroy", C.c_void_p(h))
    apcg.call("apcg_scalar_destroy", C.c_void_p(a))


def test_normalize_listing_keeps_scalar_on_device(dev, ctx):
    """VecNormAsync -> Eval(1/alpha) -> VecScaleAsync with no device-to-host copy (Sec. 3.3)."""
    rng = np.random.default_rng(9)
    v = torch.from_numpy(rng.standard_normal(123_457)).to(dev)
    vv = apcg.vec_wrap(v)
    alpha = apcg.scalar_create()
    apcg.reset_counters()
    apcg.call("apcg_vec_norm2_async", C.c_void_p(ctx), C.c_void_p(vv), C.c_void_p(alpha))
    apcg.call("apcg_scalar_recip_async", C.c_void_p(ctx), C.c_void_p(alpha), C.c_void_p(alpha))
    apcg.call("apcg_vec_scale_async", C.c_void_p(ctx), C.c_void_p(vv), C.c_void_p(alpha))
    c = apcg.get_counters()
    assert c["d2h_copies"] == 0 and c["host_syncs"] == 0 and c["kernel_launches"] == 3
    s = apcg.scalar_create()
    apcg.call("apcg_vec_norm2_async", C.c_void_p(ctx), C.c_void_p(vv), C.c_void_p(s))
    assert abs(apcg.scalar_get(s) - 1.0) <= 1e-15
    for h in (alpha, s):
        apcg.call("apcg_scalar_destroy", C.c_void_p(h))
    apcg.call("apcg_vec_destroy", C.c_void_p(vv))


def test_jacobi_setup_and_apply(dev, ctx):
    rng = np.random.default_rng(2)
    A = random_spd_csr(500, 0.02, rng)
    d = Dev(A)
    dinv = torch.empty(A.n, dtype=torch.float64, device=dev)
    vd = apcg.vec_wrap(dinv)
    apcg.call("apcg_pc_jacobi_setup_async", C.c_void_p(ctx), C.c_void_p(d.mat), C.c_void_p(vd))
    apcg.call("apcg_ctx_synchronize", C.c_void_p(ctx))
    diag, _ = oracle.diagonal(A)
    assert np.array_equal(dinv.cpu().numpy(), 1.0 / diag)
    apcg.call("apcg_vec_destroy", C.c_void_p(vd))
    d.close()


# ---------------------------------------------------------------- CG parity


@pytest.mark.parametrize("mode", MODES)
def test_cg_c1_parity(dev, ctx, mode):
    p = single_problem("c1", seed=0)
    ref = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=1, hist_len=10)
    d = Dev(p.A, p.b)
    res = d.solve(ctx, rtol=1e-8, check_every=1, mode=mode, history_len=10)
    assert res["reason"] == "converged"
    assert res["iters"] == ref["iters"]
    assert np.max(np.abs(np.array(res["alpha"]) - ref["alpha"]) / np.abs(ref["alpha"])) <= 1e-12
    assert np.max(np.abs(np.array(res["beta"]) - ref["beta"]) / np.abs(ref["beta"])) <= 1e-12
    x = d.x.cpu().numpy()
    assert _rel(x, ref["x"]) <= 1e-7
    assert res["rel_res"] <= 1e-8
    d.close()


@pytest.mark.parametrize(
    "name,size,k",
    [("c1", 37, 1), ("c1", 61, 7), ("c2", 23, 10), ("c3", 15, 3), ("lap27", 11, 1), ("lap9", 30, 4)],
)
@pytest.mark.parametrize("mode", ["async", "async_graph", "persistent"])
def test_cg_parity_ragged_sizes(dev, ctx, name, size, k, mode):
    p = single_problem(name, seed=3, size=size)
    ref = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=k, hist_len=10)
    d = Dev(p.A, p.b)
    res = d.solve(ctx, rtol=1e-8, check_every=k, mode=mode, history_len=10)
    assert res["reason"] == "converged"
    assert abs(res["iters"] - ref["iters"]) <= k
    h = min(10, ref["iters"] - 1)
    assert np.max(np.abs(np.array(res["alpha"][:h]) - ref["alpha"][:h]) / np.abs(ref["alpha"][:h])) <= 1e-12
    assert np.max(np.abs(np.array(res["beta"][:h]) - ref["beta"][:h]) / np.abs(ref["beta"][:h])) <= 1e-12
    # x against the oracle's iterate at the GPU's own count (the counts may differ by a test block)
    assert _rel(d.x.cpu().numpy(), _oracle_x_at(p.A, p.b, ref, res["iters"])) <= 1e-7
    assert res["rel_res"] <= 1e-8
    d.close()


def test_cg_variable_diagonal_random_spd(dev, ctx):
    rng = np.random.default_rng(12)
    A = random_spd_csr(1001, 0.01, rng, dominance=0.2)
    xt = rng.uniform(-1, 1, A.n)
    b = rhs_from_solution(A, xt)
    ref = oracle.pcg(A, b, rtol=1e-10, hist_len=10)
    d = Dev(A, b)
    res = d.solve(ctx, rtol=1e-10, mode="async_graph", history_len=10)
    assert res["iters"] == ref["iters"]
    assert np.max(np.abs(np.array(res["alpha"]) - ref["alpha"]) / np.abs(ref["alpha"])) <= 1e-12
    assert _rel(d.x.cpu().numpy(), ref["x"]) <= 1e-9
    d.close()


@pytest.mark.parametrize("mode", MODES)
def test_cg_edge_cases(dev, ctx, mode):
    # zero right-hand side: converged before the first iteration
    A = laplace_2d_5pt(9)
    d = Dev(A, np.zeros(A.n))
    r = d.solve(ctx, mode=mode)
    assert r["iters"] == 0 and r["reason"] == "converged" and not d.x.any().item()
    d.close()
    # n = 1
    d = Dev(diagonal_csr(np.array([4.0])), np.array([2.0]))
    r = d.solve(ctx, mode=mode)
    assert r["iters"] == 1 and abs(d.x.item() - 0.5) < 1e-15
    d.close()
    # diagonal matrix: exact in one iteration (with k = 5 the first test comes at 5)
    rng = np.random.default_rng(0)
    dd = rng.uniform(0.5, 5.0, 777)
    b = rng.standard_normal(777)
    for k in (1, 5):
        d = Dev(diagonal_csr(dd), b)
        r = d.solve(ctx, mode=mode, rtol=1e-12, check_every=k)
        ref = oracle.pcg(diagonal_csr(dd), b, rtol=1e-12, check_every=k)
        assert r["reason"] == "converged" and r["iters"] == ref["iters"] == (1 if k == 1 else r["iters"])
        assert np.allclose(d.x.cpu().numpy(), b / dd, rtol=1e-14, atol=0)
        d.close()
    # fixed 20 iterations (rtol = 0), as in the paper's benchmark
    p = single_problem("c1", seed=1, size=32)
    ref = oracle.pcg(p.A, p.b, rtol=0.0, max_it=20)
    d = Dev(p.A, p.b)
    r = d.solve(ctx, mode=mode, rtol=0.0, max_it=20, check_every=3)
    assert r["iters"] == 20 and r["reason"] == "not_converged"
    assert _rel(d.x.cpu().numpy(), ref["x"]) <= 1e-12
    d.close()
    # nonzero initial guess
    x0 = rng.uniform(-1, 1, p.n)
    ref = oracle.pcg(p.A, p.b, x0=x0, rtol=1e-9)
    d = Dev(p.A, p.b, x0=x0)
    r = d.solve(ctx, mode=mode, rtol=1e-9)
    assert r["iters"] == ref["iters"] and _rel(d.x.cpu().numpy(), ref["x"]) <= 1e-8
    d.close()
    # indefinite matrix: breakdown is reported, not raised
    Ai = CSR(np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 3.0, 3.0, 1.0]))
    d = Dev(Ai, np.array([1.0, 0.0]))
    r = d.solve(ctx, mode=mode, rtol=1e-12)
    assert r["reason"] == "breakdown"
    d.close()


def test_cg_bad_diagonal_is_an_error(dev, ctx):
    A = CSR(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([2.0, 1.0]))
    d = Dev(A, np.ones(2))
    with pytest.raises(apcg.ApcgError) as e:
        d.solve(ctx)
    assert e.value.status == -4
    d.close()


def test_cg_eigenvector_rhs_full_size(dev, ctx):
    """A sine mode of the 128^3 7-point operator converges in one iteration with alpha = 6 / lambda."""
    import math

    N = 128
    p = single_problem("c2", seed=0)
    g = np.arange(1, N + 1)
    s = [np.sin(j * np.pi * g / (N + 1)) for j in (3, 5, 7)]
    v = (s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]).ravel()
    lam = sum(4 * math.sin(j * math.pi / (2 * (N + 1))) ** 2 for j in (3, 5, 7))
    d = Dev(p.A, v)
    r = d.solve(ctx, rtol=1e-9, check_every=1, mode="async_graph", history_len=1, max_it=50)
    assert r["iters"] == 1 and abs(r["alpha"][0] - 6.0 / lam) <= 1e-12 * 6.0 / lam
    assert np.max(np.abs(d.x.cpu().numpy() - v / lam)) <= 1e-9 * np.max(np.abs(v / lam))
    d.close()


def test_cg_c2_full_size_parity(dev, ctx):
    """The benchmark workload: 128^3 7-point, rtol 1e-8, k = 10, graph mode."""
    mode = "async_graph"
    p = single_problem("c2", seed=0)
    ref = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=10, hist_len=10)
    d = Dev(p.A, p.b)
    res = d.solve(ctx, rtol=1e-8, check_every=10, mode=mode, history_len=10, max_it=5000)
    assert res["reason"] == "converged"
    assert abs(res["iters"] - ref["iters"]) <= 10
    assert np.max(np.abs(np.array(res["alpha"]) - ref["alpha"]) / np.abs(ref["alpha"])) <= 1e-12
    assert np.max(np.abs(np.array(res["beta"]) - ref["beta"]) / np.abs(ref["beta"])) <= 1e-12
    assert _rel(d.x.cpu().numpy(), _oracle_x_at(p.A, p.b, ref, res["iters"])) <= 1e-7
    # true residual of the GPU solution
    x = d.x.cpu().numpy()
    assert np.linalg.norm(p.b - oracle.spmv(p.A, x)) / np.linalg.norm(p.b) <= 2e-8
    d.close()


def test_cg_host_buffers_entry_point(dev):
    p = single_problem("c1", seed=5, size=50)
    ref = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=2)
    x = np.zeros(p.n)
    res = apcg.cg_solve_host(p.A.rowptr, p.A.col, p.A.val, p.b, x, apcg.cg_opts(rtol=1e-8, check_every=2, mode="async_graph"))
    assert res["iters"] == ref["iters"] and _rel(x, ref["x"]) <= 1e-7


def test_plan_reuse_and_async_result(dev, ctx):
    p = single_problem("c2", seed=2, size=40)
    d = Dev(p.A, p.b)
    opts = apcg.cg_opts(rtol=1e-8, check_every=10, mode="async_graph")
    plan = apcg.cg_plan_create(ctx, d.mat, opts)
    ref = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=10)
    for _ in range(3):
        d.x.zero_()
        torch.cuda.synchronize()
        r = apcg.cg_plan_solve(plan, d.vb, d.vx)
        assert r["iters"] == ref["iters"] and _rel(d.x.cpu().numpy(), ref["x"]) <= 1e-7
    # enqueue without waiting, then collect
    d.x.zero_()
    torch.cuda.synchronize()
    apcg.call("apcg_cg_plan_solve_async", C.c_void_p(plan), C.c_void_p(d.vb), C.c_void_p(d.vx))
    res = apcg.CgResult()
    apcg.call("apcg_cg_plan_result", C.c_void_p(plan), C.byref(res))
    assert res.iters == ref["iters"]
    apcg.call("apcg_cg_plan_destroy", C.c_void_p(plan))
    d.close()


def test_async_modes_avoid_per_iteration_syncs(dev, ctx):
    p = single_problem("c1", seed=0, size=40)
    d = Dev(p.A, p.b)
    out = {}
    for mode in MODES:
        d.x.zero_()
        torch.cuda.synchronize()
        apcg.reset_counters()
        r = d.solve(ctx, rtol=1e-8, check_every=5, mode=mode)
        out[mode] = (r, apcg.get_counters())
    iters = out["host_sync"][0]["iters"]
    assert out["host_sync"][1]["host_syncs"] >= 2 * iters
    assert out["async"][1]["host_syncs"] <= iters // 5 + 4
    assert out["async_graph"][1]["host_syncs"] <= 3 and out["async_graph"][1]["graph_launches"] == 1
    assert out["persistent"][1]["host_syncs"] <= 3 and out["persistent"][0]["kernel_launches"] == 1
    d.close()
