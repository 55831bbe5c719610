"""Float32 parity of the refinement's inner solver against the float32 oracle.

Iterative refinement corrects its own errors, so a wrong row in the float32
SpMV or a wrong float32 scalar would only cost extra corrections; these tests
look at the float32 path itself:

* the plan's float32 inner SpMV (the very kernel instance the inner
  iterations launch: staged through shared memory, grouped, or one entry at a
  time, by layout), element by element against ``oracle.spmv_f32`` within
  the float32 summation bound (m+1) 2 u32 sum_j |a_ij x_j| (m entries in the
  row), and its (p, w) against the float64 dot of the oracle's product within
  D u32 sum |p_i w_i| plus the product's bound, D an upper bound on the depth
  of the GPU's float32 reduction;
* the inner alpha/beta of the first correction (whose right-hand side is
  fl32(b) for x0 = 0) against ``oracle.pcg_f32`` on the same float32 system,
  within max(4 D u32, 10 S), S the oracle's own largest relative change of
  those alpha/beta when fl32(b) is moved by one float32 ulp (three sign
  patterns) -- the float32 analogue of the TFQMR bar;
* the first correction's inner iteration count (within the test cadence k,
  plus one where S is large) and the number of corrections (within one) against
  the oracle's refinement;
* the refined x against the float64 oracle's PCG solution to the same
  tolerance.
"""

import ctypes as C
import math

import numpy as np
import pytest

import oracle
from synthetic import rhs_from_solution, single_problem
from synthetic.stencils import CSR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402

from test_gpu_layout import _case  # noqa: E402

V = C.c_void_p
U32 = 2.0**-24
K_INNER = 10


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


def _depth(n):
    """Upper bound on the number of sequential float32 additions behind any GPU reduction of n rows: a lane
    adds its rows of at most ceil(n / (32 * 8 * 152)) slices (grids hold at least one 8-warp block per SM
    or one warp per slice), then fixed block trees (8 + 5 levels), the partials of at most 4096 blocks
    (16 per lane) and a second block tree."""
    return math.ceil(n / (32 * 8 * 152)) + 13 + 16 + 13


class _Plan:
    """An IR plan built from the float64 CSR (its float32 copy is fl32 of the values), with history."""

    def __init__(self, ctx, A: CSR, b=None, hist=10, k=K_INNER, rtol=1e-10):
        self.keep = [_t(A.rowptr), _t(A.col), _t(A.val)]
        self.M = apcg.mat_wrap(*self.keep)
        self.opts = apcg.ir_opts(rtol=rtol, rtol_inner=1e-4, inner_check_every=k, history_len=hist)
        self.plan = apcg.ir_plan_create(ctx, self.M, None, self.opts)
        self.n = A.n

    def staged(self):
        return apcg.load().apcg_ir_plan_test_stall_copies(V(self.plan), 0) == 0

    def spmv(self, p32):
        p = _t(p32)
        w = torch.empty_like(p)
        vp, vw = apcg.vec_wrap(p), apcg.vec_wrap(w)
        g = apcg.ir_plan_inner_spmv(self.plan, vp, vw)
        for h in (vp, vw):
            apcg.call("apcg_vec_destroy", V(h))
        return w.cpu().numpy(), g

    def solve(self, b):
        bt = _t(b)
        x = torch.zeros_like(bt)
        vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
        res = apcg.ir_plan_solve(self.plan, vb, vx)
        res.update(apcg.ir_history(self.opts))
        for h in (vb, vx):
            apcg.call("apcg_vec_destroy", V(h))
        return res, x.cpu().numpy()

    def close(self):
        apcg.call("apcg_ir_plan_destroy", V(self.plan))
        apcg.call("apcg_mat_destroy", V(self.M))


def _check_spmv(A: CSR, pl: _Plan, rng):
    v32 = A.val.astype(np.float32)
    for scale in (1.0, 1e-3):
        p32 = (scale * rng.uniform(-1, 1, A.n)).astype(np.float32)
        w, g = pl.spmv(p32)
        assert w.dtype == np.float32
        ref = oracle.spmv_f32(A, p32)
        absA = CSR(A.rowptr, A.col, np.abs(v32.astype(np.float64))).to_scipy()
        m = np.diff(A.rowptr)
        bound = (m + 1) * 2 * U32 * (absA @ np.abs(p32.astype(np.float64)))
        diff = np.abs(w.astype(np.float64) - ref.astype(np.float64))
        bad = np.nonzero(diff > bound)[0]
        assert bad.size == 0, (bad[:10], diff[bad[:10]], bound[bad[:10]])
        pw = p32.astype(np.float64) * ref.astype(np.float64)
        g_ref = float(np.sum(pw))
        g_bound = _depth(A.n) * U32 * float(np.sum(np.abs(pw))) + float(np.abs(p32.astype(np.float64)) @ (2 * bound))
        assert abs(g - g_ref) <= g_bound, (g, g_ref, g_bound)


def _sensitivity32(A: CSR, b32, k, h):
    """Largest relative change of the float32 oracle's first h alpha/beta under one-ulp moves of b32."""
    ref = oracle.pcg_f32(A, b32, rtol=1e-4, check_every=k, hist_len=h)
    worst = 0.0
    for t in range(3):
        sign = np.random.default_rng(1000 + t).choice([-1.0, 1.0], b32.size).astype(np.float32)
        o = oracle.pcg_f32(A, (b32 + sign * np.spacing(b32)).astype(np.float32), rtol=1e-4, check_every=k, hist_len=h)
        for key in ("alpha", "beta"):
            worst = max(worst, float(np.nanmax(np.abs(o[key] - ref[key]) / np.abs(ref[key]))))
    return worst, ref


def _check_first_correction(A: CSR, b, res, k=K_INNER, h=10):
    b32 = b.astype(np.float32)  # r = b - A 0 = b exactly, rounded to float32
    S, ref = _sensitivity32(A, b32, k, h)
    assert ref["reason"] == "converged"
    slack = (k - 1) + (1 if S > 1e-6 else 0)
    assert abs(res["inner_first"] - ref["iters"]) <= slack, (res["inner_first"], ref["iters"], S)
    hh = min(h, ref["iters"] - 1, res["inner_first"] - 1)
    assert hh >= 3
    bar = max(4 * _depth(A.n) * U32, 10 * S)
    for key in ("alpha", "beta"):
        g = np.array(res[key][:hh])
        r = ref[key][:hh]
        err = float(np.max(np.abs(g - r) / np.abs(r)))
        assert err <= bar, (key, err, bar, S)
        # the recorded scalars are float32 values
        assert np.all(g.astype(np.float32).astype(np.float64) == g)
    return S


CASES = ["diff27_13", "mixed_width", "lap7_21", "lap5_48", "far", "one_row"]


@pytest.mark.parametrize("name", CASES)
def test_inner_spmv_matches_float32_oracle(ctx, name):
    A, _ = _case(name)
    pl = _Plan(ctx, A)
    try:
        if name == "diff27_13":
            assert pl.staged()  # 27-entry rows with offset lists: values staged in shared memory
        if name == "far":
            assert not pl.staged()
        _check_spmv(A, pl, np.random.default_rng(11))
    finally:
        pl.close()


@pytest.mark.parametrize("name", ["diff27_13", "mixed_width", "lap7_21", "lap5_48", "far"])
def test_first_correction_matches_float32_oracle(ctx, name):
    A, _ = _case(name)
    b = rhs_from_solution(A, np.random.default_rng(3).uniform(-1, 1, A.n))
    pl = _Plan(ctx, A)
    try:
        res, x = pl.solve(b)
    finally:
        pl.close()
    assert res["reason"] == "converged"
    _check_first_correction(A, b, res)
    ref = oracle.ir(A, b, rtol=1e-10, inner_check_every=K_INNER)
    assert ref["reason"] == "converged"
    assert abs(res["outer"] - ref["outer"]) <= 1, (res["outer"], ref["outer"])
    true_rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert true_rel <= 1.05e-10


def test_refinement_matches_float64_oracle_80cube(ctx):
    """80^3 variable-coefficient 27-point (512,000 rows, 13.5 M nonzeros): the refined x against the float64
    oracle's PCG solution to the same tolerance, the first correction against the float32 oracle, and the
    number of corrections against the oracle's refinement."""
    p = single_problem("c3", seed=0, size=80)
    pl = _Plan(ctx, p.A)
    try:
        assert pl.staged()
        res, x = pl.solve(p.b)
    finally:
        pl.close()
    assert res["reason"] == "converged"
    ref64 = oracle.pcg(p.A, p.b, rtol=1e-10, check_every=10)
    assert ref64["reason"] == "converged"
    assert np.linalg.norm(x - ref64["x"]) / np.linalg.norm(ref64["x"]) <= 1e-7
    ir = oracle.ir(p.A, p.b, rtol=1e-10, inner_check_every=K_INNER)
    assert abs(res["outer"] - ir["outer"]) <= 1, (res["outer"], ir["outer"])
    _check_first_correction(p.A, p.b, res)


def test_inner_path_full_size_160cube(ctx):
    """The 160^3 system of the refinement benchmark at full size: the staged float32 SpMV element by element
    against the float32 oracle, and the first correction's inner alpha/beta and count."""
    p = single_problem("c3", seed=0)
    pl = _Plan(ctx, p.A)
    try:
        assert pl.staged()
        _check_spmv(p.A, pl, np.random.default_rng(12))
        res, x = pl.solve(p.b)
    finally:
        pl.close()
    assert res["reason"] == "converged"
    _check_first_correction(p.A, p.b, res)
    true_rel = np.linalg.norm(p.b - oracle.spmv(p.A, x)) / np.linalg.norm(p.b)
    assert true_rel <= 1.05e-10


def test_inner_spmv_rejects_bad_vectors(ctx):
    A, _ = _case("lap7_21")
    pl = _Plan(ctx, A)
    try:
        p64 = torch.zeros(A.n, dtype=torch.float64, device="cuda:0")
        w32 = torch.zeros(A.n, dtype=torch.float32, device="cuda:0")
        short = torch.zeros(A.n - 1, dtype=torch.float32, device="cuda:0")
        for p, w in ((p64, w32), (short, w32), (w32, w32)):
            vp, vw = apcg.vec_wrap(p), apcg.vec_wrap(w)
            st = apcg.load().apcg_ir_plan_inner_spmv(V(pl.plan), V(vp), V(vw), None)
            assert st == -1  # APCG_ERR_INVALID_ARG
            for h in {vp, vw}:
                apcg.call("apcg_vec_destroy", V(h))
    finally:
        pl.close()
