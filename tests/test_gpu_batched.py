"""Batched Jacobi-PCG (one cluster per system) against the oracle, per system.

Each system of a batch is compared with the oracle's solve of that system
alone: iteration count within one check interval, x within 1e-7 relative at
rtol 1e-8, and the reported relative residual below the tolerance.  At the
full batch sizes every system's true residual is checked, and a sample of
systems (largest, smallest, random) is compared with the oracle one by one.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import batch_aniso_7pt, batch_shifted_5pt
from synthetic.problems import Batch, _concat
from synthetic.stencils import CSR, diagonal_csr, laplace_2d_5pt, rhs_from_solution

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


def _dev(B: Batch, x0=None):
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    x = t(np.zeros(B.n_total) if x0 is None else x0)
    return t(B.rowptr), t(B.col), t(B.val), t(B.b), x


H = 10  # alpha/beta of the first H iterations of every system are recorded and compared


def _solve(ctx, B, rtol=1e-8, k=1, tune=False, max_it=0, hist=H):
    rowptr, col, val, b, x = _dev(B)
    opts = apcg.cg_opts(rtol=rtol, check_every=k, max_it=max_it, history_len=hist)
    plan = apcg.batch_plan_create(ctx, B.sys_row_off, rowptr, col, val, opts)
    table = apcg.batch_plan_tune(plan, b) if tune else None
    res = apcg.batch_plan_solve(plan, b, x, B.nsys)
    if hist:
        for s in range(B.nsys):
            res[s].update(apcg.batch_plan_history(plan, s, hist))
    apcg.call("apcg_batch_plan_destroy", C.c_void_p(plan))
    return res, x.cpu().numpy(), table


def _check_system(B, s, res_s, xg, rtol, k):
    """One system of a batch against the oracle: reason, count within the test cadence, alpha/beta of the
    first iterations within 1e-12 relative, and x within 1e-7 of the oracle's iterate at the GPU's count."""
    A, b, _ = B.system(s)
    r0, r1 = int(B.sys_row_off[s]), int(B.sys_row_off[s + 1])
    ref = oracle.pcg(A, b, rtol=rtol, check_every=k, hist_len=H)
    assert res_s["reason"] == ref["reason"] == "converged", (s, res_s, ref["reason"])
    assert abs(res_s["iters"] - ref["iters"]) <= k, (s, res_s["iters"], ref["iters"])
    assert res_s["rel_res"] <= rtol
    if "alpha" in res_s:
        h = min(H, ref["iters"] - 1, res_s["iters"] - 1)
        for key in ("alpha", "beta"):
            g = np.array(res_s[key][:h])
            err = float(np.max(np.abs(g - ref[key][:h]) / np.abs(ref[key][:h]))) if h > 0 else 0.0
            assert err <= 1e-12, (s, key, err)
    x_ref = ref["x"] if res_s["iters"] == ref["iters"] else oracle.pcg(A, b, rtol=0.0, max_it=res_s["iters"])["x"]
    err = np.linalg.norm(xg[r0:r1] - x_ref) / np.linalg.norm(x_ref)
    assert err <= 1e-7, (s, err)


@pytest.mark.parametrize("k", [1, 4])
def test_batched_shifted_small(ctx, k):
    B = batch_shifted_5pt(24, seed=3, side_lo=8, side_hi=60)
    res, xg, _ = _solve(ctx, B, k=k)
    for s in range(B.nsys):
        _check_system(B, s, res[s], xg, 1e-8, k)


def test_batched_aniso_small(ctx):
    B = batch_aniso_7pt(16, seed=5, side_lo=4, side_hi=22)
    res, xg, _ = _solve(ctx, B, k=2)
    for s in range(B.nsys):
        _check_system(B, s, res[s], xg, 1e-8, 2)


def test_batched_edge_cases(ctx):
    rng = np.random.default_rng(1)
    systems = []
    A1 = diagonal_csr(np.array([3.0]))
    systems.append((A1, np.array([6.0]), np.array([2.0])))  # n = 1
    A2 = laplace_2d_5pt(7)
    systems.append((A2, np.zeros(A2.n), np.zeros(A2.n)))  # zero right-hand side
    A3 = CSR(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([2.0, 1.0]))
    systems.append((A3, np.ones(2), np.zeros(2)))  # missing diagonal entry
    A4 = laplace_2d_5pt(33, shift=0.5)  # 1089 rows: ragged against every cluster shape
    xt = rng.uniform(-1, 1, A4.n)
    systems.append((A4, rhs_from_solution(A4, xt), xt))
    B = _concat("edge", systems, {})
    res, xg, _ = _solve(ctx, B)
    assert res[0]["reason"] == "converged" and res[0]["iters"] == 1 and abs(xg[0] - 2.0) < 1e-15
    assert res[1]["reason"] == "converged" and res[1]["iters"] == 0
    assert res[2]["reason"] == "bad_diagonal"
    _check_system(B, 3, res[3], xg, 1e-8, 1)


def test_batched_fixed_iterations_match_oracle(ctx):
    B = batch_shifted_5pt(10, seed=8, side_lo=20, side_hi=90)
    res, xg, _ = _solve(ctx, B, rtol=0.0, max_it=20)
    for s in range(B.nsys):
        A, b, _ = B.system(s)
        ref = oracle.pcg(A, b, rtol=0.0, max_it=20)
        r0, r1 = int(B.sys_row_off[s]), int(B.sys_row_off[s + 1])
        assert res[s]["iters"] == 20 and res[s]["reason"] == "not_converged"
        assert np.linalg.norm(xg[r0:r1] - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-12


def test_batched_autotuner_keeps_results(ctx):
    B = batch_shifted_5pt(40, seed=11, side_lo=16, side_hi=128)
    res, xg, table = _solve(ctx, B, tune=True)
    assert table and all(r["ms"] > 0 for r in table)
    assert all(r["cluster"] in (1, 2, 4, 8, 16) for r in table)
    for s in (0, 7, 39):
        _check_system(B, s, res[s], xg, 1e-8, 1)


def test_batched_full_size_shifted(ctx):
    """1024 systems, sides 16..128 (6.4 M rows): every residual, and a sample against the oracle."""
    B = batch_shifted_5pt(1024, seed=0)
    res, xg, _ = _solve(ctx, B)
    assert all(r["reason"] == "converged" and r["rel_res"] <= 1e-8 for r in res)
    for s in range(B.nsys):
        A, b, _ = B.system(s)
        r0, r1 = int(B.sys_row_off[s]), int(B.sys_row_off[s + 1])
        tr = np.linalg.norm(b - oracle.spmv(A, xg[r0:r1])) / np.linalg.norm(b)
        assert tr <= 2e-8, (s, tr)
    sizes = np.diff(B.sys_row_off)
    sample = {int(np.argmax(sizes)), int(np.argmin(sizes))} | set(np.random.default_rng(0).choice(B.nsys, 6, replace=False).tolist())
    for s in sorted(sample):
        _check_system(B, s, res[s], xg, 1e-8, 1)
