"""Batched mixed-precision refinement (one cluster per system) on the GPU.

Each system is refined to rtol 1e-10 with float32 inner Jacobi-PCG solves
(Sec. 3.3's CG) and float64 residuals and updates.  Iteration counts of the
refinement are not pinned (no closed form); the checks are what the method
guarantees: the float64 true residual b - A x of every system meets the
tolerance and equals the residual the kernel reports, and x agrees with the
float64 solution (dense Cholesky on small systems, the float64 oracle CG on the
identical float32-exact matrix at full size) within the conditioning bound.
"""

import ctypes as C

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from synthetic import batch_aniso_7pt
from synthetic.problems import Batch, _concat
from synthetic.stencils import CSR, aniso_3d_7pt_fp32exact, diagonal_csr, diffusion_3d_27pt, rhs_from_solution

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


def _solve(ctx, B: Batch, use64=False, use32=True, tune=False, **kw):
    rowptr, col, b = _t(B.rowptr), _t(B.col), _t(B.b)
    v64 = _t(B.val) if use64 else None
    v32 = _t(B.val.astype(np.float32)) if use32 else None
    x = torch.zeros(B.n_total, dtype=torch.float64, device="cuda:0")
    opts = apcg.ir_opts(**{"rtol": 1e-10, "rtol_inner": 1e-4, "inner_check_every": 1, **kw})
    plan = apcg.batch_ir_plan_create(ctx, B.sys_row_off, rowptr, col, v64, v32, opts)
    table = apcg.batch_plan_tune(plan, b) if tune else None
    res = apcg.batch_plan_solve(plan, b, x, B.nsys)
    apcg.call("apcg_batch_plan_destroy", C.c_void_p(plan))
    return res, x.cpu().numpy(), table


def _true_rel(A: CSR, b, x):
    bn = np.linalg.norm(b)
    r = np.linalg.norm(b - oracle.spmv(A, x))
    return r / bn if bn > 0 else r


def _check_small(B: Batch, s, res_s, xg, rtol=1e-10):
    A, b, _ = B.system(s)
    r0, r1 = int(B.sys_row_off[s]), int(B.sys_row_off[s + 1])
    x = xg[r0:r1]
    assert res_s["reason"] == "converged", (s, res_s)
    tr = _true_rel(A, b, x)
    assert tr <= rtol * 1.05 and abs(tr - res_s["rel_res"]) <= 1e-12, (s, tr, res_s)
    Ad = A.to_dense()
    xc = sla.cho_solve(sla.cho_factor(Ad), b)
    kappa = np.linalg.cond(Ad)
    assert np.linalg.norm(x - xc) / np.linalg.norm(xc) <= kappa * 2 * rtol, (s, kappa)
    ref = oracle.ir(A, b, rtol=rtol)
    assert ref["reason"] == "converged"
    assert abs(ref["outer"] - res_s["outer"]) <= 1, (s, ref["outer"], res_s["outer"])


@pytest.mark.parametrize("vals", ["f32_only_exact", "f64_only", "both"])
def test_batched_ir_small_aniso(ctx, vals):
    B = batch_aniso_7pt(12, seed=21, side_lo=4, side_hi=13)
    res, xg, _ = _solve(ctx, B, use64=(vals != "f32_only_exact"), use32=(vals != "f64_only"))
    for s in range(B.nsys):
        _check_small(B, s, res[s], xg)
        assert res[s]["outer"] >= 1 and res[s]["iters"] >= res[s]["outer"]


def test_batched_ir_rounded_values(ctx):
    """27-point variable coefficients (not float32-exact): float64 residual, float32 copy made in the kernel."""
    rng = np.random.default_rng(4)
    systems = []
    for m in (5, 8, 11, 9):
        A = diffusion_3d_27pt(m, 10.0 ** rng.uniform(-2, 2, m**3))
        xt = rng.uniform(-1, 1, A.n)
        systems.append((A, rhs_from_solution(A, xt), xt))
    B = _concat("diff27", systems, {})
    for use32 in (False, True):
        res, xg, _ = _solve(ctx, B, use64=True, use32=use32)
        for s in range(B.nsys):
            _check_small(B, s, res[s], xg)


def test_batched_ir_edge_cases(ctx):
    rng = np.random.default_rng(6)
    systems = []
    systems.append((diagonal_csr(np.array([4.0])), np.array([2.0]), np.array([0.5])))  # n = 1
    A1 = aniso_3d_7pt_fp32exact(5, 4, 3, 1.0, 10.0, 100.0)
    systems.append((A1, np.zeros(A1.n), np.zeros(A1.n)))  # zero right-hand side
    A2 = CSR(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([2.0, 1.0]))
    systems.append((A2, np.ones(2), np.zeros(2)))  # missing diagonal entry
    A3 = aniso_3d_7pt_fp32exact(11, 10, 9, 1.0, 3.0, 70.0)  # 990 rows: ragged against every cluster shape
    xt = rng.uniform(-1, 1, A3.n)
    systems.append((A3, rhs_from_solution(A3, xt), xt))
    A4 = CSR(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))  # empty system
    systems.append((A4, np.zeros(0), np.zeros(0)))
    B = _concat("edge", systems, {})
    res, xg, _ = _solve(ctx, B)
    assert res[0]["reason"] == "converged" and res[0]["outer"] == 1 and abs(xg[0] - 0.5) < 1e-15
    assert res[1]["reason"] == "converged" and res[1]["outer"] == 0 and res[1]["iters"] == 0
    r1 = slice(int(B.sys_row_off[1]), int(B.sys_row_off[2]))
    assert not xg[r1].any()
    assert res[2]["reason"] == "bad_diagonal"
    _check_small(B, 3, res[3], xg)
    assert res[4]["reason"] == "converged" and res[4]["outer"] == 0


def test_batched_ir_caps(ctx):
    B = batch_aniso_7pt(5, seed=9, side_lo=6, side_hi=12)
    res, _, _ = _solve(ctx, B, rtol=1e-14, max_outer=2, max_inner=5)
    for r in res:
        assert r["reason"] == "not_converged" and r["outer"] == 2 and r["iters"] <= 10


def test_batched_ir_autotuner_keeps_results(ctx):
    B = batch_aniso_7pt(30, seed=13, side_lo=6, side_hi=24)
    res, xg, table = _solve(ctx, B, tune=True, inner_check_every=4)
    assert table and all(r["ms"] > 0 and r["cluster"] in (1, 2, 4, 8, 16) for r in table)
    for s in range(B.nsys):
        A, b, _ = B.system(s)
        r0, r1 = int(B.sys_row_off[s]), int(B.sys_row_off[s + 1])
        assert res[s]["reason"] == "converged"
        assert _true_rel(A, b, xg[r0:r1]) <= 1.05e-10


def test_batched_ir_full_size(ctx):
    """4096 anisotropic 7-point systems, sides 8..32, float32-exact (32.5 M rows): every residual,
    and a sample against the float64 oracle CG on the identical matrix."""
    B = batch_aniso_7pt(4096, seed=0)
    res, xg, _ = _solve(ctx, B, inner_check_every=4)
    assert all(r["reason"] == "converged" and r["rel_res"] <= 1e-10 for r in res)
    sizes = np.diff(B.sys_row_off)
    rng = np.random.default_rng(0)
    sample = {int(np.argmax(sizes)), int(np.argmin(sizes))} | set(rng.choice(B.nsys, 6, replace=False).tolist())
    for s in sorted(sample):
        A, b, _ = B.system(s)
        r0, r1 = int(B.sys_row_off[s]), int(B.sys_row_off[s + 1])
        x = xg[r0:r1]
        tr = _true_rel(A, b, x)
        assert tr <= 1.05e-10 and abs(tr - res[s]["rel_res"]) <= 1e-12, (s, tr, res[s])
        ref = oracle.pcg(A, b, rtol=1e-12, max_it=20 * A.n)
        assert ref["reason"] == "converged"
        # Dirichlet a_x L_x + a_y L_y + a_z L_z (+ a tiny diagonal shift) has
        # kappa <= 1 / sin^2(pi / (2 (m + 1))), m the longest side, whatever the a_d;
        # both residuals are below 1e-10 ||b||, so the two solutions differ by kappa * 1.01e-10 at most
        m = int(B.meta["sides"][s].max())
        kappa = 1.0 / np.sin(np.pi / (2 * (m + 1))) ** 2
        err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= 1.1 * kappa * 1.01e-10, (s, err, kappa)
