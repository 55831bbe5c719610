"""Mixed-precision iterative refinement (float32 inner PCG, float64 outer) on the GPU.

Parity for the refinement's iteration counts is unpinned (no closed form);
what is checked is what the method guarantees: the float64 true residual of
the result meets the outer tolerance, and the result agrees with the float64
solution (dense Cholesky on small systems, the float64 CG at full size)
within the conditioning bound.  The oracle's own refinement reaches the same
tolerance on the same systems.
"""

import ctypes as C

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from synthetic import aniso_3d_7pt_fp32exact, diffusion_3d_27pt, rhs_from_solution, single_problem
from synthetic.stencils import CSR

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


def _ir(ctx, A: CSR, b, use64=True, use32=False, val32=None, **kw):
    rowptr, col = _t(A.rowptr), _t(A.col)
    v64 = _t(A.val)
    v32 = _t(np.asarray(A.val if val32 is None else val32, dtype=np.float32))
    A64 = apcg.mat_wrap(rowptr, col, v64) if use64 else None
    A32 = apcg.mat_wrap(rowptr, col, v32) if use32 else None
    bt = _t(b)
    x = torch.zeros_like(bt)
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    plan = apcg.ir_plan_create(ctx, A64, A32, apcg.ir_opts(**kw))
    res = apcg.ir_plan_solve(plan, vb, vx)
    apcg.call("apcg_ir_plan_destroy", C.c_void_p(plan))
    for h in (vb, vx):
        apcg.call("apcg_vec_destroy", C.c_void_p(h))
    for h in (A64, A32):
        if h:
            apcg.call("apcg_mat_destroy", C.c_void_p(h))
    return res, x.cpu().numpy()


@pytest.mark.parametrize("mode", ["a64_only", "a32_only_exact", "both"])
def test_ir_small_systems_reach_double_accuracy(ctx, mode):
    rng = np.random.default_rng(17)
    if mode == "a32_only_exact":
        A = aniso_3d_7pt_fp32exact(12, 9, 11, 1.0, 300.0, 4.0)
    else:
        A = diffusion_3d_27pt(11, 10.0 ** rng.uniform(-2, 2, 11**3))
    xt = rng.uniform(-1, 1, A.n)
    b = rhs_from_solution(A, xt)
    res, x = _ir(ctx, A, b, use64=(mode != "a32_only_exact"), use32=(mode != "a64_only"), rtol=1e-10)
    assert res["reason"] == "converged" and res["outer"] >= 2
    true_rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert true_rel <= 1.05e-10 and abs(true_rel - res["rel_res"]) <= 1e-12
    Ad = A.to_dense()
    xc = sla.cho_solve(sla.cho_factor(Ad), b)
    kappa = np.linalg.cond(Ad)
    assert np.linalg.norm(x - xc) / np.linalg.norm(xc) <= kappa * 2e-10
    ref = oracle.ir(A, b, rtol=1e-10)
    assert ref["reason"] == "converged"


def test_ir_zero_rhs_and_fixed_caps(ctx):
    A = aniso_3d_7pt_fp32exact(6, 6, 6, 1.0, 10.0, 100.0)
    res, x = _ir(ctx, A, np.zeros(A.n), rtol=1e-10)
    assert res["reason"] == "converged" and res["outer"] == 0 and not x.any()
    rng = np.random.default_rng(2)
    b = rhs_from_solution(A, rng.uniform(-1, 1, A.n))
    res, _ = _ir(ctx, A, b, rtol=1e-14, max_outer=2, max_inner=5)
    assert res["reason"] == "not_converged" and res["outer"] == 2 and res["inner_total"] <= 10


def test_ir_full_size_27pt_matches_float64_cg(ctx):
    """160^3 variable-coefficient 27-point: refinement to 1e-10 against float64 CG to 1e-10."""
    p = single_problem("c3", seed=0)
    res, x_ir = _ir(ctx, p.A, p.b, rtol=1e-10)
    assert res["reason"] == "converged"
    rel_ir = np.linalg.norm(p.b - oracle.spmv(p.A, x_ir)) / np.linalg.norm(p.b)
    assert rel_ir <= 1.05e-10
    # float64 CG on the same system
    rowptr, col, val, b = _t(p.A.rowptr), _t(p.A.col), _t(p.A.val), _t(p.b)
    x = torch.zeros_like(b)
    A = apcg.mat_wrap(rowptr, col, val)
    vb, vx = apcg.vec_wrap(b), apcg.vec_wrap(x)
    r64 = apcg.cg_solve(ctx, A, vb, vx, apcg.cg_opts(rtol=1e-10, check_every=10, mode="async_graph", max_it=20000))
    assert r64["reason"] == "converged"
    x64 = x.cpu().numpy()
    rel_64 = np.linalg.norm(p.b - oracle.spmv(p.A, x64)) / np.linalg.norm(p.b)
    assert rel_64 <= 2e-10
    # both are within the conditioning bound of the same solution
    assert np.linalg.norm(x_ir - x64) / np.linalg.norm(x64) <= 1e-6
    for h, fn in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (A, "apcg_mat_destroy")):
        apcg.call(fn, C.c_void_p(h))
