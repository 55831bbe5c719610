"""Failure detection with faults injected on the host (nothing faults, traps or hangs the GPU).

A NaN or infinity in the right-hand side or the start vector must end every
solver and mode with a reported breakdown (not a hang, not a CUDA error), a
NaN system inside a batch must fail alone, bad arguments must be rejected
before anything is enqueued, and the context must stay usable for the next
solve.  The only device-side waits are those of the refinement's staged
float32 SpMV on its bulk copies (mbarriers), each bounded by polls and time; a
test hook makes every one of them run out, without any fault, and the solve
must report the timeout.
"""

import ctypes as C

import numpy as np
import pytest

from synthetic import batch_aniso_7pt, batch_shifted_5pt, laplace_2d_5pt, rhs_from_solution, stencil_terms

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


def _system(N=30):
    A = laplace_2d_5pt(N, shift=0.1)
    b = rhs_from_solution(A, np.random.default_rng(1).uniform(-1, 1, A.n))
    return A, b


def _cg(ctx, A, b, x0=None, solver="cg", **kw):
    rowptr, col, val, bt = _t(A.rowptr), _t(A.col), _t(A.val), _t(b)
    x = _t(np.zeros(A.n) if x0 is None else x0)
    M = apcg.mat_wrap(rowptr, col, val)
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    try:
        fn = apcg.cg_solve if solver == "cg" else apcg.tfqmr_solve
        return fn(ctx, M, vb, vx, apcg.cg_opts(**kw)), x.cpu().numpy()
    finally:
        for h, f in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
            apcg.call(f, V(h))


@pytest.mark.parametrize("mode", ["host_sync", "async", "async_graph", "persistent"])
@pytest.mark.parametrize("where", ["b_nan", "b_inf", "x0_nan"])
def test_cg_reports_breakdown_on_non_finite_input(ctx, mode, where):
    A, b = _system()
    x0 = None
    if where == "b_nan":
        b = b.copy()
        b[17] = np.nan
    elif where == "b_inf":
        b = b.copy()
        b[3] = np.inf
    else:
        x0 = np.zeros(A.n)
        x0[5] = np.nan
    res, _ = _cg(ctx, A, b, x0=x0, mode=mode, rtol=1e-8, max_it=500)
    assert res["reason"] == "breakdown" and res["iters"] <= 1, res
    # the context is still usable
    A2, b2 = _system(12)
    ok, _ = _cg(ctx, A2, b2, mode=mode, rtol=1e-8)
    assert ok["reason"] == "converged"


@pytest.mark.parametrize("mode", ["host_sync", "async_graph", "persistent"])
def test_tfqmr_reports_breakdown_on_nan(ctx, mode):
    A, b = _system()
    b = b.copy()
    b[0] = np.nan
    res, _ = _cg(ctx, A, b, solver="tfqmr", mode=mode, rtol=1e-8, max_it=500)
    assert res["reason"] == "breakdown"
    ok, _ = _cg(ctx, *_system(12), solver="tfqmr", mode=mode, rtol=1e-8)
    assert ok["reason"] == "converged"


def test_stencil_cg_reports_breakdown_on_nan(ctx):
    dims = (20, 20, 1)
    offs, w = stencil_terms("5pt", dims)
    S = apcg.stencil_create(dims, offs, w)
    plan = apcg.cg_plan_create_stencil(ctx, S, apcg.cg_opts(rtol=1e-8, mode="async_graph", max_it=300))
    apcg.call("apcg_stencil_destroy", V(S))
    b = np.ones(400)
    b[7] = np.nan
    bt, x = _t(b), torch.zeros(400, dtype=torch.float64, device="cuda:0")
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    res = apcg.cg_plan_solve(plan, vb, vx)
    assert res["reason"] == "breakdown"
    apcg.call("apcg_cg_plan_destroy", V(plan))
    for h in (vb, vx):
        apcg.call("apcg_vec_destroy", V(h))


@pytest.mark.parametrize("ir", [False, True])
def test_batched_nan_system_fails_alone(ctx, ir):
    B = batch_aniso_7pt(9, seed=3, side_lo=4, side_hi=10) if ir else batch_shifted_5pt(9, seed=3, side_lo=8, side_hi=30)
    b = B.b.copy()
    bad = 4
    b[int(B.sys_row_off[bad]) + 2] = np.nan
    rowptr, col, bt = _t(B.rowptr), _t(B.col), _t(b)
    x = torch.zeros(B.n_total, dtype=torch.float64, device="cuda:0")
    if ir:
        plan = apcg.batch_ir_plan_create(ctx, B.sys_row_off, rowptr, col, None, _t(B.val.astype(np.float32)),
                                         apcg.ir_opts(rtol=1e-10))
    else:
        plan = apcg.batch_plan_create(ctx, B.sys_row_off, rowptr, col, _t(B.val), apcg.cg_opts(rtol=1e-8))
    res = apcg.batch_plan_solve(plan, bt, x, B.nsys)
    apcg.call("apcg_batch_plan_destroy", V(plan))
    for s, r in enumerate(res):
        assert r["reason"] == ("breakdown" if s == bad else "converged"), (s, r)


def test_bad_arguments_are_rejected_before_enqueue(ctx):
    A, b = _system(10)
    rowptr, col, val, bt = _t(A.rowptr), _t(A.col), _t(A.val), _t(b)
    M = apcg.mat_wrap(rowptr, col, val)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda:0")
    vb, vx = apcg.vec_wrap(bt), apcg.vec_wrap(x)
    short = torch.zeros(A.n - 1, dtype=torch.float64, device="cuda:0")
    vs = apcg.vec_wrap(short)
    apcg.reset_counters()
    with pytest.raises(apcg.ApcgError):  # wrong length
        apcg.cg_solve(ctx, M, vs, vx, apcg.cg_opts())
    with pytest.raises(apcg.ApcgError):  # aliasing b and x
        apcg.cg_solve(ctx, M, vb, vb, apcg.cg_opts())
    with pytest.raises(apcg.ApcgError):  # bad option
        apcg.cg_solve(ctx, M, vb, vx, apcg.cg_opts(check_every=0))
    assert apcg.get_counters()["kernel_launches"] == 0
    res = apcg.cg_solve(ctx, M, vb, vx, apcg.cg_opts(rtol=1e-8))
    assert res["reason"] == "converged"
    for h, f in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (vs, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
        apcg.call(f, V(h))


def _malformed(kind):
    A, b = _system(12)
    rowptr, col = A.rowptr.copy(), A.col.copy()
    if kind == "rowptr_decreasing":
        rowptr[40] = rowptr[41] + 1
    elif kind == "rowptr_end":
        rowptr[-1] -= 1
    elif kind == "col_high":
        col[57] = A.n + 3
    else:
        col[3] = -1
    return A, b, rowptr, col


@pytest.mark.parametrize("kind", ["rowptr_decreasing", "rowptr_end", "col_high", "col_negative"])
@pytest.mark.parametrize("solver,mode", [("cg", "host_sync"), ("cg", "async_graph"), ("cg", "persistent"),
                                         ("tfqmr", "async_graph"), ("tfqmr", "persistent"), ("ir", None)])
def test_malformed_csr_is_rejected_at_plan_creation(ctx, kind, solver, mode):
    """The arrays have their declared sizes; only their contents break the CSR rules.  Plan creation reads the
    row pointers on the host and the column indices in one bounded device pass, before any kernel reads
    through the structure, and returns an error; the context stays usable."""
    A, b, rowptr, col = _malformed(kind)
    keep = [_t(rowptr), _t(col), _t(A.val), _t(b), torch.zeros(A.n, dtype=torch.float64, device="cuda:0")]
    M = apcg.mat_wrap(keep[0], keep[1], keep[2])
    vb, vx = apcg.vec_wrap(keep[3]), apcg.vec_wrap(keep[4])
    try:
        with pytest.raises(apcg.ApcgError) as ei:
            if solver == "cg":
                apcg.cg_solve(ctx, M, vb, vx, apcg.cg_opts(rtol=1e-8, mode=mode))
            elif solver == "tfqmr":
                apcg.tfqmr_solve(ctx, M, vb, vx, apcg.cg_opts(rtol=1e-8, mode=mode))
            else:
                apcg.ir_plan_create(ctx, M, None, apcg.ir_opts(rtol=1e-10))
        assert "CSR" in str(ei.value)
    finally:
        for h, f in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
            apcg.call(f, V(h))
    ok, _ = _cg(ctx, *_system(12), solver="cg" if solver == "ir" else solver, mode=mode or "async_graph", rtol=1e-8)
    assert ok["reason"] == "converged"


def test_staged_spmv_wait_runs_out_and_reports_timeout(ctx):
    """The refinement's staged float32 SpMV waits on mbarriers for its bulk copies, each wait bounded (2^16
    polls, about 0.16 s).
    The test hook makes every copy announce 16 bytes more than it moves, so every wait runs out (nothing
    faults: the copies are unchanged): the solve must return APCG_ERR_TIMEOUT, and the same plan, with the
    hook off, and the context must solve normally afterwards."""
    from synthetic import single_problem

    A = single_problem("c3", size=13).A  # 27-entry rows with per-slice offset lists: the staged SpMV
    b = rhs_from_solution(A, np.random.default_rng(8).uniform(-1, 1, A.n))
    keep = [_t(A.rowptr), _t(A.col), _t(A.val), _t(b), torch.zeros(A.n, dtype=torch.float64, device="cuda:0")]
    M = apcg.mat_wrap(keep[0], keep[1], keep[2])
    vb, vx = apcg.vec_wrap(keep[3]), apcg.vec_wrap(keep[4])
    plan = apcg.ir_plan_create(ctx, M, None, apcg.ir_opts(rtol=1e-10))
    try:
        assert apcg.plan_layout(plan, "ir")["col_format"] == "pattern"
        apcg.call("apcg_ir_plan_test_stall_copies", V(plan), 1)
        with pytest.raises(apcg.ApcgError) as ei:
            apcg.ir_plan_solve(plan, vb, vx)
        assert ei.value.status == apcg.ERR_TIMEOUT and "bounded device wait" in str(ei.value)
        apcg.call("apcg_ir_plan_test_stall_copies", V(plan), 0)
        keep[4].zero_()
        res = apcg.ir_plan_solve(plan, vb, vx)
        assert res["reason"] == "converged" and res["rel_res"] <= 1.05e-10, res
    finally:
        apcg.call("apcg_ir_plan_destroy", V(plan))
        for h, f in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (M, "apcg_mat_destroy")):
            apcg.call(f, V(h))
    ok, _ = _cg(ctx, *_system(12), rtol=1e-8)
    assert ok["reason"] == "converged"


def test_stall_hook_needs_a_staged_plan(ctx):
    A, b = _system(12)  # 5-point rows: no staged SpMV
    keep = [_t(A.rowptr), _t(A.col), _t(A.val)]
    M = apcg.mat_wrap(*keep)
    plan = apcg.ir_plan_create(ctx, M, None, apcg.ir_opts(rtol=1e-10))
    try:
        with pytest.raises(apcg.ApcgError) as ei:
            apcg.call("apcg_ir_plan_test_stall_copies", V(plan), 1)
        assert ei.value.status == apcg.ERR_UNSUPPORTED
    finally:
        apcg.call("apcg_ir_plan_destroy", V(plan))
        apcg.call("apcg_mat_destroy", V(M))
