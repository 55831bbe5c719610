"""The column formats of the plans' sliced-ELL copy, through the C ABI.

Stencil matrices take the per-slice offset lists (APCG_COLS_PATTERN): no
column stream at all, rows that lack an offset store 0 there, and columns that
fall outside the matrix at the grid's edges are clamped.  A row whose columns
do not increase, or slices whose rows do not share their offsets, fall back to
16-bit offsets from the row, and entries farther than 32767 from the diagonal
to 32-bit indices.  Every format must give the oracle's CG scalars (alpha and
beta of the first 10 iterations within 1e-12 relative, x within 1e-7 at rtol
1e-8), TFQMR and the float32-inner refinement their usual bars, on the same
systems.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import laplace_2d_5pt, random_spd_csr, rhs_from_solution, single_problem
from synthetic.stencils import CSR

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


def _reverse_rows(A: CSR, rows) -> CSR:
    """The same matrix with the entries of the given rows stored in reverse column order (still valid CSR)."""
    col, val = A.col.copy(), A.val.copy()
    for r in rows:
        a, b = A.rowptr[r], A.rowptr[r + 1]
        col[a:b] = col[a:b][::-1]
        val[a:b] = val[a:b][::-1]
    return CSR(A.rowptr.copy(), col, val)


def _add_couplings(A: CSR, pairs, w) -> CSR:
    """A + w (e_i e_j^T + e_j e_i^T) for each pair, with w added to both diagonals (stays SPD, rows sorted)."""
    M = A.to_scipy().tolil()
    for i, j in pairs:
        M[i, j] = M[i, j] - w
        M[j, i] = M[j, i] - w
        M[i, i] = M[i, i] + w
        M[j, j] = M[j, j] + w
    M = M.tocsr()
    M.sort_indices()
    return CSR(M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def _case(name):
    rng = np.random.default_rng(5)
    if name == "lap5_48":  # 48-wide grid lines: slices straddle two lines
        return laplace_2d_5pt(48, shift=0.05), "pattern"
    if name == "lap7_21":  # 9261 rows: a ragged last slice
        return single_problem("c2", size=21).A, "pattern"
    if name == "diff27_13":
        return single_problem("c3", size=13).A, "pattern"
    if name == "one_row":
        return CSR(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0])), "pattern"
    if name == "unsorted":  # a few rows stored in reverse column order
        return _reverse_rows(laplace_2d_5pt(48, shift=0.05), [0, 17, 500, 2303]), "offset16"
    if name == "scattered":  # a 5-point Laplacian plus one random long-range coupling per 4 rows
        A = laplace_2d_5pt(48, shift=0.05)
        i = np.arange(0, A.n, 4)
        j = rng.integers(0, A.n, i.size)
        keep = np.abs(i - j) > 60
        return _add_couplings(A, zip(i[keep], j[keep]), 0.25), "offset16"
    if name == "mixed_width":  # 27-point rows plus couplings 1000 rows away: slices of 18..29 entries per row
        A = single_problem("c3", size=13).A
        return _add_couplings(A, [(i, i + 1000) for i in range(A.n // 2)], 0.1), "pattern"
    if name == "far":  # random SPD with entries beyond 32767 of the diagonal
        return random_spd_csr(40_000, 2e-4, rng, dominance=0.2), "index"
    raise ValueError(name)


CASES = ["lap5_48", "lap7_21", "diff27_13", "one_row", "unsorted", "scattered", "mixed_width", "far"]


class _Sys:
    def __init__(self, A, b, f32=False):
        self.keep = [_t(A.rowptr), _t(A.col), _t(A.val), _t(b), torch.zeros(A.n, dtype=torch.float64, device="cuda:0")]
        self.M = apcg.mat_wrap(self.keep[0], self.keep[1], self.keep[2])
        self.vb, self.vx = apcg.vec_wrap(self.keep[3]), apcg.vec_wrap(self.keep[4])
        self.M32 = None
        if f32:
            self.keep.append(_t(A.val.astype(np.float32)))
            self.M32 = apcg.mat_wrap(self.keep[0], self.keep[1], self.keep[5])

    @property
    def x(self):
        return self.keep[4].cpu().numpy()

    def close(self):
        for h, f in ((self.vb, "apcg_vec_destroy"), (self.vx, "apcg_vec_destroy"), (self.M, "apcg_mat_destroy"),
                     (self.M32, "apcg_mat_destroy")):
            if h:
                apcg.call(f, V(h))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("mode", ["host_sync", "async_graph"])
def test_cg_layout_and_parity(ctx, name, mode):
    A, fmt = _case(name)
    b = rhs_from_solution(A, np.random.default_rng(2).uniform(-1, 1, A.n))
    ref = oracle.pcg(A, b, rtol=1e-8, check_every=1, hist_len=10)
    s = _Sys(A, b)
    opts = apcg.cg_opts(rtol=1e-8, check_every=1, mode=mode, history_len=10)  # the plan writes its histories here
    plan = apcg.cg_plan_create(ctx, s.M, opts)
    try:
        lay = apcg.plan_layout(plan, "cg")
        assert lay["col_format"] == fmt, lay
        assert lay["nslices"] == (A.n + 31) // 32
        widest = int(np.diff(A.rowptr).max())
        assert lay["padded"] % 32 == 0 and lay["padded"] >= widest * 32
        res = apcg.cg_plan_solve(plan, s.vb, s.vx)
    finally:
        apcg.call("apcg_cg_plan_destroy", V(plan))
    assert res["reason"] == "converged" and abs(res["iters"] - ref["iters"]) <= 1, (res, ref["iters"])
    alpha, beta = np.array(opts._hist[0]), np.array(opts._hist[1])
    h = min(10, ref["iters"] - 1)
    if h > 0:
        assert np.max(np.abs(alpha[:h] - ref["alpha"][:h]) / np.abs(ref["alpha"][:h])) <= 1e-12
        assert np.max(np.abs(beta[:h] - ref["beta"][:h]) / np.abs(ref["beta"][:h])) <= 1e-12
    if res["iters"] == ref["iters"]:
        assert _rel(s.x, ref["x"]) <= 1e-7
    assert res["rel_res"] <= 1e-8
    s.close()


def test_pattern_layout_pads_only_missing_offsets(ctx):
    """5-point rows on a 48-wide grid: the offsets of a slice are {-48, -1, 0, 1, 48}, without -48 on the
    first grid line and without 48 on the last, and every slice holds a row with all of its offsets, so the
    pattern copy is exactly as large as padding each slice to its widest row."""
    A, _ = _case("lap5_48")
    rows = np.diff(A.rowptr)
    widest = [int(rows[32 * s:32 * s + 32].max()) for s in range((A.n + 31) // 32)]
    s = _Sys(A, np.ones(A.n))
    plan = apcg.cg_plan_create(ctx, s.M, apcg.cg_opts(mode="async_graph"))
    lay = apcg.plan_layout(plan, "cg")
    apcg.call("apcg_cg_plan_destroy", V(plan))
    s.close()
    assert lay["col_format"] == "pattern" and lay["padded"] == 32 * sum(widest), lay
    assert widest[0] == 4 and widest[1] == 5 and widest[-1] == 4


def test_no_copy_in_whole_solve_mode(ctx):
    A = laplace_2d_5pt(20)
    s = _Sys(A, np.ones(A.n))
    plan = apcg.cg_plan_create(ctx, s.M, apcg.cg_opts(mode="persistent"))
    lay = apcg.plan_layout(plan, "cg")
    apcg.call("apcg_cg_plan_destroy", V(plan))
    s.close()
    assert lay == {"col_format": "none", "group": 0, "nslices": 0, "padded": 0}


@pytest.mark.parametrize("name", ["lap7_21", "diff27_13", "unsorted", "far"])
def test_tfqmr_layout_and_solution(ctx, name):
    A, fmt = _case(name)
    b = rhs_from_solution(A, np.random.default_rng(3).uniform(-1, 1, A.n))
    ref = oracle.tfqmr(A, b, rtol=1e-8, check_every=1)
    s = _Sys(A, b)
    plan = apcg.tfqmr_plan_create(ctx, s.M, apcg.cg_opts(rtol=1e-8, check_every=1, mode="async_graph"))
    try:
        lay = apcg.plan_layout(plan, "tfqmr")
        assert lay["col_format"] == fmt, lay
        res = apcg.tfqmr_plan_solve(plan, s.vb, s.vx)
    finally:
        apcg.call("apcg_tfqmr_plan_destroy", V(plan))
    assert res["reason"] == "converged" and abs(res["iters"] - ref["iters"]) <= 1, (res, ref["iters"])
    assert _rel(s.x, ref["x"]) <= 1e-7
    s.close()


@pytest.mark.parametrize("name", ["lap7_21", "diff27_13", "mixed_width", "unsorted", "far"])
def test_ir_layout_and_accuracy(ctx, name):
    """Float32 inner PCG (rtol 1e-4) inside float64 refinement to rtol 1e-10: the GPU's true residual meets
    the tolerance and x agrees with the oracle's float64 CG solution to 1e-12 within 1e-6 (the bar of the
    refinement's full-size test; both lie within the conditioning bound of the same solution).  diff27_13
    and mixed_width run the shared-memory staged float32 SpMV; mixed_width's slices wider than 27 entries
    per row read their values from global memory instead."""
    A, fmt = _case(name)
    b = rhs_from_solution(A, np.random.default_rng(4).uniform(-1, 1, A.n))
    ref = oracle.pcg(A, b, rtol=1e-12, check_every=1)
    s = _Sys(A, b, f32=True)
    plan = apcg.ir_plan_create(ctx, s.M, s.M32, apcg.ir_opts(rtol=1e-10))
    try:
        lay = apcg.plan_layout(plan, "ir")
        assert lay["col_format"] == ("index" if fmt == "offset16" else fmt), lay  # no 16-bit offsets here
        if name == "diff27_13":  # 27-entry rows: whole groups of 9 with the offset lists
            assert lay["group"] == 9, lay
        res = apcg.ir_plan_solve(plan, s.vb, s.vx)
    finally:
        apcg.call("apcg_ir_plan_destroy", V(plan))
    assert res["reason"] == "converged", res
    x = s.x
    true_rel = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
    assert true_rel <= 1.05e-10 and abs(true_rel - res["rel_res"]) <= 1e-12
    assert _rel(x, ref["x"]) <= 1e-6
    s.close()


def test_ir_profile_times_kernels_and_leaves_x(ctx):
    A, _ = _case("diff27_13")
    b = rhs_from_solution(A, np.random.default_rng(6).uniform(-1, 1, A.n))
    s = _Sys(A, b)
    x0 = np.random.default_rng(7).uniform(-1, 1, A.n)
    s.keep[4].copy_(torch.from_numpy(x0))
    plan = apcg.ir_plan_create(ctx, s.M, None, apcg.ir_opts(rtol=1e-10))
    apcg.reset_counters()
    ms = apcg.ir_plan_profile(plan, s.vb, s.vx, 4)
    launches = apcg.get_counters()["kernel_launches"]
    with pytest.raises(apcg.ApcgError):
        apcg.ir_plan_profile(plan, s.vb, s.vx, 0)
    apcg.call("apcg_ir_plan_destroy", V(plan))
    assert len(ms) == 4 and all(t > 0 for t in ms), ms
    assert launches == 1 + 3 * 4
    assert np.array_equal(s.x, x0)
    s.close()
