"""The solve entry point that allocates no device memory.

apcg_cg_solve_noalloc exists for callers that cannot allocate device memory at
solve time (a framework that reserved the device memory for its own pool, or
a loop that must not allocate after start-up).  It keeps its scratch in a
fixed array inside the library.  Two calls in a row on different systems
must each agree with apcg_cg_solve in persistent mode (the same kernel with
an allocated workspace) within the tolerances of the other parity tests --
equal iteration counts and x within 1e-7 relative -- and with the CPU oracle
(count within the test cadence, x within 1e-7 of the oracle's iterate at the
same count).  A matrix with a zero diagonal entry or a malformed CSR
structure is refused without any iteration and leaves x as it was; an empty
system and the legacy default stream work.  This file is collected last so
that a run that stops at the first failure has run everything else.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import single_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402

ERR_INVALID_ARG, ERR_BAD_DIAGONAL = -1, -4


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    return apcg.load()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _system(name, size, seed):
    p = single_problem(name, seed=seed, size=size)
    return p, _t(p.A.rowptr), _t(p.A.col), _t(p.A.val), _t(p.b)


def _reference(rowptr, col, val, b, k):
    ctx = apcg.ctx_create()
    x = torch.zeros_like(b)
    A = apcg.mat_wrap(rowptr, col, val)
    vb, vx = apcg.vec_wrap(b), apcg.vec_wrap(x)
    res = apcg.cg_solve(ctx, A, vb, vx, apcg.cg_opts(rtol=1e-8, check_every=k, mode="persistent"))
    for h, fn in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (A, "apcg_mat_destroy"), (ctx, "apcg_ctx_destroy")):
        apcg.call(fn, C.c_void_p(h))
    return res, x.cpu().numpy()


def _raw(lib, stream, n, nnz, rowptr, col, val, b, x, opts=None):
    """The C call itself; returns (status, result)."""
    res = apcg.CgResult()
    ptr = lambda t: C.c_void_p(t.data_ptr() if t is not None and t.numel() else 0)  # noqa: E731
    st = lib.apcg_cg_solve_noalloc(C.c_void_p(stream), n, nnz, ptr(rowptr), ptr(col), ptr(val), ptr(b), ptr(x),
                                   C.byref(opts) if opts is not None else None, C.byref(res))
    return st, res


def test_noalloc_matches_allocating_solver_and_oracle_on_two_calls_in_a_row(lib):
    stream = torch.cuda.Stream()
    cases = [("c1", 64, 0, 1), ("c2", 20, 3, 4)]  # 4096 rows, then 8000 rows: the second call reuses the array
    for name, size, seed, k in cases:
        p, rowptr, col, val, b = _system(name, size, seed)
        ref, x_ref = _reference(rowptr, col, val, b, k)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        got = apcg.cg_solve_noalloc(stream, rowptr, col, val, b, x, apcg.cg_opts(rtol=1e-8, check_every=k))
        xg = x.cpu().numpy()
        assert got["reason"] == ref["reason"] == "converged"
        assert got["iters"] == ref["iters"]
        assert np.linalg.norm(xg - x_ref) / np.linalg.norm(x_ref) <= 1e-7
        assert got["rel_res"] <= 1e-8
        orc = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=k)
        assert orc["reason"] == "converged" and abs(got["iters"] - orc["iters"]) <= k
        x_orc = orc["x"] if orc["iters"] == got["iters"] else oracle.pcg(p.A, p.b, rtol=0.0, max_it=got["iters"])["x"]
        assert np.linalg.norm(xg - x_orc) / np.linalg.norm(x_orc) <= 1e-7


def test_noalloc_refuses_a_zero_diagonal_without_iterating(lib):
    p, rowptr, col, val, b = _system("c1", 40, 1)
    v = p.A.val.copy()
    i = 777
    for e in range(p.A.rowptr[i], p.A.rowptr[i + 1]):
        if p.A.col[e] == i:
            v[e] = 0.0
    x0 = np.random.default_rng(4).uniform(-1, 1, p.n)
    x = _t(x0)
    st, _ = _raw(lib, 0, p.n, p.nnz, rowptr, col, _t(v), b, x, apcg.cg_opts(rtol=1e-8))
    assert st == ERR_BAD_DIAGONAL
    assert np.array_equal(x.cpu().numpy(), x0)  # no iteration touched x
    # the array is reusable afterwards
    x = torch.zeros_like(b)
    got = apcg.cg_solve_noalloc(None, rowptr, col, val, b, x, apcg.cg_opts(rtol=1e-8))
    assert got["reason"] == "converged"


@pytest.mark.parametrize("fault", ["rowptr_start", "rowptr_decreasing", "rowptr_end", "column_negative", "column_too_large"])
def test_noalloc_refuses_a_malformed_structure(lib, fault):
    """Arrays of the declared sizes with bad contents, made on the host: the device check reads only within
    those sizes and refuses the call before any kernel reads through the structure."""
    p = single_problem("c1", seed=2, size=30)
    rp, cl = p.A.rowptr.copy(), p.A.col.copy()
    if fault == "rowptr_start":
        rp[0] = 1
    elif fault == "rowptr_decreasing":
        rp[400] = rp[402] + 3
    elif fault == "rowptr_end":
        rp[-1] = rp[-1] - 1
    elif fault == "column_negative":
        cl[123] = -5
    else:
        cl[321] = p.n + 1000
    x0 = np.full(p.n, 0.25)
    x = _t(x0)
    st, _ = _raw(lib, 0, p.n, p.nnz, _t(rp), _t(cl), _t(p.A.val), _t(p.b), x, apcg.cg_opts(rtol=1e-8))
    assert st == ERR_INVALID_ARG, apcg.last_error()
    assert "malformed" in apcg.last_error()
    assert np.array_equal(x.cpu().numpy(), x0)


def test_noalloc_empty_system_and_default_stream(lib):
    rowptr = _t(np.zeros(1, np.int32))
    empty_i, empty_d = _t(np.zeros(0, np.int32)), _t(np.zeros(0))
    st, res = _raw(lib, 0, 0, 0, rowptr, empty_i, empty_d, empty_d, empty_d, apcg.cg_opts(rtol=1e-8))
    assert st == 0 and res.reason == 0 and res.iters == 0
    p, rowptr, col, val, b = _system("c1", 24, 7)
    x = torch.zeros_like(b)
    got = apcg.cg_solve_noalloc(None, rowptr, col, val, b, x, apcg.cg_opts(rtol=1e-8, check_every=1))
    ref = oracle.pcg(p.A, p.b, rtol=1e-8, check_every=1)
    assert got["reason"] == "converged" and got["iters"] == ref["iters"]
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-7


def test_noalloc_rejects_systems_beyond_its_scratch(lib):
    res = apcg.CgResult()
    st = lib.apcg_cg_solve_noalloc(None, 65537, 65537, C.c_void_p(16), C.c_void_p(32), C.c_void_p(64), C.c_void_p(128), C.c_void_p(256), None, C.byref(res))
    assert st == ERR_INVALID_ARG
    assert "65536" in apcg.last_error()
