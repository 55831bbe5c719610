"""The solve entry point that allocates no device memory, against the allocating solver.

apcg_cg_solve_noalloc exists for callers that cannot allocate device memory at
solve time (a framework that reserved the device memory for its own pool, or
a loop that must not allocate after start-up).  It keeps its scratch in a
fixed array inside the library.  Two calls in a row on different systems
must each agree with apcg_cg_solve in persistent mode (the same kernel with
an allocated workspace) within the tolerances of the other parity tests:
equal iteration counts and x within 1e-7 relative.  This file is collected
last so that a run that stops at the first failure has run everything else.
"""

import ctypes as C

import numpy as np
import pytest

from synthetic import single_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    return apcg.load()


def _system(name, size, seed):
    p = single_problem(name, seed=seed, size=size)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    return p, t(p.A.rowptr), t(p.A.col), t(p.A.val), t(p.b)


def _reference(rowptr, col, val, b, k):
    ctx = apcg.ctx_create()
    x = torch.zeros_like(b)
    A = apcg.mat_wrap(rowptr, col, val)
    vb, vx = apcg.vec_wrap(b), apcg.vec_wrap(x)
    res = apcg.cg_solve(ctx, A, vb, vx, apcg.cg_opts(rtol=1e-8, check_every=k, mode="persistent"))
    for h, fn in ((vb, "apcg_vec_destroy"), (vx, "apcg_vec_destroy"), (A, "apcg_mat_destroy"), (ctx, "apcg_ctx_destroy")):
        apcg.call(fn, C.c_void_p(h))
    return res, x.cpu().numpy()


def test_noalloc_matches_allocating_solver_on_two_calls_in_a_row(lib):
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


def test_noalloc_rejects_systems_beyond_its_scratch(lib):
    res = apcg.CgResult()
    st = lib.apcg_cg_solve_noalloc(None, 65537, 65537, C.c_void_p(16), C.c_void_p(32), C.c_void_p(64), C.c_void_p(128), C.c_void_p(256), None, C.byref(res))
    assert st == -1
    assert "65536" in apcg.last_error()
