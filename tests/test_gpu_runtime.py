"""Device contexts, marking and managed scalars on a real GPU (Sec. 3.1-3.3).

Ordering is checked with long-running producers (large vectors) followed by
consumers on other contexts: the consumer must see the producer's final
result, and the library counters must show the waits that marking inserted
or elided.  Nothing here waits without a bound: every wait is a CUDA event
wait on work that always finishes.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from synthetic import single_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_17801_gb300 import apcg  # noqa: E402


def V(h):
    return C.c_void_p(h)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    apcg.load()
    return torch.device("cuda:0")


def _ctxs(n):
    return [apcg.ctx_create() for _ in range(n)]


def _destroy(*hs, fn="apcg_ctx_destroy"):
    for h in hs:
        apcg.call(fn, V(h))


def test_write_then_read_on_other_context_is_ordered(dev):
    a, b = _ctxs(2)
    n = 1 << 25
    x = torch.empty(n, dtype=torch.float64, device=dev)
    vx = apcg.vec_wrap(x)
    two = apcg.scalar_create()
    out = apcg.scalar_create()
    apcg.call("apcg_scalar_set_async", V(a), V(two), 2.0)
    apcg.call("apcg_vec_set_async", V(a), V(vx), C.c_double(1.0))
    for _ in range(20):
        apcg.call("apcg_vec_scale_async", V(a), V(vx), V(two))
    apcg.reset_counters()
    apcg.call("apcg_vec_norm2_async", V(b), V(vx), V(out))
    c = apcg.get_counters()
    assert c["waits_inserted"] == 1
    assert apcg.scalar_get(out) == 2.0**20 * np.sqrt(n)
    _destroy(two, out, fn="apcg_scalar_destroy")
    apcg.call("apcg_vec_destroy", V(vx))
    _destroy(a, b)


def test_read_read_is_not_ordered_and_write_after_read_is(dev):
    a, b, c = _ctxs(3)
    n = 1 << 24
    x = torch.ones(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    vx = apcg.vec_wrap(x)
    s1, s2, k = apcg.scalar_create(), apcg.scalar_create(), apcg.scalar_create()
    apcg.call("apcg_scalar_set_async", V(c), V(k), 3.0)
    apcg.call("apcg_ctx_synchronize", V(c))
    apcg.reset_counters()
    apcg.call("apcg_vec_norm2_async", V(a), V(vx), V(s1))
    apcg.call("apcg_vec_norm2_async", V(b), V(vx), V(s2))
    assert apcg.get_counters()["waits_inserted"] == 0  # read after read: no order
    apcg.call("apcg_vec_scale_async", V(c), V(vx), V(k))  # write after two reads: waits for both
    cc = apcg.get_counters()
    assert cc["waits_inserted"] + cc["waits_elided"] >= 2
    assert apcg.scalar_get(s1) == np.sqrt(n) and apcg.scalar_get(s2) == np.sqrt(n)
    apcg.call("apcg_ctx_synchronize", V(c))
    assert torch.all(x == 3.0).item()
    _destroy(s1, s2, k, fn="apcg_scalar_destroy")
    apcg.call("apcg_vec_destroy", V(vx))
    _destroy(a, b, c)


def test_global_blocking_context_completes_before_return(dev):
    (g,) = _ctxs(1)
    apcg.call("apcg_ctx_set_stream_type", V(g), apcg.STREAM_GLOBAL_BLOCKING)
    x = torch.empty(1 << 25, dtype=torch.float64, device=dev)
    vx = apcg.vec_wrap(x)
    apcg.call("apcg_vec_set_async", V(g), V(vx), C.c_double(4.0))
    assert apcg.ctx_query_idle(g)
    # the NULL context is global blocking too
    s = apcg.scalar_create()
    apcg.call("apcg_vec_norm2_async", None, V(vx), V(s))
    assert apcg.scalar_get(s) == 4.0 * np.sqrt(x.numel())
    apcg.call("apcg_scalar_destroy", V(s))
    apcg.call("apcg_vec_destroy", V(vx))
    _destroy(g)


def test_fork_join(dev):
    (parent,) = _ctxs(1)
    kids = apcg.ctx_fork(parent, 3)
    xs = [torch.empty(1 << 23, dtype=torch.float64, device=dev) for _ in kids]
    vs = [apcg.vec_wrap(x) for x in xs]
    for i, (k, v) in enumerate(zip(kids, vs)):
        apcg.call("apcg_vec_set_async", V(k), V(v), C.c_double(float(i + 1)))
    apcg.ctx_join(parent, kids, apcg.JOIN_NO_SYNC)
    apcg.call("apcg_ctx_synchronize", V(parent))
    for k in kids:  # the parent's tail was ordered after each child's work
        assert apcg.ctx_query_idle(k)
    for i, x in enumerate(xs):
        assert torch.all(x == i + 1).item()
    apcg.ctx_join(parent, kids, apcg.JOIN_DESTROY)
    for v in vs:
        apcg.call("apcg_vec_destroy", V(v))
    _destroy(parent)


def test_wait_for_context_and_caller_kernels(dev):
    """A caller launch bracketed by mark_intent_begin/end on the context's stream (Sec. 3.1.2)."""
    a, b = _ctxs(2)
    x = torch.zeros(1 << 22, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    vx = apcg.vec_wrap(x)
    xid = apcg.vec_id(vx)
    apcg.call("apcg_mark_intent_begin", V(a), xid, apcg.WRITE, b"torch fill")
    stream = torch.cuda.ExternalStream(apcg.ctx_get_stream(a))
    with torch.cuda.stream(stream):
        x.fill_(7.0)
    apcg.call("apcg_mark_intent_end", V(a), xid, apcg.WRITE, b"torch fill")
    s = apcg.scalar_create()
    apcg.call("apcg_vec_norm2_async", V(b), V(vx), V(s))
    assert apcg.scalar_get(s) == 7.0 * np.sqrt(x.numel())
    # explicit context-to-context wait
    apcg.call("apcg_ctx_wait_for_context", V(b), V(a))
    apcg.call("apcg_host_access", xid, apcg.READ)
    apcg.call("apcg_scalar_destroy", V(s))
    apcg.call("apcg_vec_destroy", V(vx))
    _destroy(a, b)


def test_scalar_released_only_after_its_work(dev):
    a, b = _ctxs(2)
    n = 1 << 25
    x = torch.ones(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    vx = apcg.vec_wrap(x)
    for _ in range(5):
        s = apcg.scalar_create()
        apcg.call("apcg_vec_dot_async", V(a), V(vx), V(vx), V(s))
        apcg.call("apcg_scalar_destroy", V(s))  # destroyed while its producer may still run
        t = apcg.scalar_create()
        apcg.call("apcg_scalar_set_async", V(b), V(t), 5.0)
        apcg.call("apcg_ctx_synchronize", V(a))
        assert apcg.scalar_get(t) == 5.0
        apcg.call("apcg_scalar_destroy", V(t))
    apcg.call("apcg_vec_destroy", V(vx))
    _destroy(a, b)


def test_context_destroyed_with_pending_work(dev):
    (a,) = _ctxs(1)
    x = torch.empty(1 << 25, dtype=torch.float64, device=dev)
    vx = apcg.vec_wrap(x)
    apcg.call("apcg_vec_set_async", V(a), V(vx), C.c_double(2.0))
    apcg.call("apcg_ctx_destroy", V(a))  # returns at once; the work still completes
    (b,) = _ctxs(1)
    s = apcg.scalar_create()
    apcg.call("apcg_vec_norm2_async", V(b), V(vx), V(s))
    assert apcg.scalar_get(s) == 2.0 * np.sqrt(x.numel())
    apcg.call("apcg_scalar_destroy", V(s))
    apcg.call("apcg_vec_destroy", V(vx))
    _destroy(b)


def test_mixed_api_cg_listing(dev):
    """The three-context mixed sync/async CG main loop of Sec. 3.3 on the public API.

    Synchronous calls use the NULL (global-blocking) context; b.front() is a
    host read of the scalar.  Initialisation: x = 0, r = b, z = D^-1 r,
    beta = (z, r), betaold = 1, p = 0, so that the first pass sets p = z.
    After 20 passes x equals the oracle's 20-iteration iterate.
    """
    p = single_problem("c1", seed=7, size=40)
    n = p.n
    ca, cb, cc = _ctxs(3)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    rowptr, col, val = t(p.A.rowptr), t(p.A.col), t(p.A.val)
    A = apcg.mat_wrap(rowptr, col, val)
    X, R, Z, P, W, D = (torch.zeros(n, dtype=torch.float64, device=dev) for _ in range(6))
    R.copy_(t(p.b))
    torch.cuda.synchronize()
    vX, vR, vZ, vP, vW, vD = (apcg.vec_wrap(v) for v in (X, R, Z, P, W, D))
    a, bs, beta, betaold, dp, host_b = (apcg.scalar_create() for _ in range(6))
    apcg.call("apcg_pc_jacobi_setup_async", None, V(A), V(vD))
    apcg.call("apcg_pc_jacobi_apply_async", None, V(vD), V(vR), V(vZ))
    apcg.call("apcg_vec_dot_async", None, V(vZ), V(vR), V(beta))
    apcg.call("apcg_scalar_set_async", None, V(betaold), 1.0)
    apcg.reset_counters()
    iters = 20
    for _ in range(iters):
        apcg.call("apcg_scalar_div_async", V(ca), V(bs), V(beta), V(betaold))
        bval = apcg.scalar_get(bs)  # b.front(): implicit synchronisation
        apcg.call("apcg_scalar_set_async", None, V(host_b), bval)
        apcg.call("apcg_vec_aypx_async", None, V(vP), V(host_b), V(vZ))
        apcg.call("apcg_mat_mult_async", None, V(A), V(vP), V(vW))
        apcg.call("apcg_vec_dot_async", V(cb), V(vP), V(vW), V(a))
        apcg.call("apcg_scalar_div_async", V(cc), V(a), V(beta), V(a))
        apcg.call("apcg_scalar_copy_async", V(ca), V(betaold), V(beta))
        apcg.call("apcg_vec_axpy_async", V(cb), V(vX), V(a), 0, V(vP))
        apcg.call("apcg_vec_axpy_async", V(cc), V(vR), V(a), 1, V(vW))
        apcg.call("apcg_pc_jacobi_apply_async", None, V(vD), V(vR), V(vZ))
        apcg.call("apcg_vec_norm2_async", V(ca), V(vZ), V(dp))
        apcg.call("apcg_vec_dot_async", V(cb), V(vZ), V(vR), V(beta))
    cnt = apcg.get_counters()
    for c in (ca, cb, cc):
        apcg.call("apcg_ctx_synchronize", V(c))
    ref = oracle.pcg(p.A, p.b, rtol=0.0, max_it=iters)
    assert np.linalg.norm(X.cpu().numpy() - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-12
    assert cnt["d2h_copies"] == iters  # only b.front(): every other scalar stays on the device
    assert cnt["waits_inserted"] >= 2 * iters
    for s in (a, bs, beta, betaold, dp, host_b):
        apcg.call("apcg_scalar_destroy", V(s))
    for v in (vX, vR, vZ, vP, vW, vD):
        apcg.call("apcg_vec_destroy", V(v))
    apcg.call("apcg_mat_destroy", V(A))
    _destroy(ca, cb, cc)


def test_launch_floor_reports_positive_times(dev):
    ctx = apcg.ctx_create()
    f = apcg.launch_floor(ctx, 20)
    assert all(0.0 < v < 1e5 for v in f.values()), f
    assert f["graph3_back_to_back_us"] <= f["graph3_sync_us"] * 1.5
    apcg.call("apcg_ctx_destroy", C.c_void_p(ctx))


def test_fp64_fma_peak_is_in_the_float64_range(dev):
    """Independent float64 FMA chains: GB300's float64 pipe is 2 lanes/SM/cycle (152 SMs, up to 2.07 GHz: at
    most 1.26 TFLOP/s); a figure far above means the kernel's FMAs were folded away, far below that it stalls."""
    ctx = apcg.ctx_create()
    g = apcg.fp64_fma_peak(ctx, 2)
    assert 300.0 < g < 1.6e3, g
    with pytest.raises(apcg.ApcgError):
        apcg.fp64_fma_peak(ctx, 0)
    apcg.call("apcg_ctx_destroy", C.c_void_p(ctx))


def test_views_keep_their_tensors_alive(dev):
    """The library holds raw device pointers; the binding keeps each wrapped tensor until its view is destroyed."""
    import gc
    import weakref

    t = torch.zeros(1000, dtype=torch.float64, device=dev)
    r, c = torch.zeros(11, dtype=torch.int32, device=dev), torch.zeros(0, dtype=torch.int32, device=dev)
    v = torch.zeros(0, dtype=torch.float64, device=dev)
    refs = [weakref.ref(x) for x in (t, r, c, v)]
    hv = apcg.vec_wrap(t)
    hm = apcg.mat_wrap(r, c, v)
    del t, r, c, v
    gc.collect()
    assert all(w() is not None for w in refs)
    apcg.call("apcg_vec_destroy", V(hv))
    apcg.call("apcg_mat_destroy", V(hm))
    gc.collect()
    assert all(w() is None for w in refs)
