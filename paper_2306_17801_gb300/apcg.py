"""Thin ctypes binding of libapcg (include/apcg.h).

Argument marshalling only: every entry point keeps its C name; device arrays
are passed as raw pointers taken from PyTorch CUDA tensors.  All computation
runs in the library's CUDA kernels.  Importing this module does not need a
GPU; loading the library needs it to have been built (``build()`` of the
repository's entry module) and raises ``ImportError`` otherwise.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libapcg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "apcg.h")

OK = 0
ERR = {
    -1: "APCG_ERR_INVALID_ARG",
    -2: "APCG_ERR_CUDA",
    -3: "APCG_ERR_NO_MEMORY",
    -4: "APCG_ERR_BAD_DIAGONAL",
    -5: "APCG_ERR_TIMEOUT",
    -6: "APCG_ERR_UNSUPPORTED",
    -7: "APCG_ERR_NOT_READY",
    -8: "APCG_ERR_BREAKDOWN",
}
ERR_TIMEOUT, ERR_UNSUPPORTED = -5, -6
STREAM_DEFAULT_BLOCKING, STREAM_GLOBAL_BLOCKING = 0, 1
READ, WRITE, READ_WRITE = 1, 2, 3
JOIN_DESTROY, JOIN_SYNC, JOIN_NO_SYNC = 0, 1, 2
F64, F32 = 0, 1
MODE_HOST_SYNC, MODE_ASYNC, MODE_ASYNC_GRAPH, MODE_PERSISTENT, MODE_AUTO = 0, 1, 2, 3, 4
MODES = {"host_sync": 0, "async": 1, "async_graph": 2, "persistent": 3, "auto": 4}
REASONS = {0: "converged", 1: "not_converged", 2: "breakdown"}


class ApcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{ERR.get(status, status)}: {msg}")
        self.status = status


class Counters(C.Structure):
    _fields_ = [
        (n, C.c_int64)
        for n in (
            "kernel_launches",
            "graph_launches",
            "waits_inserted",
            "waits_elided",
            "events_recorded",
            "host_syncs",
            "d2h_copies",
            "d2h_bytes",
            "h2d_copies",
            "h2d_bytes",
        )
    ]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class CgOpts(C.Structure):
    _fields_ = [
        ("rtol", C.c_double),
        ("atol", C.c_double),
        ("max_it", C.c_int32),
        ("check_every", C.c_int32),
        ("mode", C.c_int32),
        ("history_len", C.c_int32),
        ("alpha_hist", C.POINTER(C.c_double)),
        ("beta_hist", C.POINTER(C.c_double)),
    ]


class CgResult(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("reason", C.c_int32),
        ("rr", C.c_double),
        ("bnorm", C.c_double),
        ("rel_res", C.c_double),
        ("kernel_launches", C.c_int64),
    ]

    def as_dict(self):
        return {
            "iters": int(self.iters),
            "reason": REASONS.get(int(self.reason), int(self.reason)),
            "rr": float(self.rr),
            "bnorm": float(self.bnorm),
            "rel_res": float(self.rel_res),
            "kernel_launches": int(self.kernel_launches),
        }


class IrOpts(C.Structure):
    _fields_ = [
        ("rtol", C.c_double),
        ("atol", C.c_double),
        ("max_outer", C.c_int32),
        ("max_inner", C.c_int32),
        ("rtol_inner", C.c_float),
        ("inner_check_every", C.c_int32),
        ("history_len", C.c_int32),
        ("pad", C.c_int32),
        ("alpha_hist", C.POINTER(C.c_double)),
        ("beta_hist", C.POINTER(C.c_double)),
    ]


class IrResult(C.Structure):
    _fields_ = [
        ("outer", C.c_int32),
        ("inner_total", C.c_int32),
        ("reason", C.c_int32),
        ("inner_first", C.c_int32),
        ("rel_res", C.c_double),
        ("kernel_launches", C.c_int64),
    ]

    def as_dict(self):
        return {
            "outer": int(self.outer),
            "inner_total": int(self.inner_total),
            "reason": REASONS.get(int(self.reason), int(self.reason)),
            "inner_first": int(self.inner_first),
            "rel_res": float(self.rel_res),
            "kernel_launches": int(self.kernel_launches),
        }


COL_FORMATS = {-1: "none", 0: "index", 1: "offset16", 2: "pattern"}


class PlanLayout(C.Structure):
    _fields_ = [("col_format", C.c_int32), ("group", C.c_int32), ("nslices", C.c_int64), ("padded", C.c_int64)]

    def as_dict(self):
        return {"col_format": COL_FORMATS.get(int(self.col_format), int(self.col_format)), "group": int(self.group),
                "nslices": int(self.nslices), "padded": int(self.padded)}


class ExprTerm(C.Structure):
    _fields_ = [("op", C.c_int32), ("pad", C.c_int32), ("s", C.c_void_p), ("c", C.c_double)]


EXPR_OPS = {name: i for i, name in enumerate(
    ["scalar", "const", "add", "sub", "mul", "div", "min", "max", "neg", "recip", "sqrt", "abs", "sin", "cos", "exp", "log"])}


class BatchResult(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("reason", C.c_int32),
        ("rel_res", C.c_double),
        ("outer", C.c_int32),
        ("pad", C.c_int32),
    ]


REASONS[3] = "bad_diagonal"

P = C.c_void_p
PP = C.POINTER(C.c_void_p)
S = C.c_int32
i32, i64, u64, f64 = C.c_int32, C.c_int64, C.c_uint64, C.c_double

# name -> argument types (every function returns apcg_status unless listed in _RESTYPE)
PROTOS = {
    "apcg_last_error_string": [],
    "apcg_version": [],
    "apcg_get_counters": [C.POINTER(Counters)],
    "apcg_reset_counters": [],
    "apcg_ctx_create": [PP],
    "apcg_ctx_create_from_stream": [P, PP],
    "apcg_ctx_set_stream_type": [P, C.c_int],
    "apcg_ctx_get_stream_type": [P, C.POINTER(C.c_int)],
    "apcg_ctx_get_stream": [P, PP],
    "apcg_ctx_wait_for_context": [P, P],
    "apcg_ctx_query_idle": [P, C.POINTER(i32)],
    "apcg_ctx_synchronize": [P],
    "apcg_ctx_fork": [P, i32, PP],
    "apcg_ctx_join": [P, i32, PP, C.c_int],
    "apcg_ctx_destroy": [P],
    "apcg_register_memory": [P, C.c_size_t, C.POINTER(u64)],
    "apcg_get_pointer_attributes": [P, C.POINTER(u64), C.POINTER(C.c_size_t)],
    "apcg_unregister_memory": [P],
    "apcg_mark_intent_begin": [P, u64, C.c_int, C.c_char_p],
    "apcg_mark_intent_end": [P, u64, C.c_int, C.c_char_p],
    "apcg_host_access": [u64, C.c_int],
    "apcg_scalar_create": [C.c_int, PP],
    "apcg_scalar_set_async": [P, P, f64],
    "apcg_scalar_get": [P, C.POINTER(f64)],
    "apcg_scalar_device_ptr": [P, PP],
    "apcg_scalar_id": [P, C.POINTER(u64)],
    "apcg_scalar_div_async": [P, P, P, P],
    "apcg_scalar_recip_async": [P, P, P],
    "apcg_scalar_neg_async": [P, P, P],
    "apcg_scalar_copy_async": [P, P, P],
    "apcg_scalar_mul_async": [P, P, P, P],
    "apcg_scalar_sqrt_async": [P, P, P],
    "apcg_scalar_destroy": [P],
    "apcg_vec_wrap": [P, i64, C.c_int, PP],
    "apcg_vec_id": [P, C.POINTER(u64)],
    "apcg_vec_destroy": [P],
    "apcg_mat_csr_wrap": [P, P, P, i32, i32, i64, C.c_int, PP],
    "apcg_mat_validate": [P],
    "apcg_mat_id": [P, C.POINTER(u64)],
    "apcg_mat_destroy": [P],
    "apcg_vec_dot_async": [P, P, P, P],
    "apcg_vec_norm2_async": [P, P, P],
    "apcg_vec_axpy_async": [P, P, P, i32, P],
    "apcg_vec_aypx_async": [P, P, P, P],
    "apcg_vec_scale_async": [P, P, P],
    "apcg_vec_copy_async": [P, P, P],
    "apcg_vec_set_async": [P, P, f64],
    "apcg_vec_pointwise_mult_async": [P, P, P, P],
    "apcg_mat_mult_async": [P, P, P, P],
    "apcg_mat_mult_dot_async": [P, P, P, P, P],
    "apcg_pc_jacobi_setup_async": [P, P, P],
    "apcg_pc_jacobi_apply_async": [P, P, P, P],
    "apcg_cg_opts_default": [C.POINTER(CgOpts)],
    "apcg_cg_solve": [P, P, P, P, C.POINTER(CgOpts), C.POINTER(CgResult)],
    "apcg_cg_plan_create": [P, P, C.POINTER(CgOpts), PP],
    "apcg_cg_plan_solve": [P, P, P, C.POINTER(CgResult)],
    "apcg_cg_plan_solve_async": [P, P, P],
    "apcg_cg_plan_result": [P, C.POINTER(CgResult)],
    "apcg_cg_plan_destroy": [P],
    "apcg_cg_plan_profile": [P, P, P, i32, C.POINTER(C.c_float)],
    "apcg_cg_plan_layout": [P, C.POINTER(PlanLayout)],
    "apcg_cg_solve_host": [i32, i64, P, P, P, P, P, C.POINTER(CgOpts), C.POINTER(CgResult)],
    "apcg_cg_solve_noalloc": [P, i32, i64, P, P, P, P, P, C.POINTER(CgOpts), C.POINTER(CgResult)],
    "apcg_ir_opts_default": [C.POINTER(IrOpts)],
    "apcg_ir_plan_create": [P, P, P, C.POINTER(IrOpts), PP],
    "apcg_ir_plan_solve": [P, P, P, C.POINTER(IrResult)],
    "apcg_ir_plan_destroy": [P],
    "apcg_ir_plan_layout": [P, C.POINTER(PlanLayout)],
    "apcg_ir_plan_profile": [P, P, P, i32, C.POINTER(C.c_float)],
    "apcg_ir_plan_test_stall_copies": [P, i32],
    "apcg_ir_plan_inner_spmv": [P, P, P, C.POINTER(C.c_double)],
    "apcg_ir_solve": [P, P, P, P, P, C.POINTER(IrOpts), C.POINTER(IrResult)],
    "apcg_expr_create": [P, i32, PP],
    "apcg_expr_destroy": [P],
    "apcg_expr_describe": [P, P, P, C.c_char_p, C.c_size_t],
    "apcg_expr_execute_async": [P, P, P],
    "apcg_vec_axpy_expr_async": [P, P, P, P],
    "apcg_launch_floor": [P, i32, P],
    "apcg_fp64_fma_peak": [P, i32, C.POINTER(C.c_double)],
    "apcg_stencil_create": [i32, i32, i32, i32, P, P, PP],
    "apcg_stencil_destroy": [P],
    "apcg_stencil_apply_async": [P, P, P, P],
    "apcg_cg_plan_create_stencil": [P, P, C.POINTER(CgOpts), PP],
    "apcg_ir_plan_create_stencil": [P, P, C.POINTER(IrOpts), PP],
    "apcg_tfqmr_plan_create": [P, P, C.POINTER(CgOpts), PP],
    "apcg_tfqmr_plan_solve": [P, P, P, C.POINTER(CgResult)],
    "apcg_tfqmr_plan_destroy": [P],
    "apcg_tfqmr_plan_layout": [P, C.POINTER(PlanLayout)],
    "apcg_tfqmr_solve": [P, P, P, P, C.POINTER(CgOpts), C.POINTER(CgResult)],
    "apcg_batch_plan_create": [P, i32, P, P, P, P, C.POINTER(CgOpts), PP],
    "apcg_batch_ir_plan_create": [P, i32, P, P, P, P, P, C.POINTER(IrOpts), PP],
    "apcg_batch_plan_solve": [P, P, P, P],
    "apcg_batch_plan_tune": [P, P, C.c_char_p, C.c_size_t],
    "apcg_batch_plan_history": [P, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "apcg_batch_plan_destroy": [P],
    "apcg_cg_solve_batched": [P, i32, P, P, P, P, P, P, C.POINTER(CgOpts), P],
    "apcg_sim_create": [i32, PP],
    "apcg_sim_op": [P, i32, i32, C.POINTER(u64), C.POINTER(i32)],
    "apcg_sim_complete": [P, i32, u64],
    "apcg_sim_log": [P, C.c_char_p, C.c_size_t],
    "apcg_sim_destroy": [P],
}
_RESTYPE = {"apcg_last_error_string": C.c_char_p, "apcg_version": i32}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libapcg.so (raises ImportError when it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"libapcg.so is not built ({p} missing); run the repository's build() first")
        lib = C.CDLL(p)
        for name, args in PROTOS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _RESTYPE.get(name, S)
        _lib = lib
        return lib


def last_error() -> str:
    return load().apcg_last_error_string().decode()


# Tensors behind the views made by vec_wrap / mat_wrap, by handle: the library keeps raw device pointers, so
# the binding keeps the tensors alive until the view is destroyed (a view of freed memory would let the
# caching allocator hand the same bytes to the next tensor).
_views: dict[int, tuple] = {}
_DESTROY = {"apcg_vec_destroy", "apcg_mat_destroy"}


def call(name: str, *args):
    """Call an entry point; raise ApcgError on a non-zero status."""
    st = getattr(load(), name)(*args)
    if st != OK:
        raise ApcgError(st, last_error())
    if name in _DESTROY and args:
        h = args[0]
        _views.pop(h.value if isinstance(h, C.c_void_p) else h, None)
    return st


# ---------------------------------------------------------------- handles and helpers


def _out():
    return C.c_void_p()


def _ptr(t) -> int:
    """Raw data pointer of a tensor (or an int pointer; None is NULL)."""
    if t is None:
        return 0
    return t if isinstance(t, int) else int(t.data_ptr())


def ctx_create(stream=None):
    h = _out()
    if stream is None:
        call("apcg_ctx_create", C.byref(h))
    else:
        s = stream if isinstance(stream, int) else int(stream.cuda_stream)
        call("apcg_ctx_create_from_stream", C.c_void_p(s), C.byref(h))
    return h.value


def ctx_get_stream(ctx) -> int:
    s = _out()
    call("apcg_ctx_get_stream", C.c_void_p(ctx), C.byref(s))
    return s.value or 0


def ctx_query_idle(ctx) -> bool:
    v = i32()
    call("apcg_ctx_query_idle", C.c_void_p(ctx), C.byref(v))
    return bool(v.value)


def ctx_fork(parent, n):
    arr = (C.c_void_p * n)()
    call("apcg_ctx_fork", C.c_void_p(parent), n, arr)
    return [arr[i] for i in range(n)]


def ctx_join(parent, children, mode=JOIN_DESTROY):
    arr = (C.c_void_p * len(children))(*children)
    call("apcg_ctx_join", C.c_void_p(parent), len(children), arr, mode)


def register_memory(ptr, nbytes) -> int:
    v = u64()
    call("apcg_register_memory", C.c_void_p(_ptr(ptr)), nbytes, C.byref(v))
    return v.value


def scalar_create():
    h = _out()
    call("apcg_scalar_create", F64, C.byref(h))
    return h.value


def scalar_get(s) -> float:
    v = f64()
    call("apcg_scalar_get", C.c_void_p(s), C.byref(v))
    return v.value


def scalar_id(s) -> int:
    v = u64()
    call("apcg_scalar_id", C.c_void_p(s), C.byref(v))
    return v.value


def scalar_device_ptr(s) -> int:
    v = _out()
    call("apcg_scalar_device_ptr", C.c_void_p(s), C.byref(v))
    return v.value


def vec_wrap(t, dtype=None):
    """View a contiguous 1-D CUDA tensor (float64 or float32) as an apcg_vec."""
    import torch

    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is None:
        dtype = F64 if t.dtype == torch.float64 else F32 if t.dtype == torch.float32 else None
        if dtype is None:
            raise ValueError(f"unsupported dtype {t.dtype}")
    h = _out()
    call("apcg_vec_wrap", C.c_void_p(_ptr(t) if t.numel() else 0), t.numel(), dtype, C.byref(h))
    _views[h.value] = (t,)
    return h.value


def vec_id(v) -> int:
    x = u64()
    call("apcg_vec_id", C.c_void_p(v), C.byref(x))
    return x.value


def mat_wrap(rowptr, col, val, ncols=None):
    """View CUDA tensors rowptr (int32), col (int32), val (float64/float32) as an apcg_mat."""
    import torch

    nrows = rowptr.numel() - 1
    dtype = F64 if val.dtype == torch.float64 else F32
    h = _out()
    call(
        "apcg_mat_csr_wrap",
        C.c_void_p(_ptr(rowptr)),
        C.c_void_p(_ptr(col) if col.numel() else 0),
        C.c_void_p(_ptr(val) if val.numel() else 0),
        nrows,
        nrows if ncols is None else ncols,
        col.numel(),
        dtype,
        C.byref(h),
    )
    _views[h.value] = (rowptr, col, val)
    return h.value


def mat_id(A) -> int:
    x = u64()
    call("apcg_mat_id", C.c_void_p(A), C.byref(x))
    return x.value


def cg_opts(rtol=1e-8, atol=0.0, max_it=0, check_every=1, mode="auto", history_len=0):
    o = CgOpts()
    call("apcg_cg_opts_default", C.byref(o))
    o.rtol, o.atol, o.max_it, o.check_every = rtol, atol, max_it, check_every
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.history_len = history_len
    hist = None
    if history_len:
        hist = ((C.c_double * history_len)(), (C.c_double * history_len)())
        o.alpha_hist = C.cast(hist[0], C.POINTER(C.c_double))
        o.beta_hist = C.cast(hist[1], C.POINTER(C.c_double))
    o._hist = hist  # keep the buffers alive with the struct
    return o


def cg_solve(ctx, A, b, x, opts: CgOpts) -> dict:
    res = CgResult()
    call("apcg_cg_solve", C.c_void_p(ctx), C.c_void_p(A), C.c_void_p(b), C.c_void_p(x), C.byref(opts), C.byref(res))
    out = res.as_dict()
    if opts.history_len:
        out["alpha"] = list(opts._hist[0])
        out["beta"] = list(opts._hist[1])
    return out


def cg_plan_create(ctx, A, opts: CgOpts):
    h = _out()
    call("apcg_cg_plan_create", C.c_void_p(ctx), C.c_void_p(A), C.byref(opts), C.byref(h))
    return h.value


def cg_plan_solve(plan, b, x) -> dict:
    res = CgResult()
    call("apcg_cg_plan_solve", C.c_void_p(plan), C.c_void_p(b), C.c_void_p(x), C.byref(res))
    return res.as_dict()


def plan_layout(plan, kind: str = "cg") -> dict:
    """The sliced-ELL copy a plan's SpMV reads (kind: "cg", "tfqmr" or "ir")."""
    out = PlanLayout()
    call(f"apcg_{kind}_plan_layout", C.c_void_p(plan), C.byref(out))
    return out.as_dict()


def cg_plan_profile(plan, b, x, iters: int) -> list[float]:
    ms = (C.c_float * 3)()
    call("apcg_cg_plan_profile", C.c_void_p(plan), C.c_void_p(b), C.c_void_p(x), iters, ms)
    return [float(v) for v in ms]


def cg_solve_host(rowptr, col, val, b, x, opts: CgOpts) -> dict:
    """Solve with numpy arrays in host memory (x is updated in place)."""
    import numpy as np

    for a, dt in ((rowptr, np.int32), (col, np.int32), (val, np.float64), (b, np.float64), (x, np.float64)):
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous int32/float64")
    res = CgResult()
    call(
        "apcg_cg_solve_host",
        rowptr.shape[0] - 1,
        col.shape[0],
        rowptr.ctypes.data_as(P),
        col.ctypes.data_as(P),
        val.ctypes.data_as(P),
        b.ctypes.data_as(P),
        x.ctypes.data_as(P),
        C.byref(opts),
        C.byref(res),
    )
    return res.as_dict()


def expr_create(terms, scalars: dict):
    """Freeze a postfix expression: terms like ("scalar", name), ("const", c), ("add",), ... ;
    scalars maps names to apcg_scalar handles."""
    arr = (ExprTerm * len(terms))()
    for i, t in enumerate(terms):
        arr[i].op = EXPR_OPS[t[0]]
        if t[0] == "scalar":
            arr[i].s = scalars[t[1]]
        elif t[0] == "const":
            arr[i].c = float(t[1])
    h = _out()
    call("apcg_expr_create", arr, len(terms), C.byref(h))
    return h.value


def expr_describe(expr) -> dict:
    ni, nl = C.c_int32(), C.c_int32()
    buf = C.create_string_buffer(8192)
    call("apcg_expr_describe", C.c_void_p(expr), C.byref(ni), C.byref(nl), buf, len(buf))
    return {"instructions": ni.value, "inputs": nl.value, "text": buf.value.decode()}


def fp64_fma_peak(ctx, reps=5) -> float:
    """Measured float64 FMA throughput in GFLOP/s (apcg_fp64_fma_peak)."""
    g = C.c_double()
    call("apcg_fp64_fma_peak", C.c_void_p(ctx), int(reps), C.byref(g))
    return float(g.value)


def launch_floor(ctx, reps=200) -> dict:
    us = (C.c_double * 4)()
    call("apcg_launch_floor", C.c_void_p(ctx), int(reps), us)
    return {"empty_kernel_sync_us": us[0], "graph3_sync_us": us[1], "d2h_8B_sync_us": us[2],
            "graph3_back_to_back_us": us[3]}


def stencil_create(dims, offsets, weights):
    """A stencil operator handle; dims = (nx, ny, nz), offsets [k][3] ints, weights [k] floats."""
    import numpy as np

    offs = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, 3)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    h = _out()
    nx, ny, nz = (int(d) for d in dims)
    call("apcg_stencil_create", nx, ny, nz, offs.shape[0], offs.ctypes.data_as(P), w.ctypes.data_as(P), C.byref(h))
    return h.value


def cg_plan_create_stencil(ctx, stencil, opts: CgOpts):
    h = _out()
    call("apcg_cg_plan_create_stencil", C.c_void_p(ctx), C.c_void_p(stencil), C.byref(opts), C.byref(h))
    return h.value


def ir_plan_create_stencil(ctx, stencil, opts: IrOpts):
    h = _out()
    call("apcg_ir_plan_create_stencil", C.c_void_p(ctx), C.c_void_p(stencil), C.byref(opts), C.byref(h))
    return h.value


def tfqmr_solve(ctx, A, b, x, opts: CgOpts) -> dict:
    """Jacobi-preconditioned TFQMR (apcg_vec/apcg_mat handles)."""
    res = CgResult()
    call("apcg_tfqmr_solve", C.c_void_p(ctx), C.c_void_p(A), C.c_void_p(b), C.c_void_p(x), C.byref(opts), C.byref(res))
    out = res.as_dict()
    if opts.history_len:
        out["alpha"] = list(opts._hist[0])
        out["beta"] = list(opts._hist[1])
    return out


def tfqmr_plan_create(ctx, A, opts: CgOpts):
    h = _out()
    call("apcg_tfqmr_plan_create", C.c_void_p(ctx), C.c_void_p(A), C.byref(opts), C.byref(h))
    return h.value


def tfqmr_plan_solve(plan, b, x) -> dict:
    res = CgResult()
    call("apcg_tfqmr_plan_solve", C.c_void_p(plan), C.c_void_p(b), C.c_void_p(x), C.byref(res))
    return res.as_dict()


def batch_plan_create(ctx, sys_row_off, rowptr, col, val, opts: CgOpts):
    """sys_row_off: host int32 array [nsys+1]; rowptr/col/val: CUDA tensors of the concatenation."""
    import numpy as np

    off = np.ascontiguousarray(sys_row_off, dtype=np.int32)
    h = _out()
    call(
        "apcg_batch_plan_create", C.c_void_p(ctx), off.shape[0] - 1, off.ctypes.data_as(P), C.c_void_p(_ptr(rowptr)),
        C.c_void_p(_ptr(col)), C.c_void_p(_ptr(val)), C.byref(opts), C.byref(h),
    )
    return h.value


def batch_plan_history(plan, sys: int, history_len: int) -> dict:
    """alpha/beta of iterations 1..history_len of system sys in the plan's last solve (NaN where not reached)."""
    a, b = (C.c_double * history_len)(), (C.c_double * history_len)()
    call("apcg_batch_plan_history", C.c_void_p(plan), int(sys), a, b)
    return {"alpha": list(a), "beta": list(b)}


def batch_plan_solve(plan, b, x, nsys: int | None = None):
    """Solve all systems; returns per-system results when nsys is given (blocks), else None (enqueued only)."""
    if nsys is None:
        call("apcg_batch_plan_solve", C.c_void_p(plan), C.c_void_p(_ptr(b)), C.c_void_p(_ptr(x)), None)
        return None
    res = (BatchResult * nsys)()
    call("apcg_batch_plan_solve", C.c_void_p(plan), C.c_void_p(_ptr(b)), C.c_void_p(_ptr(x)), res)
    return [
        {"iters": int(r.iters), "reason": REASONS.get(int(r.reason), int(r.reason)), "rel_res": float(r.rel_res), "outer": int(r.outer)}
        for r in res
    ]


def batch_ir_plan_create(ctx, sys_row_off, rowptr, col, val, val32, opts: IrOpts):
    """Batched mixed-precision refinement plan; val (float64) and val32 (float32) CUDA tensors, either may be None."""
    import numpy as np

    off = np.ascontiguousarray(sys_row_off, dtype=np.int32)
    h = _out()
    call(
        "apcg_batch_ir_plan_create", C.c_void_p(ctx), off.shape[0] - 1, off.ctypes.data_as(P), C.c_void_p(_ptr(rowptr)),
        C.c_void_p(_ptr(col)), C.c_void_p(_ptr(val)), C.c_void_p(_ptr(val32)), C.byref(opts), C.byref(h),
    )
    return h.value


def batch_plan_tune(plan, b) -> list[tuple]:
    buf = C.create_string_buffer(1 << 14)
    call("apcg_batch_plan_tune", C.c_void_p(plan), C.c_void_p(_ptr(b)), buf, len(buf))
    rows = []
    for line in buf.value.decode().splitlines():
        f = line.split()
        rows.append({"n_lo": int(f[0]), "n_hi": int(f[1]), "cluster": int(f[2]), "threads": int(f[3]), "rows_per_thread": int(f[4]), "ms": float(f[5])})
    return rows


def cg_solve_noalloc(stream, rowptr, col, val, b, x, opts: CgOpts) -> dict:
    """Solve through the entry point that allocates no device memory (CUDA tensors; x updated in place)."""
    s = 0 if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    res = CgResult()
    call(
        "apcg_cg_solve_noalloc", C.c_void_p(s), rowptr.numel() - 1, col.numel(), C.c_void_p(_ptr(rowptr)),
        C.c_void_p(_ptr(col)), C.c_void_p(_ptr(val)), C.c_void_p(_ptr(b)), C.c_void_p(_ptr(x)), C.byref(opts), C.byref(res),
    )
    return res.as_dict()


def ir_opts(rtol=1e-10, atol=0.0, max_outer=50, max_inner=1000, rtol_inner=1e-4, inner_check_every=1, history_len=0):
    o = IrOpts()
    call("apcg_ir_opts_default", C.byref(o))
    o.rtol, o.atol, o.max_outer, o.max_inner = rtol, atol, max_outer, max_inner
    o.rtol_inner, o.inner_check_every = rtol_inner, inner_check_every
    o.history_len = history_len
    hist = None
    if history_len:
        hist = ((C.c_double * history_len)(), (C.c_double * history_len)())
        o.alpha_hist = C.cast(hist[0], C.POINTER(C.c_double))
        o.beta_hist = C.cast(hist[1], C.POINTER(C.c_double))
    o._hist = hist  # keep the buffers alive with the struct (a plan keeps the pointers)
    return o


def ir_history(opts: IrOpts) -> dict:
    """The inner alpha/beta of the first correction written by the last solve of a plan made with opts."""
    if not opts.history_len:
        return {"alpha": [], "beta": []}
    return {"alpha": list(opts._hist[0]), "beta": list(opts._hist[1])}


def ir_plan_inner_spmv(plan, p, w) -> float:
    """w = A32 p by the plan's float32 inner SpMV (apcg_vec handles of float32 vectors); returns (p, w)."""
    g = C.c_double()
    call("apcg_ir_plan_inner_spmv", C.c_void_p(plan), C.c_void_p(p), C.c_void_p(w), C.byref(g))
    return float(g.value)


def ir_plan_profile(plan, b, x, iters: int) -> list[float]:
    """[residual, inner K1, inner K2, inner K3] kernel times in ms (see apcg_ir_plan_profile)."""
    ms = (C.c_float * 4)()
    call("apcg_ir_plan_profile", C.c_void_p(plan), C.c_void_p(b), C.c_void_p(x), iters, ms)
    return [float(v) for v in ms]


def ir_plan_create(ctx, A64, A32, opts: IrOpts):
    h = _out()
    call("apcg_ir_plan_create", C.c_void_p(ctx), C.c_void_p(A64), C.c_void_p(A32), C.byref(opts), C.byref(h))
    return h.value


def ir_plan_solve(plan, b, x) -> dict:
    res = IrResult()
    call("apcg_ir_plan_solve", C.c_void_p(plan), C.c_void_p(b), C.c_void_p(x), C.byref(res))
    return res.as_dict()


def get_counters() -> dict:
    c = Counters()
    call("apcg_get_counters", C.byref(c))
    return c.as_dict()


def reset_counters():
    call("apcg_reset_counters")


def header_functions() -> list[str]:
    """Entry points declared in include/apcg.h."""
    import re

    txt = open(HEADER).read()
    return re.findall(r"^APCG_API\s+[\w\s\*]+?\b(apcg_\w+)\s*\(", txt, flags=re.M)


# ---------------------------------------------------------------- host-only marking simulator


class Sim:
    """The host-only simulator of the marking rules (apcg_sim_*)."""

    def __init__(self, nctx: int):
        h = _out()
        call("apcg_sim_create", nctx, C.byref(h))
        self.h = h.value

    def op(self, ctx: int, accesses):
        ids = (u64 * len(accesses))(*[a[0] for a in accesses])
        modes = (i32 * len(accesses))(*[a[1] for a in accesses])
        call("apcg_sim_op", C.c_void_p(self.h), ctx, len(accesses), ids, modes)

    def complete(self, ctx: int, seq: int):
        call("apcg_sim_complete", C.c_void_p(self.h), ctx, seq)

    def log(self) -> list[str]:
        buf = C.create_string_buffer(1 << 16)
        call("apcg_sim_log", C.c_void_p(self.h), buf, len(buf))
        return [l for l in buf.value.decode().split("\n") if l]

    def close(self):
        if self.h:
            call("apcg_sim_destroy", C.c_void_p(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
