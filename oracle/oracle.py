"""ctypes front end of the plain C oracle (``pcg_oracle.c``, ``tfqmr_oracle.c``, ``stencil_oracle.c``).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg may use it.  The library is compiled with gcc (ISO C11,
-ffp-contract=off so that no multiply-add is fused and x86 and Arm hosts give
the same bits) into ``oracle/_build``.

Every function takes numpy arrays and returns numpy arrays; see the C file for
the algorithms (textbook Jacobi-PCG, Sec. 4.1-4.2, loop order of the mixed-API
example of Sec. 3.3; Jacobi-preconditioned TFQMR, Sec. 4.3).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("pcg_oracle.c", "tfqmr_oracle.c", "stencil_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_OMP_SRC = os.path.join(_HERE, "pcg_oracle_omp.c")
_OMP_LIB = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp_lib = None

REASON = {0: "converged", 1: "not_converged", 2: "breakdown", 3: "bad_diagonal", 4: "no_memory"}


class _Res(C.Structure):
    _fields_ = [("iters", C.c_int32), ("reason", C.c_int32), ("rr", C.c_double), ("bnorm", C.c_double)]


class _TqRes(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("reason", C.c_int32),
        ("tau", C.c_double),
        ("bound", C.c_double),
        ("bnorm", C.c_double),
    ]


class _IrRes(C.Structure):
    _fields_ = [
        ("outer", C.c_int32),
        ("inner_total", C.c_int32),
        ("reason", C.c_int32),
        ("pad", C.c_int32),
        ("rel_res", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False) -> str | None:
    """Compile the multi-threaded timing variant (OpenMP); None where the compiler has no OpenMP."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_OMP_LIB) or os.path.getmtime(_OMP_LIB) < os.path.getmtime(_OMP_SRC):
        tmp = _OMP_LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", _OMP_SRC,
               "-o", tmp, "-lm"]
        if subprocess.run(cmd, capture_output=True).returncode != 0:
            return None
        os.replace(tmp, _OMP_LIB)
    return _OMP_LIB


def host_cores() -> int:
    """Cores this process may run on (the affinity mask, else the CPU count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def host_cpu_model() -> str:
    """CPU model string of this host (from /proc/cpuinfo or lscpu), or the machine type."""
    import platform

    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def pcg_omp(A, b, x0=None, rtol=1e-8, atol=0.0, max_it=None, check_every=1, threads=0) -> dict:
    """The float64 Jacobi-PCG oracle's steps split over OpenMP threads (timing only; threads=0: all)."""
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            path = build_omp()
            if path is None:
                raise RuntimeError("gcc without OpenMP: the multi-threaded oracle variant is unavailable")
            lib = C.CDLL(path)
            P = C.c_void_p
            lib.oracle_pcg_omp.argtypes = [C.c_int64, P, P, P, P, P, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                           C.c_int32, C.POINTER(_Res)]
            lib.oracle_pcg_omp.restype = C.c_int
            _omp_lib = lib
    rowptr, col, val = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n, dtype=np.float64) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    if max_it is None:
        max_it = max(10 * A.n, 10)
    res = _Res()
    _omp_lib.oracle_pcg_omp(A.n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), float(rtol), float(atol), int(max_it),
                            int(check_every), int(threads), C.byref(res))
    return dict(x=x, iters=int(res.iters), reason=REASON[res.reason], rr=float(res.rr), bnorm=float(res.bnorm))


def load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            i64, i32, f64, f32 = C.c_int64, C.c_int32, C.c_double, C.c_float
            lib.oracle_dot.argtypes = [i64, P, P]
            lib.oracle_dot.restype = f64
            lib.oracle_sum.argtypes = [i64, P]
            lib.oracle_sum.restype = f64
            lib.oracle_spmv.argtypes = [i64, P, P, P, P, P]
            lib.oracle_spmv.restype = None
            lib.oracle_spmv_f32.argtypes = [i64, P, P, P, P, P]
            lib.oracle_spmv_f32.restype = None
            lib.oracle_diagonal.argtypes = [i64, P, P, P, P]
            lib.oracle_diagonal.restype = C.c_int
            lib.oracle_pcg.argtypes = [i64, P, P, P, P, P, f64, f64, i32, i32, i32, P, P, P, P, P, i32, C.POINTER(_Res)]
            lib.oracle_pcg.restype = C.c_int
            lib.oracle_pcg_f32.argtypes = [i64, P, P, P, P, P, f32, i32, i32, i32, P, P, P, i32, C.POINTER(_Res)]
            lib.oracle_pcg_f32.restype = C.c_int
            lib.oracle_ir.argtypes = [i64, P, P, P, P, P, P, f64, i32, f32, i32, i32, C.POINTER(_IrRes)]
            lib.oracle_ir.restype = C.c_int
            lib.oracle_tfqmr.argtypes = [i64, P, P, P, P, P, f64, f64, i32, i32, i32, P, P, P, i32, C.POINTER(_TqRes)]
            lib.oracle_tfqmr.restype = C.c_int
            lib.oracle_stencil_apply.argtypes = [i32, i32, i32, i32, P, P, P, P, i32]
            lib.oracle_stencil_apply.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(A):
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    return rowptr, col, val


def dot(x, y) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(load().oracle_dot(x.shape[0], _p(x), _p(y)))


def fsum(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(load().oracle_sum(x.shape[0], _p(x)))


def spmv(A, x) -> np.ndarray:
    rowptr, col, val = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n, dtype=np.float64)
    load().oracle_spmv(A.n, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def spmv_f32(A, x, val32=None) -> np.ndarray:
    """y = A x in float32 (A's values rounded to float32, or val32), float32 accumulation in column order."""
    rowptr, col, _ = _csr(A)
    val = np.ascontiguousarray(A.val if val32 is None else val32, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(A.n, dtype=np.float32)
    load().oracle_spmv_f32(A.n, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def diagonal(A):
    rowptr, col, val = _csr(A)
    d = np.empty(A.n, dtype=np.float64)
    bad = load().oracle_diagonal(A.n, _p(rowptr), _p(col), _p(val), _p(d))
    return d, bool(bad)


def pcg(A, b, x0=None, rtol=1e-8, atol=0.0, max_it=None, check_every=1, hist_len=0, mutation=0) -> dict:
    """Jacobi-PCG in float64.  Returns x, iters, reason, rr, bnorm and histories."""
    rowptr, col, val = _csr(A)
    n = A.n
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n, dtype=np.float64) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    if max_it is None:
        max_it = max(10 * n, 10)
    H = int(hist_len)
    hs = {k: np.full(max(H, 1), np.nan) for k in ("alpha", "beta", "gamma", "rho", "rr_hist")}
    res = _Res()
    load().oracle_pcg(
        n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), float(rtol), float(atol), int(max_it), int(check_every), H,
        _p(hs["alpha"]), _p(hs["beta"]), _p(hs["gamma"]), _p(hs["rho"]), _p(hs["rr_hist"]), int(mutation), C.byref(res),
    )
    out = dict(x=x, iters=int(res.iters), reason=REASON[res.reason], rr=float(res.rr), bnorm=float(res.bnorm))
    for k, v in hs.items():
        out[k] = v[:H]
    return out


def tfqmr(A, b, x0=None, rtol=1e-8, atol=0.0, max_it=None, check_every=1, hist_len=0, mutation=0) -> dict:
    """Jacobi-preconditioned (left) TFQMR in float64.  Returns x, iters, reason, tau, bound, bnorm
    (norms of the preconditioned system) and the alpha, beta and tau_hist histories."""
    rowptr, col, val = _csr(A)
    n = A.n
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n, dtype=np.float64) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    if max_it is None:
        max_it = max(10 * n, 10)
    H = int(hist_len)
    hs = {k: np.full(max(H, 1), np.nan) for k in ("alpha", "beta", "tau_hist")}
    res = _TqRes()
    load().oracle_tfqmr(
        n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), float(rtol), float(atol), int(max_it), int(check_every), H,
        _p(hs["alpha"]), _p(hs["beta"]), _p(hs["tau_hist"]), int(mutation), C.byref(res),
    )
    out = dict(x=x, iters=int(res.iters), reason=REASON[res.reason], tau=float(res.tau), bound=float(res.bound),
               bnorm=float(res.bnorm))
    for k, v in hs.items():
        out[k] = v[:H]
    return out


def stencil_apply(dims, offsets, weights, x, mutation=0) -> np.ndarray:
    """y = S x for a constant-coefficient stencil on an nx x ny x nz grid (Dirichlet: outside terms dropped)."""
    nx, ny, nz = (int(v) for v in dims)
    offs = np.ascontiguousarray(offsets, dtype=np.int32).reshape(-1, 3)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    assert offs.shape[0] == w.shape[0]
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(nx * ny * nz, dtype=np.float64)
    load().oracle_stencil_apply(nx, ny, nz, offs.shape[0], _p(offs), _p(w), _p(x), _p(y), int(mutation))
    return y


def pcg_f32(A, bf, rtol=1e-4, max_it=1000, check_every=1, x0=None, hist_len=0, mutation=0, val32=None) -> dict:
    """Jacobi-PCG entirely in float32 on A's values rounded to float32 (or on val32).  Returns x, iters,
    reason, rr, bnorm and the alpha, beta and rho histories (float32 values widened to float64)."""
    rowptr, col, _ = _csr(A)
    val32 = np.ascontiguousarray(A.val if val32 is None else val32, dtype=np.float32)
    bf = np.ascontiguousarray(bf, dtype=np.float32)
    x = np.zeros(A.n, dtype=np.float32) if x0 is None else np.array(x0, dtype=np.float32, copy=True)
    H = int(hist_len)
    hs = {k: np.full(max(H, 1), np.nan) for k in ("alpha", "beta", "rho")}
    res = _Res()
    load().oracle_pcg_f32(
        A.n, _p(rowptr), _p(col), _p(val32), _p(bf), _p(x), float(rtol), int(max_it), int(check_every), H,
        _p(hs["alpha"]), _p(hs["beta"]), _p(hs["rho"]), int(mutation), C.byref(res),
    )
    out = dict(x=x, iters=int(res.iters), reason=REASON[res.reason], rr=float(res.rr), bnorm=float(res.bnorm))
    for k, v in hs.items():
        out[k] = v[:H]
    return out


def ir(A, b, x0=None, rtol=1e-10, max_outer=50, rtol_inner=1e-4, max_inner=1000, inner_check_every=1, val32=None) -> dict:
    """float64 iterative refinement around a float32 inner Jacobi-PCG."""
    rowptr, col, val = _csr(A)
    v32 = np.ascontiguousarray(A.val if val32 is None else val32, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n, dtype=np.float64) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    res = _IrRes()
    load().oracle_ir(
        A.n, _p(rowptr), _p(col), _p(val), _p(v32), _p(b), _p(x), float(rtol), int(max_outer), float(rtol_inner),
        int(max_inner), int(inner_check_every), C.byref(res),
    )
    return dict(x=x, outer=int(res.outer), inner_total=int(res.inner_total), reason=REASON[res.reason], rel_res=float(res.rel_res))
