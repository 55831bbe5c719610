"""Build libapcg.so in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into
``paper_2306_17801_gb300/_build/libapcg.so`` (static CUDA runtime).  A build
is skipped when the library is newer than every source and header.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libapcg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libapcg")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(SRC_DIR, "*.cu")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(SRC_DIR, "*.hpp")) + glob.glob(os.path.join(SRC_DIR, "*.cuh")) + [
        os.path.join(ROOT, "include", "apcg.h")
    ]


def source_hash() -> str:
    """sha256 over the library's sources and header (identifies a kernel build)."""
    import hashlib

    h = hashlib.sha256()
    for p in sorted(_deps()):
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _code_tokens(text: bytes) -> bytes:
    """Source text without comments and with whitespace runs collapsed (string literals kept)."""
    import re

    tok = re.compile(rb'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/|\s+', re.S)

    def keep(m):
        t = m.group(0)
        if t.startswith(b"//") or t.startswith(b"/*"):
            return b" "
        if t[:1].isspace():
            return b" "
        return t

    return re.sub(rb" +", b" ", tok.sub(keep, text)).strip()


def unit_hash(unit: str) -> str:
    """sha256 over one translation unit and every local header it includes, transitively,
    with comments and layout removed (identifies the code of the kernels defined in that
    unit: an edit of a comment keeps the hash)."""
    import hashlib
    import re

    inc = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)
    dirs = [SRC_DIR, os.path.join(ROOT, "include")]
    seen: dict[str, bytes] = {}
    todo = [os.path.join(SRC_DIR, unit)]
    while todo:
        p = todo.pop()
        if p in seen:
            continue
        with open(p, "rb") as f:
            seen[p] = f.read()
        for name in inc.findall(seen[p].decode("utf-8", "replace")):
            for d in [os.path.dirname(p)] + dirs:
                q = os.path.join(d, name)
                if os.path.exists(q):
                    todo.append(q)
                    break
    h = hashlib.sha256()
    for p in sorted(seen):
        h.update(os.path.basename(p).encode())
        h.update(_code_tokens(seen[p]))
    return h.hexdigest()[:16]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src: str, log_dir: str) -> str:
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    with open(os.path.join(log_dir, os.path.basename(src) + ".log"), "w") as f:
        f.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{p.stderr[-6000:]}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and up_to_date():
        return LIB
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, OUT_DIR), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr[-6000:]}")
    os.replace(tmp, LIB)
    if verbose:
        for s in srcs:
            print(open(os.path.join(OUT_DIR, os.path.basename(s) + ".log")).read())
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
