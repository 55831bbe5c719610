"""Named workloads: single SPD systems and batches, seeded.

Random draws use ``numpy.random.default_rng(seed)`` (PCG64).  Draw order: all
structure parameters first (grid sides, shifts, anisotropy, coefficient
field), then the exact solutions x_true, system by system in index order.
b = A x_true is formed in float64 and shared by every consumer.

Workloads (sizes as in the benchmark configurations):

* ``c1``  2-D 5-point Laplacian, 64 x 64 (n = 4096, nnz = 20,224).
* ``c2``  3-D 7-point Laplacian, 128^3 (n = 2,097,152, nnz = 14,581,760).
* ``c3``  3-D 27-point variable-coefficient diffusion, 160^3 (n = 4,096,000,
  nnz = 109,215,352), kappa = 10^U(-2,2) per cell.
* batches: 5-point + sigma I (sides U{16..128}, sigma U[1e-3, 1]) and
  anisotropic 7-point with float32-exact values (sides U{8..32} per axis,
  a_y, a_z = 10^U(0,3)).

Reduced-size variants keep the same recipe so that the oracle finishes in
seconds while the inputs still span many GPU tiles and a ragged tail.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .stencils import (
    CSR,
    aniso_3d_7pt_fp32exact,
    diffusion_3d_27pt,
    laplace_2d_5pt,
    laplace_3d_7pt,
    laplace_3d_27pt,
    laplace_2d_9pt,
    rhs_from_solution,
)


@dataclass
class Problem:
    name: str
    A: CSR
    b: np.ndarray
    x_true: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.n

    @property
    def nnz(self) -> int:
        return self.A.nnz


@dataclass
class Batch:
    """Independent systems concatenated row-wise.

    ``sys_row_off[s] .. sys_row_off[s+1]`` are the rows of system s.  ``rowptr``
    runs over the whole concatenation (global nnz positions); ``col`` holds
    column indices local to each system (0 .. n_s-1).  ``b`` and ``x_true`` are
    concatenated the same way.
    """

    name: str
    sys_row_off: np.ndarray  # int32 [B+1]
    rowptr: np.ndarray  # int32 [N+1]
    col: np.ndarray  # int32 [nnz], local
    val: np.ndarray  # float64 [nnz]
    b: np.ndarray
    x_true: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nsys(self) -> int:
        return int(self.sys_row_off.shape[0] - 1)

    @property
    def n_total(self) -> int:
        return int(self.sys_row_off[-1])

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def system(self, s: int) -> tuple[CSR, np.ndarray, np.ndarray]:
        r0, r1 = int(self.sys_row_off[s]), int(self.sys_row_off[s + 1])
        e0, e1 = int(self.rowptr[r0]), int(self.rowptr[r1])
        A = CSR((self.rowptr[r0 : r1 + 1] - e0).astype(np.int32), self.col[e0:e1].copy(), self.val[e0:e1].copy())
        return A, self.b[r0:r1].copy(), self.x_true[r0:r1].copy()


def _uniform_solution(rng, n):
    return rng.uniform(-1.0, 1.0, size=n)


def single_problem(name: str, seed: int = 0, size: int | None = None) -> Problem:
    """Build one of the single-system workloads; ``size`` overrides the grid side."""
    rng = np.random.default_rng(seed)
    meta = {"seed": seed}
    if name == "c1":
        N = size or 64
        A = laplace_2d_5pt(N)
        meta.update(grid=(N, N), stencil="5pt")
    elif name == "c2":
        N = size or 128
        A = laplace_3d_7pt(N)
        meta.update(grid=(N, N, N), stencil="7pt")
    elif name == "c3":
        N = size or 160
        kappa = 10.0 ** rng.uniform(-2.0, 2.0, size=N**3)
        A = diffusion_3d_27pt(N, kappa)
        meta.update(grid=(N, N, N), stencil="27pt-var")
    elif name == "lap27":
        N = size or 32
        A = laplace_3d_27pt(N)
        meta.update(grid=(N, N, N), stencil="27pt")
    elif name == "lap9":
        N = size or 64
        A = laplace_2d_9pt(N)
        meta.update(grid=(N, N), stencil="9pt")
    else:
        raise KeyError(name)
    x_true = _uniform_solution(rng, A.n)
    b = rhs_from_solution(A, x_true)
    return Problem(name, A, b, x_true, meta)


def _concat(name, systems, meta) -> Batch:
    rows = [A.n for A, _, _ in systems]
    sys_row_off = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(rows, out=sys_row_off[1:])
    nnz = [A.nnz for A, _, _ in systems]
    nnz_off = np.zeros(len(systems) + 1, dtype=np.int64)
    np.cumsum(nnz, out=nnz_off[1:])
    if nnz_off[-1] >= 2**31 or sys_row_off[-1] >= 2**31:
        raise ValueError("batch does not fit int32 indices")
    rowptr = np.empty(int(sys_row_off[-1]) + 1, dtype=np.int64)
    for s, (A, _, _) in enumerate(systems):
        rowptr[sys_row_off[s] : sys_row_off[s + 1]] = A.rowptr[:-1].astype(np.int64) + nnz_off[s]
    rowptr[-1] = nnz_off[-1]
    col = np.concatenate([A.col for A, _, _ in systems]).astype(np.int32)
    val = np.concatenate([A.val for A, _, _ in systems])
    b = np.concatenate([bb for _, bb, _ in systems])
    xt = np.concatenate([xx for _, _, xx in systems])
    return Batch(name, sys_row_off.astype(np.int32), rowptr.astype(np.int32), col, val, b, xt, meta)


def batch_shifted_5pt(nsys: int = 1024, seed: int = 0, side_lo: int = 16, side_hi: int = 128) -> Batch:
    """Batch of 2-D 5-point Laplacians plus sigma I, side ~ U{lo..hi}, sigma ~ U[1e-3, 1]."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=nsys)
    sigmas = rng.uniform(1e-3, 1.0, size=nsys)
    systems = []
    mats = [laplace_2d_5pt(int(N), float(s)) for N, s in zip(sides, sigmas)]
    for A in mats:
        xt = _uniform_solution(rng, A.n)
        systems.append((A, rhs_from_solution(A, xt), xt))
    return _concat("shifted5", systems, {"seed": seed, "sides": sides, "sigmas": sigmas})


def batch_aniso_7pt(nsys: int = 4096, seed: int = 0, side_lo: int = 8, side_hi: int = 32) -> Batch:
    """Batch of anisotropic 3-D 7-point operators with float32-exact values.

    Sides ~ U{lo..hi} per axis; (a_x, a_y, a_z) = (1, 10^U(0,3), 10^U(0,3)).
    """
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=(nsys, 3))
    ay = 10.0 ** rng.uniform(0.0, 3.0, size=nsys)
    az = 10.0 ** rng.uniform(0.0, 3.0, size=nsys)
    mats = [
        aniso_3d_7pt_fp32exact(int(s[0]), int(s[1]), int(s[2]), 1.0, float(y), float(z))
        for s, y, z in zip(sides, ay, az)
    ]
    systems = []
    for A in mats:
        xt = _uniform_solution(rng, A.n)
        systems.append((A, rhs_from_solution(A, xt), xt))
    return _concat("aniso7", systems, {"seed": seed, "sides": sides, "ay": ay, "az": az})


PROBLEMS = {
    "c1": dict(kind="single", name="c1", desc="2D 5-point Laplacian 64x64, n=4096"),
    "c2": dict(kind="single", name="c2", desc="3D 7-point Laplacian 128^3, n=2,097,152"),
    "c3": dict(kind="single", name="c3", desc="3D 27-point variable-kappa diffusion 160^3, n=4,096,000"),
    "c4": dict(kind="batch", name="shifted5", desc="1024 x (2D 5-point + sigma I), sides 16..128"),
    "c5": dict(kind="batch", name="aniso7", desc="4096 x anisotropic 3D 7-point, sides 8..32, fp32-exact"),
}
