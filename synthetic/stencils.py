"""Finite-difference stencil matrices in CSR form (int32 indices, float64 values).

Conventions (Sec. 4.1 names the stencils but not their scaling or boundary
treatment; these are the readings used throughout the project):

* unscaled integer stencils, no h^2 factor;
* homogeneous Dirichlet boundary by elimination: a neighbour outside the grid
  is dropped from the row, the diagonal is unchanged;
* lexicographic ordering with x fastest: row = x + nx*(y + ny*z);
* inside every row the column indices ascend.

The builders only assemble values; nothing here solves or preconditions.
"""

from __future__ import annotations

from dataclasses import dataclass
import itertools

import numpy as np
import scipy.sparse as sp


@dataclass
class CSR:
    """A square sparse matrix in compressed-row form."""

    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]

    @property
    def n(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix(
            (self.val, self.col.astype(np.int64), self.rowptr.astype(np.int64)),
            shape=(self.n, self.n),
        )

    def to_dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


def _grid_coords(dims):
    nx, ny, nz = dims
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    return n, idx, x, y, z


def _assemble(dims, offsets, offdiag_value, diag_value) -> CSR:
    """Build a stencil CSR.

    ``offsets`` is a list of (dx, dy, dz) excluding (0,0,0).  ``offdiag_value(k,
    valid, idx_nb)`` returns the value of the k-th neighbour column for every row
    (only entries where ``valid`` is true are kept).  ``diag_value`` is an array
    or scalar for the diagonal.
    """
    nx, ny, nz = dims
    n, idx, x, y, z = _grid_coords(dims)
    allofs = list(offsets) + [(0, 0, 0)]
    allofs.sort(key=lambda o: o[0] + nx * (o[1] + ny * o[2]))
    cols, vals, masks = [], [], []
    for o in allofs:
        dx, dy, dz = o
        if o == (0, 0, 0):
            valid = np.ones(n, dtype=bool)
            v = np.broadcast_to(np.asarray(diag_value, dtype=np.float64), (n,))
        else:
            valid = (
                (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & (z + dz >= 0) & (z + dz < nz)
            )
            k = offsets.index(o)
            v = np.broadcast_to(np.asarray(offdiag_value(k, valid, idx + dx + nx * (dy + ny * dz)), dtype=np.float64), (n,))
        lin = dx + nx * (dy + ny * dz)
        cols.append((idx + lin).astype(np.int32, copy=False) if n < 2**31 else None)
        vals.append(v)
        masks.append(valid)
    mask = np.stack(masks, axis=1)
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    col = np.stack(cols, axis=1)[mask]
    val = np.stack(vals, axis=1)[mask]
    return CSR(rowptr.astype(np.int32), np.ascontiguousarray(col, dtype=np.int32), np.ascontiguousarray(val, dtype=np.float64))


def _neighbours(ndim, full):
    rng = (-1, 0, 1)
    out = []
    for d in itertools.product(rng, repeat=ndim):
        if all(c == 0 for c in d):
            continue
        if not full and sum(abs(c) for c in d) != 1:
            continue
        d = tuple(d) + (0,) * (3 - ndim)
        out.append(d)
    return out


STENCIL_KINDS = {"5pt": (2, False, 4.0), "9pt": (2, True, 8.0), "7pt": (3, False, 6.0), "27pt": (3, True, 26.0)}


def stencil_terms(kind: str, dims, shift: float = 0.0):
    """Terms (offsets [k, 3], weights [k]) of the constant Laplace stencils above, in ascending order of
    the linear offset dx + nx (dy + ny dz) -- the column order of the assembled rows.

    kind: "5pt" and "9pt" (2-D, nz = 1), "7pt" and "27pt" (3-D); all neighbours -1, centre the number of
    neighbours (+ shift)."""
    ndim, full, diag = STENCIL_KINDS[kind]
    nx, ny, _ = dims
    offs = _neighbours(ndim, full) + [(0, 0, 0)]
    offs.sort(key=lambda o: o[0] + nx * (o[1] + ny * o[2]))
    w = [diag + shift if o == (0, 0, 0) else -1.0 for o in offs]
    return np.array(offs, dtype=np.int32), np.array(w, dtype=np.float64)


def stencil_matrix(kind: str, dims, shift: float = 0.0) -> CSR:
    """The assembled CSR of stencil_terms(kind, dims, shift) on a grid of the given dims."""
    ndim, full, diag = STENCIL_KINDS[kind]
    return _assemble(tuple(int(d) for d in dims), _neighbours(ndim, full), lambda k, v, j: -1.0, diag + shift)


def laplace_2d_5pt(N: int, shift: float = 0.0) -> CSR:
    """5-point Laplacian on an N x N grid: diagonal 4 (+shift), neighbours -1."""
    offs = _neighbours(2, full=False)
    return _assemble((N, N, 1), offs, lambda k, v, j: -1.0, 4.0 + shift)


def laplace_2d_9pt(N: int) -> CSR:
    """9-point Laplacian on an N x N grid: diagonal 8, all 8 neighbours -1."""
    offs = _neighbours(2, full=True)
    return _assemble((N, N, 1), offs, lambda k, v, j: -1.0, 8.0)


def laplace_3d_7pt(N: int) -> CSR:
    """7-point Laplacian on an N^3 grid: diagonal 6, neighbours -1."""
    offs = _neighbours(3, full=False)
    return _assemble((N, N, N), offs, lambda k, v, j: -1.0, 6.0)


def laplace_3d_27pt(N: int) -> CSR:
    """27-point constant stencil on an N^3 grid: diagonal 26, all 26 neighbours -1."""
    offs = _neighbours(3, full=True)
    return _assemble((N, N, N), offs, lambda k, v, j: -1.0, 26.0)


def diffusion_3d_27pt(N: int, kappa: np.ndarray) -> CSR:
    """Variable-coefficient 27-point diffusion operator on an N^3 grid.

    The coupling between cells i and j is the harmonic mean
    w_ij = 2 (k_i k_j) / (k_i + k_j) (bit-symmetric as written), the
    off-diagonal entry is -w_ij, and a neighbour outside the grid acts as a
    Dirichlet ghost cell carrying k_i (weight k_i, diagonal only).  The
    diagonal is the sum of the 26 weights, so the matrix is symmetric and
    diagonally dominant, strictly on the boundary: SPD.
    """
    kappa = np.asarray(kappa, dtype=np.float64)
    n = N**3
    assert kappa.shape == (n,)
    offs = _neighbours(3, full=True)
    diag = np.zeros(n, dtype=np.float64)
    weights = []
    _, idx, x, y, z = _grid_coords((N, N, N))
    for (dx, dy, dz) in offs:
        valid = (x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N) & (z + dz >= 0) & (z + dz < N)
        j = np.where(valid, idx + dx + N * (dy + N * dz), idx)
        kj = kappa[j]
        w = np.where(valid, 2.0 * (kappa * kj) / (kappa + kj), kappa)
        diag += w
        weights.append(w)
    return _assemble((N, N, N), offs, lambda k, v, j: -weights[k], diag)


def aniso_3d_7pt_fp32exact(nx: int, ny: int, nz: int, ax: float, ay: float, az: float) -> CSR:
    """Anisotropic 7-point operator whose values are exactly representable in float32.

    Off-diagonals are -a_d with each a_d first rounded to float32; the diagonal
    2(a_x+a_y+a_z) is summed in float64 and rounded to float32 upward, so the
    float32 copy of the matrix is the very matrix the float64 path solves and
    every row stays diagonally dominant.
    """
    a = [float(np.float32(v)) for v in (ax, ay, az)]
    d64 = 2.0 * (a[0] + a[1] + a[2])
    d32 = np.float32(d64)
    if float(d32) < d64:
        d32 = np.nextafter(d32, np.float32(np.inf))
    offs = _neighbours(3, full=False)

    def off(k, v, j):
        dx, dy, dz = offs[k]
        return -(a[0] if dx else a[1] if dy else a[2])

    return _assemble((nx, ny, nz), offs, off, float(d32))


def diagonal_csr(d: np.ndarray) -> CSR:
    """A diagonal matrix as CSR."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    return CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d.copy())


def random_spd_csr(n: int, density: float, rng: np.random.Generator, dominance: float = 1.0) -> CSR:
    """A random sparse symmetric positive-definite matrix (n small).

    Symmetric random off-diagonal pattern with values in [-1, 1]; the diagonal
    is the absolute row sum times (1 + dominance * U[0,1]) plus a little, so the
    matrix is strictly diagonally dominant with a positive diagonal: SPD.
    """
    m = sp.random(n, n, density=density, random_state=rng, data_rvs=lambda k: rng.uniform(-1.0, 1.0, k))
    m = sp.triu(m, k=1)
    m = (m + m.T).tocsr()
    rs = np.asarray(abs(m).sum(axis=1)).ravel()
    diag = rs * (1.0 + dominance * rng.uniform(0.0, 1.0, n)) + 0.1 + rng.uniform(0.0, 1.0, n)
    m = (m + sp.diags(diag)).tocsr()
    m.sort_indices()
    return CSR(m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64))


def convection_diffusion_2d(N: int, gx: float, gy: float, shift: float = 0.0) -> CSR:
    """Nonsymmetric 5-point convection-diffusion operator on an N x N grid (Dirichlet, unscaled).

    Central differences: diagonal 4 + shift, west/east couplings -1 -/+ gx,
    south/north -1 -/+ gy (gx, gy are the cell Peclet numbers over two).  For
    |gx|, |gy| < 1 every off-diagonal is negative and the matrix is a
    nonsingular M-matrix; it is symmetric only for gx = gy = 0.
    """
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    ix, iy = idx % N, idx // N
    rows, cols, vals = [idx], [idx], [np.full(n, 4.0 + shift)]
    for dx, dy, v in ((-1, 0, -1.0 - gx), (1, 0, -1.0 + gx), (0, -1, -1.0 - gy), (0, 1, -1.0 + gy)):
        ok = (ix + dx >= 0) & (ix + dx < N) & (iy + dy >= 0) & (iy + dy < N)
        rows.append(idx[ok])
        cols.append(idx[ok] + dx + dy * N)
        vals.append(np.full(int(ok.sum()), v))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    A.sort_indices()
    return CSR(A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))


def graph_laplacian_csr(n: int, rng: np.random.Generator, mean_degree: float = 6.0, hub_degrees=(),
                        shift: float = 1.0) -> CSR:
    """Weighted graph Laplacian of a random graph plus shift * I (symmetric positive definite).

    Rows of very different lengths: about n * mean_degree / 2 random edges
    among the ordinary nodes (degrees roughly Poisson, some nodes isolated, so
    their row holds only the diagonal), and hub nodes at evenly spaced indices,
    hub h joined to exactly hub_degrees[h] distinct ordinary nodes (its row has
    hub_degrees[h] + 1 entries).  Edge weights ~ U[0.5, 2].
    """
    hubs = np.array([(k + 1) * n // (len(hub_degrees) + 1) for k in range(len(hub_degrees))], dtype=np.int64)
    ordinary = np.setdiff1d(np.arange(n, dtype=np.int64), hubs)
    m = int(n * mean_degree / 2)
    i = ordinary[rng.integers(0, ordinary.size, m)]
    j = ordinary[rng.integers(0, ordinary.size, m)]
    keep = i != j
    i, j = i[keep], j[keep]
    for h, d in zip(hubs, hub_degrees):
        nb = rng.choice(ordinary, size=int(d), replace=False)
        i = np.concatenate([i, np.full(nb.size, h)])
        j = np.concatenate([j, nb])
    w = rng.uniform(0.5, 2.0, i.size)
    W = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([i, j]), np.concatenate([j, i]))), shape=(n, n)).tocsr()
    W.sum_duplicates()
    deg = np.asarray(W.sum(axis=1)).ravel()
    A = (sp.diags(deg + shift) - W).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return CSR(A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))


def sine_mode_2d(N: int, j1: int, j2: int) -> np.ndarray:
    """Discrete sine mode sin(j1 pi x/(N+1)) sin(j2 pi y/(N+1)) on the N x N grid, x fastest."""
    g = np.arange(1, N + 1, dtype=np.float64)
    sx = np.sin(j1 * np.pi * g / (N + 1))
    sy = np.sin(j2 * np.pi * g / (N + 1))
    return np.outer(sy, sx).ravel()


def sine_mode_3d(N: int, j1: int, j2: int, j3: int) -> np.ndarray:
    """Discrete sine mode on the N^3 grid, x fastest."""
    g = np.arange(1, N + 1, dtype=np.float64)
    sx = np.sin(j1 * np.pi * g / (N + 1))
    sy = np.sin(j2 * np.pi * g / (N + 1))
    sz = np.sin(j3 * np.pi * g / (N + 1))
    return (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).ravel()


def rhs_from_solution(A: CSR, x_true: np.ndarray) -> np.ndarray:
    """b = A x_true in float64 (scipy.sparse product)."""
    return np.asarray(A.to_scipy() @ np.asarray(x_true, dtype=np.float64), dtype=np.float64)
