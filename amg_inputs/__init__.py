"""Seeded synthetic inputs for the sparsified-AMG solver and its oracle.

This module is the only code shared by the CUDA path, the CPU oracle, the
tests and the benchmark.  It produces the linear systems ``A x = b`` the paper
solves (Section 5: 3D Laplacian on a uniform mesh, Table 1's 7-point 3D
Poisson problem) and nothing of the AMG method itself: no strength, coarsening,
interpolation, Galerkin product or sparsification arithmetic lives here.

Conventions (all generators):

* interior unknowns of a uniform grid, homogeneous Dirichlet boundary
  eliminated, no ``h^2`` scaling, lexicographic order with x fastest;
* CSR with ``int32`` row pointers and column indices, ``float64`` values,
  columns strictly increasing in every row, the diagonal always stored;
* the matrix is symmetric (structurally and numerically) with a positive
  diagonal; every generator but the rotated anisotropic one also gives an
  M-matrix (non-positive off-diagonals, weakly diagonally dominant, strictly
  dominant on boundary rows).

Random numbers come from one counter-based generator, SplitMix64
(G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants as published in S. Vigna's reference
``splitmix64.c``): ``mix(key + 0x9E3779B97F4A7C15)``.  Uniforms are the top 53
bits scaled by ``2**-53``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(keys) -> np.ndarray:
    """SplitMix64 output for each 64-bit key (counter-based form)."""
    z = np.asarray(keys, dtype=np.uint64) + _GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """``n`` uniforms in [0, 1): key = (seed << 40) ^ (stream << 36) ^ index."""
    idx = np.arange(n, dtype=np.uint64)
    base = (np.uint64(seed) << np.uint64(40)) ^ (np.uint64(stream) << np.uint64(36))
    bits = splitmix64(idx ^ base) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -53)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform in [-1, 1): ``b_i = 2 u_i - 1``."""
    return 2.0 * uniform01(seed, n) - 1.0


@dataclass
class CSR:
    """A square sparse matrix in CSR form (host arrays)."""

    n: int
    rowptr: np.ndarray  # int32[n+1]
    col: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _assemble(n: int, cols: np.ndarray, vals: np.ndarray, name: str) -> CSR:
    """Compress a dense (n x S) stencil table; invalid slots have col < 0.

    The S slots of each row are in increasing column order already, so the
    compressed rows stay sorted.
    """
    mask = cols >= 0
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("matrix has 2**31 or more stored entries")
    col = cols[mask].astype(np.int32, copy=False)
    val = vals[mask].astype(np.float64, copy=False)
    return CSR(n, rowptr.astype(np.int32), col, val, name)


def poisson2d_5pt(N: int) -> CSR:
    """2D 5-point Laplacian on an N x N interior grid: diagonal 4, neighbours -1."""
    n = N * N
    i = np.arange(n, dtype=np.int64)
    x = i % N
    y = i // N
    table = [(-N, y > 0), (-1, x > 0), (0, None), (1, x < N - 1), (N, y < N - 1)]
    cols = np.empty((n, len(table)), dtype=np.int64)
    vals = np.empty((n, len(table)), dtype=np.float64)
    for s, (off, ok) in enumerate(table):
        c = i + off
        if ok is not None:
            c = np.where(ok, c, -1)
        cols[:, s] = c
        vals[:, s] = 4.0 if off == 0 else -1.0
    return _assemble(n, cols, vals, f"poisson2d_5pt_{N}")


def _box3d(N: int, radius_points, value_fn, name: str) -> CSR:
    """Generic 3D box stencil on an N^3 interior grid.

    ``radius_points`` is the list of (dz, dy, dx) offsets (sorted so that the
    linear offsets increase); ``value_fn(dz, dy, dx)`` gives the coefficient.
    Zero coefficients are not stored.
    """
    n = N * N * N
    i = np.arange(n, dtype=np.int64)
    x = i % N
    y = (i // N) % N
    z = i // (N * N)
    pts = [p for p in radius_points if value_fn(*p) != 0.0]
    cols = np.empty((n, len(pts)), dtype=np.int64)
    vals = np.empty((n, len(pts)), dtype=np.float64)
    for s, (dz, dy, dx) in enumerate(pts):
        ok = np.ones(n, dtype=bool)
        for d, c in ((dx, x), (dy, y), (dz, z)):
            if d < 0:
                ok &= c > 0
            elif d > 0:
                ok &= c < N - 1
        cols[:, s] = np.where(ok, i + dz * N * N + dy * N + dx, -1)
        vals[:, s] = value_fn(dz, dy, dx)
    return _assemble(n, cols, vals, name)


_CUBE = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
_CROSS = [p for p in _CUBE if sum(abs(t) for t in p) <= 1]


def poisson3d_7pt(N: int) -> CSR:
    """3D 7-point Laplacian on an N^3 interior grid: diagonal 6, neighbours -1."""
    return _box3d(N, _CROSS, lambda dz, dy, dx: 6.0 if (dz, dy, dx) == (0, 0, 0) else -1.0,
                  f"poisson3d_7pt_{N}")


def poisson3d_27pt(N: int) -> CSR:
    """3D 27-point operator: diagonal 26, all 26 neighbours -1."""
    return _box3d(N, _CUBE, lambda dz, dy, dx: 26.0 if (dz, dy, dx) == (0, 0, 0) else -1.0,
                  f"poisson3d_27pt_{N}")


def q1_laplace3d(N: int) -> CSR:
    """Trilinear (Q1) finite-element Laplacian on a uniform mesh (paper Section 5).

    Stencil (times h): centre 8/3, face neighbours 0 (not stored), edge
    neighbours -1/6, corner neighbours -1/12; interior rows sum to zero.
    """

    def v(dz, dy, dx):
        k = abs(dz) + abs(dy) + abs(dx)
        return {0: 8.0 / 3.0, 1: 0.0, 2: -1.0 / 6.0, 3: -1.0 / 12.0}[k]

    return _box3d(N, _CUBE, v, f"q1_laplace3d_{N}")


def lognormal_cells(N: int, seed: int, sigma: float = 2.0, mu: float = 0.0) -> np.ndarray:
    """Cell coefficients k = exp(mu + sigma z), z ~ N(0,1) by Box-Muller.

    z_c = sqrt(-2 ln(1 - u1)) cos(2 pi u2) with u1, u2 from streams 1 and 2.
    """
    n = N * N * N
    u1 = uniform01(seed, n, stream=1)
    u2 = uniform01(seed, n, stream=2)
    zz = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return np.exp(mu + sigma * zz)


def fv7_lognormal(N: int, seed: int = 3, sigma: float = 2.0) -> CSR:
    """3D cell-centred finite-volume diffusion, 7-point, lognormal coefficients.

    Interior face between cells c, d: transmissibility t = 2 k_c k_d / (k_c + k_d)
    (harmonic mean); a Dirichlet boundary face at half a cell: t = 2 k_c.
    Off-diagonal = -t, diagonal = sum of the six face transmissibilities.
    """
    n = N * N * N
    k = lognormal_cells(N, seed, sigma)
    i = np.arange(n, dtype=np.int64)
    x = i % N
    y = (i // N) % N
    z = i // (N * N)
    pts = _CROSS
    cols = np.empty((n, 7), dtype=np.int64)
    vals = np.empty((n, 7), dtype=np.float64)
    diag = np.zeros(n, dtype=np.float64)
    centre = None
    for s, (dz, dy, dx) in enumerate(pts):
        if (dz, dy, dx) == (0, 0, 0):
            centre = s
            continue
        ok = np.ones(n, dtype=bool)
        for d, c in ((dx, x), (dy, y), (dz, z)):
            if d < 0:
                ok &= c > 0
            elif d > 0:
                ok &= c < N - 1
        j = np.where(ok, i + dz * N * N + dy * N + dx, 0)
        kj = k[j]
        t = np.where(ok, 2.0 * k * kj / (k + kj), 2.0 * k)
        diag += t
        cols[:, s] = np.where(ok, j, -1)
        vals[:, s] = -t
    cols[:, centre] = i
    vals[:, centre] = diag
    return _assemble(n, cols, vals, f"fv7_lognormal_{N}_s{seed}")


def q1_element_stiffness(K: np.ndarray) -> np.ndarray:
    """4 x 4 bilinear (Q1) element matrix int grad(phi_a)^T K grad(phi_b) on
    a square element (independent of its size in 2D).  Local nodes
    0 (0,0), 1 (1,0), 2 (0,1), 3 (1,1); 2 x 2 Gauss quadrature, exact here
    (each integrand is at most quadratic in each coordinate)."""
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    Ke = np.zeros((4, 4))
    for x in g:
        for y in g:
            grads = np.array([[-(1 - y), -(1 - x)], [1 - y, -x], [-y, 1 - x], [y, x]])
            Ke += 0.25 * grads @ K @ grads.T
    return Ke


def rotated_aniso_q1(N: int, theta: float = np.pi / 8, eps: float = 1e-3) -> CSR:
    """2D rotated anisotropic diffusion -div(K grad u) = f, K = Q^T D Q with
    Q = [[cos t, sin t], [-sin t, cos t]], D = diag(1, eps) (paper Section 5),
    Q1 elements on a uniform square mesh of (N + 1)^2 elements, homogeneous
    Dirichlet boundary: the N x N interior nodes, a 9-point stencil (no h
    scaling: the 2D Q1 stiffness does not depend on h).  Off-diagonals of
    either sign: not an M-matrix."""
    c, s = np.cos(theta), np.sin(theta)
    Q = np.array([[c, s], [-s, c]])
    K = Q.T @ np.diag([1.0, eps]) @ Q
    Ke = q1_element_stiffness(K)
    local = {(0, 0): 0, (1, 0): 1, (0, 1): 2, (1, 1): 3}
    st = {}
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            v = 0.0
            for ey in (0, 1):          # the four elements around the node
                for ex in (0, 1):
                    cpos = (1 - ex, 1 - ey)
                    npos = (cpos[0] + dx, cpos[1] + dy)
                    if npos in local:
                        v += Ke[local[cpos], local[npos]]
            st[(dy, dx)] = v
    n = N * N
    i = np.arange(n, dtype=np.int64)
    x = i % N
    y = i // N
    pts = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if st[(dy, dx)] != 0.0]
    cols = np.empty((n, len(pts)), dtype=np.int64)
    vals = np.empty((n, len(pts)), dtype=np.float64)
    for k, (dy, dx) in enumerate(pts):
        ok = np.ones(n, dtype=bool)
        for d, cc in ((dx, x), (dy, y)):
            if d < 0:
                ok &= cc > 0
            elif d > 0:
                ok &= cc < N - 1
        cols[:, k] = np.where(ok, i + dy * N + dx, -1)
        vals[:, k] = st[(dy, dx)]
    return _assemble(n, cols, vals, f"rotated_aniso_q1_{N}")


def _laplacian_from_edges(n: int, ei: np.ndarray, ej: np.ndarray) -> CSR:
    """Graph Laplacian of an undirected edge list (unit weights, each edge
    once) shifted by 0.5 on the diagonal: off-diagonals -1, diagonal
    degree + 0.5 (a strictly diagonally dominant M-matrix)."""
    r = np.concatenate([ei, ej, np.arange(n)])
    c = np.concatenate([ej, ei, np.arange(n)])
    deg = np.bincount(np.concatenate([ei, ej]), minlength=n).astype(np.float64)
    v = np.concatenate([-np.ones(2 * len(ei)), deg + 0.5])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), c.astype(np.int32), v.astype(np.float64))


def hub_graphs() -> CSR:
    """Block-diagonal union of four shifted graph Laplacians with very long
    rows, for the product-heavy and column-heavy rows of the setup's sparse
    products (2598 unknowns): complete bipartite graphs K(50, 100) and
    K(130, 140), a 40 x 40 grid whose extra hub node links to every 5th grid
    node, and a 24 x 24 grid whose hub links to every 3rd node."""
    ei, ej, off = [], [], 0

    def add(a, b):
        ei.append(np.asarray(a, dtype=np.int64) + off)
        ej.append(np.asarray(b, dtype=np.int64) + off)

    for s, L in ((50, 100), (130, 140)):
        a, b = np.meshgrid(np.arange(s), s + np.arange(L), indexing="ij")
        add(a.ravel(), b.ravel())
        off += s + L
    for N, step in ((40, 5), (24, 3)):
        i = np.arange(N * N)
        x, y = i % N, i // N
        add(i[x < N - 1], i[x < N - 1] + 1)
        add(i[y < N - 1], i[y < N - 1] + N)
        links = np.arange(0, N * N, step)
        add(np.full(len(links), N * N), links)
        off += N * N + 1
    A = _laplacian_from_edges(off, np.concatenate(ei), np.concatenate(ej))
    A.name = "hub_graphs"
    return A


def generate(kind: str, N: int, seed: int = 3) -> CSR:
    """Dispatch by stencil name."""
    if kind == "2d5":
        return poisson2d_5pt(N)
    if kind == "3d7":
        return poisson3d_7pt(N)
    if kind == "3d27":
        return poisson3d_27pt(N)
    if kind == "q1":
        return q1_laplace3d(N)
    if kind == "fv7":
        return fv7_lognormal(N, seed)
    if kind == "aniso":
        return rotated_aniso_q1(N)
    if kind == "hubs":
        return hub_graphs()
    raise ValueError(f"unknown stencil {kind!r}")
