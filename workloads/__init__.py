"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module defines the *problems* (sparse operators, lattice coordinates,
right-hand sides, random streams) and nothing of the solver's arithmetic: no
ordering, no factorization, no compression.  Both the CPU oracle and the GPU
path receive their inputs from here; neither imports the other.

Operators (stand-ins for the paper's workloads, Sec. 6):
  * helmholtz7   -- 7-point finite differences of -Lap u - k^2 (1 + 0.01 i) u on
                    an n^3 interior grid, Dirichlet boundary.  The damping term
                    replaces the PML of the visco-acoustic runs (Sec. 6.1).
  * yee_maxwell  -- curl-curl E - k^2 (1 + 0.01 i) E on a Yee edge lattice with
                    PEC walls; stands in for the Nedelec/MFEM system (Sec. 6.3).
  * green_planes -- point sets for blocks of exp(ik|x-y|)/(4 pi |x-y|), the
                    free-space Helmholtz Green's function named in Sec. 3.1.

Lattice coordinates are integers.  For the node lattice an unknown at grid
index (i, j, k) has coordinates (i, j, k); for the Yee lattice coordinates are
doubled, an x-edge (i + 1/2, j, k) sits at (2i + 1, 2j, 2k).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LATTICE_NODE = 0
LATTICE_EDGE = 1


@dataclass
class SparseProblem:
    """A complex CSR matrix with integer lattice coordinates per unknown."""
    name: str
    n: int                      # number of unknowns N
    rowptr: np.ndarray          # int64 [N+1]
    colind: np.ndarray          # int32 [nnz], sorted within each row
    vals: np.ndarray            # complex128 [nnz]
    coords: np.ndarray          # int32 [N, 3]
    lattice: int                # LATTICE_NODE or LATTICE_EDGE
    params: dict = field(default_factory=dict)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colind, self.rowptr), shape=(self.n, self.n))


def _csr_from_coo(n, rows, cols, vals):
    import scipy.sparse as sp
    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.sort_indices()
    return m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.complex128)


def helmholtz7(n: int, ppw: float, damping: float = 0.01, k: float | None = None) -> SparseProblem:
    """-Lap u - k^2 (1 + i*damping) u on the n^3 interior grid of the unit cube.

    h = 1/(n+1), k = 2 pi / (ppw h) unless given (k = 0 gives Poisson).
    Unknown p = i + n j + n^2 k (x fastest).  A_pp = 6/h^2 - kappa^2,
    A_pq = -1/h^2 for each face neighbour inside the grid.
    """
    h = 1.0 / (n + 1)
    if k is None:
        k = 2.0 * math.pi / (ppw * h)
    kappa2 = (k * k) * (1.0 + 1j * damping)
    N = n ** 3
    idx = np.arange(N, dtype=np.int64)
    i = idx % n
    j = (idx // n) % n
    kk = idx // (n * n)
    rows = [idx]
    cols = [idx]
    vals = [np.full(N, 6.0 / h ** 2 - kappa2, dtype=np.complex128)]
    for axis, stride in ((i, 1), (j, n), (kk, n * n)):
        for d in (-1, 1):
            ok = (axis + d >= 0) & (axis + d < n)
            rows.append(idx[ok])
            cols.append(idx[ok] + d * stride)
            vals.append(np.full(int(ok.sum()), -1.0 / h ** 2, dtype=np.complex128))
    rp, ci, va = _csr_from_coo(N, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    coords = np.stack([i, j, kk], axis=1).astype(np.int32)
    return SparseProblem(f"helmholtz7_{n}", N, rp, ci, va, coords, LATTICE_NODE,
                         dict(n=n, h=h, k=k, ppw=ppw, damping=damping))


def yee_maxwell(nc: int, ppw: float, damping: float = 0.01) -> SparseProblem:
    """(1/h^2) C^T C - k^2 (1 + i*damping) I on the Yee edge lattice of nc^3 cells.

    Edges lying in a boundary face are removed (PEC), leaving 3 nc (nc-1)^2
    unknowns.  C is the +-1 face/edge circulation incidence, so C^T C is the
    discrete curl-curl.  k = 2 pi / (ppw h), h = 1/nc.
    """
    h = 1.0 / nc
    k = 2.0 * math.pi / (ppw * h)
    kappa2 = (k * k) * (1.0 + 1j * damping)
    # enumerate interior edges, doubled coordinates
    ed = {}
    coords = []
    def add(X, Y, Z):
        ed[(X, Y, Z)] = len(coords)
        coords.append((X, Y, Z))
    r = range(1, nc)        # interior node-plane indices
    # x-edges: i in [0,nc), j,k interior ; y-edges ; z-edges -- x fastest ordering
    for kz in r:
        for jy in r:
            for ix in range(nc):
                add(2 * ix + 1, 2 * jy, 2 * kz)
    for kz in r:
        for jy in range(nc):
            for ix in r:
                add(2 * ix, 2 * jy + 1, 2 * kz)
    for kz in range(nc):
        for jy in r:
            for ix in r:
                add(2 * ix, 2 * jy, 2 * kz + 1)
    N = len(coords)
    # faces: each face is a unit square with 4 edges and orientation signs
    rows, cols, vals = [], [], []
    def face(edges):
        live = [(ed[e], s) for e, s in edges if e in ed]
        for a, sa in live:
            for b, sb in live:
                rows.append(a); cols.append(b); vals.append(sa * sb / h ** 2)
    for a in range(nc):
        for b in range(nc):
            for c in range(nc + 1):
                X, Y, Z = 2 * a, 2 * b, 2 * c
                # z-normal face at (a+1/2, b+1/2, c): +x(b) +y(a+1) -x(b+1) -y(a)
                face([((X + 1, Y, Z), 1), ((X + 2, Y + 1, Z), 1), ((X + 1, Y + 2, Z), -1), ((X, Y + 1, Z), -1)])
                # x-normal face at (c, a+1/2, b+1/2): y then z
                face([((Z, X + 1, Y), 1), ((Z, X + 2, Y + 1), 1), ((Z, X + 1, Y + 2), -1), ((Z, X, Y + 1), -1)])
                # y-normal face at (b+1/2, c, a+1/2): z then x
                face([((Y, Z, X + 1), 1), ((Y + 1, Z, X + 2), 1), ((Y + 2, Z, X + 1), -1), ((Y + 1, Z, X), -1)])
    rows = np.array(rows, dtype=np.int64); cols = np.array(cols, dtype=np.int64)
    vals = np.array(vals, dtype=np.complex128)
    diag = np.arange(N, dtype=np.int64)
    rows = np.concatenate([rows, diag]); cols = np.concatenate([cols, diag])
    vals = np.concatenate([vals, np.full(N, -kappa2, dtype=np.complex128)])
    rp, ci, va = _csr_from_coo(N, rows, cols, vals)
    # drop exact structural zeros produced by cancellation
    return SparseProblem(f"yee_maxwell_{nc}", N, rp, ci, va, np.array(coords, dtype=np.int32),
                         LATTICE_EDGE, dict(nc=nc, h=h, k=k, ppw=ppw, damping=damping))


def complex_gaussian(rng: np.random.Generator, n: int, ncols: int) -> np.ndarray:
    """Columns drawn in order; each column draws its real part, then its imaginary part."""
    out = np.empty((n, ncols), dtype=np.complex128)
    for c in range(ncols):
        re = rng.standard_normal(n)
        im = rng.standard_normal(n)
        out[:, c] = (re + 1j * im) / math.sqrt(2.0)
    return out


def rhs_point_plus_gaussian(prob: SparseProblem, seed: int = 42) -> np.ndarray:
    """Unit point source at grid node (n//2, n//2, n//2) plus a seeded complex Gaussian."""
    n = prob.params["n"]
    c = (n // 2) + n * (n // 2) + n * n * (n // 2)
    b = complex_gaussian(np.random.default_rng(seed), prob.n, 1)
    b[c, 0] += 1.0
    return b


def rhs_gaussian(prob: SparseProblem, ncols: int, seed: int) -> np.ndarray:
    return complex_gaussian(np.random.default_rng(seed), prob.n, ncols)


def rhs_dipoles(prob: SparseProblem, ncols: int, seed: int = 11) -> np.ndarray:
    """One unit edge source per column at edges drawn without replacement."""
    rng = np.random.default_rng(seed)
    where = rng.choice(prob.n, ncols, replace=False)
    b = np.zeros((prob.n, ncols), dtype=np.complex128)
    b[where, np.arange(ncols)] = 1.0
    return b


# ----------------------------------------------------------------------------
# Counter-based normal generator (splitmix64 + Box-Muller), used for the
# random sketching vectors so that two independent implementations can draw
# the same numbers.  splitmix64 is Steele, Lea and Flood (2014); Box-Muller is
# the classical polar-free transform z = sqrt(-2 ln u1) * (cos, sin)(2 pi u2).
# ----------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(_M64)
    z = x
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(_M64)
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(_M64)
    return z ^ (z >> np.uint64(31))


def counter_normal_complex(key: int, rows: np.ndarray, col: int) -> np.ndarray:
    """Complex normal (unit variance) for entries (row, col) of the stream `key`.

    counter c = key*2^40 ^ (col << 24) ^ row  is hashed twice (2c, 2c+1) to two
    53-bit uniforms in (0, 1); Box-Muller gives re, im; both are scaled by 1/sqrt(2).
    """
    with np.errstate(over="ignore"):
        c = (np.uint64(key & 0xFFFFFF) << np.uint64(40)) ^ (np.uint64(col & 0xFFFF) << np.uint64(24)) \
            ^ rows.astype(np.uint64)
        h1 = splitmix64(c * np.uint64(2))
        h2 = splitmix64(c * np.uint64(2) + np.uint64(1))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    u2 = ((h2 >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * math.pi * u2
    return (rad * np.cos(ang) + 1j * rad * np.sin(ang)) / math.sqrt(2.0)


# ----------------------------------------------------------------------------
# Green's-function blocks between two parallel planar point grids
# ----------------------------------------------------------------------------
def green_planes(m: int, spacing: float = 1.0, k: float = math.pi / 4):
    """Two m x m grids (spacing h = 1) at z = 0 and z = h; returns (X, Y, k)."""
    g = np.arange(m, dtype=np.float64) * spacing
    xx, yy = np.meshgrid(g, g, indexing="xy")
    P = np.stack([xx.ravel(), yy.ravel(), np.zeros(m * m)], axis=1)
    Q = P.copy(); Q[:, 2] = spacing
    return P, Q, k


def green_entries(P: np.ndarray, Q: np.ndarray, k: float, rows, cols) -> np.ndarray:
    d = P[np.asarray(rows)][:, None, :] - Q[np.asarray(cols)][None, :, :]
    r = np.sqrt((d * d).sum(-1))
    return np.exp(1j * k * r) / (4.0 * math.pi * r)


def butterfly_bench_sizes(nblocks: int = 200, seed: int = 3):
    """Block plane sizes m = rint(16 * 8^u), u ~ U(0,1) (log-uniform on [16, 128])."""
    u = np.random.default_rng(seed).random(nblocks)
    return np.rint(16.0 * 8.0 ** u).astype(np.int64)
