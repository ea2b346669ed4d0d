"""Seeded synthetic inputs for recycling BiCG: model operators, drift sequences, right-hand sides.

This module defines *problems*, not the solver: it holds none of the method's arithmetic.
Both the CPU oracle and the CUDA path draw their inputs from here, so that each side sees
the same matrices and vectors.

Operators (paper Section 6.1 uses a 2-D convection-diffusion model; the coefficient there
is given only in a figure, so a constant-coefficient operator of the same structure and
sparsity stands in for it):

    -Laplace(u) + c . grad(u)   on the unit square / cube, homogeneous Dirichlet boundary,
    second-order central differences, N interior points per direction, h = 1/(N+1),
    lexicographic ordering with x fastest (idx = i + N*j [+ N*N*l]).

Row stencil: diagonal 2d/h^2; neighbour in direction e at -1: -1/h^2 - c_e/(2h); at +1:
-1/h^2 + c_e/(2h).  Matrices are returned as CSR with int32 indices, columns sorted in
each row.
"""
from __future__ import annotations

import numpy as np


class CSR:
    """A CSR matrix held as three numpy arrays (int32 row_ptr / col_idx, values)."""

    __slots__ = ("n", "row_ptr", "col_idx", "val")

    def __init__(self, n, row_ptr, col_idx, val):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.val = np.ascontiguousarray(val)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def with_values(self, val):
        return CSR(self.n, self.row_ptr, self.col_idx, val)


def convdiff(N, c, dim=None):
    """Central-difference matrix of -Laplace(u) + c.grad(u) on a d-dimensional grid.

    N: interior points per direction; c: sequence of d convection coefficients.
    Returns CSR (float64) with n = N**d rows, nnz = (2d+1) N^d - 2d N^(d-1).
    """
    c = [float(v) for v in np.atleast_1d(c)]
    d = len(c) if dim is None else int(dim)
    if len(c) != d:
        raise ValueError("need one convection coefficient per dimension")
    if N < 1:
        raise ValueError("N must be positive")
    h = 1.0 / (N + 1)
    n = N ** d
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for _ in range(d):
        coords.append(rem % N)
        rem //= N
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 2.0 * d / (h * h))]
    stride = 1
    for e in range(d):
        lo = -1.0 / (h * h) - c[e] / (2.0 * h)
        hi = -1.0 / (h * h) + c[e] / (2.0 * h)
        m = coords[e] > 0
        rows.append(idx[m]); cols.append(idx[m] - stride); vals.append(np.full(int(m.sum()), lo))
        m = coords[e] < N - 1
        rows.append(idx[m]); cols.append(idx[m] + stride); vals.append(np.full(int(m.sum()), hi))
        stride *= N
    r = np.concatenate(rows)
    cc = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((cc, r))
    r, cc, v = r[order], cc[order], v[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(n, row_ptr.astype(np.int32), cc.astype(np.int32), v.astype(np.float64))


def convdiff_nnz(N, d):
    """Closed-form nonzero count of `convdiff` on an N^d grid."""
    return (2 * d + 1) * N ** d - 2 * d * N ** (d - 1)


def drift_sequence(c0, count, rel, seed):
    """Convection coefficients of a slowly changing sequence of systems.

    System 0 uses c0; each later system multiplies every component of the previous one by
    (1 + rel*u) with u ~ U[-1, 1] drawn from numpy's default_rng(seed + j).
    """
    out = [np.array(c0, dtype=np.float64)]
    for j in range(1, count):
        u = np.random.default_rng(seed + j).uniform(-1.0, 1.0, size=len(c0))
        out.append(out[-1] * (1.0 + rel * u))
    return out


def normal_vector(n, seed, complex_=False):
    """Seeded N(0,1) vector (real, or complex with independent N(0,1) parts)."""
    rng = np.random.default_rng(seed)
    if complex_:
        return rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return rng.standard_normal(n)


def random_csr(n, nnz_per_row, seed, complex_=False, empty_rows=(), long_row=None,
               diag_shift=0.0):
    """Random sparse matrix with ragged rows, for kernel edge cases.

    Row i gets a random number of entries in [0, 2*nnz_per_row]; rows listed in
    `empty_rows` get none; `long_row` (if given) gets min(n, 64*nnz_per_row) entries.
    `diag_shift` adds a diagonal entry of that value to every non-empty row.
    """
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    empty = set(int(e) for e in empty_rows)
    for i in range(n):
        if i in empty:
            continue
        cnt = int(rng.integers(0, 2 * nnz_per_row + 1))
        if long_row is not None and i == long_row:
            cnt = min(n, 64 * nnz_per_row)
        cs = rng.choice(n, size=min(cnt, n), replace=False)
        if diag_shift != 0.0 and i not in cs:
            cs = np.append(cs, i)
        cs = np.sort(cs)
        rows.append(np.full(len(cs), i)); cols.append(cs)
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cc = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    v = rng.standard_normal(len(r))
    if complex_:
        v = v + 1j * rng.standard_normal(len(r))
    if diag_shift != 0.0:
        v = np.where(r == cc, v + diag_shift, v)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(n, row_ptr.astype(np.int32), cc.astype(np.int32), v)


# ----------------------------------------------------------------------------------------
# Workloads with the shapes of the paper's experiments (seeded stand-ins: the paper's own
# coefficient field and rail-model matrices are not available).
# ----------------------------------------------------------------------------------------

def convdiff_sequence(N, c0, count, rel, seed, bt_kind="normal", dim=2):
    """A sequence of slowly changing dual systems A_j x = b_j, A_j^H xt = bt_j.

    A_j = convdiff(N, c_j) with c_j from drift_sequence(c0, count, rel, seed);
    b_j ~ N(0,1) from seed + 100 + j; bt_j ~ N(0,1) (seed + 200 + j) or ones.
    Returns a list of dicts {A, b, bt, c}.
    """
    cs = drift_sequence(c0, count, rel, seed)
    out = []
    for j, c in enumerate(cs):
        A = convdiff(N, c, dim=dim)
        b = normal_vector(A.n, seed + 100 + j)
        if bt_kind == "ones":
            bt = np.ones(A.n)
        elif bt_kind == "zeros":
            bt = np.zeros(A.n)
        else:
            bt = normal_vector(A.n, seed + 200 + j)
        out.append({"A": A, "b": b, "bt": bt, "c": c})
    return out


def irka_shifts(count, seed):
    """Shifts in conjugate pairs: sigma = -10^{U[0,3]} +/- i U[0, 1e3] (count even)."""
    if count % 2:
        raise ValueError("shift count must be even (conjugate pairs)")
    rng = np.random.default_rng(seed)
    half = count // 2
    re = -(10.0 ** rng.uniform(0.0, 3.0, size=half))
    im = rng.uniform(0.0, 1e3, size=half)
    s = re + 1j * im
    return np.concatenate([s, np.conj(s)])


def move_shifts(shifts, rel, seed):
    """Move each shift of a conjugate-paired set by a real factor (1 + rel*u), u ~ U[-1,1];
    conjugate partners get the same factor so the set stays closed under conjugation."""
    half = len(shifts) // 2
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, size=half)
    f = np.concatenate([1.0 + rel * u, 1.0 + rel * u])
    return shifts * f
