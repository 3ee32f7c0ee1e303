"""Seeded synthetic matrices shaped like the paper's test problems.

This module builds inputs only; it holds none of the RSAI arithmetic, so both
the CPU oracle (under ``oracle/``) and the CUDA path can be fed from it.

The paper's own matrices (Table 1, Section 5: Matrix Market / SuiteSparse
oil-reservoir, CFD and circuit problems, n from 541 to 170998, 4-70 nonzeros per
column, a few very dense rows/columns) are not available, so these generators
stand in for them:

* ``convdiff2d`` / ``convdiff3d``: upwind finite-difference convection-diffusion
  (-Laplace(u) + beta . grad(u) on the unit square/cube, zero Dirichlet boundary
  eliminated, h = 1/(N+1), lexicographic order with x fastest, backward
  differences for beta_i > 0 and forward ones for beta_i < 0).  Regular rows and
  columns, like orsirr/sherman/saylr.
* ``parametric2d``: A(theta) = L/h^2 + theta1*Cx + theta2*Cy on one common
  5-point structure, returned as three value arrays so that dA/dtheta_i is the
  value array of C_i.
* ``powerlaw``: random nonsymmetric matrix with power-law row lengths (a few
  very dense rows, like scircuit/powersim), strictly row diagonally dominant.

Every matrix is returned as a :class:`SparseMatrix` holding CSR (row_ptr int64,
col_idx int32, val float64) and the matching CSC, both sorted within each
row/column, 0-based.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class SparseMatrix:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col_idx: np.ndarray  # int32[nnz], ascending within a row
    val: np.ndarray  # float64[nnz]
    col_ptr: np.ndarray  # int64[n+1]
    row_idx: np.ndarray  # int32[nnz], ascending within a column
    cval: np.ndarray  # float64[nnz]
    csc_to_csr: np.ndarray  # int64[nnz]: CSR position of each CSC entry
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def with_values(self, val: np.ndarray) -> "SparseMatrix":
        """Same structure, new CSR values (the CSC copy follows)."""
        val = np.ascontiguousarray(val, dtype=np.float64)
        return dataclasses.replace(self, val=val, cval=val[self.csc_to_csr].copy())

    def max_row_nnz(self) -> int:
        return int(np.diff(self.row_ptr).max()) if self.n else 0

    def max_col_nnz(self) -> int:
        return int(np.diff(self.col_ptr).max()) if self.n else 0

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col_idx] = self.val
        return d


def from_coo(n: int, rows, cols, vals, name: str = "") -> SparseMatrix:
    """Assemble a matrix from COO triplets (duplicates are summed)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    if rows.size:
        order = np.lexsort((cols, rows))
        rows, cols, vals = rows[order], cols[order], vals[order]
        key = rows * n + cols
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        seg = np.cumsum(first) - 1
        vals = np.bincount(seg, weights=vals, minlength=int(first.sum()))
        rows, cols = rows[first], cols[first]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    col_idx = cols.astype(np.int32)
    # CSC by a stable sort on the column index: rows stay ascending per column.
    csc_to_csr = np.argsort(cols, kind="stable").astype(np.int64)
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(col_ptr, cols + 1, 1)
    col_ptr = np.cumsum(col_ptr)
    return SparseMatrix(
        n=n,
        row_ptr=row_ptr,
        col_idx=col_idx,
        val=np.ascontiguousarray(vals),
        col_ptr=col_ptr,
        row_idx=rows[csc_to_csr].astype(np.int32),
        cval=np.ascontiguousarray(vals[csc_to_csr]),
        csc_to_csr=csc_to_csr,
        name=name,
    )


def from_dense(d: np.ndarray, name: str = "") -> SparseMatrix:
    """Structure = the nonzeros of a dense square array."""
    d = np.asarray(d, dtype=np.float64)
    r, c = np.nonzero(d)
    return from_coo(d.shape[0], r, c, d[r, c], name=name)


def _stencil(N: int, dim: int, diff: float, beta, h: float):
    """COO triplets of diff*(-Laplace) + beta.grad on an N^dim grid (upwind)."""
    n = N**dim
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // N**a) % N for a in range(dim)]
    rows = [idx]
    cols = [idx]
    diag = np.full(n, 2.0 * dim * diff / h**2 + sum(abs(b) for b in beta) / h)
    vals = [diag]
    for a in range(dim):
        b = float(beta[a])
        stride = N**a
        for step in (-1, +1):
            ok = coords[a] + step >= 0 if step < 0 else coords[a] + step < N
            coef = -diff / h**2
            if step < 0 and b > 0:
                coef -= b / h  # backward difference: u_P - u_W
            if step > 0 and b < 0:
                coef -= -b / h  # forward difference: u_E - u_P
            rows.append(idx[ok])
            cols.append(idx[ok] + step * stride)
            vals.append(np.full(int(ok.sum()), coef))
    return n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def convdiff2d(N: int = 20, beta=(20.0, 20.0)) -> SparseMatrix:
    """2-D 5-point upwind convection-diffusion, h = 1/(N+1)."""
    h = 1.0 / (N + 1)
    n, r, c, v = _stencil(N, 2, 1.0, beta, h)
    return from_coo(n, r, c, v, name=f"convdiff2d_N{N}")


def convdiff3d(N: int = 64, beta=None, peclet: float = 5.0, direction=(1.0, 0.5, 0.25)) -> SparseMatrix:
    """3-D 7-point upwind convection-diffusion, h = 1/(N+1).

    With ``beta`` None, beta = scale*direction with scale chosen so that the cell
    Peclet number max_i |beta_i| h / 2 equals ``peclet`` (N=64: beta=(650,325,162.5)).
    """
    h = 1.0 / (N + 1)
    if beta is None:
        scale = 2.0 * peclet / (h * max(abs(x) for x in direction))
        beta = tuple(scale * x for x in direction)
    n, r, c, v = _stencil(N, 3, 1.0, beta, h)
    return from_coo(n, r, c, v, name=f"convdiff3d_N{N}")


@dataclasses.dataclass
class ParametricMatrix:
    """A(theta) = L + theta[0]*C[0] + theta[1]*C[1] on one structure."""

    base: SparseMatrix  # structure, values of A(theta0)
    L: np.ndarray  # CSR-ordered values of L/h^2
    C: list  # CSR-ordered values of Cx, Cy
    theta: tuple

    def values(self, theta) -> np.ndarray:
        return self.L + theta[0] * self.C[0] + theta[1] * self.C[1]

    def at(self, theta) -> SparseMatrix:
        return self.base.with_values(self.values(theta))


def parametric2d(N: int = 256, theta=(30.0, 10.0)) -> ParametricMatrix:
    """2-D Laplacian plus upwind (backward) first differences in x and y."""
    h = 1.0 / (N + 1)
    n, r, c, lv = _stencil(N, 2, 1.0, (0.0, 0.0), h)
    struct = from_coo(n, r, c, np.ones_like(lv))
    # CSR position of every (row, col) of the common 5-point structure.
    csr_key = np.repeat(np.arange(n, dtype=np.int64), np.diff(struct.row_ptr)) * n + struct.col_idx
    order = np.argsort(csr_key)

    def place(rows, cols, vals):
        out = np.zeros(struct.nnz)
        k = np.asarray(rows, dtype=np.int64) * n + np.asarray(cols, dtype=np.int64)
        p = order[np.searchsorted(csr_key[order], k)]
        np.add.at(out, p, vals)
        return out

    L = place(r, c, lv)
    idx = np.arange(n, dtype=np.int64)
    C = []
    for a in range(2):
        coord = (idx // N**a) % N
        ok = coord > 0
        rows = np.concatenate([idx, idx[ok]])
        cols = np.concatenate([idx, idx[ok] - N**a])
        vals = np.concatenate([np.full(n, 1.0 / h), np.full(int(ok.sum()), -1.0 / h)])
        C.append(place(rows, cols, vals))
    base = struct.with_values(L + theta[0] * C[0] + theta[1] * C[1])
    base.name = f"parametric2d_N{N}"
    return ParametricMatrix(base=base, L=L, C=C, theta=tuple(theta))


def powerlaw_row_lengths(n: int, rng: np.random.Generator, exponent=2.5, dmin=3, dmax=200) -> np.ndarray:
    """Off-diagonal count per row from a truncated discrete power law."""
    d = np.arange(dmin, dmax + 1)
    p = d.astype(np.float64) ** (-exponent)
    cdf = np.cumsum(p / p.sum())
    cdf[-1] = 1.0
    return d[np.searchsorted(cdf, rng.random(n), side="right")].astype(np.int64)


def powerlaw(n: int = 1_000_000, seed: int = 1503, exponent=2.5, dmin=3, dmax=200,
             dominance: float = 1.1) -> SparseMatrix:
    """Random nonsymmetric matrix with power-law row lengths.

    Row i gets d_i off-diagonal entries in distinct uniformly drawn columns
    (never i), values N(0,1); the diagonal is +-dominance * (row abs-sum), sign
    +-1 with probability 1/2, so A is strictly row diagonally dominant.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dmax = min(dmax, n - 1)
    dmin = min(dmin, dmax)
    d = powerlaw_row_lengths(n, rng, exponent, dmin, dmax)
    rows = np.repeat(np.arange(n, dtype=np.int64), d)
    cols = rng.integers(0, n - 1, size=rows.size)
    cols += cols >= rows  # skip the diagonal
    while True:  # redraw duplicates inside a row until none is left
        order = np.lexsort((cols, rows))
        rows, cols = rows[order], cols[order]
        dup = np.zeros(rows.size, dtype=bool)
        dup[1:] = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if not dup.any():
            break
        new = rng.integers(0, n - 1, size=int(dup.sum()))
        new += new >= rows[dup]
        cols[dup] = new
    vals = rng.standard_normal(rows.size)
    absum = np.bincount(rows, weights=np.abs(vals), minlength=n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    diag = sign * dominance * absum
    diag[diag == 0.0] = 1.0
    idx = np.arange(n, dtype=np.int64)
    return from_coo(n, np.concatenate([rows, idx]), np.concatenate([cols, idx]),
                    np.concatenate([vals, diag]), name=f"powerlaw_n{n}_s{seed}")


def random_batch_member(i: int, seed0: int = 1503, nmin: int = 1000, nmax: int = 50000) -> SparseMatrix:
    """Member i of the 512-matrix batch: half convection-diffusion, half power-law."""
    rng = np.random.Generator(np.random.PCG64(seed0 + i))
    n = int(rng.integers(nmin, nmax + 1))
    if rng.random() < 0.5:
        dirv = rng.standard_normal(3)
        dirv /= np.linalg.norm(dirv)
        pe = float(rng.uniform(1.0, 20.0))
        if rng.random() < 0.5:
            N = max(2, int(round(math.sqrt(n))))
            h = 1.0 / (N + 1)
            beta = 2.0 * pe / h * dirv[:2] / np.abs(dirv[:2]).max()
            return convdiff2d(N, tuple(beta))
        N = max(2, int(round(n ** (1.0 / 3.0))))
        return convdiff3d(N, direction=tuple(dirv), peclet=pe)
    return powerlaw(n, seed=seed0 + i)


def matrix_stats(A: SparseMatrix) -> dict:
    """The statistics the paper's matrix table reports (Section 5): n, nnz,
    p = nnz/n (average nonzeros per column), s = the number of irregular
    columns (at least 10p nonzeros, the definition of Section 1), p_d = the
    nonzeros of the densest column; and the same two counts for rows, whose
    density is what makes RSAI's LS problems large (Section 4)."""
    n = int(A.n)
    nnz = int(A.nnz)
    p = nnz / n if n else 0.0
    col = np.diff(A.col_ptr)
    row = np.diff(A.row_ptr)
    return {"n": n, "nnz": nnz, "p": p, "s": int(np.sum(col >= 10 * p)), "p_d": int(col.max()) if n else 0,
            "s_rows": int(np.sum(row >= 10 * p)), "p_d_rows": int(row.max()) if n else 0}


def ones_rhs(A: SparseMatrix) -> np.ndarray:
    """b = A * (1,...,1)^T, the right-hand side of the paper's solver runs."""
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return np.bincount(rows, weights=A.val, minlength=A.n)
