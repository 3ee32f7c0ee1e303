"""Shared checks of the GPU's M against the FP64 oracle (test helpers).

FP32 + FP64-refinement builds may choose a different pattern from the oracle
for a few columns (a drop test or a dominant-row choice decided by values that
differ by rounding).  Every column is still checked: the GPU's ||r_k|| and
m_k against the oracle's least-squares solution on the GPU's own pattern
(Eq. 2.3 refit in FP64), and, where the patterns agree, against the oracle's
build as well.
"""
import numpy as np

import oracle


def csc_of_csr(rp, ci, va, n):
    """(colptr, rows, vals) of a CSR matrix, rows ascending within a column."""
    rp = np.asarray(rp, np.int64)
    ci = np.asarray(ci)
    rows = np.repeat(np.arange(n), np.diff(rp))
    order = np.lexsort((rows, ci))
    cp = np.zeros(n + 1, np.int64)
    np.add.at(cp, ci.astype(np.int64) + 1, 1)
    return np.cumsum(cp), rows[order].astype(np.int32), np.asarray(va)[order]


def same_columns(cp, rows, ocp, orows):
    """Boolean per column: the two CSC patterns hold the same rows."""
    n = len(cp) - 1
    lg, lo = np.diff(cp), np.diff(ocp)
    same = lg == lo
    col = np.repeat(np.arange(n), lg)
    off = np.arange(len(rows)) - cp[col]
    ok = same[col]
    idx = ocp[col[ok]] + off[ok]
    bad = np.zeros(n, bool)
    bad[col[ok][rows[ok] != orows[idx]]] = True
    return same & ~bad


def check_fp32_every_column(A, res, rho, ref, rtol_rho=1e-5, rtol_val=1e-6, max_mismatch=0.01, atol_rho=1e-12):
    """FP32+refine M (CSR triple `res`, per-column `rho`) against the oracle
    build `ref` on every column; returns the mask of columns whose pattern
    equals the oracle's.

    ||r_k|| is measured against ||e_k|| = 1.  A column whose pattern holds an
    exact inverse column has rho ~ 0, where a relative bar means nothing: an
    FP32 factorization corrected once in FP64 leaves a residual of about
    (kappa(B) u_32)^2, so rho is held to an absolute floor of 1e-12 besides
    the relative 1e-5."""
    cp, rows, vals = csc_of_csr(*res, A.n)
    same = same_columns(cp, rows, ref.colptr, ref.rows)
    assert same.mean() >= 1.0 - max_mismatch, f"{(~same).sum()} of {A.n} patterns differ"
    # every column: the LS solution on the GPU's own pattern
    ov, orho2 = oracle.refit(A, cp, rows)
    np.testing.assert_allclose(rho, np.sqrt(orho2), rtol=rtol_rho, atol=atol_rho)
    np.testing.assert_allclose(vals, ov, rtol=rtol_val, atol=rtol_val * np.abs(ov).max())
    # columns with the oracle's pattern: the oracle's own ||r_k||
    np.testing.assert_allclose(rho[same], ref.rho[same], rtol=rtol_rho, atol=atol_rho)
    return same
