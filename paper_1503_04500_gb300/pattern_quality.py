"""How well the pattern RSAI(tol) finds matches the large entries of A⁻¹: the
check of Section 5.1 (Fig. 1), on the synthetic matrices.

The paper forms A⁻¹ densely, keeps its nnz(M) entries of largest magnitude,
and compares that pattern with the pattern of M by eye. It also counts the
columns of the truncated A⁻¹ that are irregular, i.e. hold more than
10·nnz(M)/n entries, to show that a regular sparse A can have an irregular
sparse approximate inverse.

`compare` returns those counts as numbers. The dense inverse is the
comparison's reference quantity, not part of the method; it is formed once on
the host in FP64 (O(n³), so n up to a few thousand).

    python -m paper_1503_04500_gb300.pattern_quality --size 30 --eps 0.2 --c 3 --lmax 15

builds M on the GPU (FP64 unless `--precision` says otherwise) and prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs


def largest_entries(X: np.ndarray, k: int) -> np.ndarray:
    """Boolean mask of the k entries of X largest in magnitude. Entries of equal
    magnitude are taken in column-major order (lower column first, then lower
    row), so the mask is unique."""
    nr, nc = X.shape
    key = np.abs(X).T.ravel()  # position j*nr + i holds X[i, j]
    order = np.argsort(-key, kind="stable")
    flat = np.zeros(key.size, dtype=bool)
    flat[order[: max(int(k), 0)]] = True
    return flat.reshape(nc, nr).T


def pattern_mask(n: int, row_ptr, col_idx) -> np.ndarray:
    """Dense boolean pattern of an n×n CSR matrix."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)[: int(rp[-1])]
    P = np.zeros((n, n), dtype=bool)
    P[np.repeat(np.arange(n), np.diff(rp)), ci] = True
    return P


def compare(A: inputs.SparseMatrix, row_ptr, col_idx, factor: float = 10.0) -> dict:
    """Compare the pattern of M (CSR arrays on the host) with the nnz(M) largest
    entries of A⁻¹ (Section 5.1).

    - `matched`: entries of M's pattern that are among those nnz(M) entries;
      `matched_frac` = matched / nnz(M).
    - `captured_frac`: Σ a⁻¹_ij² over M's pattern ÷ the same sum over the
      nnz(M) largest entries, i.e. the share of the best possible pattern's
      Frobenius mass that M's pattern holds (1 when they are equally good, even
      if ties make them differ).
    - `irregular_cols_*`, `irregular_rows_*`: columns (rows) with more than
      factor·nnz(M)/n entries, in the truncated A⁻¹ and in M.
    """
    n = int(A.n)
    PM = pattern_mask(n, row_ptr, col_idx)
    k = int(PM.sum())
    Ainv = np.linalg.inv(A.to_dense())
    PA = largest_entries(Ainv, k)
    sq = Ainv * Ainv
    best = float(sq[PA].sum())
    thr = factor * k / n if n else 0.0
    colM, colA = PM.sum(axis=0), PA.sum(axis=0)
    rowM, rowA = PM.sum(axis=1), PA.sum(axis=1)
    matched = int(np.count_nonzero(PM & PA))
    kth = float(np.abs(Ainv)[PA].min()) if k else 0.0
    return {
        "n": n, "nnz_A": int(A.nnz), "nnz_M": k, "matched": matched, "matched_frac": matched / k if k else 1.0,
        "captured_frac": float(sq[PM].sum()) / best if best > 0 else 1.0,
        "kth_largest_abs_Ainv": kth, "irregular_threshold": thr,
        "irregular_cols_Ainv": int(np.count_nonzero(colA > thr)),
        "irregular_cols_M": int(np.count_nonzero(colM > thr)),
        "irregular_rows_Ainv": int(np.count_nonzero(rowA > thr)),
        "irregular_rows_M": int(np.count_nonzero(rowM > thr)),
        "max_col_nnz_Ainv": int(colA.max()) if n else 0, "max_col_nnz_M": int(colM.max()) if n else 0,
        "max_row_nnz_Ainv": int(rowA.max()) if n else 0, "max_row_nnz_M": int(rowM.max()) if n else 0,
    }


def _workload(name: str, size: int, seed: int) -> inputs.SparseMatrix:
    if name == "convdiff2d":
        return inputs.convdiff2d(size, (20.0, 20.0))
    if name == "convdiff3d":
        return inputs.convdiff3d(size)
    if name == "powerlaw":
        return inputs.powerlaw(size, seed=seed)
    raise ValueError(f"unknown workload {name}")


def main(argv=None):
    from . import rsai

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="convdiff2d", choices=["convdiff2d", "convdiff3d", "powerlaw"])
    ap.add_argument("--size", type=int, default=30, help="grid side N (stencils) or n (power law)")
    ap.add_argument("--seed", type=int, default=1503)
    ap.add_argument("--eps", type=float, default=0.2)
    ap.add_argument("--c", type=int, default=3)
    ap.add_argument("--lmax", type=int, default=15)
    ap.add_argument("--drop", default="adaptive", choices=["none", "adaptive", "fixed"])
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_refine"])
    a = ap.parse_args(argv)
    A = _workload(a.workload, a.size, a.seed)
    if A.n > 8000:
        raise SystemExit(f"n = {A.n}: the dense inverse of this check is meant for n up to a few thousand")
    h = rsai.build(rsai.DeviceMatrix.from_host(A), c=a.c, l_max=a.lmax, eps=a.eps, drop=a.drop, tol=a.tol,
                   precision=a.precision)
    try:
        rp, ci, _ = h.M()
        s = h.stats()
        out = {"workload": a.workload, "size": a.size, "eps": a.eps, "c": a.c, "l_max": a.lmax, "drop": a.drop,
               "precision": a.precision, "n_c": s["n_c"], "frob": s["frob"]}
        out.update(compare(A, rp.cpu().numpy(), ci.cpu().numpy()))
    finally:
        h.free()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
