"""The pattern-quality check of Section 5.1 (Fig. 1): M's pattern against the
nnz(M) largest entries of A⁻¹, and the irregular-column count of the
truncated A⁻¹. Host analysis only; pinned by closed forms and brute force."""
import numpy as np
import pytest

from paper_1503_04500_gb300 import inputs
from paper_1503_04500_gb300 import pattern_quality as pq


def _csr_of_mask(P):
    n = P.shape[0]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(P.sum(axis=1))
    ci = np.concatenate([np.nonzero(P[i])[0] for i in range(n)]).astype(np.int32) if P.any() else np.zeros(0, np.int32)
    return rp, ci


def test_bidiagonal_inverse_ties_fill_column_zero_first():
    # A = I - S (S the down-shift) has A⁻¹ = I + S + S² + ... : the lower triangle,
    # all ones. With M = diag, k = n; every candidate has magnitude 1, so the tie
    # rule (column-major order) takes all of column 0.
    n = 20
    A = inputs.from_dense(np.eye(n) - np.eye(n, k=-1))
    rp, ci = _csr_of_mask(np.eye(n, dtype=bool))
    r = pq.compare(A, rp, ci)
    assert r["nnz_M"] == n
    assert r["matched"] == 1  # only (0, 0) lies on the diagonal
    assert r["captured_frac"] == pytest.approx(1.0)  # equal mass: every entry is 1
    assert r["irregular_threshold"] == 10.0
    assert r["irregular_cols_Ainv"] == 1 and r["max_col_nnz_Ainv"] == n
    assert r["irregular_rows_Ainv"] == 0 and r["max_row_nnz_Ainv"] == 1
    assert r["irregular_cols_M"] == 0 and r["kth_largest_abs_Ainv"] == 1.0


def test_diagonal_matrix():
    n = 15
    d = np.arange(1.0, n + 1)
    A = inputs.from_dense(np.diag(d))
    rp, ci = _csr_of_mask(np.eye(n, dtype=bool))
    r = pq.compare(A, rp, ci)
    assert r["matched"] == n and r["matched_frac"] == 1.0
    assert r["captured_frac"] == pytest.approx(1.0)
    assert r["kth_largest_abs_Ainv"] == pytest.approx(1.0 / n)
    assert r["irregular_cols_Ainv"] == 0 and r["irregular_rows_M"] == 0


def test_full_pattern_matches_everything():
    rng = np.random.default_rng(5)
    n = 9
    D = rng.standard_normal((n, n)) + n * np.eye(n)
    A = inputs.from_dense(D)
    rp, ci = _csr_of_mask(np.ones((n, n), dtype=bool))
    r = pq.compare(A, rp, ci)
    assert r["nnz_M"] == n * n and r["matched"] == n * n
    assert r["captured_frac"] == pytest.approx(1.0)
    assert r["irregular_cols_Ainv"] == 0  # threshold 10·n exceeds any column


def _brute(Ainv, PM, factor=10.0):
    n = Ainv.shape[0]
    k = int(PM.sum())
    cand = sorted(((-abs(Ainv[i, j]), j, i) for j in range(n) for i in range(n)))
    top = {(i, j) for _, j, i in cand[:k]}
    matched = sum(1 for i in range(n) for j in range(n) if PM[i, j] and (i, j) in top)
    thr = factor * k / n
    colA = [sum(1 for i in range(n) if (i, j) in top) for j in range(n)]
    rowA = [sum(1 for j in range(n) if (i, j) in top) for i in range(n)]
    mass_M = sum(Ainv[i, j] ** 2 for i in range(n) for j in range(n) if PM[i, j])
    mass_top = sum(Ainv[i, j] ** 2 for (i, j) in top)
    return {"matched": matched, "irregular_cols_Ainv": sum(c > thr for c in colA),
            "irregular_rows_Ainv": sum(c > thr for c in rowA), "max_col_nnz_Ainv": max(colA),
            "max_row_nnz_Ainv": max(rowA), "captured_frac": mass_M / mass_top if mass_top > 0 else 1.0}


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_small(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 9))
    D = np.where(rng.random((n, n)) < 0.4, rng.standard_normal((n, n)), 0.0) + 3 * np.eye(n)
    if seed % 2:  # integer entries make exact ties in A⁻¹ likely
        D = np.where(rng.random((n, n)) < 0.3, 1.0, 0.0) + np.eye(n)
        D = np.tril(D)
    A = inputs.from_dense(D)
    PM = rng.random((n, n)) < rng.uniform(0.1, 0.6)
    np.fill_diagonal(PM, True)
    rp, ci = _csr_of_mask(PM)
    r = pq.compare(A, rp, ci, factor=1.5)
    b = _brute(np.linalg.inv(D), PM, factor=1.5)
    for key, v in b.items():
        if key == "captured_frac":
            assert r[key] == pytest.approx(v, rel=1e-12)
        else:
            assert r[key] == v, key


def test_largest_entries_k_edges():
    X = np.array([[1.0, -3.0], [3.0, 0.0]])
    assert not pq.largest_entries(X, 0).any()
    assert pq.largest_entries(X, 4).all()
    # |3| twice: column 0 (row 1) before column 1 (row 0)
    assert pq.largest_entries(X, 1).tolist() == [[False, False], [True, False]]
    assert pq.largest_entries(X, 2).tolist() == [[False, True], [True, False]]


def test_oracle_pattern_on_the_2d_convection_diffusion_matrix():
    """The check on n = 400 with the Section 5.1 parameters (c = 3, ε = 0.2,
    l_max = 15), on the oracle's M (the FP64 GPU pattern equals it bit for bit)."""
    import oracle

    A = inputs.convdiff2d(20, (20.0, 20.0))
    M = oracle.build(A, c=3, l_max=15, eps=0.2, drop="adaptive", tol=1e-3)
    rp, ci, _ = M.csr()
    r = pq.compare(A, rp, ci)
    assert r["nnz_M"] == M.nnz and 0 < r["matched"] <= r["nnz_M"]
    assert 0.0 < r["captured_frac"] <= 1.0 + 1e-12
    assert r["irregular_threshold"] == pytest.approx(10 * M.nnz / A.n)
