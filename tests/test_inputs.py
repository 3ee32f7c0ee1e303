"""The synthetic generators produce the stated shapes and structure."""
import numpy as np
import pytest

from paper_1503_04500_gb300 import inputs as gen


def _check_formats(A):
    n = A.n
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.nnz == A.col_ptr[-1]
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    for r in range(min(n, 200)):
        seg = A.col_idx[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
    cols = np.repeat(np.arange(n), np.diff(A.col_ptr))
    assert np.all(A.col_idx[A.csc_to_csr] == cols)
    assert np.all(rows[A.csc_to_csr] == A.row_idx)
    assert np.array_equal(A.val[A.csc_to_csr], A.cval)


def test_convdiff2d_c1():
    A = gen.convdiff2d(20, (20.0, 20.0))
    assert (A.n, A.nnz) == (400, 1920)
    _check_formats(A)
    D = A.to_dense()
    h = 1 / 21
    assert D[0, 0] == pytest.approx(4 / h**2 + 40 / h)
    # upwind: the west neighbour carries the convection term for beta_x > 0
    assert D[1, 0] == pytest.approx(-1 / h**2 - 20 / h)
    assert D[0, 1] == pytest.approx(-1 / h**2)
    assert np.abs(D).sum(axis=0).max() == pytest.approx(5208.0)


def test_convdiff3d_c2_shape():
    A = gen.convdiff3d(64)
    assert (A.n, A.nnz) == (262144, 1810432)
    assert A.max_row_nnz() == 7
    h = 1 / 65
    D0 = A.val[A.row_ptr[0]]
    assert D0 == pytest.approx(6 / h**2 + (650 + 325 + 162.5) / h)


def test_parametric2d_linear_in_theta():
    P = gen.parametric2d(16, (30.0, 10.0))
    assert P.base.nnz == 5 * 256 - 4 * 16
    v1 = P.values((1.0, 2.0))
    v2 = P.values((3.0, -1.0))
    v3 = P.values((2.0, 0.5))
    np.testing.assert_allclose(0.5 * (v1 + v2), v3)
    _check_formats(P.at((1.0, 2.0)))


def test_powerlaw_structure():
    A = gen.powerlaw(20000, seed=1503)
    _check_formats(A)
    d = np.diff(A.row_ptr) - 1
    assert d.min() >= 3 and d.max() <= 200
    assert 7.0 < np.diff(A.row_ptr).mean() < 8.6
    D = A.val
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    diag = A.col_idx == rows
    assert diag.sum() == A.n
    off = np.bincount(rows[~diag], weights=np.abs(D[~diag]), minlength=A.n)
    np.testing.assert_allclose(np.abs(D[diag]), 1.1 * off)
    B = gen.powerlaw(20000, seed=1503)
    assert np.array_equal(A.col_idx, B.col_idx) and np.array_equal(A.val, B.val)


def test_batch_member_deterministic():
    a = gen.random_batch_member(3)
    b = gen.random_batch_member(3)
    assert a.n == b.n and np.array_equal(a.val, b.val)
    assert 500 <= a.n <= 60000


def test_transpose_swaps_formats_without_arithmetic():
    from paper_1503_04500_gb300 import rsai

    A = gen.powerlaw(500, seed=3, dmax=30)
    T = rsai.transpose(A)
    np.testing.assert_array_equal(T.to_dense(), A.to_dense().T)
    np.testing.assert_array_equal(T.cval, T.val[T.csc_to_csr])  # the map still pairs the two copies
    TT = rsai.transpose(T)
    for f in ("row_ptr", "col_idx", "val", "col_ptr", "row_idx", "cval", "csc_to_csr"):
        np.testing.assert_array_equal(getattr(TT, f), getattr(A, f))


def test_matrix_stats_counts_irregular_columns_and_rows():
    # 40 x 40: identity plus one dense column (all 40 rows) and one dense row (all 40 columns)
    n = 40
    rows = list(range(n)) + list(range(n)) + [7] * n
    cols = list(range(n)) + [3] * n + list(range(n))
    A = gen.from_coo(n, np.array(rows), np.array(cols), np.ones(len(rows)))
    st = gen.matrix_stats(A)
    nnz = n + (n - 1) + (n - 2)  # duplicates at (3,3), (7,7) and (7,3) are summed
    assert st["nnz"] == nnz and st["p"] == pytest.approx(nnz / n)
    assert st["s"] == 1 and st["p_d"] == n  # column 3 holds every row; 10p = 29.25 <= 40
    assert st["s_rows"] == 1 and st["p_d_rows"] == n
    assert gen.matrix_stats(gen.convdiff2d(8, (1.0, 1.0)))["s"] == 0  # a stencil is regular
