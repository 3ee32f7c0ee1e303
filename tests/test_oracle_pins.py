"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test would fail on a plausible mistake in the oracle: a dropped term, a
wrong sign or index, a transposed operand, a wrong tie or drop rule.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.exact_rsai import exact_rsai
from paper_1503_04500_gb300 import inputs as gen


def _residuals(A, M):
    """r_k = A m_k - e_k for every built column (dense, plain NumPy)."""
    D = A.to_dense()
    out = []
    for t, k in enumerate(M.cols):
        J, v = M.column(t)
        r = D[:, J] @ v
        r[k] -= 1.0
        out.append((J, r))
    return out


@pytest.fixture(scope="module")
def c1():
    return gen.convdiff2d(20, (20.0, 20.0))


def test_p1_closed_form_loop0(c1):
    """J = {k}: m_kk = a_kk/||a_k||^2, rho^2 = 1 - a_kk^2/||a_k||^2 (Eq. 2.3, p = 1)."""
    M = oracle.build(c1, l_max=0, drop="none")
    D = c1.to_dense()
    colnorm2 = (D**2).sum(axis=0)
    diag = np.diag(D)
    assert np.all(np.diff(M.colptr) == 1)
    assert np.all(M.rows == np.arange(c1.n))
    np.testing.assert_allclose(M.vals, diag / colnorm2, rtol=1e-14)
    np.testing.assert_allclose(M.rho**2, 1.0 - diag**2 / colnorm2, rtol=1e-12)
    assert np.all(M.loops == 0)
    # with loops allowed, columns already below eps stop at loop 0 with the same values
    M10 = oracle.build(c1, l_max=10, eps=0.3)
    stop0 = M.rho <= 0.3
    assert stop0.any()
    assert np.all(M10.loops[stop0] == 0)
    np.testing.assert_array_equal(M10.rho[stop0], M.rho[stop0])


def test_p2_full_pattern_gives_inverse():
    """A dense A: after one loop J is everything and M = A^{-1} (Eq. 2.1 minimum 0)."""
    rng = np.random.default_rng(7)
    n = 9
    D = rng.standard_normal((n, n)) + 4.0 * np.eye(n)
    A = gen.from_dense(D)
    M = oracle.build(A, c=n, l_max=n, eps=1e-10, drop="none")
    np.testing.assert_allclose(M.to_dense(), np.linalg.inv(D), rtol=0, atol=1e-12 * np.abs(np.linalg.inv(D)).max())
    assert np.all(M.rho < 1e-12)
    # frozen full pattern through refit
    colptr = np.arange(0, n * n + 1, n, dtype=np.int64)
    rows = np.tile(np.arange(n, dtype=np.int32), n)
    vals, rho2 = oracle.refit(A, colptr, rows)
    np.testing.assert_allclose(vals.reshape(n, n).T, np.linalg.inv(D), atol=1e-12)
    assert np.all(rho2 < 1e-24)


def test_p3_diagonal_exact():
    d = np.array([2.0, -3.0, 0.5, 7.0, -0.25])
    A = gen.from_dense(np.diag(d))
    for drop in ("none", "adaptive", "fixed"):
        M = oracle.build(A, drop=drop)
        np.testing.assert_array_equal(M.vals, 1.0 / d)
        assert np.all(M.rho == 0.0) and np.all(M.loops == 0)


@pytest.mark.parametrize("drop", ["none", "adaptive", "fixed"])
def test_p4_normal_equations(c1, drop):
    """Each emitted m_k minimises ||A(:,J) x - e_k||: A(:,J)^T r = 0 (Eq. 2.3)."""
    P = gen.powerlaw(600, seed=11, dmax=15)
    for A, kw in ((c1, {}), (P, dict(c=5, l_max=8, eps=0.4))):
        M = oracle.build(A, drop=drop, **kw, cols=np.arange(0, A.n, max(1, A.n // 300)))
        D = A.to_dense()
        for (J, r), rho in zip(_residuals(A, M), M.rho):
            AJ = D[:, J]
            np.testing.assert_allclose(np.linalg.norm(r), rho, rtol=1e-12)
            g = AJ.T @ r
            assert np.abs(g).max() <= 1e-12 * np.linalg.norm(AJ) * max(np.linalg.norm(r), 1e-300) + 1e-300


def test_p5_residual_nonincreasing_without_dropping(c1):
    """NONE mode: J^(l) is nested, so ||r_k|| cannot grow from loop to loop."""
    P = gen.powerlaw(300, seed=5, dmax=10)
    for A, c in ((c1, 3), (P, 4)):
        prev = None
        for lm in range(0, 6):
            M = oracle.build(A, c=c, l_max=lm, eps=1e-3, drop="none")
            if prev is not None:
                assert np.all(M.rho <= prev * (1 + 1e-12) + 1e-15)
            prev = M.rho


@pytest.mark.parametrize("drop", ["none", "adaptive", "fixed"])
def test_p6_theorem1_bound(drop):
    """nnz(m_k) <= min(g c l_max + 1, n) (Theorem 1)."""
    P = gen.powerlaw(400, seed=3, dmax=20)
    g = P.max_row_nnz()
    for c, lm in ((1, 3), (3, 4), (5, 2)):
        M = oracle.build(P, c=c, l_max=lm, eps=1e-4, drop=drop)
        assert np.diff(M.colptr).max() <= min(g * c * lm + 1, P.n)


def test_p7_pattern_envelope():
    """With a nonzero diagonal, J_k^(l) lies in the structure of (A^T A)^l e_k."""
    P = gen.powerlaw(400, seed=9, dmax=12)
    S = (P.to_dense() != 0).astype(np.int64)
    AtA = ((S.T @ S) > 0).astype(np.int64)
    for lm in (1, 2, 3):
        env = np.eye(P.n, dtype=np.int64)
        for _ in range(lm):
            env = ((AtA @ env) > 0).astype(np.int64)
        M = oracle.build(P, c=3, l_max=lm, eps=1e-6, drop="none")
        for t in range(P.n):
            J, _ = M.column(t)
            assert env[J, t].all()


@pytest.mark.parametrize("drop", ["none", "adaptive", "fixed"])
def test_p8_power_of_two_scaling(c1, drop):
    """M(2^s A) = 2^-s M(A) bit for bit, same patterns (every rule is scale-free)."""
    P = gen.powerlaw(800, seed=21, dmax=20)
    for A, kw in ((c1, {}), (P, dict(c=5, l_max=8, eps=0.4))):
        M = oracle.build(A, drop=drop, **kw)
        for s in (3, -5):
            As = A.with_values(A.val * 2.0**s)
            Ms = oracle.build(As, drop=drop, **kw)
            np.testing.assert_array_equal(Ms.colptr, M.colptr)
            np.testing.assert_array_equal(Ms.rows, M.rows)
            np.testing.assert_array_equal(Ms.vals, M.vals * 2.0**-s)
            np.testing.assert_array_equal(Ms.rho, M.rho)
            np.testing.assert_array_equal(Ms.loops, M.loops)


def _small_int_matrix(rng, n, density=0.35):
    D = rng.integers(-3, 4, size=(n, n)) * (rng.random((n, n)) < density)
    np.fill_diagonal(D, 0)
    d = np.abs(D).sum(axis=1) + rng.integers(1, 3, size=n)
    D += np.diag(np.where(rng.random(n) < 0.5, -d, d))
    return D


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("drop", ["none", "adaptive", "fixed"])
def test_p9_exact_brute_force(seed, drop):
    """Patterns equal and values within 1e-12 of exact rational RSAI."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 10))
    D = _small_int_matrix(rng, n)
    c = int(rng.integers(1, 4))
    lm = int(rng.integers(1, 5))
    eps, tol = Fraction(1, 20), Fraction(3, 100)
    ex = exact_rsai(D.tolist(), c=c, l_max=lm, eps=eps, drop=drop, tol=tol)
    M = oracle.build(gen.from_dense(D), c=c, l_max=lm, eps=float(eps), drop=drop, tol=float(tol))
    for t, (J, m, rho2, loops) in enumerate(ex):
        Jo, vo = M.column(t)
        assert list(Jo) == J, (t, Jo, J)
        np.testing.assert_allclose(vo, [float(v) for v in m], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(M.rho[t] ** 2, float(rho2), rtol=1e-10, atol=1e-15)
        assert M.loops[t] == loops


def test_p9_exact_ties():
    """A matrix with exactly tied residual entries: lowest index wins (exact and FP64)."""
    D = np.array([[4, 1, 1, 0, 0],
                  [1, 4, 0, 1, 0],
                  [1, 0, 4, 0, 1],
                  [0, 1, 0, 4, 1],
                  [0, 0, 1, 1, 4]])
    ex = exact_rsai(D.tolist(), c=1, l_max=3, eps=Fraction(1, 1000), drop="none")
    M = oracle.build(gen.from_dense(D), c=1, l_max=3, eps=1e-3, drop="none")
    # column 0 has r(1) = r(2) exactly at loop 0: row 1 must be taken first
    for t, (J, m, rho2, loops) in enumerate(ex):
        assert list(M.column(t)[0]) == J
    assert 1 in ex[0][0]


def test_drop_rules_thresholds():
    """FIXED drops |m_j| <= tol/||A||_1; ADAPTIVE uses eps/(p ||A||_1) (Eq. 4.3)."""
    P = gen.powerlaw(800, seed=4, dmax=20)
    nrm = oracle.norm1(P)
    D = P.to_dense()
    assert nrm == pytest.approx(np.abs(D).sum(axis=0).max(), rel=1e-15)
    Mf = oracle.build(P, c=5, l_max=8, eps=0.4, drop="fixed", tol=1e-3)
    assert Mf.counters[:, 4].sum() > 0  # some solves dropped entries
    Mn = oracle.build(P, c=5, l_max=8, eps=0.4, drop="none")
    assert Mf.nnz < Mn.nnz


def test_counters_closed_form(c1):
    """Work counters at loop 0: one solve on (q,p) = (nnz(a_k), 1)."""
    M = oracle.build(c1, l_max=0, drop="none")
    q = np.diff(c1.col_ptr)
    # solve: (q)(2 + 4) + 1; residual: 2 q + 2 q
    np.testing.assert_array_equal(M.counters[:, 0], q * 6.0 + 1.0)
    np.testing.assert_array_equal(M.counters[:, 1], 4.0 * q)


def test_refit_matches_build(c1):
    """Refit on the emitted pattern reproduces the emitted values (both exact LS minimisers)."""
    M = oracle.build(c1)
    vals, rho2 = oracle.refit(c1, M.colptr, M.rows)
    np.testing.assert_allclose(vals, M.vals, rtol=1e-12)
    np.testing.assert_allclose(np.sqrt(rho2), M.rho, rtol=1e-12)


def test_threads_do_not_change_results():
    P = gen.powerlaw(1000, seed=8, dmax=20)
    a = oracle.build(P, c=5, l_max=8, eps=0.4, threads=1)
    b = oracle.build(P, c=5, l_max=8, eps=0.4, threads=4)
    np.testing.assert_array_equal(a.rows, b.rows)
    np.testing.assert_array_equal(a.vals, b.vals)


def test_golden_exact_small():
    """Stored exact rational results (tests/golden/exact_small.json) vs the FP64 oracle."""
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "exact_small.json")
    with open(path) as f:
        data = json.load(f)
    assert len(data["cases"]) >= 18
    for case in data["cases"]:
        D = np.array(case["matrix"], dtype=np.float64)
        pr = case["params"]
        M = oracle.build(gen.from_dense(D), c=pr["c"], l_max=pr["l_max"], eps=float(Fraction(pr["eps"])),
                         drop=pr["drop"], tol=float(Fraction(pr["tol"])))
        for t, col in enumerate(case["columns"]):
            J, v = M.column(t)
            assert list(J) == col["J"]
            np.testing.assert_allclose(v, [float(Fraction(x)) for x in col["m"]], rtol=1e-12, atol=1e-15)
            assert M.loops[t] == col["loops"]


def test_initial_pattern_of_A_is_the_least_squares_solution_on_it(c1):
    """Algorithm 1 started from J_k^(0) = rows of column k of A and no loop
    (l_max = 0, no dropping): every column is the LS minimiser of
    ||A(:,J) m - e_k|| on that pattern, which NumPy's lstsq gives directly."""
    A = gen.convdiff2d(10, (7.0, -3.0))
    M = oracle.build(A, c=3, l_max=0, eps=1e-12, drop="none", init="A")
    D = A.to_dense()
    for t, k in enumerate(M.cols):
        J, v = M.column(t)
        expect_J = np.sort(A.row_idx[A.col_ptr[k]:A.col_ptr[k + 1]])
        np.testing.assert_array_equal(J, expect_J)
        e = np.zeros(A.n)
        e[k] = 1.0
        x, *_ = np.linalg.lstsq(D[:, J], e, rcond=None)
        np.testing.assert_allclose(v, x, rtol=1e-12, atol=1e-14 * np.abs(x).max())
        np.testing.assert_allclose(M.rho[t], np.linalg.norm(D[:, J] @ x - e), rtol=1e-12)
        assert M.loops[t] == 0
    # with loops, the initial pattern is kept unless a drop removes it: J^(0) is a subset of J
    M2 = oracle.build(A, c=3, l_max=5, eps=0.1, drop="none", init="A")
    for t, k in enumerate(M2.cols):
        J, _ = M2.column(t)
        assert set(A.row_idx[A.col_ptr[k]:A.col_ptr[k + 1]]) <= set(J)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("drop", ["none", "adaptive", "fixed"])
def test_p9_exact_brute_force_initial_pattern_of_A(seed, drop):
    """The oracle's initial pattern of A against exact rational RSAI started the same way."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(4, 9))
    D = _small_int_matrix(rng, n)
    c = int(rng.integers(1, 4))
    lm = int(rng.integers(0, 4))
    eps, tol = Fraction(1, 20), Fraction(3, 100)
    ex = exact_rsai(D.tolist(), c=c, l_max=lm, eps=eps, drop=drop, tol=tol, init="A")
    M = oracle.build(gen.from_dense(D), c=c, l_max=lm, eps=float(eps), drop=drop, tol=float(tol), init="A")
    for t, (J, m, rho2, loops) in enumerate(ex):
        Jo, vo = M.column(t)
        assert list(Jo) == J, (t, Jo, J)
        np.testing.assert_allclose(vo, [float(v) for v in m], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(M.rho[t] ** 2, float(rho2), rtol=1e-10, atol=1e-15)
        assert M.loops[t] == loops


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("drop", ["none", "adaptive", "fixed"])
def test_p9_exact_brute_force_zero_diagonal(seed, drop):
    """Structurally zero diagonal entries (a row permutation of a diagonally
    dominant matrix): r_k lives on S = I u {k} with r(k) = -1 while k is not
    in I, and m_kk = 0 on J = {k}.  Oracle against exact rational RSAI."""
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(4, 9))
    while True:
        D = _small_int_matrix(rng, n)[rng.permutation(n)]
        if np.any(np.diag(D) == 0):
            break
    assert abs(np.linalg.det(D)) > 0.5  # integer matrix, nonsingular
    c = int(rng.integers(1, 4))
    lm = int(rng.integers(1, 5))
    eps, tol = Fraction(1, 20), Fraction(3, 100)
    ex = exact_rsai(D.tolist(), c=c, l_max=lm, eps=eps, drop=drop, tol=tol)
    M = oracle.build(gen.from_dense(D), c=c, l_max=lm, eps=float(eps), drop=drop, tol=float(tol))
    for t, (J, m, rho2, loops) in enumerate(ex):
        Jo, vo = M.column(t)
        assert list(Jo) == J, (t, Jo, J)
        np.testing.assert_allclose(vo, [float(v) for v in m], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(M.rho[t] ** 2, float(rho2), rtol=1e-10, atol=1e-15)
        assert M.loops[t] == loops


@pytest.mark.parametrize("delta,band,row", [(1e-13, 1e-12, 1), (1e-13, 0.0, 2), (1e-6, 1e-12, 2), (0.0, 0.0, 1)])
def test_tie_band_reading(delta, band, row):
    """Reading of the order of Algorithm 1's dominant indices: residual entries
    within tie_band * ||r||_inf of the c-th largest count as tied and are taken
    by lowest index.  Column 0 of
    [[4,0,0],[1,4,0],[1+delta,0,4]] has r = (4m-1, m, (1+delta)m) at loop 0, so
    with c = 1 row 2 is strictly largest; rows 1 and 2 bring columns 1 and 2."""
    D = np.array([[4.0, 0.0, 0.0], [1.0, 4.0, 0.0], [1.0 + delta, 0.0, 4.0]])
    M = oracle.build(gen.from_dense(D), c=1, l_max=1, eps=1e-12, drop="none", tie_band=band)
    J, _ = M.column(0)
    assert list(J) == [0, row]
