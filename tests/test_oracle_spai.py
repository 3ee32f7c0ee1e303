"""Pins of the oracle's SPAI selection (Section 2, Eqs. 2.5-2.7), the
comparison method of Section 5.2, which shares the solve, drop and residual of
RSAI(tol) and replaces its dominant rows by the most profitable indices.

- exact rational SPAI (oracle.exact_rsai, select="spai") on small integer
  matrices: the same patterns, values and loop counts;
- the choice itself against Eq. 2.6 solved directly: for every candidate j the
  one-dimensional least-squares problem min_mu ||r + mu A e_j|| by NumPy's
  lstsq, and the c candidates with the smallest residual taken;
- the work counters recomputed from the exact trace;
- closed forms: a diagonal matrix needs no loop, and without dropping the
  residual never grows as l_max grows (J is nested).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.exact_rsai import exact_rsai
from paper_1503_04500_gb300 import inputs as gen
from test_counters_pin import Counted


def _small_int_matrix(rng, n, density=0.35):
    D = rng.integers(-3, 4, size=(n, n)) * (rng.random((n, n)) < density)
    np.fill_diagonal(D, 0)
    d = np.abs(D).sum(axis=1) + rng.integers(1, 3, size=n)
    D += np.diag(np.where(rng.random(n) < 0.5, -d, d))
    return D


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("drop", ["none", "fixed"])
def test_spai_exact_brute_force(seed, drop):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(4, 10))
    D = _small_int_matrix(rng, n)
    c = int(rng.integers(1, 4))
    lm = int(rng.integers(1, 5))
    eps, tol = Fraction(1, 20), Fraction(3, 100)
    ex = exact_rsai(D.tolist(), c=c, l_max=lm, eps=eps, drop=drop, tol=tol, select="spai")
    M = oracle.build(gen.from_dense(D), c=c, l_max=lm, eps=float(eps), drop=drop, tol=float(tol), select="spai")
    for t, (J, m, rho2, loops) in enumerate(ex):
        Jo, vo = M.column(t)
        assert list(Jo) == J, (t, Jo, J)
        np.testing.assert_allclose(vo, [float(v) for v in m], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(M.rho[t] ** 2, float(rho2), rtol=1e-10, atol=1e-15)
        assert M.loops[t] == loops


def test_spai_choice_minimises_the_one_dimensional_residual():
    """One SPAI loop from J = {k}, no dropping: the indices added are the c
    candidates whose one-dimensional problem (Eq. 2.6), solved here by lstsq,
    leaves the smallest residual."""
    A = gen.powerlaw(300, seed=12, dmax=12)
    D = A.to_dense()
    c = 3
    M = oracle.build(A, c=c, l_max=1, eps=1e-9, drop="none", select="spai")
    checked = 0
    for k in range(0, A.n, 7):
        a = D[:, k]
        m0 = a[k] / (a @ a)
        r = a * m0
        r[k] -= 1.0
        L = np.nonzero(np.abs(r) > 1e-12 * np.abs(r).max())[0]
        N = sorted(set(np.nonzero(D[L, :])[1].tolist()) - {k})
        rho = []
        for j in N:
            mu, *_ = np.linalg.lstsq(D[:, [j]], -r, rcond=None)
            rho.append(np.linalg.norm(r + D[:, j] * mu[0]))
        order = np.lexsort((np.array(N), np.array(rho)))
        want = sorted([k] + [N[i] for i in order[:c]])
        got = list(M.column(k)[0])
        # the c-th and (c+1)-th smallest may tie within rounding: then accept either order
        if len(N) > c and abs(rho[order[c - 1]] - rho[order[c]]) < 1e-12:
            continue
        assert got == want, (k, got, want)
        checked += 1
    assert checked > 30


def test_spai_counters_from_the_exact_trace():
    """qr_flops (the QR update replayed and counted), sel_flops and bytes of
    every column recomputed from the exact oracle's SPAI trace."""
    rng = np.random.default_rng(77)
    D = _small_int_matrix(rng, 9, density=0.3)
    nnz_col = (D != 0).sum(axis=0)
    nnz_row = (D != 0).sum(axis=1)
    tr = []
    ex = exact_rsai(D.tolist(), c=2, l_max=3, eps=Fraction(1, 50), drop="fixed", tol=Fraction(1, 20),
                    trace=tr, select="spai")
    M = oracle.build(gen.from_dense(D.astype(np.float64)), c=2, l_max=3, eps=0.02, drop="fixed", tol=0.05,
                     select="spai")
    grown = 0
    for k, ev in enumerate(tr):
        assert list(M.column(k)[0]) == ex[k][0]
        qr = Counted(D, k)
        sel, byts, seen = 0, 0, set()
        for e in ev:
            if e[0] == "spai":
                _, L, N, add = e
                byts += sum(4 * int(nnz_row[i]) + 16 for i in L)
                byts += sum(12 * int(nnz_col[j]) + 16 for j in N)
                sel += sum(4 * int(nnz_col[j]) + 3 for j in N)
            elif e[0] == "solve":
                seen.update(e[1])
                qr.solve(e[1], grown=(e[2] == "grown"))
                grown += e[2] == "grown"
        byts += sum(12 * int(nnz_col[j]) + 16 for j in seen) + 36 * len(ex[k][0])
        assert M.counters[k, 0] == qr.ops, k
        assert M.counters[k, 8] == sel, k
        assert M.counters[k, 2] == byts, k
    assert grown >= 5


def test_spai_diagonal_needs_no_loop():
    d = np.array([2.0, -3.0, 0.5, 7.0])
    M = oracle.build(gen.from_dense(np.diag(d)), c=2, l_max=5, eps=1e-6, drop="none", select="spai")
    np.testing.assert_array_equal(M.loops, 0)
    np.testing.assert_allclose(M.vals, 1.0 / d, rtol=1e-15)


def test_spai_residual_non_increasing_in_l_max():
    A = gen.convdiff2d(10, (20.0, 20.0))
    prev = None
    for lm in range(0, 5):
        M = oracle.build(A, c=3, l_max=lm, eps=1e-6, drop="none", select="spai")
        if prev is not None:
            assert np.all(M.rho <= prev * (1 + 1e-12) + 1e-15)
        prev = M.rho
