"""Pins of the oracle's work counters (the numerators of every roofline figure).

The counters charge the method's own work: the LS problem of each loop is
updated from the previous QR factorization when J grows (Section 3, the QR
update of the earlier SPAI work the paper follows), a solve after a drop pass
(Eq. 4.3) starts from scratch, each column of A that ever enters J_k is read
once for column k, and each dominant row once.

These tests recompute the counters without the oracle's formulas.  The exact
rational oracle (``oracle.exact_rsai``) records the J history of a column and
the dominant rows taken.  A plain Householder QR that keeps its factor between
growth loops, appends the new rows and columns after the old ones and applies
the old reflectors to the new columns only, replays those solves here and
counts every multiplication, addition, subtraction and division of its loops
over rows and of its back substitution.  The per-column scalars of a step
(the square root of the norm, the reflector head, 2 s / v^T v) are O(p) per
step and, as in the usual Householder flop count, not counted.  The replayed
solution is checked against the exact one, so the counted operations are
those of a working QR update.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.exact_rsai import exact_rsai
from paper_1503_04500_gb300 import inputs as gen

# 9x9 integer matrix, row-diagonally dominant.  With c = 2, l_max = 4,
# eps = 1/10 and FIXED tol = 1/20, column 1 runs four growth loops and two drop
# passes, and column 3 of A is dropped after the second loop and re-enters J
# in the third.
D9 = [[4, -1, 0, -1, 0, 0, 0, 0, 0],
      [0, 6, 0, 0, -2, 0, 3, 0, 0],
      [-4, 0, 7, -2, 0, 0, 0, 0, 0],
      [0, 0, 0, 4, 0, 2, 0, 0, 0],
      [0, 0, 0, 0, 1, 0, 0, 0, 0],
      [0, 2, 0, 2, 0, 14, 4, 0, 4],
      [0, -3, 0, 0, -3, -3, 17, 2, 4],
      [0, 4, 0, 2, 0, 0, 4, 12, 0],
      [0, 0, 0, 0, 0, 0, 0, 0, 1]]
PARAMS = dict(c=2, l_max=4, eps=Fraction(1, 10), drop="fixed", tol=Fraction(1, 20))


class Counted:
    """Householder QR of one column's LS problems, kept between growth loops."""

    def __init__(self, D, k):
        self.D = np.asarray(D, dtype=np.float64)
        self.k = k
        self.ops = 0
        self.rows = self.cols = None  # factor order
        self.W = None  # R above the diagonal, reflector tails below it
        self.vhead = self.tau = self.qte = None

    def _rows_of(self, J):
        return sorted({i for j in J for i in np.nonzero(self.D[:, j])[0].tolist()})

    def _reflect(self, j, c_list, q):
        """Reflector of factor column j over rows j..q-1, applied to the columns
        c_list (-1 stands for the right-hand side)."""
        W = self.W
        x = W[j:q, j].copy()
        self.ops += 2 * (q - j)  # sigma = x^T x
        sigma = float(np.dot(x, x))
        alpha = -np.sqrt(sigma) if x[0] >= 0 else np.sqrt(sigma)
        v = x.copy()
        v[0] = x[0] - alpha
        vtv = float(np.dot(v, v))
        tau = 2.0 / vtv if vtv > 0 else 0.0
        for c in c_list:
            t = self.qte if c < 0 else W[:, c]
            s = 0.0
            for i in range(q - j):  # dot product: a multiplication and an addition per row
                s += v[i] * t[j + i]
                self.ops += 2
            f = s * tau
            for i in range(q - j):  # update: a multiplication and a subtraction per row
                t[j + i] -= f * v[i]
                self.ops += 2
        W[j, j] = alpha
        W[j + 1:q, j] = v[1:]
        self.vhead[j] = v[0]
        self.tau[j] = tau

    def _apply_old(self, j, c, q0):
        """Stored reflector j (rows j..q0-1 of the old factor) applied to column c."""
        W = self.W
        v = np.concatenate(([self.vhead[j]], W[j + 1:q0, j]))
        t = W[:, c]
        s = 0.0
        for i in range(q0 - j):
            s += v[i] * t[j + i]
            self.ops += 2
        f = s * self.tau[j]
        for i in range(q0 - j):
            t[j + i] -= f * v[i]
            self.ops += 2

    def _back_substitute(self, p):
        W, y = self.W, self.qte
        x = np.zeros(p)
        for i in range(p - 1, -1, -1):
            s = y[i]
            for c in range(i + 1, p):  # a multiplication and a subtraction
                s -= W[i, c] * x[c]
                self.ops += 2
            x[i] = s / W[i, i]
            self.ops += 1
        return x

    def solve(self, J, grown):
        I = self._rows_of(J)
        if grown and self.rows is not None:
            new_rows = [i for i in I if i not in self.rows]
            new_cols = [j for j in J if j not in self.cols]
            q0, p0 = len(self.rows), len(self.cols)
            rows, cols = self.rows + new_rows, self.cols + new_cols
            W = np.zeros((len(rows), len(cols)))
            W[:q0, :p0] = self.W
            for b, j in enumerate(new_cols):
                W[:, p0 + b] = self.D[rows, j]
            qte = np.concatenate((self.qte, [1.0 if i == self.k else 0.0 for i in new_rows]))
            vhead = np.concatenate((self.vhead, np.zeros(len(new_cols))))
            tau = np.concatenate((self.tau, np.zeros(len(new_cols))))
            self.W, self.qte, self.vhead, self.tau = W, qte, vhead, tau
            for j in range(p0):
                for c in range(p0, len(cols)):
                    self._apply_old(j, c, q0)
            start = p0
        else:
            rows, cols = I, list(J)
            self.W = self.D[np.ix_(rows, cols)].copy()
            self.qte = np.array([1.0 if i == self.k else 0.0 for i in rows])
            self.vhead = np.zeros(len(cols))
            self.tau = np.zeros(len(cols))
            start = 0
        q, p = len(rows), len(cols)
        for j in range(start, p):
            self._reflect(j, list(range(j + 1, p)) + [-1], q)
        self.rows, self.cols = rows, cols
        # keep Q^T e for the next update; the solve works on a copy
        keep = self.qte.copy()
        x = self._back_substitute(p)
        self.qte = keep
        return dict(zip(cols, x))


def replay(D, k, events):
    """(qr flops, residual flops, bytes) of column k recomputed from its trace."""
    A = np.asarray(D, dtype=np.float64)
    nnz_col = (A != 0).sum(axis=0)
    nnz_row = (A != 0).sum(axis=1)
    qr = Counted(D, k)
    res_flops = 0
    seen, rows_bytes, m = set(), 0, None
    solves = [e for e in events if e[0] == "solve"]
    for t, ev in enumerate(events):
        if ev[0] == "rows":
            rows_bytes += sum(4 * int(nnz_row[i]) + 16 for i in ev[1])
            continue
        J, kind = ev[1], ev[2]
        seen.update(J)
        m = qr.solve(J, grown=(kind == "grown"))
        # a residual follows every round: after its solve, or after the re-solve of its drop pass
        idx = solves.index(ev)
        nxt = solves[idx + 1][2] if idx + 1 < len(solves) else None
        if nxt != "dropped":
            S = set(qr._rows_of(J)) | {k}
            res_flops += 2 * int(sum(nnz_col[j] for j in J)) + 2 * len(S)
    col_bytes = sum(12 * int(nnz_col[j]) + 16 for j in seen)
    p_final = len(solves[-1][1])
    return qr.ops, res_flops, col_bytes + rows_bytes + 36 * p_final, m


@pytest.fixture(scope="module")
def traced():
    tr = []
    ex = exact_rsai(D9, trace=tr, **PARAMS)
    M = oracle.build(gen.from_dense(np.array(D9, dtype=np.float64)), c=2, l_max=4, eps=0.1, drop="fixed", tol=0.05)
    return tr, ex, M


def test_fixture_has_growth_drops_and_a_reentry(traced):
    tr, ex, M = traced
    kinds = [e[2] for e in tr[1] if e[0] == "solve"]
    assert kinds.count("grown") >= 2 and kinds.count("dropped") >= 1
    Js = [set(e[1]) for e in tr[1] if e[0] == "solve"]
    # column 3 of A: in J, dropped, back in J
    inside = [3 in s for s in Js]
    first_out = inside.index(False, inside.index(True))
    assert True in inside[first_out:]
    # the FP64 oracle takes the same path as the exact one on every column
    for t, (J, m, rho2, loops) in enumerate(ex):
        assert list(M.column(t)[0]) == J and M.loops[t] == loops


@pytest.mark.parametrize("k", range(9))
def test_counters_equal_counted_qr_update_replay(traced, k):
    """qr_flops, res_flops and bytes of every column equal the counts of the
    replayed QR update; the replayed solution is the exact LS solution."""
    tr, ex, M = traced
    ops, res, by, m = replay(D9, k, tr[k])
    J, mx, rho2, loops = ex[k]
    np.testing.assert_allclose([m[j] for j in J], [float(v) for v in mx], rtol=1e-11, atol=1e-14)
    assert M.counters[k, 0] == ops
    assert M.counters[k, 1] == res
    assert M.counters[k, 2] == by


def test_update_branch_by_hand(traced):
    """Column 1's second growth loop by hand.  J = {1,3,4,6,7} has I = rows
    0..7 (q0 = 8, p0 = 5); adding Jhat = {5, 8} brings row 8 (q = 9, p = 7).
    The counted replay of that solve alone must equal
        4 (p - p0) sum_{j<p0} (q0 - j) + sum_{j=p0}^{p-1} (q - j)(2 + 4 (p - j)) + p^2."""
    tr, ex, M = traced
    A = np.array(D9, dtype=np.float64)
    solves = [e for e in tr[1] if e[0] == "solve"]
    assert [s[2] for s in solves[:3]] == ["first", "grown", "grown"]
    rows_of = lambda J: sorted({i for j in J for i in np.nonzero(A[:, j])[0].tolist()})  # noqa: E731
    q0, p0 = len(rows_of(solves[1][1])), len(solves[1][1])
    q, p = len(rows_of(solves[2][1])), len(solves[2][1])
    assert (q0, p0, q, p) == (8, 5, 9, 7)
    qr = Counted(D9, 1)
    qr.solve(solves[0][1], grown=False)
    qr.solve(solves[1][1], grown=True)
    before = qr.ops
    qr.solve(solves[2][1], grown=True)
    # written out: old reflectors on 2 new columns, rows j..7: 4*2*(8+7+6+5+4) = 240;
    # steps j = 5, 6 on 9 rows: (9-5)(2+4*2) + (9-6)(2+4*1) = 40 + 18 = 58; back substitution 49
    assert qr.ops - before == 240 + 58 + 49
