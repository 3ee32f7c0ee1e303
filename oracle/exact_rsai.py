"""Exact rational RSAI(tol) for tiny integer matrices -- TEST INFRASTRUCTURE ONLY.

A second, brute-force statement of Algorithm 1 + Eq. 4.3 in ``fractions``
arithmetic, used to pin the FP64 oracle (``rsai_oracle.c``).  It shares no
arithmetic with it: the LS problem (Eq. 2.3) is solved through the exact normal
equations B^T B x = B^T e by Gaussian elimination instead of Householder QR,
residuals and norms are exact, ties are exact, and the tests ||r|| <= eps and
|m_j| <= tau are decided exactly (on squares where a root would appear).

Readings are the same as the FP64 oracle's (S = I u {k}, drop once after every
solve then re-solve, keep-one, ties by lowest index, excluded rows R, empty
Jhat loops counted); with exact arithmetic no tie band is needed.

With ``select="spai"`` the new indices are SPAI's most profitable ones
(Section 2, Eqs. 2.5-2.7): the candidates are the nonzero columns of the rows
where r != 0, less J, ranked by s_j = (r^T A e_j)^2 / ||A e_j||^2 exactly
(the largest s_j is the smallest rho_j), ties by lowest j; no candidate ends
the column.
"""
from __future__ import annotations

from fractions import Fraction


def _solve_normal(B, e):
    """x with (B^T B) x = B^T e, exactly (B has full column rank)."""
    q, p = len(B), len(B[0])
    G = [[sum(B[i][a] * B[i][b] for i in range(q)) for b in range(p)] for a in range(p)]
    h = [sum(B[i][a] * e[i] for i in range(q)) for a in range(p)]
    for col in range(p):  # Gauss-Jordan with the first nonzero pivot
        piv = next(r for r in range(col, p) if G[r][col] != 0)
        G[col], G[piv] = G[piv], G[col]
        h[col], h[piv] = h[piv], h[col]
        for r in range(p):
            if r != col and G[r][col] != 0:
                f = G[r][col] / G[col][col]
                G[r] = [G[r][t] - f * G[col][t] for t in range(p)]
                h[r] -= f * h[col]
    return [h[a] / G[a][a] for a in range(p)]


def exact_rsai(A, c=3, l_max=10, eps=Fraction(3, 10), drop="fixed", tol=Fraction(1, 1000), init="identity",
               trace=None, select="rsai"):
    """Columns of M for a dense integer (or Fraction) matrix A (list of rows).
    ``init``: the initial pattern J_k^(0) (Algorithm 1), "identity" ({k})
    or "A" (the rows i with A[i][k] != 0).

    Returns a list of (J, m, rho2, loops) with J ascending, m exact Fractions,
    rho2 = ||r_k||^2 exact.

    ``trace`` (a list, optional) receives one event list per column, in the
    order of the algorithm: ("solve", J, kind) for every LS solve, with kind
    "first" (the initial pattern), "grown" (J = previous J + Jhat) or
    "dropped" (the re-solve after a drop pass), and ("rows", Rhat) for every
    set of dominant rows taken (RSAI), or ("spai", L, candidates, added) for
    every SPAI selection.  Work counters can be recomputed from it.
    """
    n = len(A)
    A = [[Fraction(v) for v in row] for row in A]
    norm1 = max(sum(abs(A[i][j]) for i in range(n)) for j in range(n))
    eps = Fraction(eps)
    tol = Fraction(tol)
    out = []
    for k in range(n):
        ev = []
        if trace is not None:
            trace.append(ev)

        def solve(J, kind):
            ev.append(("solve", list(J), kind))
            return _solve_plain(J)

        def _solve_plain(J):
            I = sorted({i for j in J for i in range(n) if A[i][j] != 0})
            B = [[A[i][j] for j in J] for i in I]
            e = [Fraction(int(i == k)) for i in I]
            return _solve_normal(B, e)

        def drop_pass(J, m):
            if drop == "none":
                return J, m
            tau = eps / (len(J) * norm1) if drop == "adaptive" else tol / norm1
            keep = [t for t in range(len(J)) if abs(m[t]) > tau]
            if len(keep) == len(J):
                return J, m
            if not keep:
                best = max(range(len(J)), key=lambda t: (abs(m[t]), -J[t]))
                keep = [best]
            if len(keep) == len(J):
                return J, m
            J = [J[t] for t in keep]
            return J, solve(J, "dropped")

        def residual(J, m):
            S = sorted({i for j in J for i in range(n) if A[i][j] != 0} | {k})
            r = {i: sum(A[i][j] * m[t] for t, j in enumerate(J)) - (1 if i == k else 0) for i in S}
            return r

        J = [k] if init == "identity" else [i for i in range(n) if A[i][k] != 0]
        R = set()
        loops = 0
        m = solve(J, "first")
        J, m = drop_pass(J, m)
        r = residual(J, m)
        rho2 = sum(v * v for v in r.values())
        while rho2 > eps * eps and loops < l_max:
            if select == "spai":
                L = sorted(i for i, v in r.items() if v != 0)
                if not L:
                    break
                N = sorted({j for i in L for j in range(n) if A[i][j] != 0} - set(J))
                if not N:
                    break
                score = {j: sum(r[i] * A[i][j] for i in r) ** 2 / sum(A[i][j] ** 2 for i in range(n)) for j in N}
                add = sorted(N, key=lambda j: (-score[j], j))[:c]
                ev.append(("spai", L, N, sorted(add)))
                loops += 1
                J = sorted(set(J) | set(add))
                m = solve(J, "grown")
                J, m = drop_pass(J, m)
                r = residual(J, m)
                rho2 = sum(v * v for v in r.values())
                continue
            cand = [i for i, v in r.items() if v != 0 and i not in R]
            if not cand:
                break
            cand.sort(key=lambda i: (-abs(r[i]), i))
            Rhat = cand[:c]
            ev.append(("rows", list(Rhat)))
            R.update(Rhat)
            Jhat = sorted({j for i in Rhat for j in range(n) if A[i][j] != 0} - set(J))
            loops += 1
            if not Jhat:
                continue
            J = sorted(set(J) | set(Jhat))
            m = solve(J, "grown")
            J, m = drop_pass(J, m)
            r = residual(J, m)
            rho2 = sum(v * v for v in r.values())
        out.append((J, m, rho2, loops))
    return out
