"""Write tests/golden/exact_small.json: exact rational RSAI(tol) results.

The values come from ``oracle.exact_rsai`` only (Algorithm 1 + Eq. 4.3 in
rational arithmetic, LS through the exact normal equations of Eq. 2.3).  The
matrices are small integer matrices with a nonzero diagonal, drawn from a fixed
seed.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
from fractions import Fraction

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.exact_rsai import exact_rsai  # noqa: E402


def small_int_matrix(rng, n, density=0.35):
    D = rng.integers(-3, 4, size=(n, n)) * (rng.random((n, n)) < density)
    np.fill_diagonal(D, 0)
    d = np.abs(D).sum(axis=1) + rng.integers(1, 3, size=n)
    D += np.diag(np.where(rng.random(n) < 0.5, -d, d))
    return D


def main():
    rng = np.random.default_rng(20150316)
    cases = []
    for i in range(6):
        n = int(rng.integers(5, 9))
        D = small_int_matrix(rng, n)
        for drop in ("none", "adaptive", "fixed"):
            params = dict(c=2, l_max=3, eps="1/20", drop=drop, tol="3/100")
            res = exact_rsai(D.tolist(), c=2, l_max=3, eps=Fraction(1, 20), drop=drop, tol=Fraction(3, 100))
            cases.append({
                "matrix": D.tolist(),
                "params": params,
                "columns": [{"J": J, "m": [str(v) for v in m], "rho2": str(r2), "loops": lp}
                            for (J, m, r2, lp) in res],
            })
    out = {
        "source": "exact rational RSAI(tol): Algorithm 1 (Section 3) with the dropping of Eq. 4.3 "
                  "(Section 4); LS problems of Eq. 2.3 solved exactly",
        "cases": cases,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, len(cases), "cases")


if __name__ == "__main__":
    main()
