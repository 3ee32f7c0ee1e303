"""Plain FP64 CPU oracle of RSAI(tol) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1503_04500_gb300``) and imports nothing from it; matrices are passed in
duck-typed (attributes n, row_ptr, col_idx, val, col_ptr, row_idx, cval).

Parity status of each function (how it is pinned, see ``tests/test_oracle_*``):
  build     -- pinned: closed form at loop 0, A^{-1} on full patterns, diagonal A,
               normal equations, monotone residual, Theorem 1, power-of-two
               scaling, exact rational brute force on small integer matrices.
  refit     -- pinned: same normal-equation and brute-force checks.
  backward  -- pinned: closed form 2 (AM-I) M^T for the Frobenius loss, dense
               torch autograd through lstsq, central finite differences.
  bicgstab  -- pinned: unpreconditioned iterations against scipy's bicgstab,
               exact solution on a diagonal system.
"""
from .rsai_oracle import (  # noqa: F401
    DROP_ADAPTIVE,
    DROP_FIXED,
    DROP_NONE,
    FLAG_CONVERGED,
    FLAG_NONFINITE,
    FLAG_RANK,
    OracleM,
    backward,
    bicgstab,
    build,
    build_library,
    norm1,
    refit,
    spmv,
)
