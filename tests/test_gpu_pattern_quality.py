"""The pattern-quality check of Section 5.1 (Fig. 1) on M built by the GPU:
the same numbers as on the oracle's M (the FP64 GPU pattern is the oracle's
bit for bit), and an FP32+refine M within its <= 1% pattern tolerance."""
import numpy as np
import pytest

import oracle
from paper_1503_04500_gb300 import pattern_quality as pq

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rsai = pytest.importorskip("paper_1503_04500_gb300.rsai")

# Section 5.1's parameters: c = 3, eps = 0.2, l_max = 15, the adaptive drop of Eq. 4.3
KW = dict(c=3, l_max=15, eps=0.2, drop="adaptive", tol=1e-3)


@pytest.mark.parametrize("name,size", [("convdiff2d", 20), ("convdiff2d", 30), ("powerlaw", 900)])
def test_gpu_M_pattern_quality_equals_oracle_M(name, size):
    A = pq._workload(name, size, 1503)
    ref = oracle.build(A, **KW)
    orp, oci, _ = ref.csr()
    want = pq.compare(A, orp, oci)
    for precision in ("fp64", "fp32_refine"):
        h = rsai.build(rsai.DeviceMatrix.from_host(A), precision=precision, **KW)
        rp, ci, _ = (t.cpu().numpy() for t in h.M())
        got = pq.compare(A, rp, ci)
        h.free()
        if precision == "fp64":
            assert got == want
        else:
            assert abs(got["nnz_M"] - want["nnz_M"]) <= 0.01 * want["nnz_M"]
            assert got["matched_frac"] == pytest.approx(want["matched_frac"], abs=0.01)
            assert got["captured_frac"] == pytest.approx(want["captured_frac"], abs=0.01)
            assert got["irregular_cols_Ainv"] == want["irregular_cols_Ainv"]
