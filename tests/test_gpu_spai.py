"""SPAI's most-profitable-index selection (Section 2, Eqs. 2.5-2.7) on the GPU
(RSAI_FLAG_SELECT_SPAI), against the oracle's SPAI mode: FP64 patterns
bit-identical with values, ||r_k|| and loops as the oracle's, the work counters
equal; FP32+refine through the every-column check.  Section 5.2's settings:
c = 3 indices per loop, eps = 0.3, l_max = floor(10 nnz(A) / (3 n))."""
import numpy as np
import pytest

import oracle
from paper_1503_04500_gb300 import inputs as gen
from parity_check import check_fp32_every_column

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rsai = pytest.importorskip("paper_1503_04500_gb300.rsai")


def _params(A, drop):
    return dict(c=3, l_max=int(np.floor(10 * A.nnz / (3 * A.n))), eps=0.3, tol=1e-3, drop=drop)


def _build(A, precision, kw):
    h = rsai.build(rsai.DeviceMatrix.from_host(A), precision=precision, select="spai", **kw)
    res = tuple(t.cpu().numpy() for t in h.M())
    rho, loops, flags = (t.cpu().numpy() for t in h.columns())
    st = h.stats()
    h.free()
    return res, rho, loops, flags, st


@pytest.mark.parametrize("name", ["convdiff2d_20", "powerlaw_2000"])
@pytest.mark.parametrize("drop", ["fixed", "none"])
def test_spai_gpu_matches_oracle(name, drop):
    A = gen.convdiff2d(20, (20.0, 20.0)) if name == "convdiff2d_20" else gen.powerlaw(2000, seed=17, dmax=100)
    kw = _params(A, drop)
    ref = oracle.build(A, select="spai", **kw)
    res, rho, loops, flags, st = _build(A, "fp64", kw)
    orp, oci, ova = ref.csr()
    rp, ci, va = res
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    np.testing.assert_allclose(va, ova, rtol=1e-9, atol=1e-15 * np.abs(ova).max())
    np.testing.assert_allclose(rho, ref.rho, rtol=1e-9, atol=1e-14)
    np.testing.assert_array_equal(loops, ref.loops)
    assert st["n_failed"] == 0
    if name == "convdiff2d_20":
        assert st["qr_flops"] == ref.counters[:, 0].sum()
        assert st["bytes"] == ref.counters[:, 2].sum()
        assert st["select_flops"] == ref.counters[:, 8].sum() > 0
    res32, rho32, *_ = _build(A, "fp32_refine", kw)
    check_fp32_every_column(A, res32, rho32, ref)


def test_spai_and_rsai_differ_only_in_selection():
    """With l_max = 0 no selection runs: SPAI and RSAI(tol) builds are the same M."""
    A = gen.convdiff2d(20, (20.0, 20.0))
    kw = dict(c=3, l_max=0, eps=0.3, tol=1e-3, drop="fixed")
    a = rsai.build(rsai.DeviceMatrix.from_host(A), precision="fp64", select="spai", **kw)
    b = rsai.build(rsai.DeviceMatrix.from_host(A), precision="fp64", **kw)
    for x, y in zip(a.M(), b.M()):
        assert torch.equal(x, y)
    a.free()
    b.free()
