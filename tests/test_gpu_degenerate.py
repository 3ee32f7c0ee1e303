"""Degenerate cases of Algorithm 1 on the GPU, against the FP64 oracle:
structurally zero diagonal entries (k not in I_k, so r_k lives on I_k u {k}
and r(k) = -1 at the start), n = 1, and l_max = 0 (no loop after the first
solve and its drop pass)."""
import numpy as np
import pytest

import oracle
from paper_1503_04500_gb300 import inputs as gen
from parity_check import check_fp32_every_column

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rsai = pytest.importorskip("paper_1503_04500_gb300.rsai")

KW = dict(c=3, l_max=10, eps=0.3, tol=1e-3)


def _build(A, **kw):
    h = rsai.build(rsai.DeviceMatrix.from_host(A), **kw)
    res = tuple(t.cpu().numpy() for t in h.M())
    rho, loops, flags = (t.cpu().numpy() for t in h.columns())
    st = h.stats()
    h.free()
    return res, rho, loops, flags, st


def _fp64_equal(A, ref, res, rho, loops, st, rtol=1e-10):
    orp, oci, ova = ref.csr()
    rp, ci, va = res
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    np.testing.assert_allclose(va, ova, rtol=rtol, atol=1e-15 * np.abs(ova).max())
    np.testing.assert_allclose(rho, ref.rho, rtol=rtol, atol=1e-14)
    np.testing.assert_array_equal(loops, ref.loops)
    assert st["n_failed"] == 0 and st["nnz_M"] == ref.nnz


def _rows_rolled(A, shift):
    """Rows of A moved down by `shift` (cyclically): a nonsingular matrix whose
    diagonal is structurally zero wherever A(k - shift, k) is."""
    return gen.from_dense(np.roll(A.to_dense(), shift, axis=0))


@pytest.mark.parametrize("name", ["convdiff2d_12_rolled", "powerlaw_500_rolled"])
@pytest.mark.parametrize("drop", ["fixed", "none"])
def test_structurally_zero_diagonal(name, drop):
    A = _rows_rolled(gen.convdiff2d(12, (20.0, 20.0)), 5) if name.startswith("convdiff") else \
        _rows_rolled(gen.powerlaw(500, seed=23, dmax=30), 1)
    D = A.to_dense()
    assert np.count_nonzero(np.diag(D) == 0.0) > A.n // 2  # most diagonal entries are structural zeros
    kw = dict(KW, drop=drop)
    ref = oracle.build(A, **kw)
    res, rho, loops, flags, st = _build(A, precision="fp64", **kw)
    _fp64_equal(A, ref, res, rho, loops, st)
    res32, rho32, *_ = _build(A, precision="fp32_refine", **kw)
    check_fp32_every_column(A, res32, rho32, ref)


@pytest.mark.parametrize("a", [3.0, -0.5])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_n_equals_one(a, precision):
    """A = [a]: J = {k} gives m = 1/a exactly as the oracle's, r = 0, no loop."""
    A = gen.from_dense(np.array([[a]]))
    ref = oracle.build(A, drop="fixed", **KW)
    res, rho, loops, flags, st = _build(A, precision=precision, drop="fixed", **KW)
    rp, ci, va = res
    np.testing.assert_array_equal(rp, [0, 1])
    np.testing.assert_array_equal(ci, [0])
    np.testing.assert_allclose(va, ref.vals, rtol=1e-15)
    np.testing.assert_allclose(va, [1.0 / a], rtol=1e-15)
    assert loops[0] == 0 and rho[0] <= 1e-15 and (flags[0] & 1) == 1
    assert st["n_c"] == 0 and st["nnz_M"] == 1


@pytest.mark.parametrize("drop", ["fixed", "adaptive", "none"])
def test_l_max_zero(drop):
    """l_max = 0: the first solve (and its drop pass) only; every column of M is
    m_kk = a_kk / ||a_k||^2 on J = {k}, and the loop count is 0 everywhere."""
    A = gen.convdiff2d(20, (20.0, 20.0))
    kw = dict(c=3, l_max=0, eps=0.3, tol=1e-3, drop=drop)
    ref = oracle.build(A, **kw)
    res, rho, loops, flags, st = _build(A, precision="fp64", **kw)
    _fp64_equal(A, ref, res, rho, loops, st)
    assert np.all(loops == 0)
    rp, ci, va = res
    np.testing.assert_array_equal(np.diff(rp), 1)
    np.testing.assert_array_equal(ci, np.arange(A.n))
    D = A.to_dense()
    np.testing.assert_allclose(va, np.diag(D) / (D * D).sum(axis=0), rtol=1e-14)
    res32, rho32, loops32, *_ = _build(A, precision="fp32_refine", **kw)
    check_fp32_every_column(A, res32, rho32, ref)
    assert np.all(loops32 == 0)
