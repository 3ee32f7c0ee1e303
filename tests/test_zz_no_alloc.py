"""rsai_bicgstab_noalloc, the solve for callers that cannot allocate device memory.

Such callers (code inside another framework's memory pool or plugin interface,
real-time loops that may not allocate or synchronise) get the same BiCGStab as
rsai_bicgstab with its work vectors in a fixed array inside the library.  This
file is collected last so that a run stopping at its first failure has already
run every other test; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_1503_04500_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rsai = pytest.importorskip("paper_1503_04500_gb300.rsai")


def test_noalloc_matches_allocating_solve_twice():
    """Two calls in a row through the C ABI agree with rsai_bicgstab (and each other)."""
    A = gen.convdiff2d(40, (20.0, 20.0))  # n = 1600
    dA = rsai.DeviceMatrix.from_host(A)
    h = rsai.build(dA, c=3, l_max=10, eps=0.3, tol=1e-3, drop="fixed", precision="fp64")
    M = h.M()
    b = torch.as_tensor(gen.ones_rhs(A), device="cuda")
    x_ref, it_ref, rel_ref, st_ref = rsai.bicgstab(dA, h, b, rtol=1e-8)
    assert st_ref == 0
    for call in range(2):
        x = torch.full_like(b, float("nan"))
        it, rel, st = rsai.bicgstab_noalloc(dA, M, b, x, rtol=1e-8)
        assert st == 0, call
        assert it == it_ref, call
        np.testing.assert_allclose(x.cpu().numpy(), x_ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
        assert rel == pytest.approx(rel_ref, rel=1e-6, abs=1e-15)
    # without a preconditioner, also twice
    x0_ref, it0_ref, _, _ = rsai.bicgstab(dA, None, b, rtol=1e-8)
    for call in range(2):
        x0 = torch.empty_like(b)
        it0, rel0, st0 = rsai.bicgstab_noalloc(dA, None, b, x0, rtol=1e-8)
        assert st0 == 0 and it0 == it0_ref
        np.testing.assert_allclose(x0.cpu().numpy(), x0_ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
    h.free()


def test_noalloc_rejects_oversize():
    """n beyond the fixed workspace is a clear error, not an allocation."""
    A = gen.convdiff2d(257, (1.0, 1.0))  # n = 66049 > 65536
    dA = rsai.DeviceMatrix.from_host(A)
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    lib = rsai.load()
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    csr = dA.csr()
    st = lib.rsai_bicgstab_noalloc(ctypes.byref(csr), None, b.data_ptr(), x.data_ptr(), 1e-8, 100,
                                   ctypes.byref(it), ctypes.byref(rr), None)
    assert st == 13
    assert "fixed-size workspace" in rsai.status_string(st)
