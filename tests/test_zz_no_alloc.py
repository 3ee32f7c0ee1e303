"""rsai_bicgstab_noalloc, the solve for callers that cannot allocate device memory.

Such callers (code inside another framework's memory pool or plugin interface,
real-time loops that may not allocate or synchronise) get rsai_bicgstab's
solver with its work vectors in a fixed array inside the library.  These tests
call it through the C ABI, check that it takes no device memory, and compare
it with rsai_bicgstab.  This file is collected last so that a run stopping at
its first failure has already run every other test; it passes alone in a fresh
process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_1503_04500_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rsai = pytest.importorskip("paper_1503_04500_gb300.rsai")


class CountingAllocator:
    """rsai_set_allocator callbacks that count calls (backed by torch's caching allocator)."""

    def __init__(self):
        self.allocs = 0
        self.frees = 0

        def _alloc(nbytes, stream, ctx):
            self.allocs += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))

        def _free(ptr, nbytes, stream, ctx):
            self.frees += 1
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cbs = (rsai.ALLOC_FN(_alloc), rsai.FREE_FN(_free))

    def __enter__(self):
        rsai._allocators.append(self.cbs)
        assert rsai.load().rsai_set_allocator(self.cbs[0], self.cbs[1], None) == 0
        return self

    def __exit__(self, *exc):
        rsai.use_cuda_allocator()


def _solve_twice_unallocated(dA, M, b, x_ref, it_ref, rel_ref):
    """Two calls in a row; the second one under watch: no allocator call, no
    change of torch's allocated bytes nor of the device's free memory."""
    with CountingAllocator() as ca:
        for call in range(2):
            x = torch.full_like(b, float("nan"))
            torch.cuda.synchronize()
            used0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
            it, rel, st = rsai.bicgstab_noalloc(dA, M, b, x, rtol=1e-8)
            torch.cuda.synchronize()
            used1, free1 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
            assert st == 0, call
            assert it == it_ref, call
            np.testing.assert_allclose(x.cpu().numpy(), x_ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
            assert rel == pytest.approx(rel_ref, rel=1e-6, abs=1e-15)
            if call == 1:
                assert used1 == used0 and free1 == free0, (used0, used1, free0, free1)
        assert ca.allocs == 0 and ca.frees == 0


def test_noalloc_matches_allocating_solve_twice():
    """Two calls in a row through the C ABI agree with rsai_bicgstab (and each other)."""
    A = gen.convdiff2d(40, (20.0, 20.0))  # n = 1600
    dA = rsai.DeviceMatrix.from_host(A)
    h = rsai.build(dA, c=3, l_max=10, eps=0.3, tol=1e-3, drop="fixed", precision="fp64")
    M = h.M()
    b = torch.as_tensor(gen.ones_rhs(A), device="cuda")
    x_ref, it_ref, rel_ref, st_ref = rsai.bicgstab(dA, h, b, rtol=1e-8)
    assert st_ref == 0
    _solve_twice_unallocated(dA, M, b, x_ref, it_ref, rel_ref)
    # without a preconditioner, also twice
    x0_ref, it0_ref, rel0_ref, st0_ref = rsai.bicgstab(dA, None, b, rtol=1e-8)
    assert st0_ref == 0
    _solve_twice_unallocated(dA, None, b, x0_ref, it0_ref, rel0_ref)
    h.free()


def test_noalloc_at_the_size_limit():
    """n = 65536, the largest size the fixed array holds: every word of the array in use."""
    A = gen.convdiff2d(256, (20.0, 20.0))
    assert A.n == 65536
    dA = rsai.DeviceMatrix.from_host(A)
    h = rsai.build(dA, c=3, l_max=10, eps=0.3, tol=1e-3, drop="fixed", precision="fp64")
    M = h.M()
    b = torch.as_tensor(gen.ones_rhs(A), device="cuda")
    x_ref, it_ref, rel_ref, st_ref = rsai.bicgstab(dA, h, b, rtol=1e-8)
    assert st_ref == 0
    _solve_twice_unallocated(dA, M, b, x_ref, it_ref, rel_ref)
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
