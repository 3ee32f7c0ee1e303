"""Failure paths reported as status codes (no device trap, no fault): device
memory that runs out part way through rsai_build, and a BiCGStab breakdown.

The allocation failure is made on the host: an allocator callback that
returns NULL on its N-th call, for every N a build makes.  The breakdown is a
2 x 2 system on which textbook BiCGStab (Section 5's solver) divides by
rhat^T v = 0 in its first step."""
import numpy as np
import pytest

import oracle
from paper_1503_04500_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rsai = pytest.importorskip("paper_1503_04500_gb300.rsai")

KW = dict(c=3, l_max=10, eps=0.3, tol=1e-3, drop="fixed")
RSAI_ERR_OOM = 6
RSAI_ERR_BREAKDOWN = 10


class FailingAllocator:
    """Allocator callbacks (torch's caching allocator underneath) that fail the
    `fail_at`-th allocation (1-based; 0 = never) and track what is outstanding."""

    def __init__(self, fail_at=0):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
            self.live[int(p)] = int(nbytes)
            return p

        def _free(ptr, nbytes, stream, ctx):
            assert int(ptr) in self.live, "freed a pointer the allocator did not hand out"
            del self.live[int(ptr)]
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cbs = (rsai.ALLOC_FN(_alloc), rsai.FREE_FN(_free))

    def __enter__(self):
        rsai._allocators.append(self.cbs)
        assert rsai.load().rsai_set_allocator(self.cbs[0], self.cbs[1], None) == 0
        return self

    def __exit__(self, *exc):
        rsai.use_cuda_allocator()


# nnz(M)/n = 174 here: the result pool outgrows its first estimate (and is regrown), and most
# columns reach the global bin (its slab is allocated after the CTA bin), so every allocation
# site of a build is met
STRESS = dict(c=5, l_max=6, eps=0.05, drop="none")


def test_every_failed_allocation_of_a_build_is_oom_and_leaks_nothing():
    A = gen.powerlaw(600, seed=5, dmax=40)
    KW = STRESS
    dA = rsai.DeviceMatrix.from_host(A)
    with FailingAllocator() as ok:
        h = rsai.build(dA, precision="fp64", **KW)
        want = [t.cpu().numpy() for t in h.M()]
        h.free()
    torch.cuda.synchronize()
    assert ok.live == {}
    total = ok.calls
    assert total >= 20
    for n_fail in range(1, total + 1):
        with FailingAllocator(n_fail) as fa:
            with pytest.raises(rsai.RSAIError) as e:
                rsai.build(dA, precision="fp64", **KW)
            assert e.value.status == RSAI_ERR_OOM, n_fail
            torch.cuda.synchronize()
            assert fa.live == {}, (n_fail, len(fa.live))
    # later builds (library pool and torch-backed) are unaffected and give the same M
    h = rsai.build(dA, precision="fp64", **KW)
    for a, b in zip(h.M(), want):
        np.testing.assert_array_equal(a.cpu().numpy(), b)
    h.free()
    with FailingAllocator() as fa:
        h = rsai.build(dA, precision="fp64", **KW)
        for a, b in zip(h.M(), want):
            np.testing.assert_array_equal(a.cpu().numpy(), b)
        h.free()
        torch.cuda.synchronize()
        assert fa.live == {}


def test_build_reports_oom_through_the_out_pointer_as_null():
    """The C ABI leaves *out NULL when the build fails."""
    import ctypes

    A = gen.convdiff2d(12, (20.0, 20.0))
    dA = rsai.DeviceMatrix.from_host(A)
    lib = rsai.load()
    params = rsai.default_params(**KW)
    out = ctypes.c_void_p(12345)
    with FailingAllocator(3):
        st = lib.rsai_build(ctypes.byref(dA.csr()), ctypes.byref(dA.csc()), ctypes.byref(params), None,
                            ctypes.byref(out))
    torch.cuda.synchronize()
    assert st == RSAI_ERR_OOM and not out.value


def test_bicgstab_breakdown_is_a_status():
    """A = [[0, 1], [-1, 0]], b = e_1, no preconditioner: r0 = rhat = e_1 and
    v = A e_1 = -e_2, so rhat^T v = 0 and alpha is undefined at the first step.
    The GPU solve returns RSAI_ERR_BREAKDOWN after one iteration, as the oracle
    reports a breakdown."""
    D = np.array([[0.0, 1.0], [-1.0, 0.0]])
    A = gen.from_dense(D)
    b_np = np.array([1.0, 0.0])
    ro = oracle.bicgstab(A, None, b_np, rtol=1e-8)
    assert ro.status == "breakdown_alpha" and ro.iters == 1
    dA = rsai.DeviceMatrix.from_host(A)
    x, it, rel, status = rsai.bicgstab(dA, None, torch.as_tensor(b_np, device="cuda"), rtol=1e-8)
    assert status == RSAI_ERR_BREAKDOWN and it == 1
    assert np.isfinite(x.cpu().numpy()).all()
    # the context is still usable
    y = torch.ones(2, dtype=torch.float64, device="cuda") * 2
    assert float(y.sum().item()) == 4.0
