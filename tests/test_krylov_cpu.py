"""The fixed-iteration BiCGStab used to differentiate a preconditioned solve,
pinned on the CPU: its k-th iterate is SciPy's k-th BiCGStab iterate (same
textbook recurrences, no stopping), and enough iterations solve the system."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
scipy_linalg = pytest.importorskip("scipy.sparse.linalg")

from paper_1503_04500_gb300 import inputs as gen  # noqa: E402
from paper_1503_04500_gb300.autograd import bicgstab_fixed  # noqa: E402


def _system(N=8):
    A = gen.convdiff2d(N, (5.0, 3.0)).to_dense()
    b = A @ np.ones(A.shape[0])
    return A, b


@pytest.mark.parametrize("k", [1, 2, 5])
def test_iterate_equals_scipy(k):
    A, b = _system()
    x_sp, _ = scipy_linalg.bicgstab(A, b, rtol=0.0, atol=0.0, maxiter=k)
    At = torch.as_tensor(A)
    y = bicgstab_fixed(lambda z: At @ z, torch.as_tensor(b), k).numpy()
    np.testing.assert_allclose(y, x_sp, rtol=1e-10, atol=1e-12 * np.abs(x_sp).max())


def test_enough_iterations_solve_the_system():
    A, b = _system()
    At = torch.as_tensor(A)
    y = bicgstab_fixed(lambda z: At @ z, torch.as_tensor(b), 40).numpy()
    np.testing.assert_allclose(y, np.linalg.solve(A, b), rtol=1e-8)


def test_iterate_is_differentiable_in_the_operator():
    """d/dt of ||b - A(t) y_k(t)||^2 by autograd equals a central difference."""
    A, b = _system(6)
    rng = np.random.default_rng(3)
    E = rng.standard_normal(A.shape) * (A != 0)

    def loss(t):
        At = torch.as_tensor(A) + t * torch.as_tensor(E)
        y = bicgstab_fixed(lambda z: At @ z, torch.as_tensor(b), 4)
        r = torch.as_tensor(b) - At @ y
        return torch.dot(r, r)

    t = torch.zeros((), dtype=torch.float64, requires_grad=True)
    g = torch.autograd.grad(loss(t), t)[0].item()
    h = 1e-6
    fd = (loss(torch.tensor(h, dtype=torch.float64)) - loss(torch.tensor(-h, dtype=torch.float64))).item() / (2 * h)
    assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd))
