"""Differentiating a BiCGStab solve preconditioned by M (Eq. 1.2) on the GPU:
the SpMV primitives and their adjoints against NumPy, the gradient of
loss = ||b - A M y_k||^2 against a CPU reference built from the oracle (its
pattern, its refit values and its LS adjoint) with dense torch autograd, and
the parametric 256^2 gradient against central differences."""
import numpy as np
import pytest

import oracle
from paper_1503_04500_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rsai = pytest.importorskip("paper_1503_04500_gb300.rsai")
from paper_1503_04500_gb300.autograd import Pattern, bicgstab_fixed, preconditioned_solve_loss  # noqa: E402

KW = dict(c=3, l_max=10, eps=0.3, tol=1e-3, drop="fixed")


def _dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def test_spmv_primitives_match_numpy():
    A = gen.powerlaw(3000, seed=5, dmax=40)
    rng = np.random.default_rng(1)
    x, gy = rng.standard_normal(A.n), rng.standard_normal(A.n)
    pat = Pattern.of_matrix(A)
    val = _dev(A.val)
    D = A.to_dense()
    y = rsai.spmv(pat.row_ptr, pat.col_idx, val, _dev(x)).cpu().numpy()
    np.testing.assert_allclose(y, D @ x, rtol=1e-13, atol=1e-13 * np.abs(D @ x).max())
    yt = rsai.spmv(pat.col_ptr, pat.row_idx, _dev(A.cval), _dev(gy)).cpu().numpy()
    np.testing.assert_allclose(yt, D.T @ gy, rtol=1e-13, atol=1e-13 * np.abs(D.T @ gy).max())
    gv = rsai.spmv_grad_values(pat.row_ptr, pat.col_idx, _dev(gy), _dev(x)).cpu().numpy()
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    np.testing.assert_array_equal(gv, gy[rows] * x[A.col_idx])  # one product per entry: exact
    # repeated products are identical (fixed reduction order)
    y2 = rsai.spmv(pat.row_ptr, pat.col_idx, val, _dev(x)).cpu().numpy()
    np.testing.assert_array_equal(y, y2)


def _oracle_pattern(ref):
    return ref.colptr.astype(np.int64), ref.rows.astype(np.int32)


def test_loss_gradient_matches_oracle_reference():
    P = gen.parametric2d(12, (30.0, 10.0))
    A = P.base
    iters = 5
    ref = oracle.build(A, **KW)
    colptr, Mrows = _oracle_pattern(ref)
    dA = rsai.DeviceMatrix.from_host(A)
    h = rsai.build(dA, precision="fp64", **KW)
    orp, oci, _ = ref.csr()
    rp, ci, _ = (t.cpu().numpy() for t in h.M())
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)  # same pattern as the oracle's
    b_np = gen.ones_rhs(A)

    A_val = dA.val.clone().requires_grad_(True)
    loss = preconditioned_solve_loss(A_val, h, Pattern.of_matrix(A), Pattern.of_M(h), _dev(b_np), iters)
    loss.backward()
    g_gpu = A_val.grad.cpu().numpy()

    # CPU reference: oracle values and adjoint of M(A), dense torch for the solve
    mv, _ = oracle.refit(A, colptr, Mrows)
    n = A.n
    rowsA = np.repeat(np.arange(n), np.diff(A.row_ptr))
    colsM = np.repeat(np.arange(n), np.diff(colptr))
    At = torch.tensor(A.val, requires_grad=True)
    Mt = torch.tensor(mv, requires_grad=True)
    Ad = torch.zeros(n, n, dtype=torch.float64).index_put((torch.as_tensor(rowsA), torch.as_tensor(A.col_idx.astype(np.int64))), At)
    Md = torch.zeros(n, n, dtype=torch.float64).index_put((torch.as_tensor(Mrows.astype(np.int64)), torch.as_tensor(colsM)), Mt)
    b = torch.as_tensor(b_np)
    y = bicgstab_fixed(lambda z: Ad @ (Md @ z), b, iters)
    r = b - Ad @ (Md @ y)
    L = torch.dot(r, r)
    L.backward()
    g_ref = At.grad.numpy() + oracle.backward(A, colptr, Mrows, Mt.grad.numpy(), np.zeros(n))

    np.testing.assert_allclose(loss.item(), L.item(), rtol=1e-9)
    np.testing.assert_allclose(g_gpu, g_ref, rtol=1e-7, atol=1e-9 * np.abs(g_ref).max())


def test_theta_gradient_at_full_size_central_differences():
    """Parametric 256^2 problem, y_20: dL/dtheta by autograd through the GPU
    kernels against central differences of the same (frozen-pattern) loss."""
    P = gen.parametric2d(256, (30.0, 10.0))
    A = P.base
    dA = rsai.DeviceMatrix.from_host(A)
    h = rsai.build(dA, precision="fp64", **KW)
    patA, patM = Pattern.of_matrix(A), Pattern.of_M(h)
    b = _dev(gen.ones_rhs(A))
    Lt, C1, C2 = _dev(P.L), _dev(P.C[0]), _dev(P.C[1])

    def loss(theta):
        return preconditioned_solve_loss(Lt + theta[0] * C1 + theta[1] * C2, h, patA, patM, b, 20)

    theta = torch.tensor(P.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    L0 = loss(theta)
    g = torch.autograd.grad(L0, theta)[0].cpu().numpy()
    assert np.isfinite(L0.item()) and L0.item() > 0
    with torch.no_grad():
        for i in range(2):
            step = 1e-4 * P.theta[i]
            e = torch.zeros(2, dtype=torch.float64, device="cuda")
            e[i] = step
            fd = (loss(theta + e) - loss(theta - e)).item() / (2 * step)
            assert abs(g[i] - fd) <= 1e-4 * abs(fd), (i, g[i], fd)
    h.free()
