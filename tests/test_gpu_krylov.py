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


def _pattern_of(h, n):
    """The handle's frozen pattern of M, column-wise (colptr, rows)."""
    rp, ci, _ = (t.cpu().numpy() for t in h.M())
    rows = np.repeat(np.arange(n), np.diff(rp))
    order = np.lexsort((rows, ci))
    colptr = np.zeros(n + 1, np.int64)
    np.add.at(colptr, ci.astype(np.int64) + 1, 1)
    return np.cumsum(colptr), rows[order].astype(np.int32)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-7), ("fp32_refine", 1e-5)])
def test_loss_gradient_matches_oracle_reference(precision, rtol):
    """d||b - A M y_5||^2 / dA on the 12^2 parametric problem against a CPU
    reference: the oracle's FP64 values and LS adjoint of M(A) on the handle's
    frozen pattern (the oracle's own pattern for the FP64 build), with dense
    torch autograd through the five BiCGStab iterations."""
    P = gen.parametric2d(12, (30.0, 10.0))
    A = P.base
    iters = 5
    dA = rsai.DeviceMatrix.from_host(A)
    h = rsai.build(dA, precision=precision, **KW)
    colptr, Mrows = _pattern_of(h, A.n)
    if precision == "fp64":
        ref = oracle.build(A, **KW)
        np.testing.assert_array_equal(colptr, ref.colptr)
        np.testing.assert_array_equal(Mrows, ref.rows)
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

    np.testing.assert_allclose(loss.item(), L.item(), rtol=10 * rtol)
    np.testing.assert_allclose(g_gpu, g_ref, rtol=rtol, atol=1e-2 * rtol * np.abs(g_ref).max())
    h.free()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-6), ("fp32_refine", 1e-4)])
def test_theta_gradient_at_full_size_central_differences(precision, rtol):
    """Parametric 256^2 problem (n = 65536), loss_2 = ||b - A M y_20||^2 with
    y_20 from 20 BiCGStab iterations: dL/dtheta by autograd through the GPU
    kernels (FP64 or FP32+refine) against central differences, with step
    h = 1e-6 * theta_1, of the FP64 loss that the oracle evaluates on the same
    frozen pattern (its refit of M(theta), then its BiCGStab with the stopping
    test disabled for exactly 20 iterations).

    The oracle's loss carries rounding noise (about 5e-10 of L, from the 20
    Krylov iterations), which a step this small turns into an error of about
    1e-3 of the smaller derivative.  So the derivative is the least-squares
    slope of L at theta + j h e_i, j = -3..3, and the check allows
    rtol * |slope| plus four standard errors of that slope, taken from the
    residuals of the fit."""
    P = gen.parametric2d(256, (30.0, 10.0))
    A = P.base
    dA = rsai.DeviceMatrix.from_host(A)
    h = rsai.build(dA, precision=precision, **KW)
    patA, patM = Pattern.of_matrix(A), Pattern.of_M(h)
    colptr, Mrows = _pattern_of(h, A.n)
    b_np = gen.ones_rhs(A)
    b = _dev(b_np)
    Lt, C1, C2 = _dev(P.L), _dev(P.C[0]), _dev(P.C[1])

    theta = torch.tensor(P.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    L0 = preconditioned_solve_loss(Lt + theta[0] * C1 + theta[1] * C2, h, patA, patM, b, 20)
    g = torch.autograd.grad(L0, theta)[0].cpu().numpy()
    assert np.isfinite(L0.item()) and L0.item() > 0

    nb = float(np.linalg.norm(b_np))
    colk = np.repeat(np.arange(A.n), np.diff(colptr))
    order = np.lexsort((colk, Mrows))
    Mrp = np.zeros(A.n + 1, np.int64)
    np.add.at(Mrp, Mrows.astype(np.int64) + 1, 1)
    Mrp = np.cumsum(Mrp)

    def loss_oracle(th):
        At = A.with_values(P.values(th))
        mv, _ = oracle.refit(At, colptr, Mrows)
        sol = oracle.bicgstab(At, (Mrp, colk[order].astype(np.int32), mv[order]), b_np, rtol=0.0, maxit=20)
        assert sol.iters == 20
        return (sol.relres_true * nb) ** 2

    np.testing.assert_allclose(L0.item(), loss_oracle(list(P.theta)), rtol=1e-8 if precision == "fp64" else 1e-5)
    step = 1e-6 * P.theta[0]
    js = np.arange(-3, 4, dtype=np.float64)
    for i in range(2):
        Ls = []
        for j in js:
            th = list(P.theta)
            th[i] += j * step
            Ls.append(loss_oracle(th))
        Ls = np.array(Ls)
        slope = float(js @ Ls) / (step * float(js @ js))
        resid = Ls - Ls.mean() - slope * step * js
        stderr = float(np.sqrt((resid @ resid) / (len(js) - 2))) / (step * float(np.sqrt(js @ js)))
        assert abs(g[i] - slope) <= rtol * abs(slope) + 4.0 * stderr, (precision, i, g[i], slope, stderr)
    h.free()
