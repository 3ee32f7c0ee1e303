"""Pins of the oracle's adjoint (frozen-pattern LS) and of its BiCGStab."""
import numpy as np
import pytest

import oracle
from paper_1503_04500_gb300 import inputs as gen


def _struct_rows(A):
    return np.repeat(np.arange(A.n), np.diff(A.row_ptr))


@pytest.fixture(scope="module")
def small():
    P = gen.parametric2d(8, (30.0, 10.0))
    A = P.base
    M = oracle.build(A, c=3, l_max=10, eps=0.3, drop="fixed", tol=1e-3)
    return P, A, M


def test_backward_frobenius_closed_form(small):
    """L = ||AM - I||_F^2 on a frozen pattern: dL/dA = 2 (AM - I) M^T on struct(A).

    The LS optimality of each column kills the terms through dm (envelope
    theorem), which leaves only the explicit dependence on A.
    """
    P, A, M = small
    g = oracle.backward(A, M.colptr, M.rows, np.zeros(M.nnz), np.ones(A.n))
    D = A.to_dense()
    Md = M.to_dense()
    full = 2.0 * (D @ Md - np.eye(A.n)) @ Md.T
    expect = full[_struct_rows(A), A.col_idx]
    np.testing.assert_allclose(g, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())


def test_backward_against_torch_normal_equations(small):
    """Generic loss <G, M> + <w, rho^2>: oracle adjoint vs torch autograd through
    the normal equations (B^T B) x = B^T e in FP64 (a different route than QR)."""
    torch = pytest.importorskip("torch")
    P, A, M = small
    rng = np.random.default_rng(3)
    gm = rng.standard_normal(M.nnz)
    gr = rng.standard_normal(A.n)
    g_oracle = oracle.backward(A, M.colptr, M.rows, gm, gr)

    rows = _struct_rows(A)
    vals = torch.tensor(A.val, dtype=torch.float64, requires_grad=True)
    D = torch.zeros((A.n, A.n), dtype=torch.float64)
    D = D.index_put((torch.tensor(rows), torch.tensor(A.col_idx.astype(np.int64))), vals)
    Dn = A.to_dense()
    loss = torch.zeros((), dtype=torch.float64)
    for k in range(A.n):
        J, _ = M.column(k)
        I = np.nonzero((Dn[:, J] != 0).any(axis=1))[0]
        B = D[I][:, J]
        e = torch.tensor((I == k).astype(np.float64))
        x = torch.linalg.solve(B.T @ B, B.T @ e)
        r = B @ x - e
        a, b = M.colptr[k], M.colptr[k + 1]
        loss = loss + torch.dot(torch.tensor(gm[a:b]), x) + gr[k] * torch.dot(r, r)
    loss.backward()
    np.testing.assert_allclose(g_oracle, vals.grad.numpy(), rtol=1e-8, atol=1e-10 * np.abs(g_oracle).max())


def test_backward_central_differences(small):
    """d/dtheta of sum(G * M) + sum(w * rho^2) along a random direction of A's values."""
    P, A, M = small
    rng = np.random.default_rng(5)
    gm = rng.standard_normal(M.nnz)
    gr = rng.standard_normal(A.n)
    dv = rng.standard_normal(A.nnz) * np.abs(A.val)
    g = oracle.backward(A, M.colptr, M.rows, gm, gr)

    def f(t):
        vals, rho2 = oracle.refit(A.with_values(A.val + t * dv), M.colptr, M.rows)
        return float(gm @ vals + gr @ rho2)

    h = 1e-6
    fd = (f(h) - f(-h)) / (2 * h)
    assert fd == pytest.approx(float(g @ dv), rel=1e-6)


def test_bicgstab_matches_scipy_unpreconditioned():
    """M = I: textbook BiCGStab; iteration count agrees with scipy's within one."""
    spla = pytest.importorskip("scipy.sparse.linalg")
    sp = pytest.importorskip("scipy.sparse")
    A = gen.convdiff2d(20, (20.0, 20.0))
    b = gen.ones_rhs(A)
    res = oracle.bicgstab(A, None, b, rtol=1e-8)
    S = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(A.n, A.n))
    count = [0]

    def cb(xk):
        count[0] += 1

    x, info = spla.bicgstab(S, b, rtol=1e-8, atol=0.0, maxiter=1000, callback=cb)
    assert info == 0 and res.converged
    assert abs(res.iters - count[0]) <= 1
    np.testing.assert_allclose(res.x, np.ones(A.n), rtol=1e-6)
    assert res.relres_true < 1e-7


def test_bicgstab_exact_preconditioner_one_iteration():
    """M = A^{-1} exactly (diagonal A): A M = I converges at the first half step."""
    d = np.linspace(1.0, 3.0, 50)
    A = gen.from_dense(np.diag(d))
    Minv = gen.from_dense(np.diag(1.0 / d))
    b = d.copy()
    res = oracle.bicgstab(A, (Minv.row_ptr, Minv.col_idx, Minv.val), b)
    assert res.iters == 1 and res.converged
    np.testing.assert_allclose(res.x, np.ones(50), rtol=1e-14)


def test_rsai_preconditioner_reduces_iterations():
    """Section 5 protocol on the 20x20 convection-diffusion problem."""
    A = gen.convdiff2d(20, (20.0, 20.0))
    M = oracle.build(A)
    b = gen.ones_rhs(A)
    r0 = oracle.bicgstab(A, None, b)
    r1 = oracle.bicgstab(A, M.csr(), b)
    assert r1.converged and r1.relres_true < 1e-8 * 10
    assert r1.iters < r0.iters
