"""Pins for the oracle's dense adjoint gradient: central finite differences
and exact forward-mode (tangent) derivatives."""
import numpy as np

import synth
from oracle import adjoint, operators


def _loss(nx, ny, theta, b, xt):
    A = operators.diffusion_var_matrix(nx, ny, theta).toarray()
    x = np.linalg.solve(A, b)
    return np.sum((x - xt) ** 2)


def test_adjoint_gradient_matches_central_differences():
    nx = ny = 6
    n = nx * ny
    theta = np.exp(0.5 * synth.grf(2, 6, 2.0))
    b = synth.randn(3, n)
    xt = synth.randn(4, n) * 0.1
    L, gth, lam, x = adjoint.loss_and_grad(nx, ny, theta, b, xt)
    assert abs(L - _loss(nx, ny, theta, b, xt)) < 1e-12 * L
    for p in range(0, n, 5):
        e = np.zeros(n)
        e[p] = 1e-5 * theta[p]
        fd = (_loss(nx, ny, theta + e, b, xt) - _loss(nx, ny, theta - e, b, xt)) / (2 * e[p])
        assert abs(fd - gth[p]) <= 1e-6 * max(1.0, abs(gth[p]))
    for p in range(0, n, 7):
        e = np.zeros(n)
        e[p] = 1e-5
        fd = (_loss(nx, ny, theta, b + e, xt) - _loss(nx, ny, theta, b - e, xt)) / 2e-5
        assert abs(fd - lam[p]) <= 1e-6 * max(1.0, abs(lam[p]))


def test_adjoint_gradient_equals_forward_mode_derivatives():
    # A(theta) is linear in theta (face values are averages of theta), so
    # A(theta + t delta) = A(theta) + t A(delta) exactly, and the tangent
    # (forward-mode) derivative along delta is exact: A dx = -A(delta) x,
    # dL = 2 (x - x_t)^T dx.  Along db: A dx = db.  One forward solve per
    # direction against the adjoint's single transposed solve: they must
    # agree to rounding (central differences above only reach ~1e-6).
    nx, ny = 9, 7
    n = nx * ny
    theta = np.exp(0.5 * synth.randn(5, n))
    b = synth.randn(6, n)
    xt = synth.randn(7, n) * 0.1
    L, gth, lam, x = adjoint.loss_and_grad(nx, ny, theta, b, xt)
    A = operators.diffusion_var_matrix(nx, ny, theta).toarray()
    # linearity of the operator in theta, checked on two random coefficient fields
    t1, t2 = synth.randn(8, n), synth.randn(9, n)
    assert np.allclose(operators.diffusion_var_matrix(nx, ny, t1 + 2.5 * t2).toarray(),
                       operators.diffusion_var_matrix(nx, ny, t1).toarray()
                       + 2.5 * operators.diffusion_var_matrix(nx, ny, t2).toarray(), atol=1e-13)
    for q in range(3):
        delta = synth.randn(20 + q, n)
        dx = np.linalg.solve(A, -(operators.diffusion_var_matrix(nx, ny, delta).toarray() @ x))
        dL = 2.0 * (x - xt) @ dx
        assert abs(dL - gth @ delta) <= 1e-10 * max(1.0, abs(dL))
        db = synth.randn(30 + q, n)
        dLb = 2.0 * (x - xt) @ np.linalg.solve(A, db)
        assert abs(dLb - lam @ db) <= 1e-10 * max(1.0, abs(dLb))


def test_stencil_adjoint_gradient_matches_central_differences():
    # coefficients and shift of the five-point operator: central differences
    # of the dense loss (a dropped sign or a transposed neighbour fails)
    nx, ny = 7, 5
    n = nx * ny
    coef = np.array([4.0, -0.7, -1.3, -0.9, -1.1])
    shift = synth.uniform(3, n)
    b = synth.randn(4, n)
    xt = synth.randn(5, n) * 0.1

    def loss(c, sh, bv):
        A = operators.stencil5_matrix(nx, ny, c, sh).toarray()
        x = np.linalg.solve(A, bv)
        return np.sum((x - xt) ** 2)

    L, gc, gs, lam, x = adjoint.stencil_loss_and_grad(nx, ny, coef, shift, b, xt)
    assert abs(L - loss(coef, shift, b)) <= 1e-12 * L
    for q in range(5):
        e = np.zeros(5)
        e[q] = 1e-6
        fd = (loss(coef + e, shift, b) - loss(coef - e, shift, b)) / 2e-6
        assert abs(fd - gc[q]) <= 1e-6 * max(1.0, abs(gc[q])), (q, fd, gc[q])
    for p in range(0, n, 4):
        e = np.zeros(n)
        e[p] = 1e-6
        fd = (loss(coef, shift + e, b) - loss(coef, shift - e, b)) / 2e-6
        assert abs(fd - gs[p]) <= 1e-6 * max(1.0, abs(gs[p]))
        fd = (loss(coef, shift, b + e) - loss(coef, shift, b - e)) / 2e-6
        assert abs(fd - lam[p]) <= 1e-6 * max(1.0, abs(lam[p]))


def test_csr_adjoint_gradient_matches_central_differences():
    # gradient with respect to the stored values of a general sparse matrix
    import scipy.sparse as sp
    n = 30
    A = (sp.random(n, n, density=0.15, random_state=5, format="csr") + 4.0 * sp.eye(n)).tocsr()
    b = synth.randn(12, n)
    xt = synth.randn(13, n) * 0.1

    def loss(vals):
        M = sp.csr_matrix((vals, A.indices, A.indptr), shape=A.shape).toarray()
        x = np.linalg.solve(M, b)
        return np.sum((x - xt) ** 2)

    L, gv, lam, x = adjoint.csr_loss_and_grad(A, b, xt)
    assert abs(L - loss(A.data)) <= 1e-12 * L
    for e in range(0, A.nnz, 7):
        d = np.zeros(A.nnz)
        d[e] = 1e-6
        fd = (loss(A.data + d) - loss(A.data - d)) / 2e-6
        assert abs(fd - gv[e]) <= 1e-6 * max(1.0, abs(gv[e])), (e, fd, gv[e])
