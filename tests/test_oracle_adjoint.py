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
