"""Pins for the oracle's dense adjoint gradient (central finite differences)."""
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
