"""Dense adjoint gradient of the differentiable solve.

Test infrastructure only (see oracle/__init__.py).

Loss L(theta, b) = ||x - x_t||^2 with A(theta) x = b and A(theta) the
variable-coefficient diffusion operator of oracle.operators.  The paper has
no differentiable solve; this is the plain definition the adjoint sGMRES
path is checked against:
  lam = A^{-T} dL/dx = A^{-T} 2(x - x_t),
  dL/db = lam,
  dL/dtheta = -d(lam^T A(theta) x)/dtheta.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import operators


def loss_and_grad(nx, ny, theta, b, x_t):
    A = operators.diffusion_var_matrix(nx, ny, theta).tocsc()
    lu = spla.splu(A)
    x = lu.solve(np.asarray(b, dtype=np.float64))
    gx = 2.0 * (x - x_t)
    lam = lu.solve(gx, trans="T")
    gtheta = -operators.diffusion_var_theta_grad(nx, ny, lam, x)
    return float(np.sum((x - x_t) ** 2)), gtheta, lam, x
