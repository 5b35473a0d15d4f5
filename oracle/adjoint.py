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


def stencil_loss_and_grad(nx, ny, coef, shift, b, x_t):
    """The same loss for the five-point operator of oracle.operators with
    coefficients coef = (c_P, c_E, c_W, c_N, c_S) and diagonal shift:
      lam = A^{-T} 2(x - x_t),  dL/db = lam,
      dL/dc_q = -lam^T A_q x  (A_q: the q-th neighbour pattern, unit weight),
      dL/dshift_P = -lam_P x_P.
    Returns (L, dL/dc (5,), dL/dshift (n,), lam, x)."""
    A = operators.stencil5_matrix(nx, ny, coef, shift).tocsc()
    lu = spla.splu(A)
    x = lu.solve(np.asarray(b, dtype=np.float64))
    lam = lu.solve(2.0 * (x - x_t), trans="T")
    gc = np.zeros(5)
    for q in range(5):
        e = np.zeros(5)
        e[q] = 1.0
        gc[q] = -lam @ (operators.stencil5_matrix(nx, ny, e) @ x)
    return float(np.sum((x - x_t) ** 2)), gc, -lam * x, lam, x


def csr_loss_and_grad(A, b, x_t):
    """The same loss for a general sparse A (scipy CSR, the given pattern):
      lam = A^{-T} 2(x - x_t),  dL/db = lam,  dL/dval_e = -lam_row(e) x_col(e).
    Returns (L, dL/dval (nnz, CSR order), lam, x)."""
    A = A.tocsr()
    lu = spla.splu(A.tocsc())
    x = lu.solve(np.asarray(b, dtype=np.float64))
    lam = lu.solve(2.0 * (x - x_t), trans="T")
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    return float(np.sum((x - x_t) ** 2)), -lam[rows] * x[A.indices], lam, x
