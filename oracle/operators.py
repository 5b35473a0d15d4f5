"""Model-problem operators, assembled as explicit sparse matrices.

Test infrastructure only (see oracle/__init__.py).

The paper accesses A only through products x -> Ax (§1.2, §3).  Its own
model problems are a 2-D Laplacian (§8.1.3) and SuiteSparse matrices that are
not available here; the operators below are the synthetic stand-ins.

Grid convention: nx x ny interior cells, unknown (ix, iy) at linear index
i = iy*nx + ix (x fastest).  Neighbours E=(ix+1,iy), W=(ix-1,iy),
N=(ix,iy+1), S=(ix,iy-1); Dirichlet zero outside the grid.
"""
import numpy as np
import scipy.sparse as sp


def stencil5_matrix(nx, ny, coef, shift=None):
    """Constant-coefficient 5-point operator as an n x n CSR matrix.

    (Au)_P = cP u_P + cE u_E + cW u_W + cN u_N + cS u_S (+ shift_P u_P),
    coef = (cP, cE, cW, cN, cS).  Built entry by entry from that definition.
    """
    cP, cE, cW, cN, cS = [float(c) for c in coef]
    n = nx * ny
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ix = ix.reshape(-1)
    iy = iy.reshape(-1)
    P = iy * nx + ix
    rows = [P]
    cols = [P]
    vals = [np.full(n, cP) + (0.0 if shift is None else np.asarray(shift, dtype=np.float64))]
    for dx, dy, c in ((1, 0, cE), (-1, 0, cW), (0, 1, cN), (0, -1, cS)):
        jx, jy = ix + dx, iy + dy
        ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny)
        rows.append(P[ok])
        cols.append((jy * nx + jx)[ok])
        vals.append(np.full(ok.sum(), c))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def neumann_laplacian_matrix(nx, ny):
    """5-point Laplacian of an nx x ny grid with zero-flux (Neumann)
    boundaries, h^2-scaled: the graph Laplacian of the grid, built as the
    Kronecker sum of two path-graph Laplacians.  Positive semidefinite,
    kernel = constant vectors, eigenvalues in [0, 8) (the E2 model problem,
    §8: "Laplacian in 2-D" with spectrum in [0, 8]).
    """
    def path(m):
        L = sp.diags([-np.ones(m - 1), 2.0 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1], format="lil")
        L[0, 0] = 1.0
        L[m - 1, m - 1] = 1.0
        return L.tocsr()
    return (sp.kron(sp.identity(ny), path(nx)) + sp.kron(path(ny), sp.identity(nx))).tocsr()


def diffusion_var_matrix(nx, ny, theta):
    """Variable-coefficient diffusion -div(theta grad u), h^2-scaled, as CSR.

    (Au)_P = sum over the four faces f of P of theta_f (u_P - u_Q), with
    theta_f = (theta_P + theta_Q)/2 on interior faces and theta_f = theta_P on
    boundary faces (u_Q = 0 there).  Symmetric positive definite.
    """
    theta = np.asarray(theta, dtype=np.float64).reshape(-1)
    n = nx * ny
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ix = ix.reshape(-1)
    iy = iy.reshape(-1)
    P = iy * nx + ix
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        jx, jy = ix + dx, iy + dy
        ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny)
        Q = np.where(ok, jy * nx + jx, 0)
        tf = np.where(ok, 0.5 * (theta[P] + theta[Q]), theta[P])
        diag += tf
        rows.append(P[ok])
        cols.append(Q[ok])
        vals.append(-tf[ok])
    rows.append(P)
    cols.append(P)
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def diffusion_var_theta_grad(nx, ny, lam, x):
    """d/dtheta of lam^T A(theta) x for the operator above, per cell.

    lam^T A x = sum_interior faces theta_f (lam_P - lam_Q)(x_P - x_Q)
                + sum_boundary faces theta_P lam_P x_P,
    and theta_f = (theta_P + theta_Q)/2, so an interior face passes half of
    (lam_P - lam_Q)(x_P - x_Q) to each of its two cells.
    """
    lam = np.asarray(lam, dtype=np.float64).reshape(ny, nx)
    x = np.asarray(x, dtype=np.float64).reshape(ny, nx)
    g = np.zeros((ny, nx))
    # x-faces between (ix, iy) and (ix+1, iy)
    fx = 0.5 * (lam[:, :-1] - lam[:, 1:]) * (x[:, :-1] - x[:, 1:])
    g[:, :-1] += fx
    g[:, 1:] += fx
    fy = 0.5 * (lam[:-1, :] - lam[1:, :]) * (x[:-1, :] - x[1:, :])
    g[:-1, :] += fy
    g[1:, :] += fy
    # boundary faces: one per side of a boundary cell
    nb = np.zeros((ny, nx))
    nb[:, 0] += 1
    nb[:, -1] += 1
    nb[0, :] += 1
    nb[-1, :] += 1
    g += nb * lam * x
    return g.reshape(-1)


def csr_from_scipy(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)
