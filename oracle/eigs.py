"""Sketched Rayleigh-Ritz (Algorithm 2), its stabilized form (§6.5), restarted
sRR on block Chebyshev bases (§7.2, §7.5) and Rayleigh-Ritz (§6.1).

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np
import scipy.linalg

from . import krylov


def select_order(lam, nev):
    """Indices of the nev eigenvalues with largest real part.

    Ties in the real part are broken by larger imaginary part, then by
    position (so a conjugate pair lists the member with Im > 0 first).
    """
    idx = sorted(range(len(lam)), key=lambda i: (-lam[i].real, -lam[i].imag, i))
    return idx[:nev]


def srr_from_basis(B, M, sketch, nev, tau=1e-8, symmetric=False):
    """Algorithm 2's reduction on a given basis B (n x d) and M = A B.

    C = S B, D = S A B (§6.4); C = U T (Householder); M-hat = T^{-1}(U^T D)
    (eq. (Mhat-form)); eig(M-hat) (numpy's LAPACK dgeev as one step);
    residual estimates ||D y_i - lam_i C y_i|| / ||C y_i|| (eq.
    (srr-resid-est)); the nev eigenvalues of largest real part;
    x_i = B y_i / ||B y_i||.  For real symmetric A (§6.8) the real parts of
    lam and x are kept.
    """
    d = B.shape[1]
    C = sketch(B)
    D = sketch(M)
    V, T = krylov.householder_qr(C)
    kappa = krylov.cond2(T)
    UtD = np.stack([krylov.apply_qt(V, D[:, j])[:d] for j in range(d)], axis=1)
    Mhat = np.zeros((d, d))
    for j in range(d):
        Mhat[:, j] = krylov.back_substitute(T, UtD[:, j])
    lam, Y = np.linalg.eig(Mhat)
    if symmetric:
        lam = lam.real.astype(np.complex128)
        Y = Y.real.astype(np.complex128)
    rhat = np.array([np.linalg.norm(D @ Y[:, i] - lam[i] * (C @ Y[:, i])) / np.linalg.norm(C @ Y[:, i])
                     for i in range(d)])
    order = select_order(lam, nev)
    X = B @ Y[:, order]
    X /= np.linalg.norm(X, axis=0)
    return dict(lam=lam[order], X=X, rhat=rhat[order], nconv=int(np.sum(rhat[order] <= tau)),
                kappa=kappa, Mhat=Mhat, C=C, D=D, all_lam=lam)


def srr(A, w1, d, k, sketch, nev, tau=1e-8, symmetric=False, passes=2, breakdown=1e-13):
    """Algorithm 2 with the basis of §1.2.2 eq. (partorth): b_1 = w_1/||w_1||,
    the truncated Arnoldi basis B and AB, then srr_from_basis."""
    B, M, _, d_used = krylov.trunc_arnoldi(A, w1, d, k, passes=passes, breakdown=breakdown)
    out = srr_from_basis(B, M, sketch, nev, tau, symmetric)
    out.update(B=B, M=M, d_used=d_used)
    return out


def srr_stabilized_from_basis(B, M, sketch, nev, trunc_tol=1e14, tau=1e-8, symmetric=False):
    """Stabilized sRR (§6.5, eq. (qz)) on a given basis B and M = A B.

    C = S B, D = S A B; thin SVD C = U Sigma V^T (LAPACK gesdd as one
    step), truncated to the r singular values with sigma_1 / sigma_i <=
    trunc_tol (the kept part has condition number at most trunc_tol); the
    generalized eigenproblem (U_r^T D V_r) z = theta Sigma_r z by QZ (LAPACK
    ggev through scipy.linalg.eig with two matrices, as one step); Ritz
    vectors y = V_r z in the coordinates of B; residual estimates
    ||D y - theta C y|| / ||C y|| (eq. (srr-resid-est)); the nev values of
    largest real part; x = B y / ||B y||.  For real symmetric A (§6.8) the
    real parts are kept.
    """
    C = sketch(B)
    D = sketch(M)
    U, sg, Vt = np.linalg.svd(C, full_matrices=False)
    r = int(np.sum(sg >= sg[0] / trunc_tol)) if sg[0] > 0 else 0
    if r == 0:
        raise ValueError("the sketched basis is zero")
    G = U[:, :r].T @ D @ Vt[:r].T
    theta, Z = scipy.linalg.eig(G, np.diag(sg[:r]))
    Y = Vt[:r].T @ Z
    if symmetric:
        theta = theta.real.astype(np.complex128)
        Y = Y.real.astype(np.complex128)
    rhat = np.array([np.linalg.norm(D @ Y[:, i] - theta[i] * (C @ Y[:, i])) / np.linalg.norm(C @ Y[:, i])
                     for i in range(r)])
    order = select_order(theta, nev)
    X = B @ Y[:, order]
    X /= np.linalg.norm(X, axis=0)
    return dict(lam=theta[order], X=X, rhat=rhat[order], nconv=int(np.sum(rhat[order] <= tau)), rank=r,
                sigma=sg, all_lam=theta)


def srr_stabilized(A, w1, d, k, sketch, nev, trunc_tol=1e14, tau=1e-8, symmetric=False, passes=2,
                   breakdown=1e-13):
    """Stabilized sRR on the truncated Arnoldi basis of Algorithm 2."""
    B, M, _, _ = krylov.trunc_arnoldi(A, w1, d, k, passes=passes, breakdown=breakdown)
    return srr_stabilized_from_basis(B, M, sketch, nev, trunc_tol, tau, symmetric)


def chebyshev_filter(A, Q, m, c, dx):
    """T_m((A - c I)/dx) Q by the three-term recurrence Y_0 = Q,
    Y_1 = (A - c I) Q / dx, Y_{j+1} = 2 (A - c I) Y_j / dx - Y_{j-1}
    (§4.3 with dy = 0, unscaled Chebyshev polynomials), both carried columns
    divided by the norms of the newest one after every 10th step (a column
    scaling, which leaves the span of each column's sequence unchanged)."""
    Y0 = np.array(Q, dtype=np.float64, copy=True)
    Y1 = (A @ Y0 - c * Y0) / dx
    for j in range(2, m + 1):
        Y0, Y1 = Y1, 2.0 * (A @ Y1 - c * Y1) / dx - Y0
        if j % 10 == 0:
            sc = np.linalg.norm(Y1, axis=0)
            Y0 = Y0 / sc
            Y1 = Y1 / sc
    return Y1


def srr_restarted(A, Omega, p, nev, lo, hi, restarts, sketch_for, tau=1e-8, trunc_tol=1e13, stabilized=True,
                  filter_degree=0):
    """Restarted sRR (§7.2) on block Chebyshev bases (§7.5).

    X_0 = Omega (n x b).  Restart t: Q = orth(X_t) (Householder QR of the
    start block); with filter_degree = m > 0, Q = orth(T_m((A - c)/dx) Q)
    (chebyshev_filter: a degree-m Chebyshev filter for the same interval,
    still a block of K_{m+1}(A; X_t)); B = [B_1..B_p] from
    block_chebyshev_basis(A, Q, p, c, dx)
    for the interval [lo, cut_t] that holds the unwanted part of the real
    spectrum (c, dx its centre and half-width; cut_0 = hi, then the real part
    of the b-th Ritz value of restart t-1), each column scaled to unit norm;
    sRR on (B, A B) with the sketch sketch_for(t) -- the stabilized form of
    §6.5 (default; the basis condition number passes 1/u within a few
    restarts) or Algorithm 2's reduction; X_{t+1} = the real and imaginary
    parts of the b leading Ritz vectors (the first b nonzero columns).
    Stops when the residual estimates of the nev leading pairs are all
    <= tau, or after `restarts` restarts.
    Returns the last sRR result (b leading pairs) plus ``restarts`` (the
    number run) and ``history`` (max estimate over the nev pairs, per restart).
    """
    b = Omega.shape[1]
    X = np.array(Omega, dtype=np.float64, copy=True)
    cut = hi
    history = []
    out = None
    for t in range(restarts):
        Q, _ = np.linalg.qr(X)
        c, dx = 0.5 * (lo + cut), 0.5 * (cut - lo)
        if filter_degree > 0:
            Q, _ = np.linalg.qr(chebyshev_filter(A, Q, filter_degree, c, dx))
        B = krylov.block_chebyshev_basis(A, Q, p, c, dx, 0.0)
        B = B / np.linalg.norm(B, axis=0)
        M = A @ B
        if stabilized:
            out = srr_stabilized_from_basis(B, M, sketch_for(t), b, trunc_tol=trunc_tol, tau=tau)
        else:
            out = srr_from_basis(B, M, sketch_for(t), b, tau=tau)
        history.append(float(np.max(out["rhat"][:nev])))
        if history[-1] <= tau:
            break
        cut = out["lam"][b - 1].real
        Xr = out["X"]
        X = np.hstack([Xr.real, Xr.imag])
        X = X[:, np.linalg.norm(X, axis=0) > 1e-10][:, :b]
    out = dict(out)
    out.update(restarts=len(history), history=history)
    return out


def rr_matrix(B, M):
    """M_star = B^+ (AB), the Rayleigh-Ritz matrix of §6.1 eq. (RR-eig)."""
    return np.linalg.lstsq(B, M, rcond=None)[0]


def eig_residual(A, lam, x):
    """||A x - lam x|| / ||x|| (x may be complex)."""
    Ax = A @ x.real + 1j * (A @ x.imag)
    return np.linalg.norm(Ax - lam * x) / np.linalg.norm(x)
