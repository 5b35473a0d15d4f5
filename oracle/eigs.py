"""Sketched Rayleigh-Ritz (Algorithm 2) and Rayleigh-Ritz (§6.1).

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np

from . import krylov


def select_order(lam, nev):
    """Indices of the nev eigenvalues with largest real part.

    Ties in the real part are broken by larger imaginary part, then by
    position (so a conjugate pair lists the member with Im > 0 first).
    """
    idx = sorted(range(len(lam)), key=lambda i: (-lam[i].real, -lam[i].imag, i))
    return idx[:nev]


def srr(A, w1, d, k, sketch, nev, tau=1e-8, symmetric=False, passes=2, breakdown=1e-13):
    """Algorithm 2 with the basis of §1.2.2 eq. (partorth).

    b_1 = w_1/||w_1||; truncated Arnoldi basis B and AB; C = S B, D = S AB
    (§6.4); C = U T; M-hat = T^{-1}(U^T D) (eq. (Mhat-form)); eig(M-hat)
    (numpy's LAPACK dgeev as one step); residual estimates
    ||D y_i - lam_i C y_i|| / ||C y_i|| (eq. (srr-resid-est)); the nev
    eigenvalues of largest real part; x_i = B y_i / ||B y_i||.
    For real symmetric A (§6.8) the real parts of lam and x are kept.
    """
    B, M, _, d_used = krylov.trunc_arnoldi(A, w1, d, k, passes=passes, breakdown=breakdown)
    C = sketch(B)
    D = sketch(M)
    V, T = krylov.householder_qr(C)
    kappa = krylov.cond2(T)
    UtD = np.stack([krylov.apply_qt(V, D[:, j])[:d_used] for j in range(d_used)], axis=1)
    Mhat = np.zeros((d_used, d_used))
    for j in range(d_used):
        Mhat[:, j] = krylov.back_substitute(T, UtD[:, j])
    lam, Y = np.linalg.eig(Mhat)
    if symmetric:
        lam = lam.real.astype(np.complex128)
        Y = Y.real.astype(np.complex128)
    rhat = np.array([np.linalg.norm(D @ Y[:, i] - lam[i] * (C @ Y[:, i])) / np.linalg.norm(C @ Y[:, i])
                     for i in range(d_used)])
    order = select_order(lam, nev)
    X = B @ Y[:, order]
    X /= np.linalg.norm(X, axis=0)
    return dict(lam=lam[order], X=X, rhat=rhat[order], nconv=int(np.sum(rhat[order] <= tau)),
                kappa=kappa, Mhat=Mhat, B=B, M=M, C=C, D=D, d_used=d_used, all_lam=lam)


def rr_matrix(B, M):
    """M_star = B^+ (AB), the Rayleigh-Ritz matrix of §6.1 eq. (RR-eig)."""
    return np.linalg.lstsq(B, M, rcond=None)[0]


def eig_residual(A, lam, x):
    """||A x - lam x|| / ||x|| (x may be complex)."""
    Ax = A @ x.real + 1j * (A @ x.imag)
    return np.linalg.norm(Ax - lam * x) / np.linalg.norm(x)
