"""Pins for the oracle's sketched Rayleigh-Ritz (Algorithm 2)."""
import numpy as np
import pytest

import synth
from oracle import eigs, hashing, krylov, operators, sketch


def _sk(d, seed=3, kind="sparse"):
    s = 2 * d
    return lambda X: sketch.apply(kind, seed, s, hashing.default_zeta(d), X)


def test_diagonal_spectrum_recovered_when_d_equals_n():
    # A = diag(lambda) with ten eigenvalues equispaced in [-1,-0.1] and the rest
    # equispaced in [0,1] (the spectrum shape of §8.3.4, at n = 64).  With
    # d = n the Krylov space is everything: sRR returns the exact spectrum.
    n = 64
    lam = np.concatenate([np.linspace(-1, -0.1, 10), np.linspace(0, 1, n - 10)])
    A = np.diag(lam)
    w1 = synth.randn(1, n)
    out = eigs.srr(A, w1, n, n, _sk(n), nev=n, symmetric=True)
    assert np.allclose(np.sort(out["lam"].real), np.sort(lam), atol=1e-8)


def test_laplacian_1d_closed_form():
    # tridiag(-1, 2, -1): lambda_j = 2 - 2 cos(j pi/(n+1)); with k = 2 the
    # truncated Arnoldi basis is the Lanczos basis (§4.3).
    n = 64
    A = np.diag(2 * np.ones(n)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    exact = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    out = eigs.srr(A, synth.randn(2, n), n, n, _sk(n), nev=10, symmetric=True)
    assert np.allclose(out["lam"].real, np.sort(exact)[::-1][:10], atol=1e-8)


def test_convection_diffusion_top_eigenvalue_closed_form():
    # largest eigenvalue of the N x N convection-diffusion stencil:
    # 4 + 4 sqrt(1-a^2) cos(pi h)  (Kronecker sum of tridiagonals)
    N, Pe = 8, 10.0
    h = 1.0 / (N + 1)
    a = Pe * h / 2
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, Pe))
    out = eigs.srr(A, synth.randn(3, N * N), N * N, N * N, _sk(N * N), nev=1)
    assert abs(out["lam"][0] - (4 + 4 * np.sqrt(1 - a * a) * np.cos(np.pi * h))) < 1e-9


def test_krylov_basis_mhat_matches_rr_except_last_column():
    # §6.7: on a Krylov basis, A b_i is in range(B) for i < d, so the sketched
    # and unsketched RR matrices agree in columns 1..d-1.
    N = 12
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, 20.0))
    out = eigs.srr(A, synth.randn(4, N * N), 20, 3, _sk(20), nev=3)
    Mstar = eigs.rr_matrix(out["B"], out["M"])
    Mhat = out["Mhat"]
    assert np.linalg.cond(out["B"]) < 1e4
    scale = np.abs(Mstar).max()
    assert np.allclose(Mhat[:, :-1], Mstar[:, :-1], atol=1e-10 * scale)
    assert not np.allclose(Mhat[:, -1], Mstar[:, -1], atol=1e-6 * scale)


@pytest.mark.parametrize("kind", ["sparse", "srht"])
def test_residual_estimate_brackets_true_residual(kind):
    # eq. (rescompare): (1-eps)/(1+eps) r_est <= ||AB y - lam B y||/||B y||
    # <= (1+eps)/(1-eps) r_est, eps the distortion on range([B, AB]).
    N, d = 16, 30
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, 15.0), synth.uniform(1, N * N))
    sk = _sk(d, 7, kind)
    out = eigs.srr(A, synth.randn(5, N * N), d, 4, sk, nev=6)
    Q = np.linalg.qr(np.column_stack([out["B"], out["M"]]))[0]
    eps, sv = sketch.distortion(sk(Q))
    lo, hi = sv[-1] / sv[0], sv[0] / sv[-1]
    lam_all, Y = np.linalg.eig(out["Mhat"])
    for i in range(len(lam_all)):
        By = out["B"] @ Y[:, i]
        ABy = out["M"] @ Y[:, i]
        true = np.linalg.norm(ABy - lam_all[i] * By) / np.linalg.norm(By)
        est = np.linalg.norm(out["D"] @ Y[:, i] - lam_all[i] * (out["C"] @ Y[:, i])) / np.linalg.norm(out["C"] @ Y[:, i])
        assert lo * est * (1 - 1e-6) <= true <= hi * est * (1 + 1e-6)


def test_selection_order_and_normalisation():
    lam = np.array([1 + 2j, 3, 1 - 2j, 3 + 0j, -5])
    assert eigs.select_order(lam, 3) == [1, 3, 0]
    N = 10
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, 10.0), synth.uniform(1, N * N))
    out = eigs.srr(A, synth.randn(6, N * N), 30, 4, _sk(30), nev=4)
    assert np.allclose(np.linalg.norm(out["X"], axis=0), 1)
    assert np.all(np.diff(out["lam"].real) <= 0)
    for i in range(4):
        r = eigs.eig_residual(A, out["lam"][i], out["X"][:, i])
        assert r < 1e-2
