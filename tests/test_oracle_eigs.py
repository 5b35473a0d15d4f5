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


# ---------------------------------------------------------------------------
# Stabilized sRR (§6.5, eq. (qz))
# ---------------------------------------------------------------------------
def _monomial_basis(A, w, d):
    # b_j = A^{j-1} w, each column scaled to unit norm: the badly conditioned
    # basis that §6.5 is about (kappa grows geometrically with d)
    B = np.zeros((w.shape[0], d))
    v = w / np.linalg.norm(w)
    for j in range(d):
        B[:, j] = v
        v = A @ v
        v = v / np.linalg.norm(v)
    return B


def _plain_srr_from_basis(B, M, sk, nev):
    # Algorithm 2's reduction M-hat = T^{-1} U^T (S A B) on the same basis
    C, D = sk(B), sk(M)
    V, T = krylov.householder_qr(C)
    d = B.shape[1]
    UtD = np.stack([krylov.apply_qt(V, D[:, j])[:d] for j in range(d)], axis=1)
    lam = np.linalg.eigvals(np.linalg.solve(T, UtD))
    return lam[eigs.select_order(lam, nev)], krylov.cond2(T)


@pytest.mark.parametrize("seed", [1, 3])
def test_stabilized_recovers_spectrum_past_unit_roundoff(seed):
    # diagonal A with six separated top eigenvalues above a bulk in [0, 1];
    # monomial bases of depth 40..80 with kappa_2(T) ~ 1e17 (beyond 1/u).
    # The stabilized form finds the top six to 5e-4 or better (measured:
    # 8e-5 at worst over three start vectors and two sketches), where
    # Algorithm 2's reduction on the same basis is off by 0.1 or more in the
    # real parts (measured 0.3 to 2.2).  At d = 20 (kappa ~ 1e16) both work.
    n = 2000
    top = np.array([3.0, 2.6, 2.2, 2.0, 1.7, 1.5])
    lam = np.concatenate([top, np.linspace(1.0, 0.0, n - 6)])
    A = np.diag(lam)
    w = synth.randn(seed, n)
    for d in (40, 60, 80):
        B = _monomial_basis(A, w, d)
        M = A @ B
        sk = lambda X: sketch.sparse_sign_apply(5, 4 * d, hashing.default_zeta(d), X)
        out = eigs.srr_stabilized_from_basis(B, M, sk, 6, trunc_tol=1e13, symmetric=True)
        err = np.abs(out["lam"].real - top).max()
        assert err <= 5e-4, (d, err)
        assert out["rank"] < d and out["sigma"][0] / out["sigma"][out["rank"] - 1] <= 1e13
        lp, kp = _plain_srr_from_basis(B, M, sk, 6)
        assert kp > 1e16 and np.abs(lp.real - top).max() > 0.1


def test_stabilized_equals_algorithm_2_on_a_good_basis():
    # no truncation (rank = d): (U^T S A B) V z = theta Sigma z is M-hat's
    # eigenproblem in other coordinates (y = V z), so the Ritz values agree.
    # Full orthogonalisation (k = d) keeps kappa_2(S B) near 1.
    N = 16
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, 20.0))
    w1 = synth.randn(4, N * N)
    d = 30
    sk = _sk(d, seed=9)
    a = eigs.srr(A, w1, d, d, sk, nev=8)
    b = eigs.srr_stabilized(A, w1, d, d, sk, nev=8, trunc_tol=np.inf)
    assert b["rank"] == d and b["sigma"][0] / b["sigma"][-1] < 10 and a["kappa"] < 10
    la, lb = a["all_lam"], b["all_lam"]
    assert la.shape == lb.shape
    # every Ritz value of one has a partner in the other (both ways)
    assert np.abs(la[:, None] - lb[None, :]).min(axis=1).max() <= 1e-9
    assert np.abs(lb[:, None] - la[None, :]).min(axis=1).max() <= 1e-9
    # the selected values as a set (a conjugate pair's real parts tie up to
    # rounding, so its order within the selection is not fixed)
    sa, sb = a["lam"], b["lam"]
    assert np.abs(sa[:, None] - sb[None, :]).min(axis=1).max() <= 1e-9
    ia = np.argsort(np.round(sa.real, 6) + 1e-3 * np.round(sa.imag, 6))
    ib = np.argsort(np.round(sb.real, 6) + 1e-3 * np.round(sb.imag, 6))
    assert np.allclose(a["rhat"][ia], b["rhat"][ib], rtol=1e-6, atol=1e-12)


def test_stabilized_diagonal_and_laplacian_closed_forms():
    # exact spectra at d = n (diagonal, §8.3.4 shape) and the 1-D Laplacian's
    # 2 - 2 cos(j pi / (n+1))
    n = 64
    lam = np.concatenate([np.linspace(-1, -0.1, 10), np.linspace(0, 1, n - 10)])
    out = eigs.srr_stabilized(np.diag(lam), synth.randn(1, n), n, n, _sk(n), nev=n, symmetric=True)
    assert np.allclose(np.sort(out["lam"].real), np.sort(lam), atol=1e-8)
    L = np.diag(2 * np.ones(n)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    exact = np.sort(2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))[::-1]
    out = eigs.srr_stabilized(L, synth.randn(2, n), n, n, _sk(n), nev=10, symmetric=True)
    assert np.allclose(out["lam"].real, exact[:10], atol=1e-8)
    # the residual estimate is small for converged pairs and the vectors are unit
    assert np.all(out["rhat"] <= 1e-8) and np.allclose(np.linalg.norm(out["X"], axis=0), 1)


def test_srr_on_block_chebyshev_basis_finds_separated_top():
    # sRR on a block Krylov basis (§7.1) built by the block Chebyshev
    # recurrence (§7.5) for the bulk [0, 1]: the filter amplifies the six
    # eigenvalues above it.  Known spectrum: b = 16, p = 10 finds them to
    # 1e-5 (measured 9e-7); b = 8, p = 4 does not (error 0.46).
    n = 3000
    top = np.array([3.0, 2.6, 2.2, 2.0, 1.7, 1.5])
    lam = np.concatenate([top, np.linspace(1.0, 0.0, n - 6)])
    A = np.diag(lam)
    errs = {}
    for b, p in ((8, 4), (16, 10)):
        Om = np.column_stack([synth.randn(100 + i, n) for i in range(b)])
        B = krylov.block_chebyshev_basis(A, Om, p, 0.5, 0.5, 0.0)
        d = b * p
        sk = lambda X: sketch.sparse_sign_apply(4, 2 * d, hashing.default_zeta(d), X)
        out = eigs.srr_from_basis(B, A @ B, sk, 6, symmetric=True)
        errs[b] = np.abs(out["lam"].real - top).max()
        if b == 16:
            tr = np.array([eigs.eig_residual(A, out["lam"][i], out["X"][:, i]) for i in range(6)])
            assert np.all(tr <= 1e-3)
    assert errs[16] <= 1e-5 and errs[8] > 0.1


# ---------------------------------------------------------------------------
# Restarted sRR (§7.2) on block Chebyshev bases (§7.5)
# ---------------------------------------------------------------------------
def test_restarted_srr_laplacian_2d_closed_form_with_double_eigenvalue():
    # Dirichlet 5-point Laplacian on 24 x 24: eigenvalues
    # 4 - 2 cos(i pi/25) - 2 cos(j pi/25); the top five include the double
    # eigenvalue of (i, j) = (23, 24) and (24, 23), which a block basis
    # resolves: both copies, with independent Ritz vectors
    import scipy.sparse  # noqa: F401  (operators returns scipy sparse)
    N, b, p, nev = 24, 8, 12, 5
    A = operators.stencil5_matrix(N, N, (4.0, -1.0, -1.0, -1.0, -1.0))
    h = np.pi / (N + 1)
    ev = np.sort([4 - 2 * np.cos(i * h) - 2 * np.cos(j * h) for i in range(1, N + 1) for j in range(1, N + 1)])[::-1]
    assert abs(ev[1] - ev[2]) < 1e-14 and ev[0] - ev[1] > 1e-2
    Om = np.column_stack([synth.randn(400 + i, N * N) for i in range(b)])
    d = b * p
    skf = lambda t: (lambda M: sketch.sparse_sign_apply(13 + t, 2 * d, hashing.default_zeta(d), M))
    out = eigs.srr_restarted(A, Om, p, nev, -0.1, 7.0, 40, skf, tau=8e-9)
    assert out["restarts"] < 40 and out["history"][-1] <= 8e-9
    lam = out["lam"][:nev].real
    assert np.allclose(np.sort(lam)[::-1], ev[:nev], atol=1e-9)
    X = out["X"][:, :nev].real
    for i in range(nev):
        assert eigs.eig_residual(A, lam[i], X[:, i]) <= 1e-8
    dbl = [i for i in range(nev) if abs(lam[i] - ev[1]) < 1e-8]
    # two copies whose Ritz vectors span the 2-D eigenspace (any basis of it
    # is valid, so they need not be orthogonal, only independent)
    assert len(dbl) == 2
    assert np.linalg.svd(X[:, dbl], compute_uv=False)[-1] >= 0.1


def test_restarted_srr_matches_arpack_on_clustered_spectrum():
    # the eig workload's operator at 48 x 48 (convection-diffusion, Pe = 10,
    # uniform random diagonal shift): its top eigenvalues are clustered
    # (single-vector restarts stall near 3e-3).  Block Chebyshev restarts
    # reach true residuals <= 1e-8 ||A|| and ARPACK's eigenvalues (scipy
    # eigs, 'LR', tol 1e-13) within 1e-7.
    import scipy.sparse.linalg as spla
    N, b, p, nev = 48, 12, 16, 6
    shift = synth.uniform(1, N * N)
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, 10.0), shift)
    An = 8 + shift.max()
    ref = np.sort(spla.eigs(A, k=nev + 4, which="LR", return_eigenvectors=False, tol=1e-13).real)[::-1]
    Om = np.column_stack([synth.randn(200 + i, N * N) for i in range(b)])
    d = b * p
    skf = lambda t: (lambda M: sketch.sparse_sign_apply(7 + t, 2 * d, hashing.default_zeta(d), M))
    out = eigs.srr_restarted(A, Om, p, nev, -0.5, 8.0, 30, skf, tau=1e-8 * An)
    assert out["restarts"] < 30
    lam = out["lam"][:nev]
    tr = np.array([eigs.eig_residual(A, lam[i], out["X"][:, i]) for i in range(nev)]) / An
    assert tr.max() <= 1e-8
    assert np.abs(np.sort(lam.real)[::-1] - ref[:nev]).max() <= 1e-7


def test_chebyshev_filter_is_chebyshev_polynomial_on_a_diagonal():
    # on a diagonal matrix column q of the filtered block is, up to a
    # positive scale, T_m((lam - c)/dx) * Q[:, q] (numpy's chebval)
    n, m, c, dx = 300, 37, 0.6, 0.55
    lam = np.linspace(-0.2, 1.3, n)
    A = np.diag(lam)
    Q = np.column_stack([synth.randn(60 + i, n) for i in range(3)])
    Y = eigs.chebyshev_filter(A, Q, m, c, dx)
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    T = np.polynomial.chebyshev.chebval((lam - c) / dx, coef)
    for q in range(3):
        ref = T * Q[:, q]
        scale = (Y[:, q] @ ref) / (ref @ ref)
        assert scale > 0
        assert np.linalg.norm(Y[:, q] - scale * ref) <= 1e-10 * np.linalg.norm(Y[:, q])


def test_filtered_restarted_srr_matches_arpack_in_few_restarts():
    # the 48 x 48 clustered case of the test above with a degree-60 filter of
    # the start block: ARPACK's eigenvalues within 1e-7 and true residuals
    # <= 1e-8 ||A|| in fewer restarts than without the filter
    import scipy.sparse.linalg as spla
    N, b, p, nev = 48, 12, 16, 6
    shift = synth.uniform(1, N * N)
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, 10.0), shift)
    An = 8 + shift.max()
    ref = np.sort(spla.eigs(A, k=nev + 4, which="LR", return_eigenvectors=False, tol=1e-13).real)[::-1]
    Om = np.column_stack([synth.randn(200 + i, N * N) for i in range(b)])
    d = b * p
    skf = lambda t: (lambda M: sketch.sparse_sign_apply(7 + t, 2 * d, hashing.default_zeta(d), M))
    plain = eigs.srr_restarted(A, Om, p, nev, -0.5, 8.0, 30, skf, tau=1e-8 * An)
    out = eigs.srr_restarted(A, Om, p, nev, -0.5, 8.0, 30, skf, tau=1e-8 * An, filter_degree=60)
    assert out["restarts"] < plain["restarts"]
    lam = out["lam"][:nev]
    tr = np.array([eigs.eig_residual(A, lam[i], out["X"][:, i]) for i in range(nev)]) / An
    assert tr.max() <= 1e-8
    assert np.abs(np.sort(lam.real)[::-1] - ref[:nev]).max() <= 1e-7
