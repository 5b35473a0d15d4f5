"""Pins for the oracle's basis generation, QR/least squares, sGMRES and GMRES."""
import numpy as np
import pytest
import scipy.linalg as sl

import synth
from oracle import hashing, krylov, operators, sketch


def _cd(N, Pe, shift=None):
    return operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, Pe), shift)


def test_full_arnoldi_when_k_equals_d():
    # k = d: every new vector is orthogonalised against all previous ones,
    # i.e. the Arnoldi process of §4.2: B^T B = I and AB = B_{d+1} H.
    A = _cd(12, 20.0)
    r = synth.randn(0, 144)
    B, M, Hc, du = krylov.trunc_arnoldi(A, r, 30, 30)
    assert du == 30
    assert np.allclose(B.T @ B, np.eye(30), atol=1e-12)
    assert np.allclose(M, A @ B, atol=0)
    # Hessenberg relation for the first d-1 columns (b_{d+1} not formed)
    assert np.allclose(M[:, :-1], B @ Hc[:30, :29], atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_local_orthogonality_of_truncated_basis(k):
    # w_j is orthogonalised against b_{j-1..j-k}: b_i^T b_j ~ 0 for 0<|i-j|<=k
    A = _cd(16, 40.0)
    B, M, Hc, du = krylov.trunc_arnoldi(A, synth.randn(3, 256), 40, k)
    G = B.T @ B
    for i in range(du):
        assert abs(G[i, i] - 1) < 1e-13
        for j in range(max(0, i - k), i):
            assert abs(G[i, j]) < 1e-13
    # the basis spans the Krylov space: each m_j is in span(b_1..b_{j+1})
    assert np.allclose(M[:, :-1], B @ Hc[:du, : du - 1], atol=1e-11)


def test_single_pass_is_classical_gram_schmidt():
    A = _cd(8, 5.0)
    r = synth.randn(1, 64)
    B1, _, _, _ = krylov.trunc_arnoldi(A, r, 6, 2, passes=1)
    # by hand for column 2 (0-based 1) and 3
    b0 = r / np.linalg.norm(r)
    m0 = A @ b0
    w = m0 - b0 * (b0 @ m0)
    b1 = w / np.linalg.norm(w)
    m1 = A @ b1
    w = m1 - b0 * (b0 @ m1) - b1 * (b1 @ m1)
    b2 = w / np.linalg.norm(w)
    assert np.allclose(B1[:, :3], np.column_stack([b0, b1, b2]), atol=1e-14)


def test_breakdown_on_invariant_subspace():
    # r in an invariant subspace of dimension 3 (diagonal A, r with 3 nonzeros)
    A = np.diag(np.arange(1.0, 21.0))
    r = np.zeros(20)
    r[[2, 7, 11]] = [1.0, -2.0, 0.5]
    B, M, Hc, du = krylov.trunc_arnoldi(A, r, 10, 10)
    assert du == 3


def test_householder_qr_and_ls_match_lapack():
    rng = np.random.default_rng(0)
    C = rng.standard_normal((60, 25)) @ np.diag(np.logspace(0, 6, 25))
    g = rng.standard_normal(60)
    V, T = krylov.householder_qr(C)
    U = krylov.form_u(V, 60)
    assert np.allclose(U.T @ U, np.eye(25), atol=1e-13)
    assert np.allclose(U @ T, C, rtol=0, atol=1e-9 * np.abs(C).max())
    assert np.allclose(np.tril(T, -1), 0)
    y, rhat, kappa, width = krylov.sketched_ls(C, g)
    y_ref = np.linalg.lstsq(C, g, rcond=None)[0]  # SVD-based (gelsd)
    assert np.allclose(y, y_ref, rtol=1e-8, atol=1e-14)
    assert abs(rhat - np.linalg.norm(C @ y_ref - g)) < 1e-10
    assert abs(kappa / np.linalg.cond(C) - 1) < 1e-8
    assert width == 25


def test_back_substitution_matches_solve_triangular():
    rng = np.random.default_rng(3)
    T = np.triu(rng.standard_normal((30, 30))) + 5 * np.eye(30)
    z = rng.standard_normal(30)
    assert np.allclose(krylov.back_substitute(T, z), sl.solve_triangular(T, z), atol=1e-13)


def test_stab_tol_truncates_to_leading_block():
    rng = np.random.default_rng(4)
    C = rng.standard_normal((40, 12)) @ np.diag(np.logspace(0, 11, 12))
    g = rng.standard_normal(40)
    y, rhat, kappa, width = krylov.sketched_ls(C, g, stab_tol=1e6)
    assert kappa > 1e6 and width < 12
    assert np.linalg.cond(C[:, :width]) <= 1e6 < np.linalg.cond(C[:, : width + 1])
    assert np.all(y[width:] == 0)
    y_ref = np.linalg.lstsq(C[:, :width], g, rcond=None)[0]
    assert np.allclose(y[:width], y_ref, rtol=1e-8)


def test_gmres_householder_matches_brute_force():
    # GMRES iterate = argmin over x0 + K_d(A, r0) of ||f - A x||; for tiny d
    # the explicit Krylov matrix solves that by dense least squares.
    A = _cd(5, 10.0).toarray()
    f = synth.randn(2, 25)
    x0 = synth.randn(9, 25) * 0.1
    r0 = f - A @ x0
    for d in (1, 3, 5):
        K = np.column_stack([np.linalg.matrix_power(A, p) @ r0 for p in range(d)])
        yk = np.linalg.lstsq(A @ K, r0, rcond=None)[0]
        res_ref = np.linalg.norm(r0 - A @ K @ yk)
        _, res = krylov.gmres_householder(A, f, x0, d)
        assert abs(res - res_ref) <= 1e-9 * np.linalg.norm(r0)


def test_gmres_full_dimension_is_exact():
    A = _cd(6, 3.0).toarray()
    f = synth.randn(4, 36)
    x, res = krylov.gmres_householder(A, f, np.zeros(36), 36)
    assert res <= 1e-10 * np.linalg.norm(f)
    assert np.allclose(x, np.linalg.solve(A, f), atol=1e-9)


def test_sgmres_exact_when_d_equals_n():
    # d >= n: the Krylov space is the whole space (or an invariant subspace
    # containing the solution), so one cycle solves the system.
    N = 8
    A = _cd(N, 10.0)
    f = synth.randn(0, N * N)
    sk = lambda M: sketch.sparse_sign_apply(1, 2 * N * N, hashing.default_zeta(N * N), M)
    x, hist, infos = krylov.sgmres(A, f, np.zeros(N * N), N * N, N * N, sk, tol=1e-300, maxit=1)
    kA = np.linalg.cond(A.toarray())
    assert hist[0] <= 1e-10 * kA


@pytest.mark.parametrize("kind", ["sparse", "srht"])
def test_sgmres_residual_within_fact_2_2_of_gmres(kind):
    # eq. (sgmres-residual): ||A x_B - f|| <= ||A x_hat - f|| <= (1+eps)/(1-eps)
    # ||A x_B - f||, where x_B is GMRES over the same Krylov space and eps
    # the distortion of S on range([AB, r0]), measured exactly.
    # eq. (sgmres-residual-norm): r_est in [1-eps, 1+eps] ||A x_hat - f||.
    N, d, k = 20, 25, 2
    A = _cd(N, 30.0)
    n = N * N
    f = synth.randn(0, n)
    x0 = np.zeros(n)
    s = 2 * (d + 1)
    sk = lambda M: sketch.apply(kind, 5, s, hashing.default_zeta(d), M)
    x_hat, info = krylov.sgmres_cycle(A, f, x0, d, k, sk)
    res_hat = np.linalg.norm(f - A @ x_hat)
    _, res_gm = krylov.gmres_householder(A, f, x0, d)
    B, M, _, _ = krylov.trunc_arnoldi(A, f, d, k)
    Q = np.linalg.qr(np.column_stack([M, f]))[0]
    eps, sv = sketch.distortion(sk(Q))
    assert res_gm <= res_hat * (1 + 1e-8)
    assert res_hat <= sv[0] / sv[-1] * res_gm * (1 + 1e-8)
    assert sv[-1] * res_hat * (1 - 1e-8) <= info["rhat"] <= sv[0] * res_hat * (1 + 1e-8)


def test_cond_diagnostic():
    # eq. (cond-diagnostic): kappa(T) within the distortion factors of
    # kappa(AB), with C = S AB = U T.
    N, d, k = 16, 30, 2
    A = _cd(N, 30.0)
    f = synth.randn(6, N * N)
    B, M, _, _ = krylov.trunc_arnoldi(A, f, d, k)
    sk = lambda X: sketch.sparse_sign_apply(2, 2 * d, hashing.default_zeta(d), X)
    _, T = krylov.householder_qr(sk(M))
    Q = np.linalg.qr(M)[0]
    _, sv = sketch.distortion(sk(Q))
    ratio = krylov.cond2(T) / np.linalg.cond(M)
    assert sv[-1] / sv[0] * (1 - 1e-8) <= ratio <= sv[0] / sv[-1] * (1 + 1e-8)


def test_restarted_sgmres_small_workload_converges():
    W = synth.WORKLOADS["small"]
    N = W["N"]
    A = _cd(N, W["Pe"])
    f = synth.randn(W["b_seed"], N * N)
    sk = lambda M: sketch.sparse_sign_apply(7, W["s"], W["zeta"], M)
    x, hist, infos = krylov.sgmres(A, f, np.zeros(N * N), W["d"], W["k"], sk, W["tol"])
    assert hist[-1] <= W["tol"]
    assert np.linalg.norm(f - A @ x) / np.linalg.norm(f) == pytest.approx(hist[-1])
    # each restart reduces the residual (the space always contains 0 update)
    assert all(b < a for a, b in zip(hist, hist[1:]))


# ---- Chebyshev basis (§4.3, eq. (Chebrecurse)) --------------------------------
@pytest.mark.parametrize("c,dx,dy", [(4.0, 4.0, 0.0), (1.0, 2.0, 0.0), (3.0, 2.5, 1.5), (3.0, 1.0, 2.0)])
def test_chebyshev_basis_is_chebyshev_polynomials_on_a_diagonal(c, dx, dy):
    # For A = diag(lambda) the recurrence produces, up to positive scalars,
    # i^j T_j((A - c)/f) r with f = sqrt(dx^2 - dy^2) (the foci of the
    # ellipse; f = dx for an interval; f imaginary for a tall ellipse, where
    # i^j T_j is real): compare the unit columns with numpy's chebval.
    from numpy.polynomial import chebyshev as npc
    rng = np.random.default_rng(3)
    n, d = 200, 25
    lam = c + dx * rng.uniform(-1, 1, n)
    A = np.diag(lam)
    r = rng.standard_normal(n)
    B, M, H = krylov.chebyshev_basis(A, r, d, c, dx, dy)
    f = np.sqrt(complex(dx * dx - dy * dy))
    z = (lam - c) / f
    for j in range(d + 1):
        e = np.zeros(j + 1)
        e[j] = 1.0
        v = npc.chebval(z, e) * r
        if dy > dx:
            v = v * (1j) ** j  # real: T_j has the parity of j and f is imaginary
        assert np.abs(v.imag).max() <= 1e-9 * np.abs(v).max()
        v = v.real / np.linalg.norm(v.real)
        assert np.allclose(B[:, j], v, atol=1e-10), j
    assert np.allclose(M, A @ B[:, :d])


@pytest.mark.parametrize("c,dx,dy", [(4.0, 4.0, 0.0), (0.5, 0.5, 0.0), (3.0, 2.5, 1.5), (3.0, 1.0, 2.0)])
def test_block_chebyshev_is_scaled_chebyshev_polynomials_on_a_diagonal(c, dx, dy):
    # §7.5 as printed (no rescaling): for A = diag(lambda), block j (1-based)
    # is exactly (f / (2 rho))^{j-1} T_{j-1}((A - c)/f) Omega with
    # f = sqrt(dx^2 - dy^2) (imaginary for a tall ellipse, where the product
    # is still real): compare with numpy's chebval, scalars included
    from numpy.polynomial import chebyshev as npc
    rng = np.random.default_rng(5)
    n, b, p = 150, 4, 12
    lam = c + dx * rng.uniform(-1, 1, n)
    Om = rng.standard_normal((n, b))
    B = krylov.block_chebyshev_basis(np.diag(lam), Om, p, c, dx, dy)
    assert B.shape == (n, b * p)
    rho = max(dx, dy)
    f = np.sqrt(complex(dx * dx - dy * dy))
    z = (lam - c) / f
    for j in range(1, p + 1):
        e = np.zeros(j)
        e[j - 1] = 1.0
        phi = (f / (2 * rho)) ** (j - 1) * npc.chebval(z, e)
        assert np.abs(phi.imag).max() <= 1e-12 * max(1.0, np.abs(phi).max())
        ref = phi.real[:, None] * Om
        blk = B[:, (j - 1) * b: j * b]
        assert np.allclose(blk, ref, rtol=1e-10, atol=1e-13 * np.abs(ref).max()), j


def test_block_chebyshev_columns_are_the_vector_recurrence():
    # column i of every block is the single-vector recurrence of §4.3 started
    # from column i of Omega (nonsymmetric operator), up to column scaling
    A = _cd(12, 10.0)
    Om = np.column_stack([synth.randn(40 + i, 144) for i in range(3)])
    B = krylov.block_chebyshev_basis(A, Om, 8, 4.0, 3.5, 0.0)
    for i in range(3):
        Bv, _, _ = krylov.chebyshev_basis(A, Om[:, i], 7, 4.0, 3.5, 0.0)
        cols = B[:, i::3]
        assert np.allclose(cols / np.linalg.norm(cols, axis=0), Bv, atol=1e-12)


def test_chebyshev_relation_and_tridiagonal_hbar():
    # A B_d = B_{d+1} Hbar to rounding, Hbar tridiagonal with c on the
    # diagonal, on a nonsymmetric convection-diffusion operator whose real
    # spectrum (a = Pe h / 2 < 1) lies in [4 - 4 sqrt(1 - a^2), 4 + 4 sqrt(1 - a^2)]
    N, Pe = 20, 12.0
    A = _cd(N, Pe)
    a = Pe / (N + 1) / 2
    half = 4 * np.sqrt(1 - a * a)
    r = synth.randn(4, N * N)
    B, M, H = krylov.chebyshev_basis(A, r, 40, 4.0, half, 0.0)
    assert np.allclose(np.linalg.norm(B, axis=0), 1)
    assert np.linalg.norm(A @ B[:, :40] - B @ H) <= 1e-12 * np.linalg.norm(A @ B[:, :40])
    assert np.allclose(np.diag(H), 4.0)
    assert np.count_nonzero(np.triu(H, 2)) == 0 and np.count_nonzero(np.tril(H, -2)) == 0


def test_sgmres_chebyshev_exact_when_d_equals_n():
    # the Chebyshev basis spans K_n(A; r) = R^n: one cycle solves the system
    N = 6
    A = operators.neumann_laplacian_matrix(N, N) + sp_identity(N * N)
    f = synth.randn(2, N * N)
    sk = lambda M: sketch.sparse_sign_apply(1, 2 * N * N, hashing.default_zeta(N * N), M)
    x, hist, infos = krylov.sgmres(A, f, np.zeros(N * N), N * N - 1, 2, sk, tol=1e-300, maxit=1,
                                   cheb=(5.0, 4.0, 0.0))
    assert hist[0] <= 1e-7
    assert np.allclose(x, np.linalg.solve(A.toarray(), f), atol=1e-6)


def test_sgmres_chebyshev_neumann_laplacian_converges():
    # the E2 model problem, small: consistent singular system f = A x_true
    N = 32
    A = operators.neumann_laplacian_matrix(N, N)
    f = A @ synth.randn(5, N * N)
    sk = lambda M: sketch.sparse_sign_apply(3, 120, hashing.default_zeta(60), M)
    x, hist, infos = krylov.sgmres(A, f, np.zeros(N * N), 60, 2, sk, tol=1e-8, maxit=60, cheb=(4.0, 4.0, 0.0))
    assert hist[-1] <= 1e-8
    assert all(i["width"] == 60 for i in infos)


def sp_identity(n):
    import scipy.sparse as sps
    return sps.identity(n, format="csr")
