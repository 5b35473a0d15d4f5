"""Pins for the oracle's model-problem operators."""
import numpy as np
import pytest

import synth
from oracle import operators


def test_stencil_closed_form_spectrum():
    # -Lap + (Pe,Pe).grad with central differences is a Kronecker sum of
    # tridiagonals diag(-(1+a), 2, -(1-a)); with 1-a^2 > 0 its eigenvalues are
    # 4 - 2 sqrt(1-a^2) (cos(i pi h) + cos(j pi h)), i, j = 1..N.
    N, Pe = 9, 12.0
    h = 1.0 / (N + 1)
    a = Pe * h / 2
    assert a < 1
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, Pe)).toarray()
    ev = np.sort(np.linalg.eigvals(A).real)
    c = np.cos(np.arange(1, N + 1) * np.pi * h)
    expect = np.sort((4 - 2 * np.sqrt(1 - a * a) * (c[:, None] + c[None, :])).reshape(-1))
    assert np.allclose(ev, expect, atol=1e-10)


def test_stencil_consistency_with_pde():
    # (Au)_P / h^2 -> (-Lap u + Pe (u_x + u_y))(P) for a smooth u vanishing
    # on the boundary; central differences are exact for this polynomial.
    N, Pe = 31, 7.0
    h = 1.0 / (N + 1)
    xs = (np.arange(N) + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    u = (X * (1 - X) * Y * (1 - Y)).reshape(-1)
    lap = (-2 * Y * (1 - Y) - 2 * X * (1 - X)).reshape(-1)
    ux = ((1 - 2 * X) * Y * (1 - Y)).reshape(-1)
    uy = ((1 - 2 * Y) * X * (1 - X)).reshape(-1)
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, Pe))
    lhs = (A @ u) / h ** 2
    rhs = -lap + Pe * (ux + uy)
    assert np.allclose(lhs, rhs, atol=1e-9)


def test_stencil_entries_by_hand():
    coef = (10.0, 1.0, 2.0, 3.0, 4.0)
    A = operators.stencil5_matrix(3, 3, coef, shift=np.arange(9.0)).toarray()
    # centre cell (1,1) -> index 4: E=5, W=3, N=7, S=1
    row = np.zeros(9)
    row[4] = 10 + 4
    row[5], row[3], row[7], row[1] = 1, 2, 3, 4
    assert np.array_equal(A[4], row)
    # corner (0,0): only E (index 1) and N (index 3)
    row = np.zeros(9)
    row[0], row[1], row[3] = 10.0, 1.0, 3.0
    assert np.array_equal(A[0], row)


def test_var_coef_reduces_to_laplacian():
    N = 6
    A1 = operators.diffusion_var_matrix(N, N, np.ones(N * N)).toarray()
    A2 = operators.stencil5_matrix(N, N, (4.0, -1.0, -1.0, -1.0, -1.0)).toarray()
    assert np.array_equal(A1, A2)


def test_var_coef_symmetric_positive_definite():
    N = 7
    th = np.exp(np.random.default_rng(0).standard_normal(N * N))
    A = operators.diffusion_var_matrix(N, N, th).toarray()
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_var_coef_theta_grad_finite_differences():
    nx, ny = 5, 4
    rng = np.random.default_rng(1)
    th = np.exp(rng.standard_normal(nx * ny))
    lam = rng.standard_normal(nx * ny)
    x = rng.standard_normal(nx * ny)
    g = operators.diffusion_var_theta_grad(nx, ny, lam, x)
    for p in range(nx * ny):
        e = np.zeros(nx * ny)
        e[p] = 1e-6
        fp = lam @ (operators.diffusion_var_matrix(nx, ny, th + e) @ x)
        fm = lam @ (operators.diffusion_var_matrix(nx, ny, th - e) @ x)
        assert abs((fp - fm) / 2e-6 - g[p]) < 1e-6 * max(1, abs(g[p]))


def test_grf_statistics():
    g = synth.grf(2, 128, 8.0)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12
    G = g.reshape(128, 128)
    # smooth: neighbour correlation close to exp(-1/(2 ell^2))
    c = np.mean(G[:, :-1] * G[:, 1:])
    assert c > 0.9


def test_neumann_laplacian_spectrum_and_kernel():
    # eigenvalues of the Kronecker sum of path-graph Laplacians:
    # (2 - 2 cos(pi i / nx)) + (2 - 2 cos(pi j / ny)), i < nx, j < ny
    nx, ny = 7, 5
    A = operators.neumann_laplacian_matrix(nx, ny).toarray()
    assert np.allclose(A, A.T)
    assert np.allclose(A @ np.ones(nx * ny), 0)
    li = 2 - 2 * np.cos(np.pi * np.arange(nx) / nx)
    lj = 2 - 2 * np.cos(np.pi * np.arange(ny) / ny)
    exact = np.sort((li[:, None] + lj[None, :]).ravel())
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), exact, atol=1e-12)
    assert exact.max() < 8


def test_neumann_shift_turns_the_stencil_into_the_neumann_laplacian():
    nx, ny = 6, 4
    S = operators.stencil5_matrix(nx, ny, (4.0, -1.0, -1.0, -1.0, -1.0), synth.neumann_shift(nx, ny))
    assert np.allclose(S.toarray(), operators.neumann_laplacian_matrix(nx, ny).toarray())
