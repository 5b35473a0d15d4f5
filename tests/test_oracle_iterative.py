"""Pins for the oracle's iterative sGMRES (§5.2: incremental QR of the
sketched reduced matrix, stop on the residual estimate) and its adaptive
restart on kappa_2(T_j) (§5.3).  The references are LAPACK least squares and
QR on the explicitly formed sketched matrix, and the minimal-polynomial
closed form."""
import numpy as np
import pytest

import synth
from oracle import hashing, krylov, operators, sketch


def _setup(N=16, Pe=10.0, dmax=30, k=2, seed=7):
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, Pe))
    f = synth.randn(11, N * N)
    s = 2 * (dmax + 1)
    sk = lambda M: sketch.sparse_sign_apply(seed, s, hashing.default_zeta(dmax), M)
    return A, f, sk


def _prefix_lstsq(A, f, x0, dmax, k, sk):
    # the sketched problem written out: C = S A B, g = S r_0, and for every
    # prefix j the LAPACK least-squares solution and residual norm
    r = f - A @ x0
    B, M, _, du = krylov.trunc_arnoldi(A, r, dmax, k)
    C = sk(M)
    g = sk(r)
    ys, res = [], []
    for j in range(1, du + 1):
        y = np.linalg.lstsq(C[:, :j], g, rcond=None)[0]
        ys.append(y)
        res.append(np.linalg.norm(g - C[:, :j] @ y))
    return B, C, g, ys, np.array(res)


def test_estimates_match_lstsq_on_every_prefix():
    A, f, sk = _setup()
    x0 = np.zeros_like(f)
    B, C, g, ys, res = _prefix_lstsq(A, f, x0, 30, 2, sk)
    x, info = krylov.sgmres_iterative_cycle(A, f, x0, 30, 2, sk, 0.0)
    assert info["stop"] == "dmax" and info["j"] == 30
    rh = np.array(info["rhat"])
    assert np.allclose(rh, res, rtol=1e-9, atol=1e-13 * np.linalg.norm(g))
    # the estimate is non-increasing in j (nested least-squares problems)
    assert np.all(np.diff(res) <= 1e-12 * res[0])
    assert np.all(np.diff(rh) <= 1e-12 * rh[0])
    # the solution after dmax columns is x0 + B y_lstsq
    xr = x0 + B @ ys[-1]
    assert np.linalg.norm(A @ (x - xr)) <= 1e-9 * np.linalg.norm(f)
    # kappa_2(T_j) = kappa_2(C_j) for every prefix (T_j is C_j's triangle)
    kap = np.array([np.linalg.cond(C[:, :j]) for j in range(1, 31)])
    assert np.allclose(info["kappa"], kap, rtol=1e-6)


@pytest.mark.parametrize("jstop", [1, 7, 19])
def test_stops_at_first_prefix_meeting_the_target(jstop):
    A, f, sk = _setup()
    x0 = synth.randn(12, f.shape[0]) * 0.1
    B, C, g, ys, res = _prefix_lstsq(A, f, x0, 30, 2, sk)
    # a target strictly between the estimates of prefixes jstop-1 and jstop
    hi = res[jstop - 2] if jstop > 1 else np.linalg.norm(g)
    tol_rel = np.sqrt(hi * res[jstop - 1]) / np.linalg.norm(g)
    assert res[jstop - 1] < tol_rel * np.linalg.norm(g) < hi
    x, info = krylov.sgmres_iterative_cycle(A, f, x0, 30, 2, sk, tol_rel)
    assert info["stop"] == "tol" and info["j"] == jstop
    assert len(info["rhat"]) == jstop
    xr = x0 + B[:, :jstop] @ ys[jstop - 1]
    assert np.linalg.norm(A @ (x - xr)) <= 1e-9 * np.linalg.norm(f)


def test_kappa_restart_keeps_previous_solution():
    # k = 1 and strong convection: kappa_2(S A B_j) grows with j.  With a
    # threshold between kappa(C_{j*-1}) and kappa(C_{j*}) (LAPACK SVD of the
    # explicit sketched matrix) the cycle ends with y_{j*-1}.
    A, f, sk = _setup(Pe=60.0, k=1)
    x0 = np.zeros_like(f)
    B, C, g, ys, res = _prefix_lstsq(A, f, x0, 30, 1, sk)
    kap = np.array([np.linalg.cond(C[:, :j]) for j in range(1, 31)])
    assert np.all(np.diff(kap) >= -1e-8 * kap[:-1])  # interlacing: non-decreasing
    jstar = int(np.argmax(kap > 1e3)) + 1
    assert 3 <= jstar <= 28 and kap[jstar - 1] > 1.01 * kap[jstar - 2]
    stab = np.sqrt(kap[jstar - 2] * kap[jstar - 1])
    x, info = krylov.sgmres_iterative_cycle(A, f, x0, 30, 1, sk, 0.0, stab_tol=stab)
    assert info["stop"] == "kappa" and info["j"] == jstar - 1
    xr = x0 + B[:, : jstar - 1] @ ys[jstar - 2]
    assert np.linalg.norm(A @ (x - xr)) <= 1e-9 * np.linalg.norm(f)


def test_exact_after_minimal_polynomial_degree():
    # A with 5 distinct eigenvalues: r_0 lies in A K_5(A; r_0), so the
    # sketched problem has a zero-residual solution at j = 5 and x is exact
    # (the recurrence, fully orthogonal here, breaks down right after).
    n = 200
    A = np.diag(np.repeat([1.0, 2.5, 4.0, 7.0, 9.5], n // 5))
    f = synth.randn(13, n)
    dmax = 12
    sk = lambda M: sketch.sparse_sign_apply(3, 2 * (dmax + 1), hashing.default_zeta(dmax), M)
    x, info = krylov.sgmres_iterative_cycle(A, f, np.zeros(n), dmax, dmax, sk, 1e-10)
    assert info["j"] == 5 and info["stop"] in ("tol", "breakdown")
    assert np.linalg.norm(f - A @ x) <= 1e-11 * np.linalg.norm(f)
    assert np.allclose(x, f / np.diag(A), atol=1e-11)


def test_restarted_iterative_reaches_tol_with_fewer_columns():
    W = synth.WORKLOADS["small"]
    N, dmax = W["N"], W["d"]
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, W["Pe"]))
    f = synth.randn(W["b_seed"], N * N)
    sk = lambda M: sketch.sparse_sign_apply(7, 2 * (dmax + 1), hashing.default_zeta(dmax), M)
    x, hist, infos = krylov.sgmres_iterative(A, f, np.zeros(N * N), dmax, W["k"], sk, W["tol"], maxit=60)
    assert hist[-1] <= W["tol"]
    assert np.linalg.norm(f - A @ x) <= W["tol"] * np.linalg.norm(f)
    assert infos[-1]["stop"] == "tol" and infos[-1]["j"] < dmax
    assert all(i["stop"] == "dmax" for i in infos[:-1])
    # the same cycles as Algorithm 1 until the last one: identical iterates
    # before it (the early stop changes nothing while the target is unmet)
    _, hist_full, _ = krylov.sgmres(A, f, np.zeros(N * N), dmax, W["k"], sk, W["tol"], maxit=60)
    assert len(hist_full) == len(hist)
    assert np.allclose(hist[:-1], hist_full[:-1], rtol=1e-6)


def test_argument_errors():
    A, f, sk = _setup(dmax=10)
    with pytest.raises(ValueError):
        krylov.sgmres_iterative_cycle(A, f, np.zeros_like(f), 22, 2, sk, 0.0)
    with pytest.raises(ValueError):
        krylov.sgmres_iterative_cycle(A, f, np.zeros_like(f), 0, 2, sk, 0.0)
