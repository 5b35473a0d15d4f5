"""Pins for the SRHT and the subspace-embedding behaviour of the oracle sketches."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import hashing, sketch


@pytest.mark.parametrize("n", [1, 2, 4, 32, 1024])
def test_fwht_equals_sylvester_hadamard(n):
    X = np.random.default_rng(n).standard_normal((n, 3))
    assert np.allclose(sketch.fwht(X), sl.hadamard(n) @ X, rtol=0, atol=1e-10)
    # closed form H[r, i] = (-1)^popcount(r & i)
    if n <= 32:
        H = np.array([[(-1) ** bin(r & i).count("1") for i in range(n)] for r in range(n)], dtype=float)
        assert np.array_equal(sketch.fwht(np.eye(n)), H)


def test_fwht_involution():
    x = np.random.default_rng(0).standard_normal(256)
    assert np.allclose(sketch.fwht(sketch.fwht(x)) / 256, x, atol=1e-12)


def test_srht_rows_distinct_and_golden():
    rows = hashing.srht_rows(7, 1 << 20, 600)
    assert len(set(rows.tolist())) == 600 and rows.min() >= 0 and rows.max() < (1 << 20)
    rows2 = hashing.srht_rows(0, 1 << 12, 80)
    gold = np.loadtxt("tests/golden/srht_rows_seed0_np4096_s80.txt", dtype=np.int64)
    assert np.array_equal(rows2, gold)


def test_srht_rows_full_permutation_when_s_equals_np():
    rows = hashing.srht_rows(3, 64, 64)
    assert sorted(rows.tolist()) == list(range(64))


@pytest.mark.parametrize("n", [100, 128])
def test_srht_equals_dense_definition(n):
    seed, s = 11, 20
    n_p = 1 << int(np.ceil(np.log2(n)))
    E = hashing.srht_signs(seed, n)
    rows = hashing.srht_rows(seed, n_p, s)
    H = sl.hadamard(n_p) / np.sqrt(n_p)
    Epad = np.zeros((n_p, n))
    Epad[:n, :n] = np.diag(E)
    S = np.sqrt(n_p / s) * (H @ Epad)[rows]
    X = np.random.default_rng(2).standard_normal((n, 4))
    assert np.allclose(sketch.srht_apply(seed, s, X), S @ X, atol=1e-12)


def _orthonormal(n, d, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, d)))
    return Q


@pytest.mark.parametrize("kind", ["sparse", "srht"])
def test_embedding_distortion_band(kind):
    # Def. (subspace-embed) with s = 2d (§3.3: s = 2(d+1) typically gives
    # eps ~ 1/sqrt(2)); for s x d Gaussian-like embeddings sigma(SQ) lies near
    # [1 - sqrt(d/s), 1 + sqrt(d/s)] (Marchenko-Pastur edges).
    n, d, s = 1 << 14, 40, 80
    Q = _orthonormal(n, d, 0)
    lo, hi = 1 - np.sqrt(d / s) - 0.15, 1 + np.sqrt(d / s) + 0.15
    for seed in range(10 if kind == "sparse" else 4):
        eps, sv = sketch.distortion(sketch.apply(kind, seed, s, 8, Q))
        assert lo <= sv[-1] and sv[0] <= hi, (seed, sv[0], sv[-1])


@pytest.mark.parametrize("kind", ["sparse", "srht"])
def test_fact_2_2_sketched_least_squares(kind):
    # Fact 2.2, eq. (ls-residuals): ||My* - f|| <= ||M y_hat - f||
    # <= (1+eps)/(1-eps) ||My* - f|| with eps the distortion of S on
    # range([M, f]), measured exactly from sigma(S Q), Q = orth([M, f]).
    rng = np.random.default_rng(5)
    n, d, s = 2000, 20, 60
    M = rng.standard_normal((n, d)) @ np.diag(np.logspace(0, 4, d))
    f = rng.standard_normal(n)
    ystar = np.linalg.lstsq(M, f, rcond=None)[0]
    SM = sketch.apply(kind, 3, s, 6, M)
    Sf = sketch.apply(kind, 3, s, 6, f)
    yhat = np.linalg.lstsq(SM, Sf, rcond=None)[0]
    Q = np.linalg.qr(np.column_stack([M, f]))[0]
    eps, sv = sketch.distortion(sketch.apply(kind, 3, s, 6, Q))
    assert eps < 1
    r_star = np.linalg.norm(M @ ystar - f)
    r_hat = np.linalg.norm(M @ yhat - f)
    assert r_star <= r_hat * (1 + 1e-12)
    assert r_hat <= (1 + eps) / (1 - eps) * r_star
    # the sharper per-instance form: ||M yhat - f|| <= (smax/smin) ||M y* - f||
    assert r_hat <= sv[0] / sv[-1] * r_star * (1 + 1e-12)
