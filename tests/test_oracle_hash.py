"""Pins for the sketch hash H1 and the sparse sign map of the oracle."""
import os

import numpy as np
import pytest

from oracle import hashing, sketch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mix64_published_splitmix64_sequence():
    # SplitMix64 (Steele, Lea & Flood 2014; reference C code by S. Vigna):
    # state = 1234567, each output = finalizer(state += 0x9E3779B97F4A7C15).
    # Published first five outputs for that seed:
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    st = 1234567
    got = []
    for _ in range(5):
        st = (st + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        got.append(int(hashing.mix64(np.array([st], dtype=np.uint64))[0]))
    assert got == expect


def test_key_layout_and_range_map():
    # key = seed*phi XOR (i<<8 | t<<4 | a); row = (x_lo32 * s) >> 32
    seed, i, t, a, s = 7, 12345, 3, 1, 600
    key = ((seed * 0x9E3779B97F4A7C15) & ((1 << 64) - 1)) ^ ((i << 8) | (t << 4) | a)
    x = int(hashing.mix64(np.array([key], dtype=np.uint64))[0])
    assert int(hashing.h1(seed, np.array([i]), t, a)[0]) == x
    assert int(hashing.row_of(np.array([x], dtype=np.uint64), s)[0]) == ((x & 0xFFFFFFFF) * s) >> 32
    assert hashing.sign_of(np.array([x], dtype=np.uint64))[0] == (1.0 if x >> 63 == 0 else -1.0)


@pytest.mark.parametrize("seed,s,zeta", [(0, 80, 8), (7, 600, 12), (3, 112, 14)])
def test_distinct_rows_in_range(seed, s, zeta):
    rows, signs = hashing.sparse_sign_indices(seed, 5000, s, zeta)
    assert rows.min() >= 0 and rows.max() < s
    srt = np.sort(rows, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0), "rows of one column must be distinct"
    assert set(np.unique(signs)) <= {-1.0, 1.0}


def test_row_and_sign_uniformity_chi2():
    s, zeta, n = 80, 8, 40000
    rows, signs = hashing.sparse_sign_indices(0, n, s, zeta)
    counts = np.bincount(rows.reshape(-1), minlength=s)
    expct = n * zeta / s
    chi2 = np.sum((counts - expct) ** 2 / expct)
    # 79 degrees of freedom: mean 79, sd ~12.6; 6 sd band
    assert chi2 < 79 + 6 * 12.6
    frac = np.mean(signs > 0)
    assert abs(frac - 0.5) < 6 * 0.5 / np.sqrt(n * zeta)


def test_golden_vectors_match():
    for name, seed, s, zeta in (("h1_seed0_s80_z8.txt", 0, 80, 8), ("h1_seed7_s600_z12.txt", 7, 600, 12)):
        gold = np.loadtxt(os.path.join(GOLDEN, name), dtype=np.int64)
        rows, signs = hashing.sparse_sign_indices(seed, gold.shape[0], s, zeta)
        assert np.array_equal(gold[:, :zeta], rows)
        assert np.array_equal(gold[:, zeta:], signs.astype(np.int64))


def test_sparse_matrix_matches_index_definition():
    # Dense S built entry by entry from the (row, sign) lists.
    seed, n, s, zeta = 5, 300, 40, 6
    rows, signs = hashing.sparse_sign_indices(seed, n, s, zeta)
    Sd = np.zeros((s, n))
    for i in range(n):
        for t in range(zeta):
            Sd[rows[i, t], i] += signs[i, t] / np.sqrt(zeta)
    S = sketch.sparse_sign_matrix(seed, n, s, zeta).toarray()
    assert np.array_equal(S, Sd)
    X = np.random.default_rng(0).standard_normal((n, 3))
    assert np.allclose(sketch.sparse_sign_apply(seed, s, zeta, X), Sd @ X, rtol=0, atol=1e-13)


def test_sparse_sign_is_isometric_in_expectation():
    # With the 1/sqrt(zeta) scale, E||Sx||^2 = ||x||^2 (columns have zeta
    # entries of modulus 1/sqrt(zeta); distinct signs are independent).
    n, s, zeta = 4096, 80, 8
    x = np.random.default_rng(1).standard_normal(n)
    ratios = [np.sum(sketch.sparse_sign_apply(seed, s, zeta, x) ** 2) / np.sum(x ** 2) for seed in range(200)]
    assert abs(np.mean(ratios) - 1.0) < 0.02


def test_default_zeta_natural_log():
    # zeta = ceil(2 log(1+d)): d=40 -> 8 (the small workload's zeta), 300 -> 12,
    # 200 -> 11, 100 -> 10
    assert [hashing.default_zeta(d) for d in (40, 300, 200, 100)] == [8, 12, 11, 10]
