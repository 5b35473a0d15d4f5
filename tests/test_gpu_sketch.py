"""GPU parity of sketch_apply (sparse sign and SRHT) against the CPU oracle."""
import numpy as np
import pytest

import synth
from oracle import hashing, sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def skg():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    import paper_2111_00113_gb300 as m
    return m


def _relf(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _tensor(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a.T), dtype=dtype, device="cuda").t()


def test_sparse_sign_indices_bit_exact(skg):
    # S e_i is column i of S: +-1/sqrt(zeta) at the hashed rows, exactly.
    import torch
    for seed, n, s, zeta in ((0, 4096, 80, 8), (7, 5000, 600, 12), (3, 100, 40, 14)):
        cols = np.unique(np.concatenate([np.arange(0, min(n, 70)), np.linspace(0, n - 1, 30).astype(int)]))
        E = np.zeros((n, cols.size))
        E[cols, np.arange(cols.size)] = 1.0
        got = skg.sketch_apply(_tensor(E, torch.float64), s, zeta, seed).cpu().numpy()
        S = sketch.sparse_sign_matrix(seed, n, s, zeta).toarray()
        assert np.array_equal(got, S[:, cols]), (seed, n, s, zeta)


@pytest.mark.parametrize("n,c,s,zeta", [(4096, 41, 80, 8), (2048 * 3 + 17, 9, 600, 12), (77, 1, 16, 3),
                                        (100003, 3, 200, 10), (1024 * 5 + 3, 1, 600, 12), (1024 * 9, 1, 640, 14)])
def test_sparse_sign_fp64(skg, n, c, s, zeta):
    import torch
    X = np.random.default_rng(n).standard_normal((n, c))
    got = skg.sketch_apply(_tensor(X, torch.float64), s, zeta, 11).cpu().numpy()
    ref = sketch.sparse_sign_apply(11, s, zeta, X)
    assert _relf(got, ref) <= 1e-12


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_sparse_sign_low_precision(skg, dtype):
    import torch
    n, c, s, zeta = 2048 * 5 + 3, 10, 600, 12
    X = np.random.default_rng(1).standard_normal((n, c))
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    Xt = _tensor(X, tdt)
    Xr = Xt.to(torch.float64).cpu().numpy()  # the values the GPU actually holds
    got = skg.sketch_apply(Xt, s, zeta, 5).cpu().numpy()
    ref = sketch.sparse_sign_apply(5, s, zeta, Xr)
    assert _relf(got, ref) <= 1e-5


@pytest.mark.parametrize("n,c,s,zeta", [(1024 * 5 + 3, 37, 600, 12), (1024 * 40 + 1000, 16, 33, 5),
                                        (1000, 20, 640, 14), (1024 * 3, 301, 200, 10)])
def test_sparse_sign_fp32_row_owner(skg, n, c, s, zeta):
    # FP32 data with at least 16 columns and s <= 640 (the row-owner gather):
    # ragged last chunk, ragged last column tile, partial last warp of rows
    import torch
    X = np.random.default_rng(n + c).standard_normal((n, c))
    Xt = _tensor(X, torch.float32)
    Xr = Xt.to(torch.float64).cpu().numpy()
    got = skg.sketch_apply(Xt, s, zeta, 3).cpu().numpy()
    ref = sketch.sparse_sign_apply(3, s, zeta, Xr)
    assert _relf(got, ref) <= 1e-6


def test_sparse_sign_vector_and_strided(skg):
    import torch
    n = 3000
    x = np.random.default_rng(2).standard_normal(n)
    got = skg.sketch_apply(torch.tensor(x, device="cuda"), 80, 8, 0).cpu().numpy()
    assert _relf(got, sketch.sparse_sign_apply(0, 80, 8, x)) <= 1e-12
    # leading dimension larger than n
    big = torch.zeros((4, n + 64), dtype=torch.float64, device="cuda")
    X = np.random.default_rng(3).standard_normal((n, 4))
    big[:, :n] = torch.tensor(X.T, device="cuda")
    Bv = big.t()[:n]
    assert Bv.stride(0) == 1 and Bv.stride(1) == n + 64
    got = skg.sketch_apply(Bv, 80, 8, 0).cpu().numpy()
    assert _relf(got, sketch.sparse_sign_apply(0, 80, 8, X)) <= 1e-12


@pytest.mark.parametrize("n,c,s", [(4096, 3, 80), (5000, 2, 100), (1 << 14, 1, 64), (33, 4, 16)])
def test_srht_fp64(skg, n, c, s):
    import torch
    X = np.random.default_rng(n + c).standard_normal((n, c))
    got = skg.sketch_apply(_tensor(X, torch.float64), s, 0, 9, kind="srht").cpu().numpy()
    ref = sketch.srht_apply(9, s, X)
    assert _relf(got, ref) <= 1e-12


def test_srht_fp32(skg):
    import torch
    n, c, s = 70000, 3, 200
    X = np.random.default_rng(8).standard_normal((n, c))
    Xt = _tensor(X, torch.float32)
    got = skg.sketch_apply(Xt, s, 0, 4, kind="srht").cpu().numpy()
    ref = sketch.srht_apply(4, s, Xt.to(torch.float64).cpu().numpy())
    assert _relf(got, ref) <= 1e-5


def test_full_size_sketch_sampled(skg):
    # the benchmark's sketch shape: n = 2^20, 301 columns, s = 600, zeta = 12,
    # FP32; checked on sampled columns computed one by one by the oracle.
    import torch
    n, c, s, zeta = 1 << 20, 301, 600, 12
    g = torch.Generator(device="cuda").manual_seed(0)
    Xt = torch.randn((c, n), generator=g, device="cuda", dtype=torch.float32).t()
    got = skg.sketch_apply(Xt, s, zeta, 7)
    S = sketch.sparse_sign_matrix(7, n, s, zeta)
    for j in (0, 150, 300):
        col = Xt[:, j].to(torch.float64).cpu().numpy()
        ref = S @ col
        assert _relf(got[:, j].cpu().numpy(), ref) <= 1e-5


def test_sparse_sign_single_column_unaligned(skg):
    # one FP64 column that does not start on a 16-byte boundary (a view at
    # offset 1) and has an odd length: the staging falls back to 8-byte copies
    import torch
    n, s, zeta = 1024 * 3 + 5, 300, 10
    X = np.random.default_rng(3).standard_normal(n + 1)
    Xt = torch.tensor(X, device="cuda")[1:]
    got = skg.sketch_apply(Xt, s, zeta, 4).cpu().numpy()
    ref = sketch.sparse_sign_apply(4, s, zeta, X[1:, None])[:, 0]
    assert _relf(got, ref) <= 1e-12


@pytest.mark.parametrize("kind", ["sparse", "srht"])
def test_sketch_plan_reused_across_calls(skg, kind):
    # one plan applied to blocks of different widths and types (its
    # workspace grows on the wider ones): each result is the oracle's sketch
    # of the values the GPU holds, as sketch_apply gives it
    import torch
    n, s, zeta, seed = 1024 * 6 + 77, 300, 10, 4
    plan = skg.SketchPlan(n, s, zeta, seed, kind=kind)
    rng = np.random.default_rng(3)
    for c, dt, tol in ((3, torch.float64, 1e-12), (40, torch.float32, 1e-5), (1, torch.float64, 1e-12),
                       (17, torch.bfloat16, 1e-5), (3, torch.float64, 1e-12)):
        X = rng.standard_normal((n, c))
        Xt = _tensor(X, dt)
        held = Xt.to(torch.float64).cpu().numpy()
        got = plan(Xt).cpu().numpy()
        ref = sketch.apply(kind, seed, s, zeta, held)
        assert _relf(got, ref) <= tol, (c, dt)
        assert _relf(got, skg.sketch_apply(Xt, s, zeta, seed, kind=kind).cpu().numpy()) <= tol
