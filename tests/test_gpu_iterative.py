"""GPU iterative sGMRES (§5.2: chunked basis, QR grown by the new columns,
stop at the first prefix whose estimate meets the target; §5.3 restart on
the kappa estimate) against the CPU oracle and against Algorithm 1."""
import numpy as np
import pytest

import synth
from oracle import hashing, krylov, operators, sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def skg():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    import paper_2111_00113_gb300 as m
    return m


def _relres(A, f, x):
    return np.linalg.norm(f - A @ x) / np.linalg.norm(f)


def _small():
    W = synth.WORKLOADS["small"]
    N = W["N"]
    coef = synth.conv_diff_coef(N, W["Pe"])
    return W, coef, operators.stencil5_matrix(N, N, coef), synth.randn(W["b_seed"], N * N)


def test_matches_oracle_cycle_by_cycle(skg):
    # small workload, s = 2(d+1) as in §5.2, chunks of 16 (40 = 16 + 16 + 8:
    # a partial last panel).  Per cycle: the prefix used equals the oracle's
    # (within one column: FP64 estimates in another summation order), the
    # residual within 1.5x while above tol; the last cycle meets tol.
    import torch
    W, coef, A, f = _small()
    N, d, k, tol = W["N"], W["d"], W["k"], W["tol"]
    s, zeta = 2 * (d + 1), hashing.default_zeta(d)
    sk = lambda M: sketch.sparse_sign_apply(7, s, zeta, M)
    _, hist, infos = krylov.sgmres_iterative(A, f, np.zeros(N * N), d, k, sk, tol, maxit=60)
    assert infos[-1]["j"] < d
    op = skg.Op.stencil5(N, N, coef)
    b = torch.tensor(f, device="cuda")
    x = torch.zeros_like(b)
    for c, (h, io) in enumerate(zip(hist, infos)):
        x, info = skg.sgmres_solve(op, b, d, k, s, tol, x0=x, maxit=1, zeta=zeta, seed=7, iter_chunk=16)
        rel = _relres(A, f, x.cpu().numpy())
        assert abs(info["d_used"] - io["j"]) <= 1, (c, info["d_used"], io["j"])
        if c < len(hist) - 1:
            assert rel <= 1.5 * h and h <= 1.5 * rel, (c, rel, h)
        else:
            assert rel <= tol and info["status"] == 0
    # one call: the same number of cycles, and fewer columns in the last
    x, info = skg.sgmres_solve(op, b, d, k, s, tol, zeta=zeta, seed=7, iter_chunk=16)
    assert info["status"] == 0 and abs(info["cycles"] - len(hist)) <= 1
    assert info["d_used"] < d
    assert _relres(A, f, x.cpu().numpy()) <= tol


@pytest.mark.parametrize("chunk", [16, 32, 48])
def test_without_early_stop_equals_algorithm_1(skg, chunk):
    # target unreachable in one cycle: every chunk runs and the QR grown
    # column block by column block is the one-shot QR (same reflectors, same
    # order); only the sketch's partial-sum grouping differs
    import torch
    W, coef, A, f = _small()
    N, d, k, s = W["N"], W["d"], W["k"], W["s"]
    op = skg.Op.stencil5(N, N, coef)
    b = torch.tensor(f, device="cuda")
    x1, i1 = skg.sgmres_solve(op, b, d, k, s, 1e-300, maxit=1, zeta=W["zeta"], seed=7)
    x2, i2 = skg.sgmres_solve(op, b, d, k, s, 1e-300, maxit=1, zeta=W["zeta"], seed=7, iter_chunk=chunk)
    assert i2["d_used"] == d and i2["width"] == i1["width"] == d
    assert i2["rhat_est"] == pytest.approx(i1["rhat_est"], rel=1e-9)
    assert torch.allclose(x1, x2, rtol=1e-9, atol=1e-12 * float(x1.abs().max()))


def test_kappa_restart_matches_truncated_solve(skg):
    # a small stab_tol: the kappa estimate (max/min |r_jj| over the prefix)
    # trips inside the cycle; the iterative cycle ends at that chunk and its
    # solve keeps the same leading block as Algorithm 1's kappa truncation.
    # The expected block comes from the oracle's triangle: on this workload
    # the prefix ratio jumps from 2.64 (25 columns) to 3.23 (26 columns), so
    # stab_tol = 2.9 keeps 25 columns, across the first chunk boundary.
    import torch
    W, coef, A, f = _small()
    N, d, k, s = W["N"], W["d"], W["k"], W["s"]
    B, M, _, _ = krylov.trunc_arnoldi(A, f, d, k)
    _, T = krylov.householder_qr(sketch.sparse_sign_apply(7, s, W["zeta"], M))
    dg = np.abs(np.diag(T))
    ratio = np.array([dg[:j].max() / dg[:j].min() for j in range(1, d + 1)])
    stab = 2.9
    w_ref = int(np.argmax(ratio > stab))
    assert w_ref == 25 and ratio[w_ref - 1] < 0.95 * stab and ratio[w_ref] > 1.05 * stab
    op = skg.Op.stencil5(N, N, coef)
    b = torch.tensor(f, device="cuda")
    kw = dict(maxit=1, zeta=W["zeta"], seed=7, stab_tol=stab)
    x1, i1 = skg.sgmres_solve(op, b, d, k, s, 1e-300, **kw)
    x2, i2 = skg.sgmres_solve(op, b, d, k, s, 1e-300, iter_chunk=16, **kw)
    assert i1["width"] == w_ref
    assert i2["width"] == i1["width"]
    assert i2["d_used"] <= ((i1["width"] + 1 + 15) // 16) * 16
    assert torch.allclose(x1, x2, rtol=1e-9, atol=1e-12 * float(x1.abs().max()))


def test_breakdown_gives_exact_solution(skg):
    # A with 5 distinct eigenvalues (diagonal stencil): the minimal polynomial
    # has degree 5, the recurrence (k = 16 >= 5) breaks down after b_5, and
    # the prefix j = 5 solves exactly, as in the oracle
    import torch
    n, d = 200, 40
    diag = np.repeat([1.0, 2.5, 4.0, 7.0, 9.5], n // 5)
    op = skg.Op.stencil5(n, 1, (0, 0, 0, 0, 0), torch.tensor(diag, device="cuda"))
    f = synth.randn(13, n)
    s, zeta = 2 * (d + 1), hashing.default_zeta(d)
    sk = lambda M: sketch.sparse_sign_apply(3, s, zeta, M)
    xo, io = krylov.sgmres_iterative_cycle(np.diag(diag), f, np.zeros(n), d, 16, sk, 1e-10)
    assert io["j"] == 5
    x, info = skg.sgmres_solve(op, torch.tensor(f, device="cuda"), d, 16, s, 1e-10, maxit=1, zeta=zeta, seed=3,
                               iter_chunk=16)
    assert info["status"] == 0 and info["width"] == 5
    assert np.allclose(x.cpu().numpy(), f / diag, atol=1e-11)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_low_precision_basis_converges(skg, dtype):
    # FP32/BF16 basis, FP64 residual and update: the early stop asks each
    # cycle for the reduction still needed; restarts refine to 1e-8
    import torch
    W, coef, A, f = _small()
    N, d, k = W["N"], W["d"], W["k"]
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    x, info = skg.sgmres_solve(skg.Op.stencil5(N, N, coef), torch.tensor(f, device="cuda"), d, k, 2 * (d + 1),
                               W["tol"], basis=tdt, maxit=500, iter_chunk=16)
    assert info["status"] == 0, info
    assert _relres(A, f, x.cpu().numpy()) <= W["tol"]


def test_batched_matches_single_solves(skg):
    import torch
    ops, bs, As = [], [], []
    for i, N in enumerate((40, 36, 64)):
        coef = synth.conv_diff_coef(N, 10.0)
        ops.append(skg.Op.stencil5(N, N, coef))
        As.append(operators.stencil5_matrix(N, N, coef))
        bs.append([torch.tensor(synth.randn(30 + i, N * N), device="cuda")])
    kw = dict(maxit=200, iter_chunk=16)
    xs, stat, info = skg.sgmres_solve_batched(ops, bs, 40, 2, 82, 1e-8, **kw)
    assert all(st == 0 for st in stat)
    for i in range(3):
        x, _ = skg.sgmres_solve(ops[i], bs[i][0], 40, 2, 82, 1e-8, **kw)
        assert torch.equal(x, xs[i][0])
        assert _relres(As[i], bs[i][0].cpu().numpy(), x.cpu().numpy()) <= 1e-8
