"""GPU parity of restarted sGMRES (Algorithm 1) against the CPU oracle."""
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


def _problem(N, Pe, seed):
    coef = synth.conv_diff_coef(N, Pe)
    return coef, operators.stencil5_matrix(N, N, coef), synth.randn(seed, N * N)


def _relres(A, f, x):
    return np.linalg.norm(f - A @ x) / np.linalg.norm(f)


@pytest.mark.parametrize("kind", ["sparse", "srht"])
def test_small_workload_fp64(skg, kind):
    import torch
    W = synth.WORKLOADS["small"]
    N = W["N"]
    coef, A, f = _problem(N, W["Pe"], W["b_seed"])
    op = skg.Op.stencil5(N, N, coef)
    b = torch.tensor(f, device="cuda")
    sk = lambda M: sketch.apply(kind, 7, W["s"], W["zeta"], M)
    # one cycle from x0 = 0: residual within 1.5x of the oracle's cycle
    x1, info1 = skg.sgmres_solve(op, b, W["d"], W["k"], W["s"], 1e-300, maxit=1, zeta=W["zeta"], seed=7,
                                 sketch=kind)
    xo, _ = krylov.sgmres_cycle(A, f, np.zeros(N * N), W["d"], W["k"], sk)
    r_gpu = _relres(A, f, x1.cpu().numpy())
    r_ora = _relres(A, f, xo)
    assert r_gpu <= 1.5 * r_ora and r_ora <= 1.5 * r_gpu
    assert info1["relres"] == pytest.approx(r_gpu, rel=1e-8)
    # full solve to tol
    x, info = skg.sgmres_solve(op, b, W["d"], W["k"], W["s"], W["tol"], zeta=W["zeta"], seed=7, sketch=kind)
    _, hist, _ = krylov.sgmres(A, f, np.zeros(N * N), W["d"], W["k"], sk, W["tol"])
    rel = _relres(A, f, x.cpu().numpy())
    assert info["status"] == 0
    assert rel <= W["tol"]
    assert rel <= 1.5 * max(hist[-1], 1e-300) or info["cycles"] <= len(hist)
    assert info["cycles"] <= len(hist) + 1


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_small_workload_mixed_precision(skg, dtype):
    # FP32/BF16 basis with FP64 residual and update: restarts act as
    # iterative refinement and still reach 1e-8
    import torch
    W = synth.WORKLOADS["small"]
    N = W["N"]
    coef, A, f = _problem(N, W["Pe"], W["b_seed"])
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    x, info = skg.sgmres_solve(skg.Op.stencil5(N, N, coef), torch.tensor(f, device="cuda"), W["d"], W["k"], W["s"],
                               W["tol"], zeta=W["zeta"], seed=7, basis=tdt)
    assert info["status"] == 0, info
    assert _relres(A, f, x.cpu().numpy()) <= W["tol"]


def test_graph_and_eager_agree(skg):
    import torch
    N = 48
    coef, A, f = _problem(N, 25.0, 3)
    op = skg.Op.stencil5(N, N, coef)
    b = torch.tensor(f, device="cuda")
    xg, ig = skg.sgmres_solve(op, b, 30, 2, 60, 1e-10, use_graph=True)
    xe, ie = skg.sgmres_solve(op, b, 30, 2, 60, 1e-10, use_graph=False)
    assert ig["cycles"] == ie["cycles"]
    assert torch.allclose(xg, xe, rtol=0, atol=1e-12 * xg.abs().max().item())


@pytest.mark.parametrize("dtype,kind,d", [("f64", "sparse", 47), ("f32", "sparse", 75), ("f32", "sparse", 16),
                                          ("bf16", "sparse", 40), ("f64", "srht", 33), ("f32", "sparse", 15)])
def test_pipelined_cycle_equals_sequential(skg, dtype, kind, d):
    # the pipelined cycle (each finished block of 16 basis columns sketched
    # and added to the QR on a second stream while the basis passes go on)
    # performs per column the arithmetic of the one-phase-after-another
    # cycle: the iterates agree bit for bit after every cycle.  Sizes cover a
    # last block of 1 column (d = 16), d < 16, and ragged panels.
    import torch
    N = 96
    coef, A, f = _problem(N, 30.0, 12)
    op = skg.Op.stencil5(N, N, coef)
    b = torch.tensor(f, device="cuda")
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    kw = dict(basis=tdt, sketch=kind, zeta=hashing.default_zeta(d), seed=5)
    xp = xs = None
    for c in range(3):
        xp, ip = skg.sgmres_solve(op, b, d, 2, 2 * d, 1e-300, x0=xp, maxit=1, pipeline=True, **kw)
        xs, is_ = skg.sgmres_solve(op, b, d, 2, 2 * d, 1e-300, x0=xs, maxit=1, pipeline=False, **kw)
        assert torch.equal(xp, xs), (c, float((xp - xs).abs().max()))
        assert ip["relres"] == is_["relres"]


@pytest.mark.parametrize("opts", [dict(basis="f32"), dict(basis="f64", pipeline=False), dict(basis="bf16"),
                                  dict(basis="f32", iter_chunk=16), dict(basis="f32", sketch="srht")])
def test_plan_handle_equals_one_shot_solves(skg, opts):
    # one SgmresPlan (sketch plan, buffers and cycle graph built once)
    # solves several right-hand sides and initial guesses in a row; each
    # solve equals a fresh sgmres_solve bit for bit (x, cycles, residual),
    # including a zero right-hand side and an initial guess that already
    # meets tol (no cycle), and a maxit-limited run that stops unconverged
    import torch
    N = 64
    coef, A, f = _problem(N, 30.0, 12)
    op = skg.Op.stencil5(N, N, coef)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[opts["basis"]]
    kw = dict(opts, basis=tdt, seed=5)
    d, k, s = 40, 2, 80
    rng = np.random.default_rng(7)
    rhs = [torch.tensor(f, device="cuda"), torch.tensor(rng.standard_normal(N * N), device="cuda"),
           torch.zeros(N * N, dtype=torch.float64, device="cuda")]
    plan = skg.SgmresPlan(op, d, k, s, **kw)
    for tol in (1e-8, 1e-10):
        for b in rhs:
            x1, i1 = skg.sgmres_solve(op, b, d, k, s, tol, **kw)
            x2, i2 = plan.solve(b, tol)
            assert torch.equal(x1, x2), (tol, float((x1 - x2).abs().max()))
            assert i1["cycles"] == i2["cycles"] and i1["relres"] == i2["relres"] and i1["status"] == i2["status"]
    # an initial guess that meets tol: no cycle, x returned as given
    xg, _ = skg.sgmres_solve(op, rhs[0], d, k, s, 1e-9, **kw)
    x3, i3 = plan.solve(rhs[0], 1e-6, x0=xg)
    assert i3["cycles"] == 0 and torch.equal(x3, xg)
    # maxit: a plan built for one cycle stops unconverged like sgmres_solve
    short = skg.SgmresPlan(op, d, k, s, **dict(kw, maxit=1))
    x4, i4 = short.solve(rhs[1], 1e-12)
    x5, i5 = skg.sgmres_solve(op, rhs[1], d, k, s, 1e-12, **dict(kw, maxit=1))
    assert i4["status"] == i5["status"] == 5 and torch.equal(x4, x5)


@pytest.mark.parametrize("dtype,d,N", [("f32", 75, 96), ("f64", 40, 96), ("f32", 33, 61)])
def test_pipelined_chebyshev_cycle_equals_sequential(skg, dtype, d, N):
    # the Chebyshev basis in the pipelined cycle: each block's column norms
    # and Hbar columns are finalised on the sketch stream before its sketch;
    # the iterates equal the sequential cycle's bit for bit (N = 61: the
    # scalar recurrence path, 33 columns: a last block of one column)
    import torch
    coef, A, f = _problem(N, 5.0, 3)
    op = skg.Op.stencil5(N, N, coef)
    b = torch.tensor(f, device="cuda")
    tdt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    kw = dict(basis=tdt, zeta=hashing.default_zeta(d), seed=5, cheb=(4.0, 4.0, 1.0))
    xp = xs = None
    for c in range(3):
        xp, ip = skg.sgmres_solve(op, b, d, 2, 2 * d, 1e-300, x0=xp, maxit=1, pipeline=True, **kw)
        xs, is_ = skg.sgmres_solve(op, b, d, 2, 2 * d, 1e-300, x0=xs, maxit=1, pipeline=False, **kw)
        assert torch.equal(xp, xs), (c, float((xp - xs).abs().max()))
        assert ip["relres"] == is_["relres"]


def test_initial_guess_and_zero_rhs(skg):
    import torch
    N = 32
    coef, A, f = _problem(N, 10.0, 4)
    op = skg.Op.stencil5(N, N, coef)
    xs = np.linalg.solve(A.toarray(), f)
    x, info = skg.sgmres_solve(op, torch.tensor(f, device="cuda"), 20, 2, 40, 1e-8,
                               x0=torch.tensor(xs, device="cuda"))
    assert info["cycles"] == 0 and info["relres"] <= 1e-8
    x, info = skg.sgmres_solve(op, torch.zeros(N * N, dtype=torch.float64, device="cuda"), 20, 2, 40, 1e-8)
    assert info["relres"] == 0 and float(x.abs().max()) == 0.0


def test_noconv_returns_best_x(skg):
    import torch
    N = 64
    coef, A, f = _problem(N, 10.0, 0)
    x, info = skg.sgmres_solve(skg.Op.stencil5(N, N, coef), torch.tensor(f, device="cuda"), 10, 2, 20, 1e-12,
                               maxit=3)
    assert info["status"] == 5 and info["cycles"] == 3
    assert _relres(A, f, x.cpu().numpy()) == pytest.approx(info["relres"], rel=1e-8)
    with pytest.raises(skg.SkError):
        skg.sgmres_solve(skg.Op.stencil5(N, N, coef), torch.tensor(f, device="cuda"), 10, 2, 20, 1e-12, maxit=3,
                         raise_on_noconv=True)


def test_exact_when_d_equals_n(skg):
    # full Arnoldi (k = d = n = 16, the largest supported k): one cycle solves
    import torch
    N = 4
    coef, A, f = _problem(N, 10.0, 0)
    n = N * N
    x, info = skg.sgmres_solve(skg.Op.stencil5(N, N, coef), torch.tensor(f, device="cuda"), n, n, 2 * n, 1e-300,
                               maxit=1, zeta=hashing.default_zeta(n))
    kA = np.linalg.cond(A.toarray())
    assert _relres(A, f, x.cpu().numpy()) <= 1e-10 * kA


def test_ragged_medium_size(skg):
    # n = 200*157 (not a multiple of the 2048-row chunk), FP32 basis
    import torch
    nx, ny = 200, 157
    coef = synth.conv_diff_coef(200, 40.0)
    A = operators.stencil5_matrix(nx, ny, coef)
    f = synth.randn(5, nx * ny)
    x, info = skg.sgmres_solve(skg.Op.stencil5(nx, ny, coef), torch.tensor(f, device="cuda"), 60, 2, 120, 1e-6,
                               basis=torch.float32)
    assert info["status"] == 0
    assert _relres(A, f, x.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("dtype,kind", [("f64", "sparse"), ("f32", "sparse"), ("bf16", "sparse"), ("f64", "srht")])
def test_scale_workload_full_size(skg, dtype, kind):
    # the benchmark configuration: 1024^2 convection-diffusion, Pe=50,
    # d=300, k=2, s=600, zeta=12, tol 1e-6.  The FP64 residual of the
    # returned x, recomputed on the CPU from the assembled oracle matrix, is
    # <= tol.  Against the FP64 oracle's run of the same workload and sketch
    # (tests/golden/scale_oracle.json and scale_srht_oracle.json, written by
    # make_scale_reference.py from the oracle only):
    #   FP64 basis: the same number of restarts (+-1) and a final residual
    #     within 1.5x of the oracle's after as many cycles;
    #   FP32 basis: within the oracle's cycles + 2;
    #   BF16 basis: converges (its kappa(T) threshold of 1e2 truncates every
    #     cycle's triangle, so each refinement step gains less).
    import json
    import os
    import torch
    W = synth.WORKLOADS["scale"]
    N = W["N"]
    coef, A, f = _problem(N, W["Pe"], W["b_seed"])
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    maxit = 400 if dtype == "bf16" else 100
    x, info = skg.sgmres_solve(skg.Op.stencil5(N, N, coef), torch.tensor(f, device="cuda"), W["d"], W["k"], W["s"],
                               W["tol"], zeta=W["zeta"], seed=7, basis=tdt, sketch=kind, maxit=maxit)
    assert info["status"] == 0, info
    rel = _relres(A, f, x.cpu().numpy())
    assert rel <= W["tol"]
    name = "scale_oracle.json" if kind == "sparse" else "scale_srht_oracle.json"
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        ref = json.load(fh)
    assert ref["relres"][-1] <= W["tol"]
    if dtype == "f64":
        assert abs(info["cycles"] - ref["cycles"]) <= 1, (info["cycles"], ref["cycles"])
        c = min(info["cycles"], len(ref["relres"])) - 1
        assert rel <= 1.5 * ref["relres"][c]
    elif dtype == "f32":
        assert info["cycles"] <= ref["cycles"] + 2, (info["cycles"], ref["cycles"])


def test_maximum_basis_size_one_cycle(skg):
    # the largest basis sgmres_solve accepts (d = 768: the LS solve keeps
    # 33 d doubles in shared memory) with s = 2d = 1536 rows (beyond the
    # row-owner gather: the general gather kernel), FP64.  At this size the
    # k = 2 basis reaches kappa ~ 1e16, so both sides truncate the triangle,
    # each with its own kappa estimate (exact kappa_2 in the oracle, the
    # diagonal ratio on the GPU): both must solve the system in one cycle.
    import torch
    N, d, k, s = 96, 768, 2, 1536
    coef, A, f = _problem(N, 20.0, 6)
    zeta = hashing.default_zeta(d)
    op = skg.Op.stencil5(N, N, coef)
    x1, info = skg.sgmres_solve(op, torch.tensor(f, device="cuda"), d, k, s, 1e-300, maxit=1, zeta=zeta, seed=7)
    sk = lambda M: sketch.sparse_sign_apply(7, s, zeta, M)
    xo, oinfo = krylov.sgmres_cycle(A, f, np.zeros(N * N), d, k, sk)
    r_gpu = _relres(A, f, x1.cpu().numpy())
    r_ora = _relres(A, f, xo)
    assert info["d_used"] == oinfo["d_used"] == d
    assert r_ora <= 1e-9
    assert r_gpu <= max(1.5 * r_ora, 1e-9), (r_gpu, r_ora, info["width"], oinfo["width"])
    with pytest.raises(skg.SkError):
        skg.sgmres_solve(op, torch.tensor(f, device="cuda"), d + 1, k, 2 * d + 2, 1e-8, maxit=1)


def test_csr_operator_fp64_cycle_and_fp32_solve(skg):
    # a general sparse (CSR) nonsymmetric operator: the convection-diffusion
    # matrix plus a random sparse perturbation (scalar path of every pass).
    # FP64: one cycle within 1.5x of the oracle's; FP32 basis: converges to 1e-8.
    import scipy.sparse as sp
    import torch
    N, d, k, s = 48, 40, 2, 80
    coef, A0, f = _problem(N, 15.0, 9)
    P = sp.random(N * N, N * N, density=2e-4, random_state=3, format="csr")
    A = (A0 + 0.05 * P).tocsr()
    rp, ci, va = operators.csr_from_scipy(A)
    op = skg.Op.csr(torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"),
                    torch.tensor(va, device="cuda"))
    zeta = hashing.default_zeta(d)
    b = torch.tensor(f, device="cuda")
    x1, info = skg.sgmres_solve(op, b, d, k, s, 1e-300, maxit=1, zeta=zeta, seed=7)
    xo, _ = krylov.sgmres_cycle(A, f, np.zeros(N * N), d, k, lambda M: sketch.sparse_sign_apply(7, s, zeta, M))
    r_gpu, r_ora = _relres(A, f, x1.cpu().numpy()), _relres(A, f, xo)
    assert r_gpu <= 1.5 * r_ora and r_ora <= 1.5 * r_gpu, (r_gpu, r_ora)
    x, info = skg.sgmres_solve(op, b, d, k, s, 1e-8, zeta=zeta, seed=7, basis=torch.float32, maxit=500)
    assert info["status"] == 0, info
    assert _relres(A, f, x.cpu().numpy()) <= 1e-8
