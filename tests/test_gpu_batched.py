"""GPU batched sGMRES: independent jobs of uneven size."""
import numpy as np
import pytest

import synth
from oracle import operators

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def skg():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    import paper_2111_00113_gb300 as m
    return m


def _rel(A, f, x):
    return np.linalg.norm(f - A @ x) / np.linalg.norm(f)


@pytest.mark.parametrize("dtype,mode,elems", [("f64", "workers", 0), ("f32", "workers", 0),
                                              ("f64", "grouped", 0), ("f32", "grouped", 0),
                                              ("f32", "grouped", 5000)])
def test_batched_equals_single_solves(skg, dtype, mode, elems):
    # every job of the batch runs the same kernel bodies with the same block
    # shapes as a single solve: the solutions agree bit for bit, and all
    # reach tol.  Grouped: every launch serves all resident jobs (jobs of
    # 24^2 .. 64^2 cells, the three stencil paths mixed); elems =
    # 5000 admits one or two jobs at a time, so jobs start at different
    # cycles of the batch.
    import torch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    sides = [24, 64, 34, 33, 48]   # 34: the vector path across grid rows; 33: the scalar path
    pes = [5.0, 40.0, 80.0, 20.0, 10.0]
    ops, bs, mats, fs = [], [], [], []
    for i, (N, Pe) in enumerate(zip(sides, pes)):
        coef = synth.conv_diff_coef(N, Pe)
        ops.append(skg.Op.stencil5(N, N, coef))
        mats.append(operators.stencil5_matrix(N, N, coef))
        f = [synth.randn(synth.batch_rhs_seed(i, r), N * N) for r in range(2)]
        fs.append(f)
        bs.append([torch.tensor(v, device="cuda") for v in f])
    d, k, s, tol = 30, 2, 60, 1e-8
    xs, stat, info = skg.sgmres_solve_batched(ops, bs, d, k, s, tol, basis=tdt, batch_workers=3, batch_mode=mode,
                                              batch_elems=elems)
    assert all(st == 0 for st in stat), stat
    for i in range(len(ops)):
        for r in range(2):
            x1, i1 = skg.sgmres_solve(ops[i], bs[i][r], d, k, s, tol, basis=tdt)
            assert torch.equal(x1, xs[i][r])
            assert _rel(mats[i], fs[i][r], xs[i][r].cpu().numpy()) <= tol
            ji = info["jobs"][i * 2 + r]
            assert ji["cycles"] == i1["cycles"] and ji["relres"] == i1["relres"]
            assert ji["width"] == i1["width"] and ji["d_used"] == i1["d_used"]
    assert info["relres"] <= tol
    if mode == "grouped" and elems == 0:
        # all ten jobs resident: one launch per phase serves them all, far
        # fewer launches than the jobs' (shared) launches summed
        assert info["launches"] < 0.5 * sum(j["launches"] for j in info["jobs"])


def test_grouped_edge_jobs(skg):
    # one grouped batch holding: a zero right-hand side (x = 0 at once, no
    # cycle), a job whose initial guess already meets tol (no cycle), jobs
    # stopped by maxit (ENOCONV, the cycles' x kept), and a CSR operator next
    # to stencils; each job's status, x and diagnostics equal a single solve's
    import torch
    N = 32
    coef = synth.conv_diff_coef(N, 30.0)
    A = operators.stencil5_matrix(N, N, coef).tocsr()
    st_op = skg.Op.stencil5(N, N, coef)
    csr_op = skg.Op.csr(torch.tensor(A.indptr, dtype=torch.int32, device="cuda"),
                        torch.tensor(A.indices, dtype=torch.int32, device="cuda"),
                        torch.tensor(A.data, dtype=torch.float64, device="cuda"))
    f = torch.tensor(synth.randn(11, N * N), device="cuda")
    xs_exact = torch.tensor(np.linalg.solve(A.toarray(), f.cpu().numpy()), device="cuda")
    ops = [st_op, csr_op, st_op]
    bs = [[torch.zeros(N * N, dtype=torch.float64, device="cuda"), f], [f, f], [f, f]]
    x0s = [[torch.zeros_like(f), torch.zeros_like(f)], [xs_exact, torch.zeros_like(f)],
           [torch.zeros_like(f), torch.zeros_like(f)]]
    d, k, s, tol = 20, 2, 40, 1e-9
    for basis in (torch.float64, torch.float32):
        for maxit in (2, 10000):
            xs, stat, info = skg.sgmres_solve_batched(ops, bs, d, k, s, tol, x0s=x0s, basis=basis, maxit=maxit,
                                                      batch_mode="grouped")
            for i in range(3):
                for r in range(2):
                    j = i * 2 + r
                    x1, i1 = skg.sgmres_solve(ops[i], bs[i][r], d, k, s, tol, x0=x0s[i][r].clone(), basis=basis,
                                              maxit=maxit)
                    assert stat[j] == i1["status"], (i, r, maxit, stat[j], i1["status"])
                    assert torch.equal(x1, xs[i][r]), (i, r, maxit)
                    assert info["jobs"][j]["cycles"] == i1["cycles"]
            assert stat[0] == 0 and info["jobs"][0]["cycles"] == 0 and torch.count_nonzero(xs[0][0]) == 0
            assert stat[2] == 0 and info["jobs"][2]["cycles"] == 0
            if maxit == 2:
                assert stat[1] == 5 and info["jobs"][1]["cycles"] == 2


def test_batched_workload_full(skg):
    # 256 systems, side ~ U{128..512}, Pe ~ U(1,100) (seed 4), 4 right-hand
    # sides each; d = 100, k = 2, s = 200; FP32 basis with FP64 refinement
    # to 1e-6, at most 500 restarts.  A few jobs stagnate (restarted
    # GMRES(100) does so in FP64 as well, near 5e-3): they return ENOCONV
    # with their best x.  The FP64 residual of a sample of converged jobs is
    # recomputed on the CPU.
    import torch
    W = synth.WORKLOADS["batched"]
    sides, pes = synth.batch_systems(W["seed"], W["nsys"])
    ops, bs = [], []
    for i in range(W["nsys"]):
        N = int(sides[i])
        ops.append(skg.Op.stencil5(N, N, synth.conv_diff_coef(N, pes[i])))
        g = torch.Generator(device="cuda").manual_seed(synth.batch_rhs_seed(i, 0))
        bs.append([torch.randn(N * N, generator=g, dtype=torch.float64, device="cuda") for r in range(W["nrhs"])])
    xs, stat, info = skg.sgmres_solve_batched(ops, bs, W["d"], W["k"], W["s"], W["tol"], zeta=W["zeta"],
                                              basis=torch.float32, batch_workers=16, maxit=500)
    ok = [st == 0 for st in stat]
    assert sum(ok) >= 0.99 * len(stat)
    assert all(st in (0, 5) for st in stat)
    checked = 0
    for i in (0, 17, 128, 200, 255):
        N = int(sides[i])
        A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, pes[i]))
        for r in (0, 3):
            rel = _rel(A, bs[i][r].cpu().numpy(), xs[i][r].cpu().numpy())
            if ok[i * W["nrhs"] + r]:
                assert rel <= W["tol"]
                checked += 1
            else:
                assert rel < 0.1
    assert checked >= 8


def _batched_golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "batched_oracle.json")) as fh:
        return json.load(fh)


def test_batched_jobs_match_oracle_history(skg):
    # jobs of the batched workload of different sizes (129^2 .. 485^2), one
    # right-hand side each drawn on the host, FP64 basis, the oracle's sketch;
    # tests/golden/batched_oracle.json holds the FP64 oracle's residual after
    # every cycle (written by make_batched_reference.py from the oracle only).
    # Cycle by cycle (restarting from the returned x is the next cycle of
    # the same run): each job's residual within 1.5x of the oracle's; then
    # the uninterrupted batched solve: cycles within +-1 of the oracle's and
    # the final residual within 1.5x of the oracle's at that cycle.  FP32
    # basis: every job reaches tol within the oracle's cycles + 2.
    import torch
    ref = _batched_golden()
    W = synth.WORKLOADS["batched"]
    sides, pes = synth.batch_systems(W["seed"], W["nsys"])
    ops, bs, mats, fs, hist = [], [], [], [], []
    for job in ref["jobs"]:
        i = job["system"]
        N = int(sides[i])
        assert N == job["N"]
        coef = synth.conv_diff_coef(N, pes[i])
        ops.append(skg.Op.stencil5(N, N, coef))
        mats.append(operators.stencil5_matrix(N, N, coef))
        f = synth.randn(synth.batch_rhs_seed(i, 0), N * N)
        fs.append(f)
        bs.append([torch.tensor(f, device="cuda")])
        hist.append(job["relres"])
    kw = dict(zeta=W["zeta"], seed=7, basis=torch.float64)
    d, k, s = W["d"], W["k"], W["s"]
    xs = None
    for c in range(max(len(h) for h in hist)):
        xs, stat, _ = skg.sgmres_solve_batched(ops, bs, d, k, s, 1e-300, x0s=xs, maxit=1, batch_workers=3, **kw)
        for j in range(len(ops)):
            if c < len(hist[j]):
                rel = _rel(mats[j], fs[j], xs[j][0].cpu().numpy())
                assert rel <= 1.5 * hist[j][c] and hist[j][c] <= 1.5 * rel, (j, c, rel, hist[j][c])
    xs, stat, info = skg.sgmres_solve_batched(ops, bs, d, k, s, W["tol"], batch_workers=3, **kw)
    assert all(st == 0 for st in stat), stat
    for j, ji in enumerate(info["jobs"]):
        assert abs(ji["cycles"] - len(hist[j])) <= 1, (j, ji["cycles"], len(hist[j]))
        rel = _rel(mats[j], fs[j], xs[j][0].cpu().numpy())
        assert rel <= W["tol"]
        assert rel <= 1.5 * hist[j][min(ji["cycles"], len(hist[j])) - 1]
        assert ji["relres"] == pytest.approx(rel, rel=1e-6)
    xs, stat, info = skg.sgmres_solve_batched(ops, bs, d, k, s, W["tol"], batch_workers=3,
                                              **dict(kw, basis=torch.float32))
    assert all(st == 0 for st in stat), stat
    for j, ji in enumerate(info["jobs"]):
        assert ji["cycles"] <= len(hist[j]) + 2, (j, ji["cycles"], len(hist[j]))
        assert _rel(mats[j], fs[j], xs[j][0].cpu().numpy()) <= W["tol"]
