"""Oracle reference runs of jobs from the batched workload (stored values).

The batched workload: 256 convection-diffusion systems, side ~ U{128..512},
Pe ~ U(1,100) (seed 4), d = 100, k = 2, s = 200, zeta = 10, sparse sign
sketch seed 7, tol 1e-6.  For the systems in JOBS (spread over the size
range), right-hand side r = 0 drawn on the host as N(0,1) with seed
1000 + 4 i, x0 = 0, the plain FP64 oracle (Algorithm 1 restarted, §3.5)
records the relative residual after every cycle.

Writes tests/golden/batched_oracle.json.  Runs the jobs in parallel
processes (a few minutes):
    OPENBLAS_NUM_THREADS=1 python tests/golden/make_batched_reference.py
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import krylov, operators, sketch  # noqa: E402

JOBS = (196, 102, 228, 204, 236, 30)
MAXIT = 150


def run(i):
    W = synth.WORKLOADS["batched"]
    sides, pes = synth.batch_systems(W["seed"], W["nsys"])
    N = int(sides[i])
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, pes[i]))
    f = synth.randn(synth.batch_rhs_seed(i, 0), N * N)
    S = sketch.sparse_sign_matrix(7, N * N, W["s"], W["zeta"])
    _, hist, _ = krylov.sgmres(A, f, np.zeros(N * N), W["d"], W["k"], lambda M: S @ M, W["tol"], maxit=MAXIT)
    print(i, N, len(hist), hist[-1], flush=True)
    return dict(system=i, N=N, Pe=float(pes[i]), relres=[float(v) for v in hist], cycles=len(hist))


def main():
    W = synth.WORKLOADS["batched"]
    ctx = mp.get_context("spawn")
    with ctx.Pool(3) as pool:
        res = pool.map(run, JOBS)
    out = dict(workload="batched", d=W["d"], k=W["k"], s=W["s"], zeta=W["zeta"], seed=7, tol=W["tol"],
               rhs="synth.randn(synth.batch_rhs_seed(i, 0), N*N)", maxit=MAXIT, jobs=res)
    with open(os.path.join(HERE, "batched_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
