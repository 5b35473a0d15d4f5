"""Rounding sensitivity of the full-size Laplacian workload (stored values).

The oracle run of make_laplace_reference.py repeated with its sketches
perturbed at the level of rounding: every entry is multiplied by
(1 + 1e-15 z_i), z ~ N(0,1) from numpy's PCG64 with the run's seed, as a
different summation order of the sketch would do.  Seeds 101-104 perturb
g = S r only; seeds 201-204 perturb every sketch (g and S A B).  Each cycle
gains only 10-20 % on this singular, consistent problem, so such
differences compound; the spread of the perturbed runs' histories is the
band any correct implementation of Algorithm 1 can land in.

Writes tests/golden/laplace_spread.json with one residual history per seed.
Each run takes several minutes (single-threaded numpy/scipy); the seeds run
in parallel processes:
    OPENBLAS_NUM_THREADS=1 python tests/golden/make_laplace_spread.py
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

SEEDS = (101, 102, 103, 104, 201, 202, 203, 204)
REL = 1e-15


def run(seed):
    W = synth.WORKLOADS["laplace"]
    N = W["N"]
    A = operators.neumann_laplacian_matrix(N, N)
    f = A @ synth.grf(W["x_seed"], N, W["ell"])
    S = sketch.sparse_sign_matrix(7, N * N, W["s"], W["zeta"])
    rng = np.random.default_rng(seed)

    def sk(M):
        out = S @ M
        if out.ndim == 1 or seed >= 200:
            out = out * (1.0 + REL * rng.standard_normal(out.shape))
        return out

    x = np.zeros(N * N)
    fn = np.linalg.norm(f)
    hist = []
    while True:
        x, _ = krylov.sgmres_cycle(A, f, x, W["d"], W["k"], sk, cheb=W["cheb"])
        hist.append(float(np.linalg.norm(f - A @ x) / fn))
        print(seed, len(hist), hist[-1], flush=True)
        if hist[-1] <= W["tol"] or len(hist) >= 80:
            break
    return seed, hist


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(4) as pool:
        res = pool.map(run, SEEDS)
    out = dict(workload="laplace",
               perturbation="sketch entries times (1 + %g z), z ~ N(0,1): g = S r only (seeds 1xx), every "
                            "sketch (seeds 2xx)" % REL,
               runs={str(s): h for s, h in res}, cycles={str(s): len(h) for s, h in res})
    with open(os.path.join(HERE, "laplace_spread.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
