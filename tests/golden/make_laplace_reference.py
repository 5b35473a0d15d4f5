"""Oracle reference run of the full-size Laplacian workload with the
Chebyshev basis (stored expected values).

1024 x 1024 Neumann Laplacian, f = A x_true with x_true = GRF(seed 5,
length 64 cells), x0 = 0, d = 300, s = 600, zeta = 12, sparse sign sketch
seed 7, Chebyshev basis c = 4, dx = 4, dy = 0 (§4.3, the spectrum [0, 8] of
the §8 Laplacian example), tol 1e-6, plain FP64 oracle (Algorithm 1
restarted, §3.5).  Writes tests/golden/laplace_oracle.json with the relative
residual after each cycle.

Run from the repository root (takes tens of minutes):
    OPENBLAS_NUM_THREADS=1 python tests/golden/make_laplace_reference.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import krylov, operators, sketch  # noqa: E402


def main():
    W = synth.WORKLOADS["laplace"]
    N = W["N"]
    A = operators.neumann_laplacian_matrix(N, N)
    f = A @ synth.grf(W["x_seed"], N, W["ell"])
    S = sketch.sparse_sign_matrix(7, N * N, W["s"], W["zeta"])
    x = np.zeros(N * N)
    fn = np.linalg.norm(f)
    hist, secs, kappas = [], [], []
    while True:
        t = time.time()
        x, info = krylov.sgmres_cycle(A, f, x, W["d"], W["k"], lambda M: S @ M, cheb=W["cheb"])
        secs.append(time.time() - t)
        hist.append(float(np.linalg.norm(f - A @ x) / fn))
        kappas.append(float(info["kappa"]))
        print(len(hist), hist[-1], secs[-1], flush=True)
        if hist[-1] <= W["tol"] or len(hist) >= 80:
            break
    out = dict(workload="laplace", N=N, x_seed=W["x_seed"], ell=W["ell"], d=W["d"], s=W["s"], zeta=W["zeta"],
               seed=7, cheb=list(W["cheb"]), tol=W["tol"], relres=hist, kappa=kappas, cycle_seconds=secs,
               cycles=len(hist))
    with open(os.path.join(HERE, "laplace_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
