"""Oracle reference run of the full-size sGMRES workload (stored expected values).

1024 x 1024 convection-diffusion (Pe = 50), b ~ N(0,1) seed 0, x0 = 0,
d = 300, k = 2, s = 600, zeta = 12, sketch seed 7, tol 1e-6, plain FP64
oracle (Algorithm 1 restarted, §3.5).  Writes the relative residual after
each cycle and the wall time of each cycle on this host (single-threaded
numpy/scipy):

  --sketch sparse (default)  sparse sign embedding (§2.3.2)  -> scale_oracle.json
  --sketch srht              SRHT (§2.3.1, Walsh-Hadamard)   -> scale_srht_oracle.json

Run from the repository root (takes several minutes; the SRHT run longer):
    OPENBLAS_NUM_THREADS=1 python tests/golden/make_scale_reference.py [--sketch srht]
"""
import argparse
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
    ap = argparse.ArgumentParser()
    ap.add_argument("--sketch", default="sparse", choices=["sparse", "srht"])
    args = ap.parse_args()
    W = synth.WORKLOADS["scale"]
    N = W["N"]
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, W["Pe"]))
    f = synth.randn(W["b_seed"], N * N)
    if args.sketch == "sparse":
        S = sketch.sparse_sign_matrix(7, N * N, W["s"], W["zeta"])
        sk = lambda M: S @ M  # noqa: E731
        name = "scale_oracle.json"
    else:
        sk = lambda M: sketch.srht_apply(7, W["s"], M)  # noqa: E731
        name = "scale_srht_oracle.json"
    x = np.zeros(N * N)
    fn = np.linalg.norm(f)
    hist, secs, kappas = [], [], []
    while True:
        t = time.time()
        x, info = krylov.sgmres_cycle(A, f, x, W["d"], W["k"], sk)
        secs.append(time.time() - t)
        hist.append(float(np.linalg.norm(f - A @ x) / fn))
        kappas.append(float(info["kappa"]))
        print(len(hist), hist[-1], secs[-1], flush=True)
        if hist[-1] <= W["tol"] or len(hist) >= 60:
            break
    out = dict(workload="scale", sketch=args.sketch, N=N, Pe=W["Pe"], d=W["d"], k=W["k"], s=W["s"],
               zeta=W["zeta"], seed=7, tol=W["tol"], relres=hist, kappa=kappas, cycle_seconds=secs,
               cycles=len(hist))
    with open(os.path.join(HERE, name), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
