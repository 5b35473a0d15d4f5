"""Oracle reference run of restarted sRR on the full-size eigen workload.

512 x 512 convection-diffusion (Pe = 10) plus diag(U(0,1) seed 1); the 10
eigenvalues of largest real part by restarted sRR (§7.2) on block Chebyshev
bases (§7.5): start block of b = 16 columns randn(500 + i), p = 12 blocks
(d = 192, s = 384), each start block filtered by a degree-150 Chebyshev
polynomial for [lo, cut], lo = -0.5, cut_0 = hi = 9.0, stabilized sRR with
truncation 1e13, sparse sign sketch seed 7 + t at restart t, stop when the
10 leading residual estimates are <= 1e-8 ||A||_2, at most 40 restarts.
Stored: the Ritz values, estimates, true residuals / ||A||_2, restarts and
the estimate history.

Run from the repository root (about a minute):
    OPENBLAS_NUM_THREADS=1 python tests/golden/make_eig_restarted_reference.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import eigs, hashing, operators, sketch  # noqa: E402

B_COLS, P_BLOCKS, DEGREE, LO, HI, MAXR = 16, 12, 150, -0.5, 9.0, 40


def main():
    W = synth.WORKLOADS["eig"]
    N, nev = W["N"], W["nev"]
    shift = synth.uniform(W["shift_seed"], N * N)
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, W["Pe"]), shift).tocsr()
    with open(os.path.join(HERE, "eig_oracle.json")) as fh:
        anorm = json.load(fh)["anorm"]
    Om = np.column_stack([synth.randn(500 + i, N * N) for i in range(B_COLS)])
    d = B_COLS * P_BLOCKS
    skf = lambda t: (lambda M: sketch.sparse_sign_apply(7 + t, 2 * d, hashing.default_zeta(d), M))  # noqa: E731
    out = eigs.srr_restarted(A, Om, P_BLOCKS, nev, LO, HI, MAXR, skf, tau=1e-8 * anorm, filter_degree=DEGREE)
    lam = out["lam"][:nev]
    tr = [float(eigs.eig_residual(A, lam[i], out["X"][:, i]) / anorm) for i in range(nev)]
    res = dict(workload="eig", b=B_COLS, p=P_BLOCKS, filter_degree=DEGREE, lo=LO, hi=HI, max_restarts=MAXR,
               anorm=anorm, restarts=out["restarts"], history=out["history"],
               lam_re=[float(v) for v in lam.real], lam_im=[float(v) for v in lam.imag],
               rhat=[float(v) for v in out["rhat"][:nev]], true_res=tr)
    with open(os.path.join(HERE, "eig_restarted_oracle.json"), "w") as fh:
        json.dump(res, fh, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
