"""Oracle reference run of the full-size sRR eigen workload (stored values).

512 x 512 convection-diffusion (Pe = 10) plus diag(U(0,1) seed 1); the 10
eigenvalues of largest real part by Algorithm 2 with the k = 4 truncated
Arnoldi basis (d = 200, s = 400, zeta = 11, sparse sign sketch seed 7,
start vector randn(1 ^ 0x5EED)), plain FP64 oracle.  Stored: the selected
Ritz values, their residual estimates (eq. (srr-resid-est)), the true
residuals ||A x - lambda x|| / ||x|| of the oracle's Ritz vectors, ||A||_2,
and the rounding sensitivity of the Ritz values: the same reduction with
S A B formed as (S B_{d+1}) Hbar (the Arnoldi relation A B_d = B_{d+1} Hbar,
mathematically the same matrix) instead of S (A B).

Run from the repository root (about a minute):
    OPENBLAS_NUM_THREADS=1 python tests/golden/make_eig_reference.py
"""
import json
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import eigs, krylov, operators, sketch  # noqa: E402


def main():
    W = synth.WORKLOADS["eig"]
    N = W["N"]
    shift = synth.uniform(W["shift_seed"], N * N)
    A = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, W["Pe"]), shift)
    w1 = synth.randn(synth.SRR_START_SEED, N * N)
    d, k, s, nev, zeta = W["d"], W["k"], W["s"], W["nev"], W["zeta"]
    S = sketch.sparse_sign_matrix(7, N * N, s, zeta)
    sk = lambda M: S @ M  # noqa: E731
    out = eigs.srr(A, w1, d, k, sk, nev)
    lam = out["lam"]
    true_res = [float(eigs.eig_residual(A, lam[i], out["X"][:, i])) for i in range(nev)]
    # the other arithmetic route: one more basis vector and the Arnoldi coefficients
    B1, _, Hc, du = krylov.trunc_arnoldi(A, w1, d + 1, k)
    assert du == d + 1
    C = S @ B1[:, :d]
    D2 = (S @ B1[:, : d + 1]) @ Hc[: d + 1, :d]
    V, T = krylov.householder_qr(C)
    UtD = np.stack([krylov.apply_qt(V, D2[:, j])[:d] for j in range(d)], axis=1)
    Mhat2 = np.stack([krylov.back_substitute(T, UtD[:, j]) for j in range(d)], axis=1)
    lam2_all = np.linalg.eigvals(Mhat2)
    lam2 = lam2_all[eigs.select_order(lam2_all, nev)]
    anorm = float(spla.svds(A, k=1, return_singular_vectors=False)[0])
    res = dict(workload="eig", N=N, Pe=W["Pe"], d=d, k=k, s=s, zeta=zeta, nev=nev, seed=7,
               lam_re=[float(v) for v in lam.real], lam_im=[float(v) for v in lam.imag],
               rhat=[float(v) for v in out["rhat"]], true_res=true_res, anorm=anorm,
               kappa_T=float(out["kappa"]),
               route_lam_re=[float(v) for v in lam2.real], route_lam_im=[float(v) for v in lam2.imag],
               route_dlam=[float(abs(a - b)) for a, b in zip(lam, lam2)])
    with open(os.path.join(HERE, "eig_oracle.json"), "w") as fh:
        json.dump(res, fh, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
