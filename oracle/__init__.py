"""Plain FP64 CPU oracle for sketched GMRES and sketched Rayleigh-Ritz.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle follows Nakatsukasa & Tropp, "Fast & Accurate Randomized
Algorithms for Linear Systems and Eigenvalue Problems" (2021/2022), step by
step, in float64, with numpy/scipy primitives (matmul, sparse matvec, SVD,
dense eig) as single steps and no blocking, fusion or reordering beyond what
the paper states.  It shares no code with the CUDA library under
``paper_2111_00113_gb300/``; the two sides meet only through the seeded input
generators in ``synth/``.

Modules
  hashing   counter-based sketch hash H1 (sparse-sign rows/signs, SRHT signs
            and sampled rows)                              -- §2.3.1, §2.3.2
  sketch    sparse sign embedding, SRHT, distortion       -- §2, Def. (subspace-embed)
  operators 5-point convection-diffusion and variable-coefficient
            diffusion operators (the model problems)
  krylov    k-truncated Arnoldi with double Gram-Schmidt, Householder QR,
            sGMRES (Algorithm 1) with restarting (§3.5), iterative sGMRES
            with early stopping (§5.2, §5.3), Householder-Arnoldi GMRES
            (§4.2), the Chebyshev basis (§4.3)
  eigs      sketched Rayleigh-Ritz (Algorithm 2), stabilized sRR (§6.5),
            Rayleigh-Ritz (§6.1)
  adjoint   dense adjoint gradient of ||x(theta)-x_t||^2

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, brute force, library routines on special cases,
the bounds of Fact 2.2); see tests/test_oracle_*.py.
"""
