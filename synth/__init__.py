"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method: it only draws random inputs
(numpy PCG64 streams) and states the model problems' parameters.  Both the
CPU oracle and the CUDA library receive the arrays made here.

Workloads (shapes of the paper's model problems, §8.1.3/§8.3: 2-D five-point
operators with n ~ 1e6 unknowns, nonsymmetric sparse operators and random
spectra; the paper's SuiteSparse/Matrix Market matrices are not available):

  small      64x64 convection-diffusion, Pe=10, b ~ N(0,1) seed 0,
             d=40, k=2, s=80, zeta=8, tol 1e-8, FP64
  scale      1024x1024 convection-diffusion, Pe=50, b ~ N(0,1) seed 0,
             d=300, k=2, s=600, zeta=12, tol 1e-6 (FP64 plain and FP32/BF16
             basis forms; sparse-sign and SRHT sketches)
  eig        512x512 convection-diffusion, Pe=10, + diag(U(0,1) seed 1),
             nev=10, d=200, k=4, s=400, zeta=11, FP32 basis / FP64 Ritz
  batched    256 systems, side ~ U{128..512}, Pe ~ U(1,100) (seed 4),
             4 right-hand sides ~ N(0,1) each, d=100, k=2, s=200, zeta=10
  laplace    1024x1024 Neumann Laplacian (spectrum in [0, 8], kernel = the
             constants), f = A x_true with x_true = GRF(seed 5, length 64
             cells) (f is consistent and smooth, so the small eigenvalues
             matter), d=300, k=2, s=600, zeta=12, tol 1e-6; Chebyshev
             basis with c = 4, dx = 4, dy = 0 (the paper's §8 Laplacian
             experiment: "eigenvalues in [0, 8]")
  adjoint    512x512 variable-coefficient diffusion, theta = exp(GRF,
             length scale 32 cells, seed 2), b ~ N(0,1) seed 3,
             x_target = A(theta = 1)^{-1} b, d=300, k=2, s=600, zeta=12,
             tol 1e-10 with an FP64 basis, 1e-7 with an FP32 basis (whose
             refinement floors near 2e-8 on this operator; restarted
             sGMRES(100) stagnates near 1e-3)
"""
import numpy as np


def randn(seed, n):
    return np.random.default_rng(seed).standard_normal(n)


def uniform(seed, n):
    return np.random.default_rng(seed).random(n)


def conv_diff_coef(N, Pe, diff=1.0):
    """Five-point coefficients (cP, cE, cW, cN, cS) of -diff*Lap(u) + (Pe,Pe).grad(u).

    Unit square, N x N interior grid, h = 1/(N+1), central differences for
    both terms, whole row multiplied by h^2:
      (Au)_P = 4 diff u_P - (diff - a) u_E - (diff + a) u_W
                          - (diff - a) u_N - (diff + a) u_S,   a = Pe*h/2.
    """
    h = 1.0 / (N + 1)
    a = Pe * h / 2.0
    return (4.0 * diff, -(diff - a), -(diff + a), -(diff - a), -(diff + a))


def grf(seed, N, ell):
    """Smooth periodic Gaussian random field on an N x N grid, unit variance.

    White N(0,1) noise circularly convolved with a Gaussian kernel of width
    ell/sqrt(2) cells (covariance ~ exp(-r^2 / (2 ell^2))), then rescaled to
    zero mean and unit sample variance.
    """
    w = np.random.default_rng(seed).standard_normal((N, N))
    k = np.fft.fftfreq(N) * N
    kx, ky = np.meshgrid(k, k, indexing="xy")
    sig = ell / np.sqrt(2.0)
    # Fourier transform of a unit-mass Gaussian kernel of width sig (cells)
    filt = np.exp(-2.0 * (np.pi * sig / N) ** 2 * (kx ** 2 + ky ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    g -= g.mean()
    g /= g.std()
    return g.reshape(-1)


def neumann_shift(nx, ny):
    """Diagonal correction that turns the 5-point stencil (4, -1, -1, -1, -1)
    with zero Dirichlet neighbours into the zero-flux (Neumann) Laplacian:
    -1 for every missing neighbour of a boundary cell."""
    ix = np.tile(np.arange(nx), ny)
    iy = np.repeat(np.arange(ny), nx)
    missing = (ix == 0).astype(float) + (ix == nx - 1) + (iy == 0) + (iy == ny - 1)
    return -missing


def batch_systems(seed, nsys, side_lo=128, side_hi=512, pe_lo=1.0, pe_hi=100.0):
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=nsys)
    pes = rng.uniform(pe_lo, pe_hi, size=nsys)
    return sides, pes


def batch_rhs_seed(sys_index, r):
    return 1000 + 4 * sys_index + r


SRR_START_SEED = 1 ^ 0x5EED

WORKLOADS = {
    "small": dict(N=64, Pe=10.0, b_seed=0, d=40, k=2, s=80, zeta=8, tol=1e-8),
    "scale": dict(N=1024, Pe=50.0, b_seed=0, d=300, k=2, s=600, zeta=12, tol=1e-6),
    "eig": dict(N=512, Pe=10.0, shift_seed=1, nev=10, d=200, k=4, s=400, zeta=11),
    "batched": dict(nsys=256, seed=4, nrhs=4, d=100, k=2, s=200, zeta=10, tol=1e-6),
    "laplace": dict(N=1024, x_seed=5, ell=64.0, d=300, k=2, s=600, zeta=12, tol=1e-6, cheb=(4.0, 4.0, 0.0)),
    "adjoint": dict(N=512, grf_seed=2, ell=32.0, b_seed=3, target_seed=3, d=300, k=2, s=600, zeta=12, tol=1e-10,
                    tol_f32=1e-7),
}
