"""GPU differentiable solve: parameter gradients and the adjoint sGMRES.

Checked against the oracle's direct adjoint (oracle/adjoint.py), assembled
matrices and central finite differences of the GPU forward solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import adjoint, operators

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def skg():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    import paper_2111_00113_gb300 as m
    return m


def _t(a):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def test_param_grad_diffusion_stencil_csr(skg):
    rng = np.random.default_rng(0)
    nx, ny = 37, 29
    n = nx * ny
    th = np.exp(rng.standard_normal(n))
    lam, x = rng.standard_normal(n), rng.standard_normal(n)
    g = skg.Op.diffusion_var(nx, ny, _t(th)).param_grad(_t(lam), _t(x)).cpu().numpy()
    assert np.allclose(g, operators.diffusion_var_theta_grad(nx, ny, lam, x), rtol=1e-12, atol=1e-12)
    # stencil coefficients: d(lam^T A x)/dc_q = lam^T A_q x with A_q the q-th neighbour pattern
    coef = (4.0, -0.9, -1.1, -0.8, -1.2)
    shift = rng.random(n)
    op = skg.Op.stencil5(nx, ny, coef, _t(shift))
    g = op.param_grad(_t(lam), _t(x)).cpu().numpy()
    for q in range(5):
        e = np.zeros(5)
        e[q] = 1.0
        Aq = operators.stencil5_matrix(nx, ny, e)
        assert abs(g[q] - lam @ (Aq @ x)) <= 1e-10 * max(1, abs(g[q]))
    assert np.allclose(g[5:], lam * x, rtol=0, atol=1e-14)
    # CSR values
    A = sp.random(n, n, density=0.01, random_state=1, format="csr") + sp.eye(n)
    rp, ci, va = operators.csr_from_scipy(A)
    opc = skg.Op.csr(_t(rp).to(int), _t(ci).to(int), _t(va))
    g = opc.param_grad(_t(lam), _t(x)).cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.allclose(g, lam[rows] * x[ci], rtol=0, atol=1e-14)


def _loss_grad_gpu(skg, nx, ny, theta, b, xt, tol, d=100, **opts):
    import torch
    th = _t(theta).requires_grad_(True)
    bb = _t(b).requires_grad_(True)
    d = min(d, nx * ny)
    x = skg.diffusion_solve(th, bb, nx, ny, d=d, k=2, s=2 * d, tol=tol, **opts)
    L = torch.sum((x - _t(xt)) ** 2)
    L.backward()
    return L.item(), th.grad.cpu().numpy(), bb.grad.cpu().numpy()


@pytest.mark.parametrize("N", [16, 64])
def test_adjoint_matches_direct_oracle(skg, N):
    theta = np.exp(0.5 * synth.grf(2, N, N / 8.0))
    b = synth.randn(3, N * N)
    xt = synth.randn(4, N * N) * 0.01
    L, gth, gb = _loss_grad_gpu(skg, N, N, theta, b, xt, 1e-12)
    Lr, gth_r, lam_r, x_r = adjoint.loss_and_grad(N, N, theta, b, xt)
    assert abs(L - Lr) <= 1e-9 * Lr
    assert np.linalg.norm(gth - gth_r) <= 1e-7 * np.linalg.norm(gth_r)
    assert np.linalg.norm(gb - lam_r) <= 1e-7 * np.linalg.norm(lam_r)


def test_adjoint_central_differences(skg):
    import torch
    N = 16
    theta = np.exp(0.5 * synth.grf(5, N, 2.0))
    b = synth.randn(6, N * N)
    xt = synth.randn(7, N * N) * 0.01
    L, gth, gb = _loss_grad_gpu(skg, N, N, theta, b, xt, 1e-13)

    def loss(th, bv):
        with torch.no_grad():
            x = skg.diffusion_solve(_t(th), _t(bv), N, N, d=100, k=2, s=200, tol=1e-13)
            return float(torch.sum((x - _t(xt)) ** 2))

    for p in (0, 17, 100, 255):
        e = np.zeros(N * N)
        h = 1e-5 * theta[p]
        e[p] = h
        fd = (loss(theta + e, b) - loss(theta - e, b)) / (2 * h)
        assert abs(fd - gth[p]) <= 1e-6 * max(1.0, abs(gth[p])), (p, fd, gth[p])
        e[p] = 1e-5
        fd = (loss(theta, b + e) - loss(theta, b - e)) / 2e-5
        assert abs(fd - gb[p]) <= 1e-6 * max(1.0, abs(gb[p]))


def test_adjoint_workload_full_size_directional(skg):
    # 512 x 512, theta = exp(GRF, length 32 cells, seed 2), b ~ N(0,1) seed 3,
    # x_target = A(theta = 1)^{-1} b.  FP64 basis at tol 1e-10: a random
    # directional derivative of the loss against central differences of the
    # forward solve.  FP32 basis (FP64 refinement) at tol 1e-7: its gradient
    # against the FP64 one.
    import torch
    W = synth.WORKLOADS["adjoint"]
    N = W["N"]
    theta = np.exp(synth.grf(W["grf_seed"], N, W["ell"]))
    b = synth.randn(W["b_seed"], N * N)
    kw = dict(d=W["d"], k=W["k"], s=W["s"], zeta=W["zeta"], maxit=2000)
    with torch.no_grad():
        xt = skg.diffusion_solve(_t(np.ones(N * N)), _t(b), N, N, tol=W["tol"], **kw).cpu().numpy()
    L, gth, gb = _loss_grad_gpu(skg, N, N, theta, b, xt, W["tol"], d=W["d"], zeta=W["zeta"], maxit=2000)
    v = synth.randn(11, N * N) * theta * 1e-3

    def loss(th):
        with torch.no_grad():
            x = skg.diffusion_solve(_t(th), _t(b), N, N, tol=W["tol"], **kw)
            return float(torch.sum((x - _t(xt)) ** 2))

    fd = (loss(theta + v) - loss(theta - v)) / 2.0
    an = float(gth @ v)
    assert abs(fd - an) <= 1e-3 * abs(an), (fd, an)
    L32, g32, gb32 = _loss_grad_gpu(skg, N, N, theta, b, xt, W["tol_f32"], d=W["d"], zeta=W["zeta"], maxit=2000,
                                    basis=torch.float32)
    assert abs(L32 - L) <= 1e-3 * L
    assert np.linalg.norm(g32 - gth) <= 5e-2 * np.linalg.norm(gth)
    assert np.linalg.norm(gb32 - gb) <= 5e-2 * np.linalg.norm(gb)


def test_stencil_solve_gradients_match_oracle(skg):
    # the differentiable solve for the five-point operator: gradients with
    # respect to the five coefficients, the diagonal shift and b against the
    # oracle's dense adjoint (oracle/adjoint.py stencil_loss_and_grad)
    import torch
    N = 24
    coef = np.array(synth.conv_diff_coef(N, 20.0))
    shift = synth.uniform(8, N * N)
    b = synth.randn(9, N * N)
    xt = synth.randn(10, N * N) * 0.01
    c = torch.tensor(coef, dtype=torch.float64, requires_grad=True)
    sh = _t(shift).requires_grad_(True)
    bb = _t(b).requires_grad_(True)
    x = skg.stencil_solve(c, bb, N, N, shift=sh, d=100, k=2, s=200, tol=1e-13)
    L = torch.sum((x - _t(xt)) ** 2)
    L.backward()
    Lr, gc, gs, lam, _ = adjoint.stencil_loss_and_grad(N, N, coef, shift, b, xt)
    assert abs(L.item() - Lr) <= 1e-9 * Lr
    assert np.allclose(c.grad.numpy(), gc, rtol=1e-7, atol=1e-9 * np.abs(gc).max())
    assert np.linalg.norm(sh.grad.cpu().numpy() - gs) <= 1e-7 * np.linalg.norm(gs)
    assert np.linalg.norm(bb.grad.cpu().numpy() - lam) <= 1e-7 * np.linalg.norm(lam)


def test_csr_transpose_and_sell_apply(skg):
    # the SELL-32 copy applies A exactly like the CSR rows (same order per
    # row), and the device-built transpose applies A^T, on a matrix with
    # uneven rows (a row count not a multiple of 32, empty rows)
    rng = np.random.default_rng(4)
    n = 1000 + 13
    A = sp.random(n, n, density=0.004, random_state=6, format="lil")
    A[5, :] = 0
    A[::37, 3] = 1.5
    A = (A + sp.eye(n)).tocsr()
    rp, ci, va = operators.csr_from_scipy(A)
    op = skg.Op.csr(_t(rp).to(int), _t(ci).to(int), _t(va))
    x = rng.standard_normal(n)
    assert np.allclose(op.apply(_t(x)).cpu().numpy(), A @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(op.T.apply(_t(x)).cpu().numpy(), A.T @ x, rtol=1e-14, atol=1e-14)


def test_csr_solve_gradients_match_oracle(skg):
    # the differentiable solve for a general sparse operator (convection-
    # diffusion plus a random sparse perturbation): gradients with respect
    # to the stored values and b against the oracle's dense adjoint
    import torch
    N = 20
    A0 = operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, 15.0))
    P = sp.random(N * N, N * N, density=3e-3, random_state=7, format="csr")
    A = (A0 + 0.05 * P).tocsr()
    A.sort_indices()
    rp, ci, va = operators.csr_from_scipy(A)
    b = synth.randn(14, N * N)
    xt = synth.randn(15, N * N) * 0.01
    val = _t(va).requires_grad_(True)
    bb = _t(b).requires_grad_(True)
    x = skg.csr_solve(val, bb, _t(rp).to(torch.int32), _t(ci).to(torch.int32), d=100, k=2, s=200, tol=1e-13)
    L = torch.sum((x - _t(xt)) ** 2)
    L.backward()
    Lr, gv, lam, _ = adjoint.csr_loss_and_grad(A, b, xt)
    assert abs(L.item() - Lr) <= 1e-9 * Lr
    assert np.linalg.norm(val.grad.cpu().numpy() - gv) <= 1e-7 * np.linalg.norm(gv)
    assert np.linalg.norm(bb.grad.cpu().numpy() - lam) <= 1e-7 * np.linalg.norm(lam)
