"""GPU parity of the operators and the k-truncated Arnoldi basis."""
import numpy as np
import pytest

import synth
from oracle import hashing, krylov, operators, sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def skg():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    import paper_2111_00113_gb300 as m
    return m


def _cd(N, Pe, shift=None):
    return synth.conv_diff_coef(N, Pe), operators.stencil5_matrix(N, N, synth.conv_diff_coef(N, Pe), shift)


def test_operator_apply_matches_assembled_matrices(skg):
    import torch
    rng = np.random.default_rng(0)
    for nx, ny in ((64, 64), (37, 5), (1, 9)):
        coef, A = _cd(max(nx, ny), 10.0)
        A = operators.stencil5_matrix(nx, ny, coef, rng.random(nx * ny))
        x = rng.standard_normal(nx * ny)
        op = skg.Op.stencil5(nx, ny, coef, torch.tensor(rng.random(nx * ny) * 0, device="cuda"))
        op = skg.Op.stencil5(nx, ny, coef, torch.tensor(A.diagonal() - coef[0], device="cuda"))
        y = op.apply(torch.tensor(x, device="cuda")).cpu().numpy()
        assert np.allclose(y, A @ x, rtol=0, atol=1e-13)
        # transpose
        yT = op.T.apply(torch.tensor(x, device="cuda")).cpu().numpy()
        assert np.allclose(yT, A.T @ x, rtol=0, atol=1e-13)
    th = np.exp(synth.grf(2, 32, 4.0))
    Av = operators.diffusion_var_matrix(32, 32, th)
    x = rng.standard_normal(1024)
    op = skg.Op.diffusion_var(32, 32, torch.tensor(th, device="cuda"))
    assert np.allclose(op.apply(torch.tensor(x, device="cuda")).cpu().numpy(), Av @ x, rtol=0, atol=1e-12)
    rp, ci, va = operators.csr_from_scipy(Av)
    opc = skg.Op.csr(torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"), torch.tensor(va, device="cuda"))
    assert np.allclose(opc.apply(torch.tensor(x, device="cuda")).cpu().numpy(), Av @ x, rtol=0, atol=1e-12)


def _stencil_np(x2, coef):
    # 5-point product on an ny x nx grid (row-major, zero outside), written
    # with array shifts: y = cP x + cE x[:, i+1] + cW x[:, i-1] + cN x[j+1] + cS x[j-1]
    cP, cE, cW, cN, cS = coef
    y = cP * x2
    y[:, :-1] += cE * x2[:, 1:]
    y[:, 1:] += cW * x2[:, :-1]
    y[:-1, :] += cN * x2[1:, :]
    y[1:, :] += cS * x2[:-1, :]
    return y


def test_stencil_grid_index_math(skg):
    # the kernels find a cell's grid row by multiplying with a precomputed
    # reciprocal of nx; over grids up to 2^24 cells and widths that are
    # prime, odd, a power of two, 1 and the whole row, every product matches
    # the stencil evaluated on the 2-D array (FP64 and the FP32 basis path)
    import torch
    rng = np.random.default_rng(3)
    coef = (4.1, -0.7, -1.3, -0.9, -1.1)
    for nx, ny in ((4093, 4099), (1, 4097), (4096, 4096), (3, 1 << 20), (1 << 20, 3), (12345, 7)):
        x2 = rng.standard_normal((ny, nx))
        ref = _stencil_np(x2, coef).ravel()
        op = skg.Op.stencil5(nx, ny, coef)
        y = op.apply(torch.tensor(x2.ravel(), device="cuda")).cpu().numpy()
        assert np.max(np.abs(y - ref)) <= 1e-12 * (1 + np.max(np.abs(ref))), (nx, ny)
    # the basis passes (vector path with the cells of a group in one row when
    # nx % 4 == 0, across rows when only n % 4 == 0, scalar otherwise):
    # b_1 = (A b_0 - h b_0) / nu is A r up to the combination with r
    for nx, ny in ((4093, 1031), (2048, 2049), (1022, 1024), (6, 50)):
        r = rng.standard_normal(nx * ny)
        out = skg.trunc_arnoldi_basis(skg.Op.stencil5(nx, ny, coef), torch.tensor(r, device="cuda"), 1, 1,
                                      dtype=torch.float64)
        B = out["B"].cpu().numpy()
        H = out["Hbar"].cpu().numpy()
        Ar = _stencil_np(r.reshape(ny, nx), coef).ravel()
        rn = np.linalg.norm(r)
        lhs = Ar / rn
        rhs = H[0, 0] * B[:, 0] + H[1, 0] * B[:, 1]
        assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs), (nx, ny)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_basis_fp64_matches_oracle(skg, k):
    import torch
    N, d = 64, 40
    coef, A = _cd(N, 10.0)
    r = synth.randn(0, N * N)
    s, zeta = 80, 8
    out = skg.trunc_arnoldi_basis(skg.Op.stencil5(N, N, coef), torch.tensor(r, device="cuda"), d, k,
                                  s=s, zeta=zeta, seed=7)
    B_ref, M_ref, H_ref, du_ref = krylov.trunc_arnoldi(A, r, d, k)
    assert out["d_used"] == du_ref == d
    B = out["B"].cpu().numpy()
    H = out["Hbar"].cpu().numpy()
    # leading columns agree closely; rounding differences grow along the recurrence
    for j in range(d):
        tol = 1e-12 * (10.0 ** (j / 8))
        assert np.linalg.norm(B[:, j] - B_ref[:, j]) <= max(tol, 1e-12), j
        if j >= 15:
            break
    # the Arnoldi relation A B_d = B_{d+1} Hbar holds for the GPU's own basis
    AB = A @ B[:, :d]
    assert np.linalg.norm(AB - B @ H) <= 1e-12 * np.linalg.norm(AB)
    assert np.allclose(H[: d + 1, :d - 1], H_ref[: d + 1, :d - 1], rtol=0, atol=1e-8 * np.abs(H_ref).max())
    # local orthonormality of the window
    G = B.T @ B
    for i in range(d + 1):
        assert abs(G[i, i] - 1) < 1e-12
        for j in range(max(0, i - k), i):
            assert abs(G[i, j]) < 1e-12
    # sketches: SB = S B_d and SAB = S A B_d (formed from the Arnoldi relation)
    S = sketch.sparse_sign_matrix(7, N * N, s, zeta)
    SB = out["SB"].cpu().numpy()
    SAB = out["SAB"].cpu().numpy()
    assert np.linalg.norm(SB - S @ B[:, :d]) <= 1e-12 * np.linalg.norm(SB)
    assert np.linalg.norm(SAB - S @ AB) <= 1e-11 * np.linalg.norm(SAB)


def test_basis_single_pass_and_breakdown(skg):
    import torch
    # invariant subspace: diagonal operator (stencil with zero off-diagonals
    # and a diagonal shift), start vector with 3 nonzeros -> d_used = 3
    n = 50
    shift = np.arange(1.0, n + 1)
    op = skg.Op.stencil5(n, 1, (0, 0, 0, 0, 0), torch.tensor(shift, device="cuda"))
    r = np.zeros(n)
    r[[2, 7, 11]] = [1.0, -2.0, 0.5]
    out = skg.trunc_arnoldi_basis(op, torch.tensor(r, device="cuda"), 10, 10)
    B_ref, M_ref, H_ref, du_ref = krylov.trunc_arnoldi(np.diag(shift), r, 10, 10)
    assert out["d_used"] == du_ref == 3
    # one classical pass
    N = 32
    coef, A = _cd(N, 5.0)
    r = synth.randn(1, N * N)
    out = skg.trunc_arnoldi_basis(skg.Op.stencil5(N, N, coef), torch.tensor(r, device="cuda"), 8, 2, cgs_passes=1)
    B_ref, _, _, _ = krylov.trunc_arnoldi(A, r, 8, 2, passes=1)
    assert np.allclose(out["B"].cpu().numpy()[:, :8], B_ref, atol=1e-10)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_basis_low_precision_relation(skg, dtype):
    import torch
    N, d, k = 128, 30, 2
    coef, A = _cd(N, 20.0)
    r = synth.randn(2, N * N)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    out = skg.trunc_arnoldi_basis(skg.Op.stencil5(N, N, coef), torch.tensor(r, device="cuda"), d, k, dtype=tdt)
    B = out["B"].to(torch.float64).cpu().numpy()
    H = out["Hbar"].cpu().numpy()
    u = 6e-8 if dtype == "f32" else 4e-3
    AB = A @ B[:, :d]
    assert np.linalg.norm(AB - B @ H) <= 50 * u * np.linalg.norm(AB)
    assert np.allclose(np.linalg.norm(B, axis=0), 1, atol=10 * u)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [2, 4])
def test_persistent_matches_multikernel(skg, dtype, k):
    # the cooperative one-launch basis and the three-launch-per-step basis run
    # the same recurrence; their bases agree to rounding, and each satisfies
    # the Arnoldi relation on its own
    import torch
    N, d = 96, 30
    coef, A = _cd(N, 30.0)
    r = synth.randn(7, N * N)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    op = skg.Op.stencil5(N, N, coef)
    rt = torch.tensor(r, device="cuda")
    a = skg.trunc_arnoldi_basis(op, rt, d, k, dtype=tdt, persistent=True)
    b = skg.trunc_arnoldi_basis(op, rt, d, k, dtype=tdt, persistent=False)
    Ba = a["B"].to(torch.float64).cpu().numpy()
    Bb = b["B"].to(torch.float64).cpu().numpy()
    tol = 1e-11 if dtype == "f64" else 1e-4
    assert np.linalg.norm(Ba[:, :10] - Bb[:, :10]) <= tol * 10
    H = a["Hbar"].cpu().numpy()
    AB = A @ Ba[:, :d]
    u = 1e-15 if dtype == "f64" else 6e-8
    assert np.linalg.norm(AB - Ba @ H) <= 1e3 * u * np.linalg.norm(AB)


def test_persistent_diffusion_and_shift(skg):
    import torch
    N, d, k = 64, 20, 4
    th = np.exp(synth.grf(2, N, 8.0))
    Av = operators.diffusion_var_matrix(N, N, th)
    r = synth.randn(3, N * N)
    op = skg.Op.diffusion_var(N, N, torch.tensor(th, device="cuda"))
    out = skg.trunc_arnoldi_basis(op, torch.tensor(r, device="cuda"), d, k)
    B_ref, _, H_ref, _ = krylov.trunc_arnoldi(Av, r, d, k)
    B = out["B"].cpu().numpy()
    assert np.linalg.norm(B[:, :8] - B_ref[:, :8]) <= 1e-10
    assert np.linalg.norm(Av @ B[:, :d] - B @ out["Hbar"].cpu().numpy()) <= 1e-12 * np.linalg.norm(Av @ B[:, :d])
    shift = synth.uniform(1, N * N)
    coef, As = _cd(N, 10.0, shift)
    op = skg.Op.stencil5(N, N, coef, torch.tensor(shift, device="cuda"))
    out = skg.trunc_arnoldi_basis(op, torch.tensor(r, device="cuda"), d, k)
    B_ref, _, _, _ = krylov.trunc_arnoldi(As, r, d, k)
    assert np.linalg.norm(out["B"].cpu().numpy()[:, :8] - B_ref[:, :8]) <= 1e-10


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_low_precision_stencil_rectangular(skg, dtype, k):
    # FP32/BF16 bases on a rectangular stencil grid (vector path, nx % 4 == 0,
    # ny = 37) with a diagonal shift: the leading columns follow the FP64
    # oracle's recurrence and the Arnoldi relation holds to the storage
    # precision.
    import torch
    passes = 2
    nx, ny, d = 64, 37, 24
    coef = synth.conv_diff_coef(64, 25.0)
    shift = synth.uniform(5, nx * ny)
    A = operators.stencil5_matrix(nx, ny, coef, shift)
    r = synth.randn(6, nx * ny)
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    op = skg.Op.stencil5(nx, ny, coef, torch.tensor(shift, device="cuda"))
    out = skg.trunc_arnoldi_basis(op, torch.tensor(r, device="cuda"), d, k, dtype=tdt, cgs_passes=passes)
    assert out["d_used"] == d
    B = out["B"].to(torch.float64).cpu().numpy()
    H = out["Hbar"].cpu().numpy()
    B_ref, _, _, _ = krylov.trunc_arnoldi(A, r, d, k, passes=passes)
    u = 6e-8 if dtype == "f32" else 4e-3
    assert np.linalg.norm(B[:, :4] - B_ref[:, :4]) <= 1e3 * u
    AB = A @ B[:, :d]
    assert np.linalg.norm(AB - B @ H) <= 50 * u * np.linalg.norm(AB)
    assert np.allclose(np.linalg.norm(B, axis=0), 1, atol=10 * u)


def test_single_pass_needs_fp64_basis(skg):
    import torch
    N = 32
    coef, _ = _cd(N, 10.0)
    op = skg.Op.stencil5(N, N, coef)
    r = torch.tensor(synth.randn(1, N * N), device="cuda")
    with pytest.raises(skg.SkError, match="cgs_passes"):
        skg.trunc_arnoldi_basis(op, r, 8, 2, dtype=torch.float32, cgs_passes=1)


def test_persistent_barrier_timeout_is_reported(skg):
    # Failure detection without a GPU fault: the cooperative kernel's grid
    # barriers are bounded; with barrier_spins = -1 a CTA that is not the last
    # to arrive gives up at its first poll, sets the error word, and every CTA
    # leaves the kernel.  The call reports SK_ETIMEOUT and the context stays
    # usable.
    import torch
    from paper_2111_00113_gb300 import _native as N
    n = 256
    coef, _ = _cd(n, 10.0)
    op = skg.Op.stencil5(n, n, coef)
    r = torch.tensor(synth.randn(4, n * n), device="cuda")
    seen = []
    for _ in range(5):
        try:
            skg.trunc_arnoldi_basis(op, r, 10, 2, dtype=torch.float32, persistent=True, barrier_spins=-1)
            seen.append(N.SK_OK)
        except skg.SkError as e:
            assert e.status == N.SK_ETIMEOUT, e
            seen.append(e.status)
    assert N.SK_ETIMEOUT in seen
    out = skg.trunc_arnoldi_basis(op, r, 10, 2, dtype=torch.float32, persistent=True)
    assert out["d_used"] == 10
    torch.cuda.synchronize()
