"""GB300 (sm_103a) sketched GMRES and sketched Rayleigh-Ritz.

Thin Python binding over the C ABI of libsk.so (include/sk.h): the functions
below marshal torch CUDA tensors into device pointers and call the library,
whose CUDA kernels do all the work.  PyTorch provides device memory and the
current stream only.  There is no CPU path: without the built library or a
GPU these functions raise.

Layout: a matrix argument such as the basis B (n x c) is column-major.  A
torch tensor qualifies if ``B.stride(0) == 1`` (e.g. ``torch.empty(c, n).t()``);
other 2-D tensors are copied into that layout first.
"""
import ctypes as C

import torch

from . import _native as N
from ._native import SkError  # noqa: F401

_DT = {torch.float64: N.SK_F64, torch.float32: N.SK_F32, torch.bfloat16: N.SK_BF16}
_KIND = {"sparse": N.SK_SPARSE_SIGN, "srht": N.SK_SRHT}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev_f64(t, n=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ValueError("expected a CUDA tensor")
    t = t.to(torch.float64).contiguous()
    if n is not None and t.numel() != n:
        raise ValueError("expected %d entries, got %d" % (n, t.numel()))
    return t


def colmajor(B):
    """Column-major view (stride(0) == 1) of a 1-D or 2-D CUDA tensor."""
    if B.dim() == 1:
        return B.contiguous().view(-1, 1)
    if B.stride(0) == 1 and B.stride(1) >= B.shape[0]:
        return B
    return B.t().contiguous().t()


def empty_colmajor(n, c, dtype=torch.float64, device="cuda"):
    return torch.empty((c, n), dtype=dtype, device=device).t()


def default_zeta(d):
    import math
    return int(math.ceil(2.0 * math.log1p(d)))


class Op:
    """A library operator (sk_op); keeps the borrowed device arrays alive."""

    def __init__(self, handle, n, keep, nx=None, ny=None, kind=None):
        self._h = handle
        self.n = n
        self._keep = keep
        self.nx, self.ny, self.kind = nx, ny, kind

    @staticmethod
    def stencil5(nx, ny, coef, shift=None):
        h = C.c_void_p()
        cf = (C.c_double * 5)(*[float(c) for c in coef])
        sh = _dev_f64(shift, nx * ny) if shift is not None else None
        N.check(N.lib.sk_op_stencil5(C.byref(h), nx, ny, cf, _ptr(sh)))
        return Op(h, nx * ny, [sh], nx, ny, "stencil5")

    @staticmethod
    def diffusion_var(nx, ny, theta):
        h = C.c_void_p()
        th = _dev_f64(theta, nx * ny)
        N.check(N.lib.sk_op_diffusion_var(C.byref(h), nx, ny, _ptr(th)))
        return Op(h, nx * ny, [th], nx, ny, "diffusion")

    @staticmethod
    def csr(rowptr, colind, val):
        h = C.c_void_p()
        rp = rowptr.to(torch.int32).contiguous()
        ci = colind.to(torch.int32).contiguous()
        va = _dev_f64(val)
        n = rp.numel() - 1
        N.check(N.lib.sk_op_csr(C.byref(h), n, va.numel(), _ptr(rp), _ptr(ci), _ptr(va)))
        return Op(h, n, [rp, ci, va], kind="csr")

    @property
    def T(self):
        h = C.c_void_p()
        N.check(N.lib.sk_op_transpose(self._h, C.byref(h)))
        return Op(h, self.n, self._keep, self.nx, self.ny, self.kind)

    def apply(self, x, out=None):
        x = _dev_f64(x, self.n)
        y = torch.empty_like(x) if out is None else out
        N.check(N.lib.sk_op_apply(self._h, _ptr(x), _ptr(y), _stream()))
        return y

    def __matmul__(self, x):
        return self.apply(x)

    def param_grad(self, lam, x, alpha=1.0):
        """alpha times the gradient of lam^T A x with respect to the
        operator's parameters (the adjoint of a solve uses alpha = -1).

        diffusion: (n,) d/dtheta; stencil5: 5 coefficient entries (+ n shift
        entries if the op has a shift); CSR: (nnz,) d/dval.
        """
        lam = _dev_f64(lam, self.n)
        x = _dev_f64(x, self.n)
        if self.kind == "diffusion":
            m = self.n
        elif self.kind == "stencil5":
            m = 5 + (self.n if self._keep[0] is not None else 0)
        else:
            m = self._keep[2].numel()
        g = torch.empty(m, dtype=torch.float64, device=lam.device)
        N.check(N.lib.sk_op_param_grad(self._h, _ptr(lam), _ptr(x), float(alpha), _ptr(g), _stream()))
        return g

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib.sk_op_destroy(h)
            except Exception:
                pass
            self._h = None


def _sketch_struct(kind, n, s, zeta, seed):
    return N.SkSketch(_KIND[kind], int(n), int(s), int(zeta), int(seed))


def sketch_apply(B, s, zeta=0, seed=7, kind="sparse"):
    """S @ B (s x c, FP64, column-major) for a CUDA tensor B (n or n x c)."""
    vec = B.dim() == 1
    Bc = colmajor(B)
    if Bc.dtype not in _DT:
        raise ValueError("dtype must be float64, float32 or bfloat16")
    n, c = Bc.shape
    ldb = Bc.stride(1) if c > 1 else n  # a single column has no meaningful column stride
    out = empty_colmajor(s, c, torch.float64, Bc.device)
    sk = _sketch_struct(kind, n, s, zeta, seed)
    N.check(N.lib.sketch_apply(C.byref(sk), _ptr(Bc), ldb, c, _DT[Bc.dtype], _ptr(out), _stream()))
    return out[:, 0] if vec else out


class SketchPlan:
    """A sketch whose index tables (sparse sign) or signs and rows (SRHT) are
    built once on the device and reused: plan(B) = S @ B as sketch_apply."""

    def __init__(self, n, s, zeta=0, seed=7, kind="sparse"):
        self.n, self.s = int(n), int(s)
        self._h = C.c_void_p()
        sk = _sketch_struct(kind, n, s, zeta, seed)
        N.check(N.lib.sk_sketch_plan_create(C.byref(sk), C.byref(self._h), _stream()))

    def __call__(self, B, out=None):
        vec = B.dim() == 1
        Bc = colmajor(B)
        if Bc.dtype not in _DT:
            raise ValueError("dtype must be float64, float32 or bfloat16")
        n, c = Bc.shape
        if n != self.n:
            raise ValueError("B has %d rows, the plan %d" % (n, self.n))
        ldb = Bc.stride(1) if c > 1 else n
        if out is None:
            out = empty_colmajor(self.s, c, torch.float64, Bc.device)
        N.check(N.lib.sk_sketch_plan_apply(self._h, _ptr(Bc), ldb, c, _DT[Bc.dtype], _ptr(out), _stream()))
        return out[:, 0] if vec else out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib.sk_sketch_plan_destroy(h)
            except Exception:
                pass
            self._h = None


def sketch_apply_noalloc(B, s, zeta=0, seed=7):
    """sketch_apply (sparse sign) that allocates no device memory.

    For callers that must not allocate on their hot path (e.g. code running
    inside another framework's engine, which owns the memory budget).  Uses
    libsk's fixed 32 MiB device scratch array; concurrent calls race.  The
    output tensor is the caller's to allocate beforehand in real use; this
    wrapper allocates it with torch for convenience.
    """
    vec = B.dim() == 1
    Bc = colmajor(B)
    n, c = Bc.shape
    ldb = Bc.stride(1) if c > 1 else n
    out = empty_colmajor(s, c, torch.float64, Bc.device)
    sk = _sketch_struct("sparse", n, s, zeta, seed)
    N.check(N.lib.sketch_apply_noalloc(C.byref(sk), _ptr(Bc), ldb, c, _DT[Bc.dtype], _ptr(out), _stream()))
    return out[:, 0] if vec else out


def make_opts(basis=torch.float64, sketch="sparse", zeta=0, seed=7, stab_tol=0.0, maxit=10000, cgs_passes=2,
              tau=1e-8, symmetric=False, breakdown=0.0, use_graph=True, persistent=False, batch_workers=0,
              cheb=None, barrier_spins=0, iter_chunk=0, pipeline=True, trunc_tol=0.0, batch_mode="auto",
              batch_elems=0):
    """Solver options.  cheb=(c, dx, dy) selects the Chebyshev basis (§4.3)
    for a spectrum inside [c - dx, c + dx] x [-dy, dy].  iter_chunk > 0
    selects iterative sGMRES (§5.2): the cycle grows the basis iter_chunk
    columns at a time and stops at the first prefix whose residual estimate
    meets the target.  pipeline=False runs the cycle's phases one after
    another instead of overlapping the sketch and QR of finished basis
    blocks with the basis passes.  batch_mode ("auto", "grouped",
    "workers") and batch_elems (resident elements of a grouped batch, 0 =
    2^22) shape sgmres_solve_batched."""
    o = N.SkOpts()
    N.lib.sk_opts_default(C.byref(o))
    o.sketch = _KIND[sketch]
    o.zeta = int(zeta)
    o.seed = int(seed)
    o.stab_tol = float(stab_tol)
    o.maxit = int(maxit)
    o.basis = _DT[basis]
    o.cgs_passes = int(cgs_passes)
    o.tau = float(tau)
    o.symmetric = int(bool(symmetric))
    o.breakdown = float(breakdown)
    o.use_graph = int(bool(use_graph))
    o.persistent = int(bool(persistent))
    o.batch_workers = int(batch_workers)
    o.barrier_spins = int(barrier_spins)
    o.iter_chunk = int(iter_chunk)
    o.pipeline = int(bool(pipeline))
    o.srr_trunc_tol = float(trunc_tol)
    o.batch_mode = {"auto": 0, "grouped": 1, "workers": 2}[batch_mode]
    o.batch_elems = int(batch_elems)
    if cheb is not None:
        o.basis_kind = 1
        o.cheb_c, o.cheb_dx, o.cheb_dy = (float(v) for v in cheb)
    return o


def workspace_bytes(A, d, k, s, **opts):
    """Device bytes sgmres_solve allocates for this operator and shape."""
    o = make_opts(**opts)
    return int(N.lib.sk_workspace_bytes(A._h, d, k, s, C.byref(o)))


def trunc_arnoldi_basis(A, r0, d, k, dtype=torch.float64, s=None, zeta=0, seed=7, kind="sparse", cgs_passes=2,
                        persistent=False, cheb=None, barrier_spins=0):
    """k-truncated Arnoldi basis (§1.2.2 eq. (partorth)).

    Returns dict(B (n x (d+1), column-major), Hbar ((d+1) x d), SB, SAB (s x d
    or None), d_used).
    """
    r0 = _dev_f64(r0, A.n)
    B = empty_colmajor(A.n, d + 1, dtype, r0.device)
    Hbar = empty_colmajor(d + 1, d, torch.float64, r0.device)
    SB = SAB = None
    skp = None
    if s is not None:
        skp = _sketch_struct(kind, A.n, s, zeta if zeta else default_zeta(d), seed)
        SB = empty_colmajor(s, d, torch.float64, r0.device)
        SAB = empty_colmajor(s, d, torch.float64, r0.device)
    du = C.c_int(0)
    o = make_opts(basis=dtype, cgs_passes=cgs_passes, persistent=persistent, cheb=cheb,
                  barrier_spins=barrier_spins)
    N.check(N.lib.trunc_arnoldi_basis(A._h, _ptr(r0), d, k, _DT[dtype], _ptr(B), _ptr(Hbar),
                                      C.byref(skp) if skp is not None else None, _ptr(SB), _ptr(SAB),
                                      C.byref(o), C.byref(du), _stream()))
    return dict(B=B, Hbar=Hbar, SB=SB, SAB=SAB, d_used=du.value)


def sgmres_solve(A, b, d, k, s, tol, x0=None, raise_on_noconv=False, **opts):
    """Restarted sGMRES (Algorithm 1, §3.5).  Returns (x, info dict)."""
    b = _dev_f64(b, A.n)
    x = torch.zeros_like(b) if x0 is None else _dev_f64(x0, A.n).clone()
    o = make_opts(**opts)
    info = N.SkInfo()
    allow = (N.SK_OK,) if raise_on_noconv else (N.SK_OK, N.SK_ENOCONV)
    st = N.check(N.lib.sgmres_solve(A._h, _ptr(b), _ptr(x), d, k, s, float(tol), C.byref(o), C.byref(info),
                                    _stream()), allow=allow)
    out = info.as_dict()
    out["status"] = st
    return x, out


class SgmresPlan:
    """A reusable restarted-sGMRES solver for one operator and shape: the
    sketch plan, buffers and captured cycle graph are built once; each
    solve(b) computes what sgmres_solve(A, b, d, k, s, tol) computes, without
    the per-call setup.  The operator must outlive the plan."""

    def __init__(self, A, d, k, s, **opts):
        self.A, self.n = A, A.n
        self._h = C.c_void_p()
        o = make_opts(**opts)
        N.check(N.lib.sgmres_plan_create(A._h, d, k, s, C.byref(o), C.byref(self._h), _stream()))

    def solve(self, b, tol, x0=None, raise_on_noconv=False):
        b = _dev_f64(b, self.n)
        x = torch.zeros_like(b) if x0 is None else _dev_f64(x0, self.n).clone()
        info = N.SkInfo()
        allow = (N.SK_OK,) if raise_on_noconv else (N.SK_OK, N.SK_ENOCONV)
        st = N.check(N.lib.sgmres_plan_solve(self._h, _ptr(b), _ptr(x), float(tol), C.byref(info), _stream()),
                     allow=allow)
        out = info.as_dict()
        out["status"] = st
        return x, out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                N.lib.sgmres_plan_destroy(h)
            except Exception:
                pass
            self._h = None


def sgmres_solve_batched(ops, bs, d, k, s, tol, x0s=None, **opts):
    """Batched restarted sGMRES over independent jobs.

    ops: list of nsys Op; bs: list of nsys lists of nrhs CUDA tensors.
    Returns (xs like bs, per-job status list, aggregate info dict); the
    aggregate dict carries "jobs", the per-job info dicts in the order of
    the flattened (system, right-hand side) list.
    """
    nsys = len(ops)
    nrhs = len(bs[0])
    flat_b = [_dev_f64(bs[i][r], ops[i].n) for i in range(nsys) for r in range(nrhs)]
    if x0s is None:
        flat_x = [torch.zeros_like(t) for t in flat_b]
    else:
        flat_x = [_dev_f64(x0s[i][r], ops[i].n).clone() for i in range(nsys) for r in range(nrhs)]
    PA = (C.c_void_p * nsys)(*[op._h.value for op in ops])
    PB = (C.c_void_p * (nsys * nrhs))(*[t.data_ptr() for t in flat_b])
    PX = (C.c_void_p * (nsys * nrhs))(*[t.data_ptr() for t in flat_x])
    stat = (C.c_int * (nsys * nrhs))()
    jinfo = (N.SkInfo * (nsys * nrhs))()
    o = make_opts(**opts)
    info = N.SkInfo()
    N.check(N.lib.sgmres_solve_batched(nsys, PA, nrhs, PB, PX, d, k, s, float(tol), C.byref(o), stat, jinfo,
                                       C.byref(info), _stream()), allow=(N.SK_OK, N.SK_ENOCONV))
    xs = [[flat_x[i * nrhs + r] for r in range(nrhs)] for i in range(nsys)]
    out = info.as_dict()
    out["jobs"] = [jinfo[j].as_dict() for j in range(nsys * nrhs)]
    return xs, list(stat), out


def _batch_sample(ops, bs, sample):
    nsys = len(ops)
    order = sorted(range(nsys), key=lambda i: -ops[i].n)
    pick = sorted(set(order[int(q * (nsys - 1) / max(1, min(sample, nsys) - 1))] for q in range(min(sample, nsys))))
    return [ops[i] for i in pick], [bs[i][:1] for i in pick]


def autotune_batch(ops, bs, d, k, s, tol, candidates=(1 << 21, 1 << 22, 1 << 23), sample=256, **opts):
    """Pick the grouped batch's resident-element budget (batch_elems) by
    timing a sample of the jobs (spread evenly over the size range, one
    right-hand side each).  Returns (best, {batch_elems: seconds})."""
    import time
    sops, sbs = _batch_sample(ops, bs, sample)
    timings = {}
    for e in candidates:
        torch.cuda.synchronize()
        t = time.perf_counter()
        sgmres_solve_batched(sops, sbs, d, k, s, tol, batch_mode="grouped", batch_elems=e, **opts)
        torch.cuda.synchronize()
        timings[e] = time.perf_counter() - t
    best = min(timings, key=timings.get)
    return best, timings


def autotune_batch_workers(ops, bs, d, k, s, tol, candidates=(4, 8, 16, 32, 48), sample=48, **opts):
    """Pick the number of worker threads of batch_mode="workers" (one job
    per thread and stream) by timing a sample of jobs spread evenly over
    the size range.  Returns (best, {workers: seconds})."""
    import time
    sops, sbs = _batch_sample(ops, bs, sample)
    timings = {}
    for w in candidates:
        torch.cuda.synchronize()
        t = time.perf_counter()
        sgmres_solve_batched(sops, sbs, d, k, s, tol, batch_mode="workers", batch_workers=w, **opts)
        torch.cuda.synchronize()
        timings[w] = time.perf_counter() - t
    best = min(timings, key=timings.get)
    return best, timings


def srr_eigs(A, w1, nev, d, k, s, **opts):
    """Sketched Rayleigh-Ritz (Algorithm 2).  Returns dict(lam, X, rhat, nconv, info)."""
    w1 = _dev_f64(w1, A.n)
    o = make_opts(**opts)
    lre = (C.c_double * nev)()
    lim = (C.c_double * nev)()
    rh = (C.c_double * nev)()
    Xr = empty_colmajor(A.n, nev, torch.float64, w1.device)
    Xi = empty_colmajor(A.n, nev, torch.float64, w1.device)
    nconv = C.c_int(0)
    info = N.SkInfo()
    N.check(N.lib.srr_eigs(A._h, _ptr(w1), nev, d, k, s, C.byref(o), lre, lim, _ptr(Xr), _ptr(Xi), rh,
                           C.byref(nconv), C.byref(info), _stream()))
    lam = torch.tensor([complex(a, b) for a, b in zip(lre, lim)], dtype=torch.complex128)
    return dict(lam=lam, X=torch.complex(Xr, Xi), rhat=torch.tensor(list(rh)), nconv=nconv.value,
                info=info.as_dict())


def srr_basis(A, B, nev, s, **opts):
    """Sketched Rayleigh-Ritz on a given basis B (n x d CUDA tensor, float64/
    float32/bfloat16): A B is formed on the GPU, then Algorithm 2's reduction,
    or the stabilized form of §6.5 with opts trunc_tol > 0.  Returns
    dict(lam, X, rhat, nconv, rank)."""
    Bc = colmajor(B)
    if Bc.dtype not in _DT:
        raise ValueError("dtype must be float64, float32 or bfloat16")
    n, d = Bc.shape
    o = make_opts(**opts)
    lre = (C.c_double * nev)()
    lim = (C.c_double * nev)()
    rh = (C.c_double * nev)()
    Xr = empty_colmajor(n, nev, torch.float64, Bc.device)
    Xi = empty_colmajor(n, nev, torch.float64, Bc.device)
    nconv = C.c_int(0)
    rank = C.c_int(0)
    N.check(N.lib.srr_basis(A._h, _ptr(Bc), Bc.stride(1) if d > 1 else n, d, _DT[Bc.dtype], nev, s, C.byref(o),
                            lre, lim, _ptr(Xr), _ptr(Xi), rh, C.byref(nconv), C.byref(rank), _stream()))
    lam = torch.tensor([complex(a, b) for a, b in zip(lre, lim)], dtype=torch.complex128)
    return dict(lam=lam, X=torch.complex(Xr, Xi), rhat=torch.tensor(list(rh)), nconv=nconv.value, rank=rank.value)


def srr_restarted(A, Omega, p, nev, lo, hi, max_restarts, filter_degree=0, **opts):
    """Restarted sRR (§7.2) on block Chebyshev bases (§7.5) from the start
    block Omega (n x b, float64); [lo, hi] brackets the real spectrum;
    filter_degree > 0 filters each start block by a Chebyshev polynomial of
    that degree first.
    Returns dict(lam, X, rhat, nconv, restarts, history, status)."""
    Om = colmajor(_dev_f64(Omega) if Omega.dim() == 1 else Omega.to(torch.float64))
    n, b = Om.shape
    o = make_opts(**opts)
    lre = (C.c_double * nev)()
    lim = (C.c_double * nev)()
    rh = (C.c_double * nev)()
    hist = (C.c_double * max_restarts)()
    Xr = empty_colmajor(n, nev, torch.float64, Om.device)
    Xi = empty_colmajor(n, nev, torch.float64, Om.device)
    nconv = C.c_int(0)
    nres = C.c_int(0)
    st = N.check(N.lib.srr_restarted(A._h, _ptr(Om), b, p, nev, float(lo), float(hi), max_restarts,
                                     int(filter_degree), C.byref(o), lre,
                                     lim, _ptr(Xr), _ptr(Xi), rh, C.byref(nconv), C.byref(nres), hist, _stream()),
                 allow=(N.SK_OK, N.SK_ENOCONV))
    lam = torch.tensor([complex(a, b) for a, b in zip(lre, lim)], dtype=torch.complex128)
    return dict(lam=lam, X=torch.complex(Xr, Xi), rhat=torch.tensor(list(rh)), nconv=nconv.value,
                restarts=nres.value, history=list(hist)[:nres.value], status=st)


def _adjoint(op, x, gx, d, k, s, tol, opts):
    """Backward of x = A^{-1} b: lam = A^{-T} dL/dx by sGMRES with A^T (the
    library's transposed operator, the same kernels), then dL/db = lam and
    dL/dparams = -d(lam^T A x)/dparams (sk_op_param_grad with alpha = -1)."""
    gx = gx.detach().to(torch.float64).contiguous()
    if float(gx.abs().max()) == 0.0:
        lam = torch.zeros_like(gx)
    else:
        lam, info = sgmres_solve(op.T, gx, d, k, s, tol, **opts)
        if info["status"] != N.SK_OK:
            raise SkError(info["status"], "adjoint solve did not reach tol (relres %g)" % info["relres"])
    return lam, op.param_grad(lam, x, alpha=-1.0)


def _forward(op, b, d, k, s, tol, opts):
    x, info = sgmres_solve(op, b.detach(), d, k, s, tol, **opts)
    if info["status"] != N.SK_OK:
        raise SkError(info["status"], "forward solve did not reach tol (relres %g)" % info["relres"])
    return x, info


class DiffusionSolve(torch.autograd.Function):
    """x = A(theta)^{-1} b by sGMRES, differentiable in theta and b.

    A(theta) is the variable-coefficient diffusion operator on an nx x ny grid
    (Op.diffusion_var).  The backward pass is the adjoint: one sGMRES solve
    with A^T for lam = A^{-T} dL/dx (the same library kernels), then
    dL/db = lam and dL/dtheta = -d(lam^T A x)/dtheta (Op.param_grad).
    The paper has no differentiable solve; this is the adjoint method built on
    Algorithm 1.
    """

    @staticmethod
    def forward(ctx, theta, b, nx, ny, d, k, s, tol, opts):
        op = Op.diffusion_var(nx, ny, theta.detach())
        x, info = _forward(op, b, d, k, s, tol, opts)
        ctx.save_for_backward(theta.detach(), x)
        ctx.cfg = (nx, ny, d, k, s, tol, opts)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        theta, x = ctx.saved_tensors
        nx, ny, d, k, s, tol, opts = ctx.cfg
        lam, gtheta = _adjoint(Op.diffusion_var(nx, ny, theta), x, gx, d, k, s, tol, opts)
        return gtheta, lam, None, None, None, None, None, None, None


def diffusion_solve(theta, b, nx, ny, d=100, k=2, s=200, tol=1e-10, **opts):
    """Differentiable x = A(theta)^{-1} b (see DiffusionSolve)."""
    return DiffusionSolve.apply(theta, b, nx, ny, d, k, s, tol, opts)


class StencilSolve(torch.autograd.Function):
    """x = A(c, shift)^{-1} b by sGMRES for the five-point stencil operator
    (Op.stencil5), differentiable in the five coefficients c, the diagonal
    shift (if given) and b.  Backward: the adjoint solve with the transposed
    stencil, then dL/dc and dL/dshift from sk_op_param_grad (alpha = -1)."""

    @staticmethod
    def forward(ctx, coef, shift, b, nx, ny, d, k, s, tol, opts):
        cf = [float(v) for v in coef.detach().cpu()]
        sh = shift.detach() if shift is not None else None
        op = Op.stencil5(nx, ny, cf, sh)
        x, info = _forward(op, b, d, k, s, tol, opts)
        ctx.save_for_backward(x)
        ctx.cfg = (cf, sh, nx, ny, d, k, s, tol, opts, coef.device, coef.dtype)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        cf, sh, nx, ny, d, k, s, tol, opts, cdev, cdt = ctx.cfg
        lam, g = _adjoint(Op.stencil5(nx, ny, cf, sh), x, gx, d, k, s, tol, opts)
        gc = g[:5].to(device=cdev, dtype=cdt)
        gs = g[5:] if sh is not None else None
        return gc, gs, lam, None, None, None, None, None, None, None


def stencil_solve(coef, b, nx, ny, shift=None, d=100, k=2, s=200, tol=1e-10, **opts):
    """Differentiable x = A(coef, shift)^{-1} b (see StencilSolve); coef is a
    tensor of the five coefficients (centre, E, W, N, S)."""
    return StencilSolve.apply(coef, shift, b, nx, ny, d, k, s, tol, opts)


class CsrSolve(torch.autograd.Function):
    """x = A(val)^{-1} b by sGMRES for a general sparse operator (Op.csr with a
    fixed pattern rowptr/colind), differentiable in the stored values and b.
    Backward: the adjoint solve with the library's CSR transpose, then
    dL/dval = -lam_row x_col (sk_op_param_grad, alpha = -1, on A's entries)."""

    @staticmethod
    def forward(ctx, val, b, rowptr, colind, d, k, s, tol, opts):
        op = Op.csr(rowptr, colind, val.detach())
        x, info = _forward(op, b, d, k, s, tol, opts)
        ctx.save_for_backward(val.detach(), x)
        ctx.cfg = (rowptr, colind, d, k, s, tol, opts)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        val, x = ctx.saved_tensors
        rowptr, colind, d, k, s, tol, opts = ctx.cfg
        lam, gval = _adjoint(Op.csr(rowptr, colind, val), x, gx, d, k, s, tol, opts)
        return gval, lam, None, None, None, None, None, None, None


def csr_solve(val, b, rowptr, colind, d=100, k=2, s=200, tol=1e-10, **opts):
    """Differentiable x = A(val)^{-1} b for a CSR pattern (see CsrSolve)."""
    return CsrSolve.apply(val, b, rowptr, colind, d, k, s, tol, opts)

