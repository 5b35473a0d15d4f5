"""The C-ABI library loads and exports every entry point include/sk.h declares.

No GPU needed: only symbol lookup and host-side argument validation (which
returns before any CUDA call).
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sk.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+([a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g._build_module().build()
    from paper_2111_00113_gb300 import _native
    return _native


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sketch_apply", "trunc_arnoldi_basis", "sgmres_solve", "srr_eigs"):
        assert must in names


def test_every_declared_symbol_is_exported(native):
    lib = C.CDLL(native.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) <= set(native.EXPORTED) | set(_declared())


def test_invalid_arguments_rejected_on_host(native):
    lib = native.lib
    h = C.c_void_p()
    coef = (C.c_double * 5)(4, -1, -1, -1, -1)
    assert lib.sk_op_stencil5(C.byref(h), 0, 5, coef, None) == native.SK_EINVAL
    assert b"nx, ny" in lib.sk_last_error()
    assert lib.sk_op_stencil5(None, 5, 5, coef, None) == native.SK_EINVAL
    bad = (C.c_double * 5)(4, float("nan"), -1, -1, -1)
    assert lib.sk_op_stencil5(C.byref(h), 5, 5, bad, None) == native.SK_EINVAL
    assert lib.sk_op_stencil5(C.byref(h), 5, 5, coef, None) == native.SK_OK
    assert lib.sk_op_n(h) == 25
    hT = C.c_void_p()
    assert lib.sk_op_transpose(h, C.byref(hT)) == native.SK_OK
    info = native.SkInfo()
    o = native.SkOpts()
    lib.sk_opts_default(C.byref(o))
    assert o.cgs_passes == 2 and o.maxit == 10000 and o.seed == 7 and o.use_graph == 1
    dummy = C.c_void_p(16)
    # s < d+1, k > d, tol <= 0, NULL b: all rejected before any launch
    assert lib.sgmres_solve(h, dummy, dummy, 10, 2, 10, 1e-6, None, C.byref(info), None) == native.SK_EINVAL
    assert lib.sgmres_solve(h, dummy, dummy, 10, 11, 40, 1e-6, None, C.byref(info), None) == native.SK_EINVAL
    assert lib.sgmres_solve(h, dummy, dummy, 10, 2, 40, 0.0, None, C.byref(info), None) == native.SK_EINVAL
    assert lib.sgmres_solve(h, None, dummy, 10, 2, 40, 1e-6, None, C.byref(info), None) == native.SK_EINVAL
    sk = native.SkSketch(0, 25, 8, 4, 1)
    assert lib.sketch_apply(C.byref(sk), dummy, 10, 1, 0, dummy, None) == native.SK_EINVAL  # ldb < n
    # option combinations rejected before any device work
    o1 = native.SkOpts()
    lib.sk_opts_default(C.byref(o1))
    o1.basis, o1.cgs_passes = native.SK_F32, 1  # one Gram-Schmidt pass needs an FP64 basis
    assert lib.sgmres_solve(h, dummy, dummy, 10, 2, 40, 1e-6, C.byref(o1), C.byref(info), None) == native.SK_EINVAL
    assert b"cgs_passes" in lib.sk_last_error()
    o2 = native.SkOpts()
    lib.sk_opts_default(C.byref(o2))
    o2.basis_kind, o2.cheb_c = 1, 4.0  # Chebyshev basis without an interval
    assert lib.sgmres_solve(h, dummy, dummy, 10, 2, 40, 1e-6, C.byref(o2), C.byref(info), None) == native.SK_EINVAL
    assert b"Chebyshev" in lib.sk_last_error()
    o2.basis_kind = 7  # unknown basis kind
    assert lib.sgmres_solve(h, dummy, dummy, 10, 2, 40, 1e-6, C.byref(o2), C.byref(info), None) == native.SK_EINVAL
    o3 = native.SkOpts()
    lib.sk_opts_default(C.byref(o3))
    assert o3.basis_kind == 0 and o3.barrier_spins == 0 and o3.persistent == 0 and o3.iter_chunk == 0
    # iterative sGMRES: the chunk is a positive multiple of the QR panel
    # width (16), at most 1024, with the truncated-Arnoldi basis only
    for bad_chunk in (8, -16, 2048):
        o3.iter_chunk = bad_chunk
        assert lib.sgmres_solve(h, dummy, dummy, 10, 2, 40, 1e-6, C.byref(o3), C.byref(info), None) == native.SK_EINVAL
        assert b"iter_chunk" in lib.sk_last_error()
    o3.iter_chunk, o3.basis_kind, o3.cheb_c, o3.cheb_dx = 16, 1, 4.0, 4.0
    assert lib.sgmres_solve(h, dummy, dummy, 10, 2, 40, 1e-6, C.byref(o3), C.byref(info), None) == native.SK_EINVAL
    assert b"truncated-Arnoldi" in lib.sk_last_error()
    # batched: grouped by default where the options allow it; batch_mode = 1
    # with an SRHT sketch is refused on the host (FP64 basis: no device work)
    o4 = native.SkOpts()
    lib.sk_opts_default(C.byref(o4))
    assert o4.batch_mode == 0 and o4.batch_elems == 0
    o4.batch_mode, o4.sketch = 1, native.SK_SRHT
    PA = (C.c_void_p * 1)(h)
    PB = (C.c_void_p * 1)(dummy)
    st = (C.c_int * 1)()
    assert lib.sgmres_solve_batched(1, PA, 1, PB, PB, 10, 2, 40, 1e-6, C.byref(o4), st, None, C.byref(info),
                                    None) == native.SK_EINVAL
    assert b"grouped" in lib.sk_last_error() and b"sparse sign" in lib.sk_last_error()
    lib.sk_op_destroy(hT)
    lib.sk_op_destroy(h)


def test_workspace_bytes_accounts_for_the_basis(native):
    # sk_workspace_bytes on the bench workload (1024^2, d = 300, s = 600):
    # the basis n x (d+1) dominates; the FP64 form adds the FP64 basis and
    # the stored A b_j; invalid shapes give 0.  Host-only (no device needed).
    lib = native.lib
    h = C.c_void_p()
    coef = (C.c_double * 5)(4, -0.9, -1.1, -0.9, -1.1)
    assert lib.sk_op_stencil5(C.byref(h), 1024, 1024, coef, None) == native.SK_OK
    o = native.SkOpts()
    lib.sk_opts_default(C.byref(o))
    n, d, s = 1 << 20, 300, 600
    o.basis = native.SK_F32
    b32 = lib.sk_workspace_bytes(h, d, 2, s, C.byref(o))
    assert n * (d + 1) * 4 < b32 < 1.15 * n * (d + 1) * 4
    o.basis = native.SK_F64
    b64 = lib.sk_workspace_bytes(h, d, 2, s, C.byref(o))
    assert b64 - b32 >= n * (d + 1) * 4 + n * 8
    assert lib.sk_workspace_bytes(h, d, 2, d, C.byref(o)) == 0  # s < d + 1
    assert lib.sk_workspace_bytes(h, 0, 1, s, C.byref(o)) == 0
    lib.sk_op_destroy(h)
