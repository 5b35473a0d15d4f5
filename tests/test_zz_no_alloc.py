"""sketch_apply_noalloc: the sparse sign sketch without device allocation.

Some callers cannot allocate device memory on their hot path (code running
inside another framework's engine, which owns the memory budget and where
cudaMalloc may synchronise the device; latency-critical loops).  This file is
collected last on purpose: it exercises the library's shared fixed scratch
array after everything else has run, and also passes alone in a fresh process.
The output is compared with the allocating sketch_apply over two calls in a
row (the scratch keeps the previous call's contents; the second call must not
see them).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(native, S, B, ldb, ncols, dtype, out, stream):
    return native.lib.sketch_apply_noalloc(C.byref(S), C.c_void_p(B.data_ptr()), ldb, ncols, dtype,
                                           C.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_sketch_apply_two_calls():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    import paper_2111_00113_gb300 as skg
    from paper_2111_00113_gb300 import _native as native

    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [  # (n, ncols, s, zeta, seed, dtype): different shapes so stale scratch would show
        (2048 * 7 + 5, 9, 600, 12, 3, torch.float64),
        (100003, 4, 200, 10, 11, torch.float32),
    ]
    for n, c, s, zeta, seed, dt in cases:
        X = torch.randn((c, n), dtype=torch.float64, device="cuda").to(dt).t()
        ref = skg.sketch_apply(X, s, zeta, seed)
        out = torch.full((c, s), float("nan"), dtype=torch.float64, device="cuda").t()
        S = native.SkSketch(native.SK_SPARSE_SIGN, n, s, zeta, seed)
        dcode = native.SK_F64 if dt == torch.float64 else native.SK_F32
        st = _call_noalloc(native, S, X, X.stride(1), c, dcode, out, stream)
        assert st == native.SK_OK, native.lib.sk_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
        tol = 1e-12 if dt == torch.float64 else 1e-5
        assert err <= tol, (n, c, s, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2111_00113_gb300 import _native as native
    n = 1 << 24  # 8192 chunks x 2048 x 12 x 2 bytes of tables alone exceed 32 MiB
    S = native.SkSketch(native.SK_SPARSE_SIGN, n, 600, 12, 7)
    dummy = C.c_void_p(256)
    st = native.lib.sketch_apply_noalloc(C.byref(S), dummy, n, 1, native.SK_F32, dummy, None)
    assert st == native.SK_EINVAL
    assert b"bytes of scratch" in native.lib.sk_last_error()
