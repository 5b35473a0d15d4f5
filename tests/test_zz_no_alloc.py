"""sketch_apply_noalloc: the sparse sign sketch without device allocation.

Some callers cannot allocate device memory on their hot path (code running
inside another framework's engine, which owns the memory budget and where
cudaMalloc may synchronise the device; latency-critical loops).  This file is
collected last on purpose: it exercises the library's shared fixed scratch
array after everything else has run, and also passes alone in a fresh process.
Each output is compared with the FP64 CPU oracle's sketch (oracle/sketch.py)
of the values the GPU holds, and with the allocating sketch_apply, over
calls in a row of different shapes (the scratch keeps the previous call's
contents; a later call must not see them).
"""
import ctypes as C

import numpy as np
import pytest

from oracle import sketch

pytestmark = pytest.mark.gpu


def _call_noalloc(native, S, B, ldb, ncols, dtype, out, stream):
    return native.lib.sketch_apply_noalloc(C.byref(S), C.c_void_p(B.data_ptr()), ldb, ncols, dtype,
                                           C.c_void_p(out.data_ptr()), stream)


def _relf(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_oracle_and_sketch_apply():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    import paper_2111_00113_gb300 as skg
    from paper_2111_00113_gb300 import _native as native

    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    codes = {torch.float64: native.SK_F64, torch.float32: native.SK_F32, torch.bfloat16: native.SK_BF16}
    cases = [  # (n, ncols, s, zeta, seed, dtype): different shapes so stale scratch would show
        (1024 * 7 + 5, 9, 600, 12, 3, torch.float64),   # row-owner gather, FP64
        (100003, 4, 200, 10, 11, torch.float32),        # general gather, FP32
        (1024 * 5 + 3, 1, 600, 12, 5, torch.float64),   # one FP64 column (g = S r kernel)
        (1024 * 3 + 17, 6, 300, 9, 2, torch.bfloat16),  # BF16 storage
        (1024 * 7 + 5, 9, 600, 12, 3, torch.float64),   # the first shape again
    ]
    gen = torch.Generator(device="cuda").manual_seed(0)
    for n, c, s, zeta, seed, dt in cases:
        X = torch.randn((c, n), generator=gen, dtype=torch.float64, device="cuda").to(dt).t()
        held = X.to(torch.float64).cpu().numpy()  # the values the GPU holds
        ref = sketch.sparse_sign_apply(seed, s, zeta, held)
        out = torch.full((c, s), float("nan"), dtype=torch.float64, device="cuda").t()
        S = native.SkSketch(native.SK_SPARSE_SIGN, n, s, zeta, seed)
        st = _call_noalloc(native, S, X, X.stride(1) if c > 1 else n, c, codes[dt], out, stream)
        assert st == native.SK_OK, native.lib.sk_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        tol = 1e-12 if dt == torch.float64 else 1e-5
        assert _relf(got, ref) <= tol, (n, c, s, dt, _relf(got, ref))
        alloc = skg.sketch_apply(X, s, zeta, seed).reshape(s, c).cpu().numpy()
        assert _relf(got, alloc) <= tol, (n, c, s, dt)


def test_noalloc_hash_failure_then_success():
    # s = zeta = 14: the last slot of a column must hit the one remaining row
    # within 16 attempts, which fails for some of 4096 columns: SK_EHASH.  The
    # status word lives in the shared scratch; the next valid call clears it.
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2111_00113_gb300 import _native as native
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 4096
    X = torch.randn((3, n), dtype=torch.float64, device="cuda").t()
    out = torch.empty((3, 14), dtype=torch.float64, device="cuda").t()
    bad = native.SkSketch(native.SK_SPARSE_SIGN, n, 14, 14, 1)
    assert _call_noalloc(native, bad, X, X.stride(1), 3, native.SK_F64, out, stream) == native.SK_EHASH
    out2 = torch.empty((3, 80), dtype=torch.float64, device="cuda").t()
    good = native.SkSketch(native.SK_SPARSE_SIGN, n, 80, 8, 1)
    assert _call_noalloc(native, good, X, X.stride(1), 3, native.SK_F64, out2, stream) == native.SK_OK
    torch.cuda.synchronize()
    ref = sketch.sparse_sign_apply(1, 80, 8, X.cpu().numpy())
    assert _relf(out2.cpu().numpy(), ref) <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2111_00113_gb300 import _native as native
    n = 1 << 24  # 16384 chunks x 1024 rows x 12 entries x 2 bytes of tables alone exceed 32 MiB
    S = native.SkSketch(native.SK_SPARSE_SIGN, n, 600, 12, 7)
    dummy = C.c_void_p(256)
    st = native.lib.sketch_apply_noalloc(C.byref(S), dummy, n, 1, native.SK_F32, dummy, None)
    assert st == native.SK_EINVAL
    assert b"bytes of scratch" in native.lib.sk_last_error()
