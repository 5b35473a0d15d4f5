"""ctypes declarations of the C ABI in include/sk.h (libsk.so, built in-tree).

Argument marshalling only: every computation happens in libsk's CUDA kernels.
Importing this module never falls back to anything else; if libsk.so is
missing or cannot be loaded, the import raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsk.so")

SK_OK, SK_EINVAL, SK_ENOMEM, SK_ECUDA, SK_ENAN, SK_ENOCONV, SK_EILLCOND, SK_ETIMEOUT, SK_EHASH = range(9)
SK_F64, SK_F32, SK_BF16 = 0, 1, 2
SK_SPARSE_SIGN, SK_SRHT = 0, 1

EXPORTED = [
    "sk_op_stencil5", "sk_op_diffusion_var", "sk_op_csr", "sk_op_transpose", "sk_op_apply", "sk_op_n",
    "sk_op_destroy", "sketch_apply", "sketch_apply_noalloc", "sk_opts_default", "trunc_arnoldi_basis", "sgmres_solve", "srr_eigs",
    "sk_last_error", "sk_status_string", "sk_op_param_grad", "sgmres_solve_batched", "srr_basis", "srr_restarted",
    "sk_workspace_bytes", "sk_sketch_plan_create", "sk_sketch_plan_apply", "sk_sketch_plan_destroy",
    "sgmres_plan_create", "sgmres_plan_solve", "sgmres_plan_destroy",
]


class SkSketch(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int64), ("s", C.c_int), ("zeta", C.c_int), ("seed", C.c_uint64)]


class SkOpts(C.Structure):
    _fields_ = [
        ("sketch", C.c_int), ("zeta", C.c_int), ("seed", C.c_uint64), ("stab_tol", C.c_double),
        ("maxit", C.c_int), ("basis", C.c_int), ("cgs_passes", C.c_int), ("tau", C.c_double),
        ("symmetric", C.c_int), ("breakdown", C.c_double), ("use_graph", C.c_int), ("persistent", C.c_int),
        ("batch_workers", C.c_int), ("basis_kind", C.c_int), ("cheb_c", C.c_double), ("cheb_dx", C.c_double),
        ("cheb_dy", C.c_double), ("barrier_spins", C.c_int), ("iter_chunk", C.c_int), ("srr_trunc_tol", C.c_double),
        ("pipeline", C.c_int), ("batch_mode", C.c_int), ("batch_elems", C.c_longlong),
    ]


class SkInfo(C.Structure):
    _fields_ = [
        ("cycles", C.c_int), ("matvecs", C.c_int), ("d_used", C.c_int), ("width", C.c_int),
        ("relres", C.c_double), ("rhat_est", C.c_double), ("kappa_T_max", C.c_double),
        ("ms", C.c_float * 6), ("launches", C.c_longlong),
    ]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "ms" else getattr(self, k)) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsk.so is not built (run __graft_entry__.build() or python -m "
                           "paper_2111_00113_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    I = C.c_int
    I64 = C.c_int64
    D = C.c_double
    st = C.c_int
    sig = {
        "sk_op_stencil5": (st, [C.POINTER(P), I, I, C.POINTER(D), P]),
        "sk_op_diffusion_var": (st, [C.POINTER(P), I, I, P]),
        "sk_op_csr": (st, [C.POINTER(P), I64, I64, P, P, P]),
        "sk_op_transpose": (st, [P, C.POINTER(P)]),
        "sk_op_apply": (st, [P, P, P, P]),
        "sk_op_n": (I64, [P]),
        "sk_op_param_grad": (st, [P, P, P, D, P, P]),
        "sk_op_destroy": (None, [P]),
        "sketch_apply": (st, [C.POINTER(SkSketch), P, I64, I, I, P, P]),
        "sketch_apply_noalloc": (st, [C.POINTER(SkSketch), P, I64, I, I, P, P]),
        "sk_opts_default": (None, [C.POINTER(SkOpts)]),
        "trunc_arnoldi_basis": (st, [P, P, I, I, I, P, P, C.POINTER(SkSketch), P, P, C.POINTER(SkOpts),
                                     C.POINTER(I), P]),
        "sgmres_solve": (st, [P, P, P, I, I, I, D, C.POINTER(SkOpts), C.POINTER(SkInfo), P]),
        "sgmres_solve_batched": (st, [I, C.POINTER(P), I, C.POINTER(P), C.POINTER(P), I, I, I, D,
                                      C.POINTER(SkOpts), C.POINTER(C.c_int), C.POINTER(SkInfo),
                                      C.POINTER(SkInfo), P]),
        "srr_eigs": (st, [P, P, I, I, I, I, C.POINTER(SkOpts), C.POINTER(D), C.POINTER(D), P, P,
                          C.POINTER(D), C.POINTER(I), C.POINTER(SkInfo), P]),
        "srr_basis": (st, [P, P, I64, I, I, I, I, C.POINTER(SkOpts), C.POINTER(D), C.POINTER(D), P, P,
                           C.POINTER(D), C.POINTER(I), C.POINTER(I), P]),
        "srr_restarted": (st, [P, P, I, I, I, D, D, I, I, C.POINTER(SkOpts), C.POINTER(D), C.POINTER(D), P, P,
                               C.POINTER(D), C.POINTER(I), C.POINTER(I), C.POINTER(D), P]),
        "sk_workspace_bytes": (C.c_size_t, [P, I, I, I, C.POINTER(SkOpts)]),
        "sk_sketch_plan_create": (st, [C.POINTER(SkSketch), C.POINTER(P), P]),
        "sk_sketch_plan_apply": (st, [P, P, I64, I, I, P, P]),
        "sk_sketch_plan_destroy": (None, [P]),
        "sgmres_plan_create": (st, [P, I, I, I, C.POINTER(SkOpts), C.POINTER(P), P]),
        "sgmres_plan_solve": (st, [P, P, P, D, C.POINTER(SkInfo), P]),
        "sgmres_plan_destroy": (None, [P]),
        "sk_last_error": (C.c_char_p, []),
        "sk_status_string": (C.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class SkError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (lib.sk_status_string(status).decode(), msg))


def check(status, allow=(SK_OK,)):
    if status not in allow:
        raise SkError(status, lib.sk_last_error().decode())
    return status
