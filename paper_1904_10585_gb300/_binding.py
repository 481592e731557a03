"""ctypes binding of libpf (include/pf.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all
arithmetic runs in the CUDA kernels behind it.  If the shared library is
missing the import fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpf.so")

PF_MAX_P = 64

# pf_status
PF_OK = 0
PF_ERR_INVALID_ARG = 1
PF_ERR_OOM = 2
PF_ERR_CUDA = 3
PF_ERR_CHOL_BREAKDOWN = 4
PF_ERR_NAN = 5
PF_ERR_NOT_CONVERGED = 6
PF_ERR_DEVICE_TIMEOUT = 7
PF_ERR_UNSUPPORTED = 8

PF_OP_DENSE = 0
PF_OP_LOWRANK_SPARSE = 1
PF_PREC_FP64 = 0
PF_PREC_TF32 = 1
PF_PREC_BF16 = 2

PF_DENSE_SLICED = 0
PF_DENSE_FP64 = 1

PF_PROBLEM_MAXCUT = 0
PF_PROBLEM_COMPLETION = 1
PF_PROBLEM_NCE = 2
PF_PROBLEM_SVT = 3
PF_PROBLEM_NNLS = 4


class pf_options(C.Structure):
    _fields_ = [("p", C.c_int32), ("degree", C.c_int32), ("degree_max", C.c_int32),
                ("q", C.c_int32), ("eta", C.c_double), ("precision", C.c_int32),
                ("adaptive", C.c_int32), ("p_min", C.c_int32), ("adapt_guard", C.c_int32),
                ("adapt_every", C.c_int32), ("dense_product", C.c_int32)]


class pf_operator(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int64),
                ("A", C.c_void_p), ("lda", C.c_int64),
                ("A_lp", C.c_void_p), ("lda_lp", C.c_int64), ("lp_scale", C.c_double),
                ("Uf", C.c_void_p), ("lduf", C.c_int64), ("lam", C.c_void_p), ("r", C.c_int32),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("vals", C.c_void_p),
                ("nnz", C.c_int64), ("sparse_scale", C.c_double), ("shift", C.c_double)]


class pf_problem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int64),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("vals_f64", C.c_void_p), ("vals_f32", C.c_void_p), ("nnz", C.c_int64),
                ("t", C.c_double), ("mu", C.c_double),
                ("U", C.c_void_p), ("ldu", C.c_int64),
                ("V", C.c_void_p), ("ldv", C.c_int64),
                ("theta", C.c_void_p),
                ("Z", C.c_void_p), ("ldz", C.c_int64),
                ("Z_lp", C.c_void_p), ("ldz_lp", C.c_int64),
                ("lam", C.c_void_p), ("S", C.c_void_p), ("iter", C.c_int64),
                ("accel_l", C.c_int32), ("accel_lam", C.c_double), ("hist", C.c_void_p),
                ("p_active", C.c_int32), ("guard", C.c_void_p), ("ldg", C.c_int64),
                ("t_rowptr", C.c_void_p), ("t_colind", C.c_void_p), ("t_perm", C.c_void_p),
                ("fac", C.c_void_p), ("ldfac", C.c_int64), ("fsv", C.c_void_p),
                ("rank_cap", C.c_int32), ("Z_tf32", C.c_void_p), ("ldz_tf32", C.c_int64)]


class pf_iter_info(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("obj", C.c_double), ("kkt", C.c_double),
                ("pinf", C.c_double), ("dinf", C.c_double), ("gap", C.c_double),
                ("theta_max", C.c_double), ("theta_min", C.c_double),
                ("r_plus", C.c_int32), ("flags", C.c_int32), ("degree", C.c_int32),
                ("precision", C.c_int32), ("jacobi_sweeps", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pf_result(C.Structure):
    _fields_ = [("iters", C.c_int64), ("kkt", C.c_double), ("obj", C.c_double),
                ("last", pf_iter_info)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libpf.so not found at {LIB_PATH}: build the CUDA library first "
            "(python -m paper_1904_10585_gb300.build); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sigs = {
        "pf_create": (C.c_int, [C.POINTER(pf_options), C.c_int64, P, C.POINTER(P)]),
        "pf_destroy": (C.c_int, [P]),
        "pf_filter": (C.c_int, [P, C.POINTER(pf_operator), C.c_double, C.c_double, C.c_int32,
                                P, C.c_int64]),
        "pf_rayleigh_ritz": (C.c_int, [P, C.POINTER(pf_operator), P, C.c_int64, P, C.c_int64,
                                       P, P]),
        "pf_apply": (C.c_int, [P, C.POINTER(pf_operator), P, C.c_int64, P, C.c_int64]),
        "pf_kernel_launch_count": (C.c_int64, []),
        "pf_apply_dense_noalloc": (C.c_int, [P, C.c_int64, P, C.c_int64, P, C.c_int64, C.c_int64,
                                             C.c_int32, P]),
        "pf_problem_init": (C.c_int, [P, C.POINTER(pf_problem)]),
        "pf_prox_step": (C.c_int, [P, C.POINTER(pf_problem), C.POINTER(pf_iter_info)]),
        "pf_solve": (C.c_int, [P, C.POINTER(pf_problem), C.c_int64, C.c_double, C.c_int32,
                               C.POINTER(pf_result)]),
        "pf_get_info": (C.c_int, [P, C.POINTER(pf_iter_info)]),
        "pf_enqueue_steps": (C.c_int, [P, C.POINTER(pf_problem), C.c_int64]),
        "pf_report_async": (C.c_int, [P, P]),
        "pf_ladder_update": (C.c_int, [P, C.POINTER(pf_problem), C.c_double]),
        "pf_set_tracing": (C.c_int, [P, C.c_int32]),
        "pf_phase_times": (C.c_int, [P, C.POINTER(C.c_double)]),
        "pf_set_wait_limit": (C.c_int, [C.c_uint64]),
        "pf_status_string": (C.c_char_p, [C.c_int]),
        "pf_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("pf_create", "pf_destroy", "pf_filter", "pf_rayleigh_ritz", "pf_apply",
            "pf_problem_init", "pf_prox_step", "pf_solve", "pf_get_info", "pf_enqueue_steps",
            "pf_report_async",
            "pf_kernel_launch_count", "pf_apply_dense_noalloc", "pf_ladder_update",
            "pf_set_tracing",
            "pf_phase_times", "pf_set_wait_limit", "pf_status_string", "pf_last_error")

# pf_phase (include/pf.h)
PF_NUM_PHASES = 6
PF_PHASE_INTERVAL = 0
PF_PHASE_FILTER = 1
PF_PHASE_ORTH = 2
PF_PHASE_RR = 3
PF_PHASE_EIG = 4
PF_PHASE_UPDATE = 5
PHASE_NAMES = ("interval", "filter", "orth", "rayleigh_ritz", "eigensolve", "update")


class PFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{pf_status_string(status)} ({status}): {msg}")
        self.status = status


def _check(status: int, ctx=None, allow=()):
    if status != PF_OK and status not in allow:
        msg = pf_last_error(ctx) if ctx else ""
        raise PFError(status, msg)
    return status


def pf_status_string(status: int) -> str:
    return _lib.pf_status_string(status).decode()


def pf_last_error(ctx) -> str:
    return _lib.pf_last_error(ctx).decode()


def pf_create(opt: pf_options, n_max: int, stream: int = 0):
    out = C.c_void_p()
    _check(_lib.pf_create(C.byref(opt), int(n_max), C.c_void_p(stream or None), C.byref(out)))
    return out


def pf_destroy(ctx) -> None:
    _check(_lib.pf_destroy(ctx))


def pf_filter(ctx, op: pf_operator, a: float, b: float, degree: int, U: int, ldu: int) -> None:
    _check(_lib.pf_filter(ctx, C.byref(op), float(a), float(b), int(degree), C.c_void_p(U),
                          int(ldu)), ctx)


def pf_rayleigh_ritz(ctx, op: pf_operator, Q: int, ldq: int, V: int, ldv: int, theta: int,
                     resid: int = 0) -> None:
    _check(_lib.pf_rayleigh_ritz(ctx, C.byref(op), C.c_void_p(Q), int(ldq), C.c_void_p(V),
                                 int(ldv), C.c_void_p(theta), C.c_void_p(resid or None)), ctx)


def pf_apply(ctx, op: pf_operator, X: int, ldx: int, Y: int, ldy: int) -> None:
    _check(_lib.pf_apply(ctx, C.byref(op), C.c_void_p(X), int(ldx), C.c_void_p(Y), int(ldy)), ctx)


def pf_kernel_launch_count() -> int:
    return int(_lib.pf_kernel_launch_count())


def pf_apply_dense_noalloc(A: int, lda: int, X: int, ldx: int, Y: int, ldy: int, n: int, p: int,
                           stream: int = 0) -> None:
    """Y = A X without any device allocation (the library's fixed scratch
    array holds the partial sums); for callers that cannot allocate."""
    _check(_lib.pf_apply_dense_noalloc(C.c_void_p(A), int(lda), C.c_void_p(X), int(ldx),
                                       C.c_void_p(Y), int(ldy), int(n), int(p),
                                       C.c_void_p(stream or None)))


def pf_problem_init(ctx, prob: pf_problem) -> None:
    _check(_lib.pf_problem_init(ctx, C.byref(prob)), ctx)


def pf_prox_step(ctx, prob: pf_problem, want_info: bool = True):
    info = pf_iter_info()
    _check(_lib.pf_prox_step(ctx, C.byref(prob), C.byref(info) if want_info else None), ctx)
    return info if want_info else None


def pf_solve(ctx, prob: pf_problem, max_iter: int, tol: float = 0.0, check_every: int = 10,
             allow_not_converged: bool = True) -> pf_result:
    res = pf_result()
    allow = (PF_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    _check(_lib.pf_solve(ctx, C.byref(prob), int(max_iter), float(tol), int(check_every),
                         C.byref(res)), ctx, allow)
    return res


def pf_enqueue_steps(ctx, prob: pf_problem, n_steps: int) -> None:
    _check(_lib.pf_enqueue_steps(ctx, C.byref(prob), int(n_steps)), ctx)


def pf_report_async(ctx, info_addr: int) -> None:
    """Enqueue the latest step report into host memory at `info_addr`
    (a pinned buffer of sizeof(pf_iter_info) bytes)."""
    _check(_lib.pf_report_async(ctx, C.c_void_p(info_addr)), ctx)


def pf_get_info(ctx) -> pf_iter_info:
    info = pf_iter_info()
    _check(_lib.pf_get_info(ctx, C.byref(info)), ctx)
    return info


def pf_ladder_update(ctx, prob: pf_problem, kkt: float) -> None:
    _check(_lib.pf_ladder_update(ctx, C.byref(prob), float(kkt)), ctx)


def pf_set_tracing(ctx, on: bool) -> None:
    _check(_lib.pf_set_tracing(ctx, 1 if on else 0), ctx)


def pf_phase_times(ctx) -> dict:
    """Device milliseconds per phase of the most recent traced call."""
    ms = (C.c_double * PF_NUM_PHASES)()
    _check(_lib.pf_phase_times(ctx, ms), ctx)
    return {name: float(ms[i]) for i, name in enumerate(PHASE_NAMES)}


def pf_set_wait_limit(ns: int) -> None:
    _check(_lib.pf_set_wait_limit(int(ns)))


def raw_call(name: str, *args) -> int:
    """Call an entry point and return its status without raising (tests of
    the error paths)."""
    return getattr(_lib, name)(*args)
