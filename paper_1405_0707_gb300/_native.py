"""ctypes binding of include/expm_block.h: the same names, argument marshalling only.

Every step of the computation runs in the CUDA library; nothing here computes.  Loading
fails loudly (RuntimeError) when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

EXPM_OK = 0
EXPM_INVALID_ARG = 1
EXPM_NOT_CONVERGED = 2
EXPM_BREAKDOWN = 3
EXPM_NUMERICAL = 4
EXPM_CUDA_ERROR = 5
EXPM_NO_MEMORY = 6
EXPM_INTERNAL = 7
EXPM_TIMEOUT = 8
EXPM_AUTO_RATIO = 36.0     # the AUTO rule's ratio (include/expm_block.h)
EXPM_OP_CONV_DIFF = 0
EXPM_OP_TOEPLITZ_SYM = 1
EXPM_OP_CSR = 2
EXPM_PREC_FP64 = 0
EXPM_PREC_MIXED = 1
EXPM_ALG_AUTO = 0
EXPM_ALG_SBFOM = 1
EXPM_ALG_PSBFOM = 2
EXPM_MAX_POLES = 16

# Every exported function the header declares (checked by the CPU test suite).
EXPORTS = ("expm_cf_coeffs", "expm_plan_create", "expm_plan_destroy", "expm_block",
           "expm_block_host", "expm_op_apply", "expm_prec_apply", "expm_arnoldi",
           "expm_plan_profile", "expm_plan_get_profile", "expm_status_str",
           "expm_prec_apply_noalloc", "expm_block_batched", "expm_block_adjoint", "expm_ritz_basis",
           "expm_block_batched_host", "expm_peak_fma", "expm_batch_create", "expm_batch_run",
           "expm_batch_destroy")
STAGES = ("gemm", "tridiag", "cgs", "reduce", "qr", "poles", "update", "other", "stencil")


class expm_op_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ndim", C.c_int32), ("side", C.c_int32 * 3),
                ("diff", C.c_double), ("vel", C.c_double * 3), ("n", C.c_int64),
                ("toeplitz_col", C.POINTER(C.c_double)), ("toeplitz_bw", C.c_int64),
                ("csr_rowptr", C.POINTER(C.c_int64)), ("csr_colind", C.POINTER(C.c_int32)),
                ("csr_val", C.POINTER(C.c_double))]


class expm_opts(C.Structure):
    _fields_ = [("m", C.c_int32), ("max_cycles", C.c_int32), ("tol", C.c_double),
                ("precision", C.c_int32), ("fixed_cycles", C.c_int32), ("algorithm", C.c_int32),
                ("certify", C.c_int32), ("nu_cf", C.c_int32), ("k_defl", C.c_int32),
                ("row_ctas_per_sm", C.c_int32), ("cgs_ctas_per_sm", C.c_int32),
                ("inner_tol", C.c_double), ("inner_maxit", C.c_int32),
                ("grid_sms", C.c_int32)]


class expm_info(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("block_steps", C.c_int32), ("matvecs", C.c_int64),
                ("converged", C.c_int32), ("breakdown", C.c_int32), ("npoles", C.c_int32),
                ("resid", C.c_double * EXPM_MAX_POLES), ("normB", C.c_double),
                ("algorithm", C.c_int32), ("normA_bound", C.c_double),
                ("true_resid", C.c_double * EXPM_MAX_POLES), ("kept", C.c_int32),
                ("inner_iters", C.c_int64)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libexpm_block.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build() or python -m paper_1405_0707_gb300.build)")
    lib = C.CDLL(path)
    p, d, i32, i64 = C.c_void_p, C.c_double, C.c_int, C.c_int64
    lib.expm_status_str.restype = C.c_char_p
    lib.expm_status_str.argtypes = [C.c_int]
    lib.expm_cf_coeffs.restype = C.c_int
    lib.expm_cf_coeffs.argtypes = [C.c_int, C.POINTER(d), C.POINTER(d), C.POINTER(d), C.POINTER(d)]
    lib.expm_plan_create.restype = C.c_int
    lib.expm_plan_create.argtypes = [C.POINTER(expm_op_desc), C.c_int, C.POINTER(expm_opts), p,
                                     C.POINTER(p)]
    lib.expm_plan_destroy.restype = None
    lib.expm_plan_destroy.argtypes = [p]
    for name in ("expm_block", "expm_block_host"):
        f = getattr(lib, name)
        f.restype = C.c_int
        f.argtypes = [p, d, p, i64, i32, p, i64, C.POINTER(expm_info)]
    for name in ("expm_op_apply", "expm_prec_apply"):
        f = getattr(lib, name)
        f.restype = C.c_int
        f.argtypes = [p, d, p, i64, i32, p, i64]
    for name in ("expm_block_batched", "expm_block_batched_host"):
        f = getattr(lib, name)
        f.restype = C.c_int
        f.argtypes = [C.POINTER(p), C.c_int, C.POINTER(d), C.POINTER(p), C.POINTER(i64), C.POINTER(C.c_int),
                      C.POINTER(p), C.POINTER(i64), C.POINTER(expm_info)]
    lib.expm_block_adjoint.restype = C.c_int
    lib.expm_block_adjoint.argtypes = [p, d, p, i64, i32, p, i64, p, i64, C.POINTER(d), C.POINTER(expm_info)]
    lib.expm_arnoldi.restype = C.c_int
    lib.expm_arnoldi.argtypes = [p, d, p, i64, i32, p, i64, p, i64]
    lib.expm_prec_apply_noalloc.restype = C.c_int
    lib.expm_prec_apply_noalloc.argtypes = [C.POINTER(expm_op_desc), d, p, i64, i32, p, i64, p]
    lib.expm_ritz_basis.restype = C.c_int
    lib.expm_ritz_basis.argtypes = [C.POINTER(d), i64, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(d), i64,
                                    C.POINTER(C.c_int)]
    lib.expm_batch_create.restype = C.c_int
    lib.expm_batch_create.argtypes = [C.POINTER(p), C.c_int, C.POINTER(d), C.POINTER(p), C.POINTER(i64),
                                      C.POINTER(C.c_int), C.POINTER(p), C.POINTER(i64), p, C.POINTER(p)]
    lib.expm_batch_run.restype = C.c_int
    lib.expm_batch_run.argtypes = [p, C.POINTER(expm_info)]
    lib.expm_batch_destroy.restype = None
    lib.expm_batch_destroy.argtypes = [p]
    lib.expm_peak_fma.restype = C.c_int
    lib.expm_peak_fma.argtypes = [C.c_int, i64, C.POINTER(d), p]
    lib.expm_plan_profile.restype = C.c_int
    lib.expm_plan_profile.argtypes = [p, C.c_int]
    lib.expm_plan_get_profile.restype = C.c_int
    lib.expm_plan_get_profile.argtypes = [p, C.POINTER(d), C.POINTER(C.c_int64), C.c_int,
                                          C.POINTER(C.c_int64)]
    _lib = lib
    return lib


class ExpmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().expm_status_str(code).decode()
        super().__init__(f"{where}: status {code} ({msg})")


def check(code, where, allow=(EXPM_OK,)):
    if code not in allow:
        raise ExpmError(code, where)
    return code


# ---------------------------------------------------------------- thin wrappers (same names)
def expm_cf_coeffs(nu=14):
    lib = load()
    k = nu // 2
    tau = (C.c_double * (2 * k))()
    om = (C.c_double * (2 * k))()
    w0 = C.c_double()
    sg = C.c_double()
    check(lib.expm_cf_coeffs(nu, tau, om, C.byref(w0), C.byref(sg)), "expm_cf_coeffs")
    taus = [complex(tau[2 * i], tau[2 * i + 1]) for i in range(k)]
    oms = [complex(om[2 * i], om[2 * i + 1]) for i in range(k)]
    return taus, oms, w0.value, sg.value


def expm_plan_create(op: expm_op_desc, p_max: int, opts: expm_opts, stream: int = 0):
    lib = load()
    out = C.c_void_p()
    check(lib.expm_plan_create(C.byref(op), p_max, C.byref(opts), C.c_void_p(stream), C.byref(out)),
          "expm_plan_create")
    return out


def expm_plan_destroy(plan):
    load().expm_plan_destroy(plan)


def expm_block(plan, t, dB, ldb, p, dZ, ldz, allow_not_converged=True):
    info = expm_info()
    allow = (EXPM_OK, EXPM_NOT_CONVERGED) if allow_not_converged else (EXPM_OK,)
    code = check(load().expm_block(plan, t, C.c_void_p(dB), ldb, p, C.c_void_p(dZ), ldz,
                                   C.byref(info)), "expm_block", allow)
    return code, info


def expm_block_host(plan, t, hB, ldb, p, hZ, ldz, allow_not_converged=True):
    info = expm_info()
    allow = (EXPM_OK, EXPM_NOT_CONVERGED) if allow_not_converged else (EXPM_OK,)
    code = check(load().expm_block_host(plan, t, C.c_void_p(hB), ldb, p, C.c_void_p(hZ), ldz,
                                        C.byref(info)), "expm_block_host", allow)
    return code, info


def expm_block_batched(plans, ts, dBs, ldbs, ps, dZs, ldzs, allow_not_converged=True, host=False):
    """Independent solves in one call (see include/expm_block.h); returns (code, [info]).
    host: the pointers are host buffers (expm_block_batched_host)."""
    k = len(plans)
    infos = (expm_info * k)()
    arr = lambda T, xs: (T * k)(*xs)
    allow = (EXPM_OK, EXPM_NOT_CONVERGED) if allow_not_converged else (EXPM_OK,)
    fn = load().expm_block_batched_host if host else load().expm_block_batched
    code = check(fn(
        arr(C.c_void_p, [pl.value if isinstance(pl, C.c_void_p) else pl for pl in plans]), k,
        arr(C.c_double, ts), arr(C.c_void_p, dBs), arr(C.c_int64, ldbs), arr(C.c_int, ps),
        arr(C.c_void_p, dZs), arr(C.c_int64, ldzs), infos),
        "expm_block_batched_host" if host else "expm_block_batched", allow)
    return code, list(infos)


def expm_block_adjoint(plan, t, dG, ldg, p, dZ, ldz, dGB, ldgb, want_dt=True):
    """(dL/dt or None, info); dL/dB written to dGB when dGB is not 0."""
    info = expm_info()
    gt = C.c_double()
    check(load().expm_block_adjoint(plan, t, C.c_void_p(dG), ldg, p, C.c_void_p(dZ), ldz,
                                    C.c_void_p(dGB), ldgb, C.byref(gt) if want_dt else None,
                                    C.byref(info)), "expm_block_adjoint", (EXPM_OK, EXPM_NOT_CONVERGED))
    return (gt.value if want_dt else None), info


def expm_op_apply(plan, t, dV, ldv, p, dW, ldw):
    check(load().expm_op_apply(plan, t, C.c_void_p(dV), ldv, p, C.c_void_p(dW), ldw), "expm_op_apply")


def expm_prec_apply(plan, t, dV, ldv, p, dW, ldw):
    check(load().expm_prec_apply(plan, t, C.c_void_p(dV), ldv, p, C.c_void_p(dW), ldw),
          "expm_prec_apply")


def expm_arnoldi(plan, t, dV1, ldv1, p, dVout, ldvo, dHout, ldh):
    check(load().expm_arnoldi(plan, t, C.c_void_p(dV1), ldv1, p, C.c_void_p(dVout), ldvo,
                              C.c_void_p(dHout), ldh), "expm_arnoldi")


def expm_plan_profile(plan, enable):
    check(load().expm_plan_profile(plan, int(enable)), "expm_plan_profile")


def expm_plan_get_profile(plan):
    """{stage: (ms, launches)}, total launches."""
    k = len(STAGES)
    ms = (C.c_double * k)()
    nl = (C.c_int64 * k)()
    tot = C.c_int64()
    check(load().expm_plan_get_profile(plan, ms, nl, k, C.byref(tot)), "expm_plan_get_profile")
    return {STAGES[i]: (ms[i], nl[i]) for i in range(k)}, tot.value


def expm_prec_apply_noalloc(op, t, dV, ldv, p, dW, ldw, stream=0):
    """Allocation-free W = (tA)^{-1} V (no plan); see include/expm_block.h."""
    check(load().expm_prec_apply_noalloc(C.byref(op), t, C.c_void_p(dV), ldv, p, C.c_void_p(dW), ldw,
                                         C.c_void_p(stream)), "expm_prec_apply_noalloc")


def expm_ritz_basis(Hm, k, largest, align):
    """Host-only: the deflated restart's orthonormal Ritz basis P (mp x kept) of the mp x mp
    array Hm; see include/expm_block.h."""
    import numpy as np
    H = np.asfortranarray(np.asarray(Hm, dtype=np.float64))
    mp = H.shape[0]
    P = np.zeros((mp, mp), order="F")
    kept = C.c_int()
    check(load().expm_ritz_basis(H.ctypes.data_as(C.POINTER(C.c_double)), mp, mp, int(k), int(bool(largest)),
                                 int(align), P.ctypes.data_as(C.POINTER(C.c_double)), mp, C.byref(kept)),
          "expm_ritz_basis")
    return P[:, :kept.value].copy()


def expm_peak_fma(kind, iters=1 << 16, stream=0):
    """Measured FMA throughput in TFLOP/s: kind 0 = FP64, 1 = FP32 (see include/expm_block.h)."""
    out = C.c_double()
    check(load().expm_peak_fma(int(kind), int(iters), C.byref(out), C.c_void_p(stream)), "expm_peak_fma")
    return out.value


def expm_batch_create(plans, ts, dBs, ldbs, ps, dZs, ldzs, stream=0):
    """One CUDA graph for many independent solves (see include/expm_block.h); returns the handle."""
    k = len(plans)
    arr = lambda T, xs: (T * k)(*xs)
    out = C.c_void_p()
    check(load().expm_batch_create(arr(C.c_void_p, [pl.value if isinstance(pl, C.c_void_p) else pl for pl in plans]),
                                   k, arr(C.c_double, ts), arr(C.c_void_p, dBs), arr(C.c_int64, ldbs),
                                   arr(C.c_int, ps), arr(C.c_void_p, dZs), arr(C.c_int64, ldzs), C.c_void_p(stream),
                                   C.byref(out)), "expm_batch_create")
    return out


def expm_batch_run(batch, count, allow_not_converged=True):
    infos = (expm_info * count)()
    allow = (EXPM_OK, EXPM_NOT_CONVERGED) if allow_not_converged else (EXPM_OK,)
    code = check(load().expm_batch_run(batch, infos), "expm_batch_run", allow)
    return code, list(infos)


def expm_batch_destroy(batch):
    load().expm_batch_destroy(batch)
