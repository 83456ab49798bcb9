"""The C-ABI library loads and exports every function include/*.h declares; its host-only
CF table agrees with the oracle's; argument validation rejects bad input before any GPU
work.  No GPU needed."""
import glob
import os
import re

import numpy as np
import pytest

from oracle import cf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w]+\s*\*?\s+(expm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1405_0707_gb300 import _native as N
    try:
        return N.load(build_if_missing=True)
    except RuntimeError as e:  # pragma: no cover - no toolkit
        pytest.skip(str(e))


def test_exports_every_declared_symbol(lib):
    from paper_1405_0707_gb300 import _native as N
    names = _declared()
    assert len(names) >= 9
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(N.EXPORTS) <= names


def test_library_cf_table_matches_oracle(lib):
    from paper_1405_0707_gb300 import _native as N
    tau, om, w0, sig = N.expm_cf_coeffs(14)
    tab = cf.load_table()
    tau, om = np.array(tau), np.array(om)
    # two independent high-precision constructions, rounded to FP64: equal up to one
    # rounding of a value that sits within 0.004 ulp of a tie
    for a, b in ((tau.real, tab["tau"].real), (tau.imag, tab["tau"].imag),
                 (om.real, tab["omega"].real), (om.imag, tab["omega"].imag)):
        assert np.all(np.abs(a - b) <= np.spacing(np.abs(b)))
    assert w0 == tab["omega0"]
    assert abs(sig - tab["sigma"]) <= 1e-15 * tab["sigma"]


def test_invalid_arguments_rejected_on_host(lib):
    from paper_1405_0707_gb300 import _native as N
    op = N.expm_op_desc()
    op.kind, op.ndim, op.diff = N.EXPM_OP_CONV_DIFF, 2, 0.1
    op.side[0], op.side[1], op.side[2] = 16, 16, 1
    op.vel[0], op.vel[1] = 1.0, 1.0
    opts = N.expm_opts()
    opts.m, opts.max_cycles, opts.tol, opts.precision = 4, 10, 1e-10, 0
    import ctypes as C
    out = C.c_void_p()
    # p_max out of range, m p too large, bad ndim, cell Peclet >= 1, bad nu
    assert lib.expm_plan_create(C.byref(op), 0, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
    assert lib.expm_plan_create(C.byref(op), 33, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
    opts.m = 200
    assert lib.expm_plan_create(C.byref(op), 8, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
    opts.m = 4
    op.ndim = 4
    assert lib.expm_plan_create(C.byref(op), 8, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
    op.ndim = 2
    op.vel[0] = 100.0      # cell Peclet 100/(17*0.2) > 1
    assert lib.expm_plan_create(C.byref(op), 8, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
    d = (C.c_double * 32)()
    assert lib.expm_cf_coeffs(13, d, d, d, d) == N.EXPM_INVALID_ARG
    assert lib.expm_block(None, 1.0, None, 1, 1, None, 1, None) == N.EXPM_INVALID_ARG
    assert lib.expm_status_str(N.EXPM_BREAKDOWN) == b"block Arnoldi breakdown"


def test_toeplitz_descriptor_checks():
    """Toeplitz descriptors are validated on the host before any device work (Example 5.4's
    operator must be symmetric negative definite): every case below is rejected."""
    import ctypes as C
    from paper_1405_0707_gb300 import _native as N
    lib = N.load(build_if_missing=True)
    opts = N.expm_opts()
    opts.m, opts.max_cycles, opts.tol, opts.precision = 4, 10, 1e-10, 0
    out = C.c_void_p()

    def create(col, n, bw=None):
        a = np.ascontiguousarray(np.asarray(col, dtype=np.float64))
        op = N.expm_op_desc()
        op.kind, op.ndim, op.n = N.EXPM_OP_TOEPLITZ_SYM, 1, n
        op.toeplitz_col = a.ctypes.data_as(C.POINTER(C.c_double))
        op.toeplitz_bw = len(a) - 1 if bw is None else bw
        return lib.expm_plan_create(C.byref(op), 2, C.byref(opts), None, C.byref(out))

    k = np.arange(1, 257)
    good = np.r_[-2.0, 1.0 / (1.0 + k) ** 2]
    assert create([-1.0, 0.6], 100) == N.EXPM_INVALID_ARG          # symbol max -1 + 1.2 > 0
    st = create([-1.0, 0.49], 100)                                  # max -0.02: accepted (refined grid)
    assert st != N.EXPM_INVALID_ARG
    if st == N.EXPM_OK:
        lib.expm_plan_destroy(out)
    assert create([-1.0, 0.5], 100) == N.EXPM_INVALID_ARG          # max 0: semidefinite
    assert create([0.5, 0.1], 100) == N.EXPM_INVALID_ARG           # a_0 >= 0
    assert create(good, 200) == N.EXPM_INVALID_ARG                 # bw > n - 1
    assert create([-2.0, np.nan], 100) == N.EXPM_INVALID_ARG       # not finite
    assert create([-2.0], (1 << 21) + 1) == N.EXPM_INVALID_ARG     # beyond the FFT size limit
    assert create([-2.0], 1) == N.EXPM_INVALID_ARG                 # n < 2
    assert create(good, 1000, bw=-1) == N.EXPM_INVALID_ARG
    # a NULL column
    op = N.expm_op_desc()
    op.kind, op.ndim, op.n, op.toeplitz_bw = N.EXPM_OP_TOEPLITZ_SYM, 1, 100, 3
    assert lib.expm_plan_create(C.byref(op), 2, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
    # an unknown operator kind
    op.kind = 7
    assert lib.expm_plan_create(C.byref(op), 2, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
