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


def test_binding_constants_match_the_header():
    """The binding's status codes and AUTO ratio mirror include/expm_block.h's values."""
    from paper_1405_0707_gb300 import _native as N
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "expm_block.h")).read(), flags=re.S)
    ratio = re.search(r"#define\s+EXPM_AUTO_RATIO\s+([0-9.]+)", src)
    assert ratio and float(ratio.group(1)) == N.EXPM_AUTO_RATIO
    codes = dict(re.findall(r"\b(EXPM_(?:OK|INVALID_ARG|NOT_CONVERGED|BREAKDOWN|NUMERICAL|CUDA_ERROR|NO_MEMORY|"
                            r"INTERNAL|TIMEOUT))\s*=\s*(\d+)", src))
    assert len(codes) == 9
    for name, v in codes.items():
        assert getattr(N, name) == int(v), name


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
    # p_max out of range, m p too large, bad ndim, cell Peclet >= 1, negative grid_sms, bad nu
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
    op.vel[0] = 1.0
    opts.grid_sms = -1     # a negative share of the SMs
    assert lib.expm_plan_create(C.byref(op), 8, C.byref(opts), None, C.byref(out)) == N.EXPM_INVALID_ARG
    opts.grid_sms = 0
    d = (C.c_double * 32)()
    assert lib.expm_cf_coeffs(13, d, d, d, d) == N.EXPM_INVALID_ARG
    assert lib.expm_block(None, 1.0, None, 1, 1, None, 1, None) == N.EXPM_INVALID_ARG
    assert lib.expm_status_str(N.EXPM_BREAKDOWN) == b"block Arnoldi breakdown"


def test_csr_descriptor_checks(lib):
    """General sparse descriptors are validated on the host before any device work: the CSR
    structure, finite values, and the Gershgorin certificate of the operator's contract (a
    negative diagonal, weakly diagonally dominant rows).  Every case below is rejected."""
    import ctypes as C
    from paper_1405_0707_gb300 import _native as N
    from paper_1405_0707_gb300 import inputs
    n = 40
    ip0, ix0, d0 = inputs.sparse_dd_matrix(n, nnz_row=5, seed=3)
    opts = N.expm_opts()
    opts.m, opts.max_cycles, opts.tol, opts.precision = 4, 10, 1e-10, 0
    out = C.c_void_p()

    def create(ip, ix, d, nn=n, certify=0):
        op = N.expm_op_desc()
        op.kind, op.ndim, op.n = N.EXPM_OP_CSR, 1, nn
        for k in range(3):
            op.side[k] = 1
        ip = np.ascontiguousarray(ip, dtype=np.int64)
        ix = np.ascontiguousarray(ix, dtype=np.int32)
        d = np.ascontiguousarray(d, dtype=np.float64)
        op.csr_rowptr = ip.ctypes.data_as(C.POINTER(C.c_int64))
        op.csr_colind = ix.ctypes.data_as(C.POINTER(C.c_int32))
        op.csr_val = d.ctypes.data_as(C.POINTER(C.c_double))
        opts.certify = certify
        return lib.expm_plan_create(C.byref(op), 2, C.byref(opts), None, C.byref(out))

    diag = ix0 == np.repeat(np.arange(n), np.diff(ip0))
    bad = d0.copy()
    bad[np.flatnonzero(diag)[3]] *= 0.3            # row 3 no longer diagonally dominant
    assert create(ip0, ix0, bad) == N.EXPM_INVALID_ARG
    bad = d0.copy()
    bad[np.flatnonzero(diag)[7]] *= -1.0           # positive diagonal entry
    assert create(ip0, ix0, bad) == N.EXPM_INVALID_ARG
    bad = d0.copy()
    bad[5] = np.nan
    assert create(ip0, ix0, bad) == N.EXPM_INVALID_ARG
    bix = ix0.copy()
    bix[9] = n                                     # column index out of range
    assert create(ip0, bix, d0) == N.EXPM_INVALID_ARG
    bip = ip0.copy()
    bip[10], bip[11] = bip[11], bip[10]            # decreasing offsets
    assert create(bip, ix0, d0) == N.EXPM_INVALID_ARG
    bip = ip0.copy()
    bip[0] = 1
    assert create(bip, ix0, d0) == N.EXPM_INVALID_ARG
    assert create(ip0, ix0, d0, nn=0) == N.EXPM_INVALID_ARG
    assert create(ip0, ix0, d0, certify=1) == N.EXPM_INVALID_ARG   # certify mode takes no CSR


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


def test_noalloc_rejects_bad_arguments_on_host(lib):
    """The allocation-free apply rejects non-finite t, diff or velocity and sizes beyond its
    fixed scratch before any device work (the device pointers below are never touched)."""
    import ctypes as C
    from paper_1405_0707_gb300 import _native as N

    def call(sides, t=0.1, diff=0.1, vel=(1.0, 1.0), ld=None, p=2):
        op = N.expm_op_desc()
        op.kind, op.ndim, op.diff = N.EXPM_OP_CONV_DIFF, len(sides), diff
        for d in range(3):
            op.side[d] = sides[d] if d < len(sides) else 1
            op.vel[d] = vel[d] if d < len(sides) else 0.0
        n = int(np.prod(sides))
        ld = n if ld is None else ld
        return lib.expm_prec_apply_noalloc(C.byref(op), t, C.c_void_p(16), ld, p, C.c_void_p(32), ld, None)

    inf, nan = float("inf"), float("nan")
    assert call((64, 64), t=inf) == N.EXPM_INVALID_ARG
    assert call((64, 64), t=nan) == N.EXPM_INVALID_ARG
    assert call((64, 64), t=-1.0) == N.EXPM_INVALID_ARG
    assert call((64, 64), diff=inf) == N.EXPM_INVALID_ARG
    assert call((64, 64), vel=(nan, 0.0)) == N.EXPM_INVALID_ARG
    assert call((64, 64), p=33) == N.EXPM_INVALID_ARG
    assert call((1 << 21,), vel=(0.0,)) == N.EXPM_INVALID_ARG          # a side beyond the scratch
    assert call((1 << 20, 1 << 20), vel=(0.0, 0.0)) == N.EXPM_INVALID_ARG   # tables beyond it
    assert call((2 ** 31 - 1, 2 ** 31 - 1), vel=(0.0, 0.0)) == N.EXPM_INVALID_ARG
    assert call((256, 256), p=12) == N.EXPM_INVALID_ARG                # 2 Ny^2 + Ny + 2n + n p > 2^20


@pytest.mark.parametrize("largest", [True, False])
def test_library_ritz_basis_matches_oracle(lib, largest):
    """The library's host eigen-solver for the deflated restart (Hessenberg reduction, Francis
    QR, Schur back substitution) against the oracle's deflation_basis (numpy's LAPACK eig),
    both with the block-aligned selection: the same count and the same subspace.  Matrices: a
    band Hessenberg H_m from the oracle's block Arnoldi on a nonsymmetric operator (complex
    Ritz pairs), and a dense random matrix."""
    from oracle import operators as ops, psbfom as ps
    from paper_1405_0707_gb300 import _native as N
    A = ops.cd_matrix((30, 26), 0.1, (3.0, -2.0), 1.0)
    V1, _ = ps.qr_positive(np.random.default_rng(4).standard_normal((A.shape[0], 4)))
    _, H, _, _ = ps.block_arnoldi_ruhe(ps.lu_inverse(A), V1, 10)
    mats = [(H[:40, :40], 4), (np.random.default_rng(5).standard_normal((57, 57)), 3),
            (np.random.default_rng(6).standard_normal((12, 12)), 1)]
    for Hm, align in mats:
        for k in (1, 5, 8, 17):
            if k > Hm.shape[0]:
                continue
            P = N.expm_ritz_basis(Hm, k, largest, align)
            Po = ps.deflation_basis(Hm, k, largest, align=align)
            assert P.shape[1] == Po.shape[1], (Hm.shape, k, align, P.shape, Po.shape)
            if P.shape[1] == 0:
                continue
            assert P.shape[1] % align == 0
            assert np.linalg.norm(P.T @ P - np.eye(P.shape[1])) <= 1e-12
            # same subspace: the projectors agree
            assert np.linalg.norm(P @ P.T - Po @ Po.T) <= 1e-8, (Hm.shape, k, align)
            # invariant under H_m
            M = P.T @ Hm @ P
            assert np.linalg.norm(Hm @ P - P @ M) <= 1e-10 * np.linalg.norm(Hm)


def test_library_ritz_basis_known_spectrum(lib):
    """Eigenvalues known by construction (real values and 2 x 2 rotation-scaling blocks under an
    orthogonal similarity): the kept Ritz values are exactly the wanted ones."""
    from paper_1405_0707_gb300 import _native as N
    from tests.test_oracle_deflation import known_spectrum_matrix
    H, _ = known_spectrum_matrix([9.0, 7.0, 3.0, 1.0], [(8.0, 1.0), (2.0, 5.0), (0.5, 0.5)], 3)
    for (k, align, largest), want in [((2, 2, True), [9, 7]),
                                      ((4, 2, True), [9, complex(8, 1), complex(8, -1), 7]),
                                      ((3, 3, False), [complex(0.5, 0.5), complex(0.5, -0.5), 1])]:
        P = N.expm_ritz_basis(H, k, largest, align)
        got = np.sort_complex(np.linalg.eigvals(P.T @ H @ P))
        assert np.allclose(got, np.sort_complex(np.asarray(want, dtype=complex)), atol=1e-10), got
    # invalid arguments
    with pytest.raises(N.ExpmError):
        N.expm_ritz_basis(H, 0, True, 1)
    with pytest.raises(N.ExpmError):
        N.expm_ritz_basis(np.full((4, 4), np.nan), 1, True, 1)


@pytest.mark.parametrize("nu", [10, 12, 16])
def test_library_cf_table_other_degrees(lib, nu):
    """expm_cf_coeffs for the degrees a plan may choose (opts.nu_cf) against the oracle's
    stored tables of the same degree (two independent high-precision constructions)."""
    from paper_1405_0707_gb300 import _native as N
    tau, om, w0, sig = N.expm_cf_coeffs(nu)
    tab = cf.load_table(nu=nu)
    tau, om = np.array(tau), np.array(om)
    for a, b in ((tau.real, tab["tau"].real), (tau.imag, tab["tau"].imag),
                 (om.real, tab["omega"].real), (om.imag, tab["omega"].imag)):
        assert np.all(np.abs(a - b) <= 2 * np.spacing(np.abs(b))), (nu, np.max(np.abs(a - b) / np.spacing(np.abs(b))))
    # omega_0 = r(-inf) comes out of the same least-squares solve as the residues: the
    # library solves it in double-double on O(1) entries, so each component carries an
    # absolute error of some units of 2^-106.  At nu = 16, omega_0 ~ 2e-16 lies far below
    # that scale and only the absolute accuracy (2^-96, ~1e-29) is meaningful.
    assert abs(w0 - tab["omega0"]) <= 2 * np.spacing(abs(tab["omega0"])) + 2.0 ** -96
    assert abs(sig - tab["sigma"]) <= 1e-12 * tab["sigma"]
