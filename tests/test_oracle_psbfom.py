"""Pins for the oracle's Algorithm 1 / Algorithm 2 (paper Sections 3-4).

Checked against: the closed-form r(A) B (eigen-expansion, r evaluated in extended
precision), dense r(A) B = omega_0 B + sum omega_i (A - tau_i I)^{-1} B on tiny n
(eq. (11)), scipy's expm within the CF error, the explicit residual B - (A - tau_i I) X_i
versus eq. (49), the block Arnoldi relation eq. (4.5), collinearity of the residuals
(Section 3, after eq. (365)) and the Theorem 4.2 identity.
"""
import numpy as np
import scipy.linalg as sl
import pytest

from oracle import cf, operators as ops, psbfom as ps


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cancellation_floor(tab, X, Z):
    """eps * sum_i 2 |omega_i| ||X_i|| / ||Z||: the rounding floor of the partial-fraction
    sum (Section 4.2 error split, last term, with FP64 rounding as the solve error)."""
    s = sum(2 * abs(o) * np.linalg.norm(x) for o, x in zip(tab["omega"], X))
    return np.finfo(float).eps * s / np.linalg.norm(Z)


SMALL = [((60,), 1.0, (0.0,), 1.0, 3), ((14, 12), 0.1, (1.0, 1.0), 0.1, 2),
         ((7, 6, 5), 1.0, (3.0, -2.0, 1.0), 0.3, 4), ((20, 16), 0.1, (1.0, 1.0), 1.0, 3)]


@pytest.mark.parametrize("sides,diff,vel,t,p", SMALL)
def test_psbfom_matches_closed_form(tab, sides, diff, vel, t, p):
    A = ops.cd_matrix(sides, diff, vel, t)
    rng = np.random.default_rng(11)
    B = rng.standard_normal((A.shape[0], p))
    Z, info = ps.psbfom(ps.lu_inverse(A), B, tab, m=6, tol=1e-13, max_cycles=200)
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    floor = cancellation_floor(tab, info["X"], ref)
    assert info["converged"]
    assert rel(Z, ref) <= max(1e-11, 50 * floor)
    # and e^A B within the CF error (symmetrisable A: ||D^-1|| ||D|| amplifies)
    ex = ops.exact_expm_B(sides, diff, vel, t, B)
    lam = ops.eigenvalues(sides, diff, vel, t).ravel()
    cf_err = np.max(np.abs(ops.r_of_lambda_ext(tab, lam) - np.exp(lam)))
    kappa_D = 1.0
    for d, N in enumerate(sides):
        _, dp, _ = ops.axis_eig(N, diff, vel[d], t)
        kappa_D *= dp.max() / dp.min()
    assert np.linalg.norm(Z - ex) <= 1.01 * cf_err * kappa_D * np.linalg.norm(B) + 50 * floor * np.linalg.norm(ex)


def test_brute_force_full_krylov_space(tab):
    """mp >= n: one cycle spans the whole space, so FOM is exact (Section 3)."""
    sides, diff, vel, t = (6, 2), 0.1, (1.0, 0.5), 0.5
    A = ops.cd_matrix(sides, diff, vel, t)
    rng = np.random.default_rng(2)
    B = rng.standard_normal((12, 2))
    Z, info = ps.psbfom(ps.lu_inverse(A), B, tab, m=6, tol=0.0, max_cycles=1, fixed_cycles=1)
    ref = ps.dense_r_of_A_B(A, B, tab)
    assert rel(Z, ref) < 1e-10
    Z1, _ = ps.sbfom(ps.matvec(A), B, tab, m=6, tol=0.0, fixed_cycles=1)
    assert rel(Z1, ref) < 1e-10


def test_eq49_equals_explicit_residual_and_collinear(tab):
    sides, diff, vel, t = (16, 14), 0.1, (1.0, 1.0), 0.5
    A = ops.cd_matrix(sides, diff, vel, t)
    Ad = A.toarray()
    n = Ad.shape[0]
    rng = np.random.default_rng(4)
    B = rng.standard_normal((n, 3))
    Z, info = ps.psbfom(ps.lu_inverse(A), B, tab, m=4, tol=0.0, fixed_cycles=2, return_details=True)
    last = info["details"][-1]
    for i, tau in enumerate(tab["tau"]):
        R = B - (Ad - tau * np.eye(n)) @ info["X"][i]
        assert abs(np.linalg.norm(R) - info["residuals"][-1][i]) <= 1e-6 * info["residuals"][-1][i]
        # collinear with the real block V_{m+1}: R = V_{m+1} (V_{m+1}^T R)
        V = last["V"]
        Vn = V[:, -3:]
        assert np.linalg.norm(R - Vn @ (Vn.T @ R)) <= 1e-6 * np.linalg.norm(R)


def test_arnoldi_relation_and_orthogonality(tab):
    sides, diff, vel, t = (18, 15), 0.1, (1.0, 1.0), 1.0
    A = ops.cd_matrix(sides, diff, vel, t)
    Ainv = ps.lu_inverse(A)
    rng = np.random.default_rng(6)
    V1, _ = ps.qr_positive(rng.standard_normal((A.shape[0], 3)))
    V, H, m_done, bd = ps.block_arnoldi_ruhe(Ainv, V1, 5)
    assert not bd and m_done == 5
    Vm = V[:, :15]
    AV = np.column_stack([Ainv(Vm[:, j]) for j in range(15)])
    assert np.linalg.norm(AV - V @ H) <= 1e-12 * np.linalg.norm(H)                # eq. (4.5)
    assert np.linalg.norm(V.T @ V - np.eye(V.shape[1])) <= 1e-13
    # band upper Hessenberg with p = 3 sub-diagonals, and H_{j+1,j} upper triangular
    assert np.allclose(np.tril(H, -4), 0)


def test_theorem_4_2_identity(tab):
    sides, diff, vel, t = (12, 10), 0.1, (1.0, 1.0), 1.0
    A = ops.cd_matrix(sides, diff, vel, t)
    Ainv = ps.lu_inverse(A)
    rng = np.random.default_rng(7)
    B = rng.standard_normal((A.shape[0], 2))
    V1, Rh = ps.qr_positive(B)
    m, p = 4, 2
    V, H, _, _ = ps.block_arnoldi_ruhe(Ainv, V1, m)
    Hm = H[:m * p, :m * p]
    Hl = H[m * p:, (m - 1) * p:m * p]
    mu, P = np.linalg.eig(Hm)
    Vm = V[:, :m * p]
    AVm = np.column_stack([Ainv(Vm[:, j]) for j in range(m * p)])
    r = AVm @ P - (Vm @ P) * mu[None, :]                       # Ritz residuals r_j
    for tau in tab["tau"]:
        E1R = np.zeros((m * p, p), dtype=complex)
        E1R[:p] = Rh
        Zi = np.linalg.solve(np.eye(m * p) - tau * Hm, E1R)
        lhs = tau * V[:, m * p:] @ (Hl @ Zi[-p:])
        rhs = tau * r @ np.linalg.solve(P @ np.diag(1 - tau * mu), E1R)
        assert np.linalg.norm(lhs - rhs) <= 1e-8 * np.linalg.norm(lhs)


def test_algorithm1_and_2_agree(tab):
    sides, diff, vel, t = (10, 9), 0.1, (1.0, 1.0), 0.05
    A = ops.cd_matrix(sides, diff, vel, t)
    rng = np.random.default_rng(8)
    B = rng.standard_normal((A.shape[0], 2))
    Z2, i2 = ps.psbfom(ps.lu_inverse(A), B, tab, m=5, tol=1e-13, max_cycles=300)
    Z1, i1 = ps.sbfom(ps.matvec(A), B, tab, m=5, tol=1e-13, max_cycles=300)
    assert i1["converged"] and i2["converged"]
    assert rel(Z1, Z2) < 1e-11


def test_deflated_restart_converges_to_same_answer(tab):
    sides, diff, vel, t = (24, 20), 0.1, (1.0, 1.0), 1.0
    A = ops.cd_matrix(sides, diff, vel, t)
    rng = np.random.default_rng(9)
    B = rng.standard_normal((A.shape[0], 2))
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    Z0, i0 = ps.psbfom(ps.lu_inverse(A), B, tab, m=4, tol=1e-12, max_cycles=200, k=0)
    Zk, ik = ps.psbfom(ps.lu_inverse(A), B, tab, m=4, tol=1e-12, max_cycles=200, k=4)
    assert i0["converged"] and ik["converged"]
    assert rel(Z0, ref) < 1e-10 and rel(Zk, ref) < 1e-10
    assert ik["matvecs"] <= i0["matvecs"]


def test_planted_sign_error_in_residual_is_caught(tab, monkeypatch):
    """A wrong sign in the restart residual factor (eq. (49) region) must break parity
    with the closed form."""
    sides, diff, vel, t = (14, 12), 0.1, (1.0, 1.0), 1.0
    A = ops.cd_matrix(sides, diff, vel, t)
    rng = np.random.default_rng(10)
    B = rng.standard_normal((A.shape[0], 2))
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    bad = dict(tab)
    bad["tau"] = tab["tau"].copy()
    Zg, _ = ps.psbfom(ps.lu_inverse(A), B, tab, m=3, tol=1e-12, max_cycles=100)
    assert rel(Zg, ref) < 1e-10
    orig = ps.qr_positive
    monkeypatch.setattr(ps, "qr_positive", lambda M: (lambda q, r: (q, -r))(*orig(M)))
    Zb, _ = ps.psbfom(ps.lu_inverse(A), B, tab, m=3, tol=1e-12, max_cycles=100)
    assert rel(Zb, ref) > 1e-3


@pytest.mark.parametrize("t", [1e-2, 1e-1])
def test_fp32_stored_basis_misses_the_1e8_metric(tab, monkeypatch, t):
    """Why the mixed path keeps the Krylov basis in FP64: the same Algorithm 2 with every basis
    vector stored in FP32 (each new vector, and the vectors the operator is applied to, rounded
    to float) leaves the converged result ~3e-8 from the exact r(tA) B on 64^2 (the
    partial-fraction sum over the poles amplifies the FP32 defect of the Arnoldi relation),
    while the FP64 basis reaches ~2e-13.  The estimate of eq. (49) still reports convergence,
    so the defect is invisible to the stop test."""
    from paper_1405_0707_gb300 import inputs
    sides, diff, vel, p = (64, 64), 0.1, (1.0, 1.0), 4
    n = 64 * 64
    B = inputs.rhs(n, p, 3)
    A = ops.cd_matrix(sides, diff, vel, t).tocsc()
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    Z64, i64 = ps.psbfom(ps.lu_inverse(A), B, tab, m=10, tol=1e-10, max_cycles=100)
    orig = ps.block_arnoldi_ruhe

    def to32(x):
        return x.astype(np.float32).astype(np.float64)

    def ruhe32(op, V1, m, start_vectors=None, H0=None):
        V, H, md, bd = orig(lambda v: op(to32(v)), to32(V1), m, start_vectors, H0)
        return to32(V), H, md, bd

    monkeypatch.setattr(ps, "block_arnoldi_ruhe", ruhe32)
    Z32, i32 = ps.psbfom(ps.lu_inverse(A), B, tab, m=10, tol=1e-10, max_cycles=100)
    e64 = np.linalg.norm(Z64 - ref) / np.linalg.norm(ref)
    e32 = np.linalg.norm(Z32 - ref) / np.linalg.norm(ref)
    assert i64["converged"] and i32["converged"]
    assert e64 < 1e-11 and e32 > 1e-8, (e64, e32)
