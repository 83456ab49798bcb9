"""GPU parity of the whole path (Algorithm 2) through the C ABI.

* against the oracle's literal Algorithm 2 run for the same number of cycles (the same
  iterate, so the only difference is rounding, amplified by the partial-fraction
  cancellation: tolerance max(1e-10, 20 x floor), floor = eps sum 2|omega_i| ||X_i|| / ||Z||);
* against the closed-form r(tA) B and e^{tA} B at convergence;
* edge cases: p = 1, p = p_max, ragged n, ld > n, NOT_CONVERGED, host buffers.
"""
import numpy as np
import pytest

from oracle import cf, operators as ops, psbfom as ps
from paper_1405_0707_gb300 import inputs
from tests.gpu_util import cancellation_floor, need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


SMALL = [((300,), 1.0, (0.0,), 1.0, 3, 5),
         ((37, 29), 0.1, (1.0, 1.0), 1e-1, 4, 4),
         ((40, 33), 0.1, (1.0, 1.0), 1.0, 1, 6),
         ((11, 9, 7), 1.0, (3.0, -2.0, 1.0), 0.3, 2, 5)]


@pytest.mark.parametrize("sides,diff,vel,t,p,m", SMALL)
def test_fixed_cycles_parity_with_oracle(tab, sides, diff, vel, t, p, m):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, 31)
    for cycles in (1, 3):
        plan = Plan(sides, diff, vel, p_max=p, m=m, fixed_cycles=cycles, algorithm=2)
        Zg, info = plan.expm_block(t, to_dev(B))
        Zg = to_np(Zg)
        Zo, io = ps.psbfom(ps.lu_inverse(ops.cd_matrix(sides, diff, vel, t)), B, tab, m=m,
                           fixed_cycles=cycles)
        floor = cancellation_floor(tab, io["X"], Zo)
        assert info.cycles == cycles
        assert rel(Zg, Zo) <= max(1e-10, 20 * floor), (cycles, rel(Zg, Zo), floor)
        # eq. (49) residual norms agree with the oracle's
        ro = io["residuals"][-1]
        rg = np.array([info.resid[i] for i in range(7)])
        assert np.allclose(rg, ro, rtol=1e-6, atol=1e-12 * np.linalg.norm(B))


@pytest.mark.parametrize("sides,diff,vel,t,p,m", SMALL)
def test_converged_matches_closed_form(tab, sides, diff, vel, t, p, m):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, 32)
    plan = Plan(sides, diff, vel, p_max=p, m=m, tol=1e-12, max_cycles=300)
    Zg, info = plan.expm_block(t, to_dev(B))
    assert info.converged == 1
    Zg = to_np(Zg)
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    _, io = ps.psbfom(ps.lu_inverse(ops.cd_matrix(sides, diff, vel, t)), B, tab, m=m, tol=1e-12,
                      max_cycles=300)
    floor = cancellation_floor(tab, io["X"], ref)
    assert rel(Zg, ref) <= max(1e-10, 50 * floor)


def test_edge_cases(tab):
    need_gpu()
    import torch
    from paper_1405_0707_gb300 import Plan, colmajor
    from paper_1405_0707_gb300 import _native as N
    sides, diff, vel, t = (23, 19), 0.1, (1.0, 1.0), 0.5
    n = 23 * 19
    plan = Plan(sides, diff, vel, p_max=5, m=3, tol=1e-11, max_cycles=200)
    ref_all = ops.exact_r_of_A_B(sides, diff, vel, t, tab, inputs.rhs(n, 5, 3))
    # p = 1 and p = p_max against the closed form
    for p in (1, 5):
        B = inputs.rhs(n, 5, 3)[:, :p]
        Zg, info = plan.expm_block(t, to_dev(B))
        assert info.converged and rel(to_np(Zg), ref_all[:, :p]) < 1e-9
    # leading dimensions larger than n
    B = inputs.rhs(n, 5, 3)
    Bd = colmajor(n, 5, ld=n + 7)
    Bd.copy_(to_dev(B))
    Zd = colmajor(n, 5, ld=n + 3)
    plan.expm_block(t, Bd, Zd)
    assert rel(to_np(Zd), ref_all) < 1e-9
    # host-buffer entry point gives the same numbers
    hB = torch.from_numpy(np.ascontiguousarray(B.T)).T.pin_memory() if False else torch.from_numpy(np.ascontiguousarray(B.T)).T
    hZ = torch.empty((5, n), dtype=torch.float64).T
    plan.expm_block_host(t, hB, hZ)
    assert rel(hZ.numpy(), to_np(Zd)) < 1e-15
    # NOT_CONVERGED with one cycle still writes Z and fills info
    one = Plan(sides, diff, vel, p_max=5, m=1, tol=1e-14, max_cycles=1)
    Zg, info = one.expm_block(t, to_dev(B))
    assert info.cycles == 1 and info.converged == 0
    assert np.all(np.isfinite(to_np(Zg)))
    # bad arguments
    with pytest.raises(N.ExpmError):
        plan.expm_block(-1.0, to_dev(B))
    with pytest.raises(ValueError):
        plan.expm_block(t, to_dev(np.ones((n + 1, 2))))


@pytest.mark.parametrize("sides,diff,vel,t,p,m", [((300,), 1.0, (0.0,), 1e-3, 3, 5),
                                                  ((37, 29), 0.1, (1.0, 1.0), 1e-2, 4, 4),
                                                  ((11, 9, 7), 1.0, (3.0, -2.0, 1.0), 0.01, 2, 5)])
def test_algorithm1_parity_with_oracle(tab, sides, diff, vel, t, p, m):
    """Algorithm 1 (SBFOM, Krylov operator tA) against the oracle's literal Algorithm 1."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, 41)
    for cycles in (1, 4):
        plan = Plan(sides, diff, vel, p_max=p, m=m, fixed_cycles=cycles, algorithm=1)
        Zg, info = plan.expm_block(t, to_dev(B))
        Zo, io = ps.sbfom(ps.matvec(ops.cd_matrix(sides, diff, vel, t)), B, tab, m=m, fixed_cycles=cycles)
        assert info.algorithm == 1 and info.cycles == cycles
        floor = cancellation_floor(tab, io["X"], Zo)
        assert rel(to_np(Zg), Zo) <= max(1e-10, 20 * floor)
        rg = np.array([info.resid[i] for i in range(7)])
        assert np.allclose(rg, io["residuals"][-1], rtol=1e-6, atol=1e-12 * np.linalg.norm(B))


def test_auto_selection_follows_norm_ratio(tab):
    """AUTO runs Algorithm 2 only when the Gershgorin bound of ||tA|| is >= EXPM_AUTO_RATIO max|tau|
    (eq. (43)); both choices converge to the closed form here."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300 import _native as N
    sides, diff, vel, p = (48, 40), 0.1, (1.0, 1.0), 2
    n = 48 * 40
    B = inputs.rhs(n, p, 5)
    plan = Plan(sides, diff, vel, p_max=p, m=8, tol=1e-11, max_cycles=400)
    taumax = np.abs(tab["tau"]).max()
    for t in (1e-3, 3e-2, 1.0):
        Zg, info = plan.expm_block(t, to_dev(B))
        h2 = [1.0 / (s + 1) ** 2 for s in sides]
        bound = t * sum(4 * diff / h for h in h2)
        assert abs(info.normA_bound - bound) <= 1e-12 * bound
        assert info.algorithm == (2 if bound >= N.EXPM_AUTO_RATIO * taumax else 1)
        ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
        assert info.converged == 1 and rel(to_np(Zg), ref) < 1e-9, (t, rel(to_np(Zg), ref))


def test_nearly_dependent_rhs_takes_the_shifted_qr_pass(tab):
    """kappa(B) ~ 1e7: the first Cholesky-QR pass is ill-conditioned, the shifted pass and
    the third pass run; the result must still match the closed form."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t = (41, 35), 0.1, (1.0, 1.0), 1.0
    n = 41 * 35
    rng = np.random.default_rng(12)
    b = rng.standard_normal((n, 3))
    B = np.column_stack([b[:, 0], b[:, 1], b[:, 0] + 1e-7 * b[:, 2]])
    assert np.linalg.cond(B) > 1e6
    plan = Plan(sides, diff, vel, p_max=3, m=6, tol=1e-12, max_cycles=200)
    Zg, info = plan.expm_block(t, to_dev(B))
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    assert info.converged == 1
    assert rel(to_np(Zg), ref) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("alg", [1, 2])
def test_zero_and_repeated_rhs_columns(tab, alg, precision):
    """A zero column and an exactly repeated column in B (rank-deficient block): the zero
    column stays zero through every block (zero Cholesky pivots are skipped) and the others
    match the closed form; an invariant subspace is reported in info.breakdown, not as an
    error."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t = (41, 35), 0.1, (1.0, 1.0), 0.1
    n = 41 * 35
    b = inputs.rhs(n, 2, 13)
    B = np.column_stack([b[:, 0], np.zeros(n), b[:, 0], b[:, 1]])
    plan = Plan(sides, diff, vel, p_max=4, m=6, tol=1e-12, max_cycles=200, algorithm=alg, precision=precision)
    Zg, info = plan.expm_block(t, to_dev(B))
    Zg = to_np(Zg)
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    assert info.converged == 1
    assert np.all(Zg[:, 1] == 0.0)
    assert rel(Zg, ref) < 1e-9


def test_invariant_subspace_is_not_an_error(tab):
    """B spanned by two eigenvectors of a 1-D Laplacian: the block Krylov space is invariant
    after one step; the solve must finish (info.breakdown = 1) with the exact answer."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, t = 200, 1e-3
    j = np.arange(1, n + 1)
    B = np.column_stack([np.sin(np.pi * j * 3 / (n + 1)), np.sin(np.pi * j * 7 / (n + 1))])
    plan = Plan((n,), 1.0, (0.0,), p_max=2, m=5, tol=1e-12, max_cycles=20, algorithm=2)
    Zg, info = plan.expm_block(t, to_dev(B))
    ref = ops.exact_r_of_A_B((n,), 1.0, (0.0,), t, tab, B)
    assert info.converged == 1 and info.breakdown == 1
    assert rel(to_np(Zg), ref) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("sides,diff,vel,t,p,alg", [((37, 29), 0.1, (1.0, 1.0), 0.1, 3, 1),
                                                    ((40, 33), 0.1, (1.0, 1.0), 1.0, 2, 2),
                                                    ((11, 9, 7), 1.0, (3.0, -2.0, 1.0), 0.3, 2, 2)])
def test_certify_true_residual_matches_eq49(tab, precision, sides, diff, vel, t, p, alg):
    """Certify mode recomputes ||B - (tA - tau_i I) X_i||_F in FP64 from the accumulated X_i
    (eq. (3)); it must equal the collinear-residual estimate of eq. (49) / eq. (365) that
    drives the stop test, for both precisions, must not change Z, and must equal the explicit
    residual of the oracle's X_i after the same number of cycles."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, 91)
    kw = dict(p_max=p, m=5, fixed_cycles=3, algorithm=alg, precision=precision)
    Zc, ic = Plan(sides, diff, vel, certify=True, **kw).expm_block(t, to_dev(B))
    Zp, ip = Plan(sides, diff, vel, **kw).expm_block(t, to_dev(B))
    assert rel(to_np(Zc), to_np(Zp)) < 1e-14
    nb = np.linalg.norm(B)
    for i in range(7):
        est, true = ic.resid[i], ic.true_resid[i]
        assert abs(true - est) <= 1e-6 * est + 1e-11 * nb, (i, est, true)
    # against the oracle: the same fixed cycles of its literal algorithm, then the explicit
    # residual ||B - (tA - tau_i I) X_i||_F of its own X_i with its own sparse matrix
    A = ops.cd_matrix(sides, diff, vel, t)
    if alg == 2:
        _, io = ps.psbfom(ps.lu_inverse(A), B, tab, m=5, fixed_cycles=3)
    else:
        _, io = ps.sbfom(ps.matvec(A), B, tab, m=5, fixed_cycles=3)
    # the mixed path's FP32 projections perturb its unconverged iterate at the FP32 level,
    # so its residuals agree with the FP64 oracle's to ~1e-6 rather than to FP64 rounding
    rtol = 1e-6 if precision == "fp64" else 1e-4
    for i, (z, X) in enumerate(zip(tab["tau"], io["X"])):
        ro = np.linalg.norm(B - (A @ X - z * X))
        assert abs(ic.true_resid[i] - ro) <= rtol * ro + 1e-11 * nb, (i, ic.true_resid[i], ro)


def test_example_5_1a_replay_on_gpu(tab):
    """The paper's Example 5.1a operator (-2500 gallery('poisson', 99), p = 3, m = 30,
    tol = 1e-8) on the GPU: Algorithm 2 converges within Table 5.1's Mat-Vec count (123) and
    error (5.76e-10 against expm); Algorithm 1 needs several times more Mat-Vecs."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t = (99, 99), 0.25, (0.0, 0.0), 1.0
    B = np.random.default_rng(2014).standard_normal((9801, 3))
    ex = ops.exact_expm_B(sides, diff, vel, t, B)
    Z2, i2 = Plan(sides, diff, vel, p_max=3, m=30, tol=1e-8, algorithm=2).expm_block(t, to_dev(B))
    Z1, i1 = Plan(sides, diff, vel, p_max=3, m=30, tol=1e-8, max_cycles=2000, algorithm=1).expm_block(t, to_dev(B))
    assert i2.converged and i1.converged
    assert i2.matvecs <= 123 and rel(to_np(Z2), ex) <= 5.76e-10
    assert i1.matvecs >= 6 * i2.matvecs and rel(to_np(Z1), ex) <= 4.5e-8


@pytest.mark.parametrize("nu", [10, 16])
def test_cf_degree_option(tab, nu):
    """opts.nu_cf: the plan uses the CF table of that degree.  The result matches r_nu(tA) B
    from the oracle's table of the same degree, and for nu = 10 it is measurably farther from
    e^{tA} B than the degree-14 result (sigma_10 ~ 2e-10 against 1.8e-14)."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    tabn = cf.load_table(nu=nu)
    sides, diff, vel, t, p = (37, 29), 0.1, (1.0, 1.0), 0.1, 3
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, 61)
    Z, info = Plan(sides, diff, vel, p_max=p, m=6, tol=1e-13, max_cycles=400, nu=nu).expm_block(t, to_dev(B))
    assert info.converged == 1 and info.npoles == nu // 2
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tabn, B)
    assert rel(to_np(Z), ref) <= 1e-10, rel(to_np(Z), ref)
    if nu == 10:
        ref14 = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
        assert rel(ref, ref14) > 10 * rel(to_np(Z), ref)
