"""GPU parity of the symmetric Toeplitz operator (Example 5.4) through the C ABI.

* products tT V (circulant embedding + four-step FFT) against the oracle's FFT product,
  element by element, on ragged n, odd p, bw = 0 and a dense column (bw = n - 1);
* the Gohberg-Semencul inverse against the oracle's (which is pinned to a dense solve);
* Algorithm 1 and Algorithm 2 on the Toeplitz operator against the oracle's literal runs
  for the same number of cycles, and against the Taylor truth at convergence;
* the 2^20 x 16 workload: sampled columns against the Taylor truth, mixed against FP64.
"""
import numpy as np
import pytest

from oracle import cf, operators as ops, psbfom as ps, toeplitz as TZ
from paper_1405_0707_gb300 import inputs
from tests.gpu_util import cancellation_floor, need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


def full_col(a, n):
    c = np.zeros(n)
    c[:len(a)] = a
    return c


def dense_col(n):
    """a_0 = -2, a_k = 1/(1+k)^2 for every k < n (bw = n - 1)."""
    k = np.arange(n, dtype=np.float64)
    a = 1.0 / (1.0 + k) ** 2
    a[0] = -2.0
    return a


PRODUCT_CASES = [(64, inputs.toeplitz_column(10), 1, 1.0),
                 (1000, inputs.toeplitz_column(256), 5, 0.7),
                 (3001, inputs.toeplitz_column(256), 16, 1.0),
                 (4097, np.array([-1.5]), 3, 2.0),        # bw = 0: T = a_0 I
                 (700, dense_col(700), 4, 1.0)]           # bw = n - 1


@pytest.mark.parametrize("n,a,p,t", PRODUCT_CASES)
def test_product_matches_oracle(n, a, p, t):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    plan = Plan.toeplitz(a, n, p_max=max(p, 2), algorithm=1)
    V = inputs.rhs(n, p, 41)
    Wg = to_np(plan.op_apply(t, to_dev(V)))
    Wo = TZ.matvec(full_col(a, n), V, t)
    scale = t * np.abs(a).sum() * 2 * np.abs(V).max()
    assert np.abs(Wg - Wo).max() <= 1e-13 * scale
    assert rel(Wg, Wo) <= 1e-13


@pytest.mark.parametrize("n,a,p,t", [(3001, inputs.toeplitz_column(256), 16, 1.0), (700, dense_col(700), 5, 1.0)])
def test_mixed_transforms_match_oracle(n, a, p, t):
    """The mixed plan's transforms run in double-float (FP32 pairs, unit roundoff u = 2^-48).
    A radix-8/4/2 four-step FFT of length N has about log2(N) rounding steps per output and
    the product three transforms, so with N <= 2^13 here the bound ~ 3 * 13 * u * ||.||
    stays under 2e-13 relative; the test allows 1e-12.  Products and the Gohberg-Semencul
    inverse both go through these passes."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    V = inputs.rhs(n, p, 47)
    plan = Plan.toeplitz(a, n, p_max=p, algorithm=2, precision="mixed")
    Wg = to_np(plan.op_apply(t, to_dev(V)))
    Wo = TZ.matvec(full_col(a, n), V, t)
    assert rel(Wg, Wo) <= 1e-12
    Ig = to_np(plan.prec_apply(t, to_dev(V)))
    Io = TZ.gsf_apply(TZ.gsf_generator(full_col(a, n)), V, t)
    assert rel(Ig, Io) <= 1e-11       # amplified by cond(T) <= 1e2 for these columns


@pytest.mark.parametrize("n,a,p,t", [(1000, inputs.toeplitz_column(256), 3, 0.5),
                                     (3001, inputs.toeplitz_column(256), 8, 1.0),
                                     (500, dense_col(500), 2, 1.0)])
def test_gsf_inverse_matches_oracle(n, a, p, t):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    plan = Plan.toeplitz(a, n, p_max=p, algorithm=2)
    V = inputs.rhs(n, p, 42)
    Wg = to_np(plan.prec_apply(t, to_dev(V)))
    x = TZ.gsf_generator(full_col(a, n))
    Wo = TZ.gsf_apply(x, V, t)
    assert rel(Wg, Wo) <= 1e-12
    # and it inverts the product
    Vg = to_np(plan.op_apply(t, to_dev(Wg)))
    assert rel(Vg, V) <= 1e-12


@pytest.mark.parametrize("alg", [1, 2])
def test_fixed_cycles_parity(tab, alg):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, p, m, t = 3000, 4, 8, 1.0
    a = inputs.toeplitz_column(256)
    col = full_col(a, n)
    B = inputs.rhs(n, p, 43)
    if alg == 1:
        op = lambda W: TZ.matvec(col, W, t)
    else:
        x = TZ.gsf_generator(col)
        op = lambda W: TZ.gsf_apply(x, W, t)
    for cycles in (1, 2):
        plan = Plan.toeplitz(a, n, p_max=p, m=m, fixed_cycles=cycles, algorithm=alg)
        Zg, info = plan.expm_block(t, to_dev(B))
        assert info.algorithm == alg and info.cycles == cycles
        run = ps.sbfom if alg == 1 else ps.psbfom
        Zo, io = run(op, B, tab, m=m, fixed_cycles=cycles)
        floor = cancellation_floor(tab, io["X"], Zo)
        assert rel(to_np(Zg), Zo) <= max(1e-10, 20 * floor), (cycles, rel(to_np(Zg), Zo), floor)
        ro = io["residuals"][-1]
        rg = np.array([info.resid[i] for i in range(7)])
        assert np.allclose(rg, ro, rtol=1e-6, atol=1e-12 * np.linalg.norm(B))


def truth_bound(tab, a_full, B, Z, tol):
    """CF error plus the solver's share (error analysis of Section 4.2), relative to ||Z||."""
    lo, hi = TZ.symbol_range(a_full[:min(len(a_full), 4097)])
    dist = [abs(complex(min(max(tt.real, lo), hi), 0.0) - tt) for tt in tab["tau"]]
    solver = sum(abs(w) / d for w, d in zip(tab["omega"], dist)) * tol
    return (1.1 * tab["sigma"] + solver) * np.linalg.norm(B) / np.linalg.norm(Z)


@pytest.mark.parametrize("alg,n,p", [(0, 2047, 3), (1, 3000, 6), (2, 3000, 6), (2, 1025, 1)])
def test_converged_matches_taylor(tab, alg, n, p):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    a = inputs.toeplitz_column(256)
    col = full_col(a, n)
    B = inputs.rhs(n, p, 44)
    tol = 1e-13
    plan = Plan.toeplitz(a, n, p_max=p, tol=tol, algorithm=alg)
    Zg, info = plan.expm_block(1.0, to_dev(B))
    assert info.converged == 1
    if alg == 0:
        assert info.algorithm == 1          # ||tA|| <= 2.36 << EXPM_AUTO_RATIO max|tau|
    truth = TZ.taylor_expm_B(col, B, 1.0)
    assert rel(to_np(Zg), truth) <= truth_bound(tab, col, B, truth, tol)


def test_diagonal_case_exact(tab):
    """bw = 0: T = a_0 I, so r(t a_0) B; checked against e^{t a_0} B within the CF error."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, p, t = 5000, 2, 0.8
    plan = Plan.toeplitz([-1.5], n, p_max=p, tol=1e-13, algorithm=2)
    B = inputs.rhs(n, p, 45)
    Zg, info = plan.expm_block(t, to_dev(B))
    assert info.converged == 1
    assert rel(to_np(Zg), np.exp(-1.5 * t) * B) <= 1.1 * tab["sigma"] / np.exp(-1.5 * t) + 1e-12


def test_certify_true_residuals(tab):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, p = 2000, 3
    a = inputs.toeplitz_column(256)
    B = inputs.rhs(n, p, 46)
    for alg in (1, 2):
        plan = Plan.toeplitz(a, n, p_max=p, tol=1e-12, algorithm=alg, certify=True)
        Zg, info = plan.expm_block(1.0, to_dev(B))
        assert info.converged == 1
        nb = np.linalg.norm(B)
        for i in range(7):
            # the recurrence residual (eq. (49) / eq. (365)) is the true residual up to rounding
            assert abs(info.true_resid[i] - info.resid[i]) <= 1e-6 * info.resid[i] + 1e-13 * nb
            assert info.true_resid[i] <= 1e-12 * nb * 1.01


def test_workload_sampled_columns_and_mixed(tab):
    """The 2^20 x 16 workload as timed: two sampled columns against the Taylor truth, and the
    mixed path against the FP64 path (the metric's 1e-8 requirement)."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    w = inputs.WORKLOADS["toeplitz-1m"]
    n, p, t = w["n"], w["p"], w["t"][0]
    a = inputs.toeplitz_column(w["bw"], w["c"])
    B = inputs.rhs(n, p, w["seed"])
    Bd = to_dev(B)
    res = {}
    for prec in ("fp64", "mixed"):
        plan = Plan.toeplitz(a, n, p_max=p, m=w["m"], tol=w["tol"], precision=prec)
        Zg, info = plan.expm_block(t, Bd)
        assert info.converged == 1 and info.algorithm == 1
        res[prec] = to_np(Zg)
        plan.close()
    assert rel(res["mixed"], res["fp64"]) <= 1e-8
    cols = [0, p - 1]
    col = full_col(a, n)
    truth = TZ.taylor_expm_B(col, B[:, cols], t)
    assert rel(res["fp64"][:, cols], truth) <= truth_bound(tab, col, B[:, cols], truth, w["tol"]) * 2


def test_invalid_descriptors_rejected():
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300._native import ExpmError
    for a, n in [([-1.0, 0.6], 100),              # symbol max -1 + 1.2 > 0: not negative definite
                 ([0.5, 0.1], 100),               # a_0 >= 0
                 (inputs.toeplitz_column(256), 200),   # bw > n - 1
                 ([-2.0, np.nan], 100),
                 ([-2.0], (1 << 21) + 1)]:        # beyond the FFT size limit
        with pytest.raises(ExpmError):
            Plan.toeplitz(a, n, p_max=2)


# --------------------------------------------------------------------------- Example 5.4 regime
@pytest.mark.parametrize("n", [4096, 1 << 17])
def test_fractional_generator_and_inverse(n):
    """The large-norm operator (symmetric part of Example 5.4's fractional diffusion matrix,
    kappa ~ 1e6 at n = 4096 and ~ 1e9 at n = 2^17): plan creation solves the generator by
    conjugate gradients with T. Chan's circulant preconditioner, and the Gohberg-Semencul
    inverse then matches the oracle's (Levinson generator) to the conditioning limit."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    a = inputs.fractional_column(n)
    plan = Plan.toeplitz(a, n, p_max=2, algorithm=2)
    V = inputs.rhs(n, 2, 41)
    W = to_np(plan.prec_apply(1.0, to_dev(V)))
    ref = TZ.gsf_apply(TZ.gsf_generator(a), V, 1.0)
    kappa = (abs(a[0]) + 2 * np.abs(a[1:]).sum()) / 27.0     # ||T|| / |lambda_max| (lambda_max ~ -27)
    assert rel(W, ref) <= 1e-14 * kappa, (rel(W, ref), kappa)
    # and T (T^{-1} V) = V through the oracle's FFT product
    assert rel(TZ.matvec(a, W), V) <= 1e-14 * kappa


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fractional_expm_matches_eigendecomposition(tab, precision):
    """Algorithm 2 with the paper's m = 30, k = 30 deflated restart and p = 2 on the fractional
    operator (n = 2048, ||tA|| ~ 2e5 >> |tau_i|, the regime the preconditioner is for) against
    the exact r(tA) B and e^{tA} B by the oracle's eigendecomposition."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, t = 2048, 0.01
    a = inputs.fractional_column(n)
    B = inputs.rhs(n, 2, 42)
    Z, info = Plan.toeplitz(a, n, p_max=2, m=30, k_defl=30, tol=1e-10, precision=precision).expm_block(t, to_dev(B))
    assert info.converged == 1 and info.algorithm == 2
    ref = TZ.eig_function(a, B, lambda lam: ops.r_of_lambda_ext(tab, lam), t)
    assert rel(to_np(Z), ref) <= 1e-9, rel(to_np(Z), ref)
    ex = TZ.eig_function(a, B, np.exp, t)
    assert rel(to_np(Z), ex) <= 1e-9 + 1.1 * tab["sigma"] * np.linalg.norm(B) / np.linalg.norm(ex)


def test_fractional_workload_full_size(tab):
    """The toeplitz-frac workload at its size (n = 2^17, ||tA|| ~ 2e8): both precisions converge,
    the mixed result is within the metric's 1e-8 of the FP64 GPU path, certify mode's true FP64
    residuals equal the eq. (49) estimates, and the FP64 result agrees with the oracle's
    literal Algorithm 2 (Levinson generator, its own Gohberg-Semencul products) to the
    conditioning limit of the inverse (Theorem 4.3)."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    w = inputs.WORKLOADS["toeplitz-frac"]
    n, p, t = w["n"], w["p"], w["t"][0]
    a = inputs.fractional_column(n, w["frac"], w["d"])
    B = inputs.rhs(n, p, w["seed"])
    kw = dict(p_max=p, m=w["m"], k_defl=w["k_defl"], tol=w["tol"], max_cycles=100)
    Z64, i64 = Plan.toeplitz(a, n, certify=True, **kw).expm_block(t, to_dev(B))
    Zm, im = Plan.toeplitz(a, n, precision="mixed", **kw).expm_block(t, to_dev(B))
    assert i64.converged == 1 and im.converged == 1 and i64.algorithm == 2
    assert rel(to_np(Zm), to_np(Z64)) <= 1e-8
    # the true FP64 residuals ||B - (tA - tau_i I) X_i||_F of every pole: forming tA X_i alone
    # rounds at eps ||tA|| ||X_i|| ~ 1e-9 ||B|| here (||tA|| ~ 2e8), far above the eq. (49)
    # estimate of a converged solve, so the check is against ||B||
    nb = np.linalg.norm(B)
    for i in range(7):
        assert i64.true_resid[i] <= 1e-8 * nb, (i, i64.true_resid[i] / nb)
    x = TZ.gsf_generator(a)
    Zo, io = ps.psbfom(lambda V: TZ.gsf_apply(x, V, t), B, tab, m=w["m"], tol=w["tol"], max_cycles=100,
                       k=w["k_defl"], align=p)
    kappa = (abs(a[0]) + 2 * np.abs(a[1:]).sum()) / 27.0
    assert rel(to_np(Z64), Zo) <= max(1e-10, 1e-15 * kappa), (rel(to_np(Z64), Zo), kappa)
