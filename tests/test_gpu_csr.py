"""General sparse operators (EXPM_OP_CSR) through the C ABI: the sparse product of Algorithm 1,
the inexact inverse of Algorithm 2 (inner BiCGStab, Section 4.1), and whole solves against
the oracle's closed forms.

* The product t A V against scipy's, entry by entry within the FP64 rounding of a row's sum.
* The inner solve meets its stopping rule: ||V - tA W|| <= inner_tol ||V|| per column.
* The convection-diffusion stencil assembled as a CSR matrix: Z against the oracle's exact
  r(tA) B (DST eigen-expansion) and against the stencil plan's Z, with both algorithms in
  both precisions.
* A seeded nonsymmetric sparse matrix: Z against the oracle's dense r(tA) B (eq. (11) by dense
  solves), both algorithms.
* Theorem 4.3: a looser inner tolerance costs accuracy in proportion, the error staying within
  kappa(A) times the tolerance.
"""
import numpy as np
import pytest

from oracle import cf, operators as ops, psbfom as ps
from paper_1405_0707_gb300 import inputs
from tests.gpu_util import need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


def random_csr(n, seed=None):
    import scipy.sparse as sp
    ip, ix, d = inputs.sparse_dd_matrix(n) if seed is None else inputs.sparse_dd_matrix(n, seed=seed)
    return sp.csr_matrix((d, ix, ip), shape=(n, n))


def test_csr_product_matches_scipy():
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    A = random_csr(3001)
    V = inputs.rhs(3001, 5, 11)
    t = 2.5e-4
    W = to_np(Plan.csr(A, p_max=5, m=2).op_apply(t, to_dev(V)))
    ref = t * (A @ V)
    bound = t * (abs(A) @ np.abs(V))
    assert np.all(np.abs(W - ref) <= 16 * 2.0 ** -53 * bound)


@pytest.mark.parametrize("eta", [1e-8, 1e-13])
def test_csr_inner_solve_meets_its_tolerance(eta):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    A = random_csr(2500)
    V = inputs.rhs(2500, 4, 12)
    V[:, 2] *= 1e-3                     # columns of different scales stop on their own norms
    t = 1e-4
    W = to_np(Plan.csr(A, p_max=4, m=2, inner_tol=eta).prec_apply(t, to_dev(V)))
    R = V - t * (A @ W)
    for c in range(4):
        assert np.linalg.norm(R[:, c]) <= 1.05 * eta * np.linalg.norm(V[:, c]), c


@pytest.mark.parametrize("sides,diff,vel,t,p", [((40, 37), 0.1, (1.0, -0.5), 0.05, 3),
                                                 ((20, 18, 16), 1.0, (2.0, -1.0, 0.5), 0.02, 2)])
@pytest.mark.parametrize("alg", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_csr_stencil_matches_closed_form(tab, sides, diff, vel, t, p, alg, precision):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    A = ops.cd_matrix(sides, diff, vel)
    B = inputs.rhs(n, p, 21)
    Zc, ic = Plan.csr(A, p_max=p, m=10, tol=1e-11, max_cycles=400, algorithm=alg, precision=precision,
                      inner_tol=1e-13).expm_block(t, to_dev(B))
    assert ic.converged == 1 and ic.algorithm == alg
    assert (ic.inner_iters > 0) == (alg == 2)
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    assert rel(to_np(Zc), ref) <= 1e-9, rel(to_np(Zc), ref)
    Zs, _ = Plan(sides, diff, vel, p_max=p, m=10, tol=1e-11, max_cycles=400, algorithm=alg,
                 precision=precision).expm_block(t, to_dev(B))
    assert rel(to_np(Zc), to_np(Zs)) <= 1e-9


@pytest.mark.parametrize("alg", [0, 1, 2])
def test_csr_random_matrix_matches_dense_reference(tab, alg):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, p, t = 1200, 3, 1e-4
    A = random_csr(n)
    B = inputs.rhs(n, p, 5)
    Z, info = Plan.csr(A, p_max=p, m=10, tol=1e-12, max_cycles=200, algorithm=alg,
                       inner_tol=1e-14).expm_block(t, to_dev(B))
    assert info.converged == 1
    ref = ps.dense_r_of_A_B((t * A).toarray(), B, tab)
    assert rel(to_np(Z), ref) <= 1e-10, rel(to_np(Z), ref)


def test_csr_inexact_inverse_error_follows_theorem_4_3(tab):
    """Theorem 4.3: ||X_i - X~_i|| / ||X_i|| <~ kappa(A) ||(I - tau_i A^{-1})^{-1}|| eta.  The
    final error grows as the inner tolerance loosens and stays within kappa(A) eta times a
    modest factor (here ||(I - tau_i A^{-1})^{-1}|| <= 1 by the spectrum's half-plane)."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, p, t = 1200, 2, 1e-4
    A = random_csr(n)
    B = inputs.rhs(n, p, 6)
    ref = ps.dense_r_of_A_B((t * A).toarray(), B, tab)
    kappa = np.linalg.cond(A.toarray())
    errs = {}
    for eta in (1e-6, 1e-9, 1e-13):
        Z, info = Plan.csr(A, p_max=p, m=10, tol=1e-13, max_cycles=200, algorithm=2,
                           inner_tol=eta).expm_block(t, to_dev(B))
        errs[eta] = rel(to_np(Z), ref)
        assert errs[eta] <= 10 * kappa * eta + 1e-11, (eta, errs[eta], kappa)
    assert errs[1e-13] < errs[1e-6]


def test_csr_full_size_product_and_inner_solve():
    """At the benchmarked size (csr3d-96: the 96^3 7-point pattern with random values, p = 16):
    the product against scipy's entry by entry, and the inner solve's stopping rule per column
    with the residual formed on the host by scipy."""
    need_gpu()
    import scipy.sparse as sp
    from paper_1405_0707_gb300 import Plan
    w = inputs.WORKLOADS["csr3d-96"]
    ip, ix, dv = inputs.sparse_stencil_matrix(w["csr_sides"])
    n, p, t = 96 ** 3, w["p"], w["t"][0]
    A = sp.csr_matrix((dv, ix, ip), shape=(n, n))
    V = inputs.rhs(n, p, w["seed"])
    plan = Plan.csr(A, p_max=p, m=2, inner_tol=1e-12)
    W = to_np(plan.op_apply(t, to_dev(V)))
    assert np.all(np.abs(W - t * (A @ V)) <= 16 * 2.0 ** -53 * t * (abs(A) @ np.abs(V)))
    X = to_np(plan.prec_apply(t, to_dev(V)))
    R = V - t * (A @ X)
    for c in range(p):
        assert np.linalg.norm(R[:, c]) <= 1.05e-12 * np.linalg.norm(V[:, c]), c


def test_csr_plans_reject_what_they_do_not_support():
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300._native import ExpmError
    from paper_1405_0707_gb300.api import Batch
    A = random_csr(500)
    with pytest.raises(ExpmError):
        Plan.csr(A, p_max=2, m=4, certify=True)
    pl = Plan.csr(A, p_max=2, m=4, stream=torch.cuda.Stream())
    B = to_dev(inputs.rhs(500, 2, 3))
    with pytest.raises(ExpmError):
        Batch([pl], [1e-4], [B])
