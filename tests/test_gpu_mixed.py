"""Mixed precision (FP32 transforms refined to FP64 accuracy, FP32 projections, FP64
updates) against the plain FP64 GPU path and the oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import cf, operators as ops, psbfom as ps
from paper_1405_0707_gb300 import inputs
from tests.gpu_util import cancellation_floor, need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

# (at t = 1 the 11 x 9 x 7 operator has ||e^{tA}|| ~ e^-30: Z would sit at the rounding
#  floor of the partial-fraction sum, so the 3-D case uses t = 0.3)
CASES = [((37, 29), 0.1, (1.0, 1.0), 1e-1, 3),
         ((70, 66), 0.1, (1.0, -0.5), 1.0, 5),
         ((11, 9, 7), 1.0, (3.0, -2.0, 1.0), 0.3, 2),
         ((256, 256), 0.1, (1.0, 1.0), 1e-1, 8)]


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


@pytest.mark.parametrize("sides,diff,vel,t,p", CASES)
def test_refined_fp32_inverse_matches_fp64(sides, diff, vel, t, p):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    V = inputs.rhs(n, p, 77)
    W64 = to_np(Plan(sides, diff, vel, p_max=p, m=2).prec_apply(t, to_dev(V)))
    W32 = to_np(Plan(sides, diff, vel, p_max=p, m=2, precision="mixed").prec_apply(t, to_dev(V)))
    kappa = 1.0
    for d in range(1, len(sides)):
        _, dp, _ = ops.axis_eig(sides[d], diff, vel[d], t)
        kappa *= dp.max() / dp.min()
    assert rel(W32, W64) <= 1e-13 * max(1.0, kappa)


@pytest.mark.parametrize("sides,diff,vel,t,p", CASES[:3])
def test_mixed_converged_matches_fp64_and_closed_form(tab, sides, diff, vel, t, p):
    """Converged to tol 1e-12, the mixed path agrees with the FP64 path and with r(tA)B.
    (Unconverged iterates of the two are not comparable: FP32 projections perturb the basis
    at the 1e-7 level, which moves an unconverged iterate by about its own residual.)"""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, 78)
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    for alg in (0,):          # AUTO: Algorithm 1 on the first case, Algorithm 2 on the others
        Z64, i64 = Plan(sides, diff, vel, p_max=p, m=5, tol=1e-12, max_cycles=400,
                        algorithm=alg).expm_block(t, to_dev(B))
        Z32, i32 = Plan(sides, diff, vel, p_max=p, m=5, tol=1e-12, max_cycles=400, algorithm=alg,
                        precision="mixed").expm_block(t, to_dev(B))
        assert i64.converged and i32.converged, alg
        assert rel(to_np(Z32), to_np(Z64)) <= 1e-9, (alg, rel(to_np(Z32), to_np(Z64)))
        assert rel(to_np(Z32), ref) <= 1e-9


@pytest.mark.parametrize("t", [1e-3, 1e-2, 1e-1])
def test_mixed_meets_metric_tolerance_on_bench_workload(tab, t):
    """The metric's criterion: rel.err <= 1e-8 against the plain FP64 GPU path, on the
    256 x 256 workload at every t, both converged to tol 1e-10."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    w = inputs.WORKLOADS["cd2d-256"]
    n = 65536
    B = to_dev(inputs.rhs(n, w["p"], w["seed"]))
    Z64, i64 = Plan(w["sides"], w["diff"], w["vel"], p_max=8, m=10, tol=1e-10).expm_block(t, B)
    Z32, i32 = Plan(w["sides"], w["diff"], w["vel"], p_max=8, m=10, tol=1e-10,
                    precision="mixed").expm_block(t, B)
    assert i64.converged and i32.converged
    assert rel(to_np(Z32), to_np(Z64)) <= 1e-8
    # and against the closed form r(tA)B
    ref = ops.exact_r_of_A_B(w["sides"], w["diff"], w["vel"], t, tab, inputs.rhs(n, w["p"], w["seed"]))
    assert rel(to_np(Z32), ref) <= 1e-8


@pytest.mark.parametrize("sides,p", [((70, 66), 1), ((70, 66), 5), ((256, 256), 8), ((97, 83), 12),
                                     ((97, 83), 16)])
def test_mixed_arnoldi_relation_is_fp64_exact(sides, p):
    """The mixed block step (FP32 projections, double-float first update, FP32 second-pass
    correction, FP32-factor Cholesky-QR applied exactly) keeps the block Arnoldi relation
    (tA)^{-1} V_m = V_{m+1} H~_m (Section 3) to FP64 rounding, while V is orthonormal only to
    the FP32 level.  W = (tA)^{-1} V_m comes from the plan's own inverse."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, m, t = int(np.prod(sides)), 6, 0.05
    V1, _ = ps.qr_positive(inputs.rhs(n, p, 8))
    plan = Plan(sides, 0.1, (1.0, -0.5), p_max=p, m=m, precision="mixed")
    Vg, Hg = plan.arnoldi(t, to_dev(V1))
    W = np.column_stack([to_np(plan.prec_apply(t, Vg[:, j * p:(j + 1) * p])) for j in range(m)])
    Vn, Hn = to_np(Vg), to_np(Hg)
    assert np.linalg.norm(W - Vn @ Hn) <= 1e-12 * np.linalg.norm(W)
    assert np.linalg.norm(Vn.T @ Vn - np.eye((m + 1) * p)) <= 1e-5
    assert np.all(Hn[np.tril_indices_from(Hn, -p - 1)] == 0.0)
