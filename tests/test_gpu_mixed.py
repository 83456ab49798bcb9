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


# 3-D grids that take each transform and line-solve kernel of the FP32 inverse: every axis
# <= 96 (shared-memory transform, N padded to 48/80/96), an axis of 100 (tiled transform with
# merged (x, z) rows), x lines <= 128 with >= 1024 modes (thread-per-line solve) and x = 130
# (shared-memory line solve), with ragged 128-row slabs throughout
CASES_3D = [((45, 37, 33), 1.0, (2.0, -1.0, 0.5), 0.05, 3),
            ((97, 33, 35), 1.0, (1.0, 1.0, -1.0), 0.02, 2),
            ((40, 100, 30), 1.0, (-1.5, 0.5, 1.0), 0.05, 2),
            ((130, 20, 60), 1.0, (0.5, -0.5, 2.0), 0.02, 1)]


@pytest.mark.parametrize("sides,diff,vel,t,p", CASES_3D)
def test_refined_fp32_inverse_3d_transform_paths(sides, diff, vel, t, p):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    V = inputs.rhs(n, p, 78)
    W64 = to_np(Plan(sides, diff, vel, p_max=p, m=2).prec_apply(t, to_dev(V)))
    W32 = to_np(Plan(sides, diff, vel, p_max=p, m=2, precision="mixed").prec_apply(t, to_dev(V)))
    kappa = 1.0
    for d in range(1, len(sides)):
        _, dp, _ = ops.axis_eig(sides[d], diff, vel[d], t)
        kappa *= dp.max() / dp.min()
    assert rel(W32, W64) <= 1e-13 * max(1.0, kappa)
    # and A (A^{-1} V) = V through the oracle's independent sparse matrix
    assert rel(ops.cd_matrix(sides, diff, vel, t) @ W32, V) <= 1e-11 * max(1.0, kappa)


@pytest.mark.parametrize("sides,diff,vel,t,p", CASES + CASES_3D[:2] + [((517,), 1.0, (0.0,), 1.0, 3)])
def test_double_float_stencil_matches_sparse_matrix(sides, diff, vel, t, p):
    """Mixed plans apply tA in double-float (pairs of floats from the bit pattern): every entry
    within 2^-43 of the sum of the magnitudes of its terms, |tA| |V|.  Each pair multiply-add
    leaves up to ~2^-47 of its term (the rounded cross terms and the low word's sum), and the
    coefficients' pairs carry 2^-48: an FP32 emulation of the kernel on the 256^2 case reaches
    0.99 * 2^-45 with 5 terms; 2^-43 covers 7 terms with room."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n = int(np.prod(sides))
    V = inputs.rhs(n, p, 4321)
    W = to_np(Plan(sides, diff, vel, p_max=p, m=2, precision="mixed").op_apply(t, to_dev(V)))
    A = ops.cd_matrix(sides, diff, vel, t)
    ref = A @ V
    bound = abs(A) @ np.abs(V)
    assert np.all(np.abs(W - ref) <= 2.0 ** -43 * bound)


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


@pytest.mark.parametrize("single_pass", ["1", "0"])
@pytest.mark.parametrize("sides,p", [((70, 66), 1), ((70, 66), 5), ((256, 256), 8), ((97, 83), 12),
                                     ((97, 83), 16)])
def test_mixed_arnoldi_relation_is_fp64_exact(sides, p, single_pass, monkeypatch):
    """The mixed block step (FP32 projections, double-float first update, FP32 second-pass
    correction, FP32-factor Cholesky-QR applied exactly) keeps the block Arnoldi relation
    (tA)^{-1} V_m = V_{m+1} H~_m (Section 3) to FP64 rounding, while V is orthonormal only to
    the FP32 level.  W = (tA)^{-1} V_m comes from the plan's own inverse.  Both with the single
    accurate Cholesky-QR pass (taken for these well-conditioned blocks) and with the plan
    switch that keeps every block on the three-pass FP32 scheme it falls back to."""
    need_gpu()
    monkeypatch.setenv("EXPM_QR_SINGLE_PASS", single_pass)
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


@pytest.mark.parametrize("alg", [1, 2])
def test_mixed_single_pass_on_and_off_agree(tab, alg, monkeypatch):
    """A converged mixed solve with the single accurate Cholesky-QR pass and with it switched
    off (every block through the FP32 three-pass fallback): both match r(tA)B and each other."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t, p = (70, 66), 0.1, (1.0, -0.5), (0.02 if alg == 1 else 1.0), 6
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, 81)
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    out = {}
    for sp in ("1", "0"):
        monkeypatch.setenv("EXPM_QR_SINGLE_PASS", sp)
        Z, info = Plan(sides, diff, vel, p_max=p, m=6, tol=1e-12, max_cycles=400, algorithm=alg,
                       precision="mixed").expm_block(t, to_dev(B))
        assert info.converged == 1, sp
        out[sp] = to_np(Z)
        assert rel(out[sp], ref) <= 1e-9, (sp, rel(out[sp], ref))
    assert rel(out["0"], out["1"]) <= 1e-9


@pytest.mark.parametrize("delta", [1e-4, 1e-6])
def test_mixed_block_nearly_dependent_mid_cycle(tab, delta):
    """B = [b0, b1, (tA)^{-1} b0 + delta b2]: the first block step's W = (tA)^{-1} V_1 then has a
    direction that lies in span(V_1) up to O(delta), so after the Gram-Schmidt passes its Gram
    matrix has a pivot far below 1e-5 of the largest diagonal entry.  The mixed path must
    reject the single accurate Cholesky-QR pass there and finish on the shifted FP32 passes
    (on real data, in the middle of a cycle), and still match r(tA)B and the FP64 path."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t = (41, 35), 0.1, (1.0, 1.0), 1.0
    n = int(np.prod(sides))
    b = inputs.rhs(n, 3, 82)
    Ainv = ps.lu_inverse(ops.cd_matrix(sides, diff, vel, t))
    B = np.column_stack([b[:, 0], b[:, 1], Ainv(b[:, 0]) * 10.0 + delta * b[:, 2]])
    # the deficiency of the first Krylov block, computed on the host: the smallest singular
    # value of the projected W relative to its largest
    V1, _ = ps.qr_positive(B)
    W = np.column_stack([Ainv(V1[:, c]) for c in range(3)])
    W = W - V1 @ (V1.T @ W)
    sv = np.linalg.svd(W, compute_uv=False)
    assert (sv[-1] / sv[0]) ** 2 < 1e-5
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    Zm, im = Plan(sides, diff, vel, p_max=3, m=6, tol=1e-12, max_cycles=300, algorithm=2,
                  precision="mixed").expm_block(t, to_dev(B))
    Zd, idd = Plan(sides, diff, vel, p_max=3, m=6, tol=1e-12, max_cycles=300,
                   algorithm=2).expm_block(t, to_dev(B))
    assert im.converged == 1 and idd.converged == 1
    assert rel(to_np(Zm), ref) <= 1e-9, rel(to_np(Zm), ref)
    assert rel(to_np(Zm), to_np(Zd)) <= 1e-9
