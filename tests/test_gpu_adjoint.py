"""Hand-written adjoint of Z = r(tA) B (torch.autograd.Function), through the C ABI.

dL/dB = r(tA^T) G is checked against the oracle's closed form with A^T (velocity negated) and
against central finite differences of the computed map; dL/dt = <G, A Z> is checked against
central finite differences in t (it differentiates e^{tA}; the gap to the derivative of
r(tA) is of the order of the CF error of r', far below the FD tolerance).
"""
import numpy as np
import pytest

from oracle import cf, operators as ops
from paper_1405_0707_gb300 import inputs
from tests.gpu_util import need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


def _loss_setup(sides, diff, vel, t, p, seed, precision, m=8, tol=1e-13):
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300.autograd import expm_block, transpose_plan
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, seed)
    t0, B0 = inputs.grad_target(n, p, seed, t)
    plan = Plan(sides, diff, vel, p_max=p, m=m, tol=tol, max_cycles=400, precision=precision)
    plan_T = transpose_plan(plan)
    Y, _ = plan.expm_block(t0, to_dev(B0))
    Y = Y.clone()

    def loss(tv, Bt):
        Z = expm_block(tv, Bt, plan, plan_T)
        return ((Z - Y) ** 2).sum(), Z
    return torch, plan, plan_T, B, Y, loss


@pytest.mark.parametrize("sides,diff,vel,t,p,precision", [((37, 29), 0.1, (1.0, 1.0), 0.1, 3, "fp64"),
                                                          ((40, 33), 0.1, (1.0, -0.5), 1.0, 2, "mixed"),
                                                          ((11, 9, 7), 1.0, (3.0, -2.0, 1.0), 0.3, 2, "fp64")])
def test_adjoint_matches_closed_form_and_finite_differences(tab, sides, diff, vel, t, p, precision):
    torch, plan, plan_T, B, Y, loss = _loss_setup(sides, diff, vel, t, p, 17, precision)
    tv = torch.tensor(t, dtype=torch.float64, device="cuda", requires_grad=True)
    Bt = to_dev(B).clone().requires_grad_(True)
    L, Z = loss(tv, Bt)
    L.backward()
    gB, gt = to_np(Bt.grad), float(tv.grad)
    G = 2.0 * (to_np(Z) - to_np(Y))
    # dL/dB = r(tA^T) G by the closed form of A^T (velocity negated)
    ref = ops.exact_r_of_A_B(sides, diff, tuple(-v for v in vel), t, tab, G)
    assert rel(gB, ref) <= 1e-9
    # central differences along a random direction in B (L is quadratic in B: exact up to
    # rounding) and in t
    rng = np.random.default_rng(3)
    D = rng.standard_normal(B.shape)
    h = 1e-4
    with torch.no_grad():
        Lp, _ = loss(tv, to_dev(B + h * D))
        Lm, _ = loss(tv, to_dev(B - h * D))
    fd = (float(Lp) - float(Lm)) / (2 * h)
    assert abs(fd - np.sum(gB * D)) <= 1e-6 * abs(fd) + 1e-9
    ht = 1e-6 * t
    with torch.no_grad():
        Lp, _ = loss(torch.tensor(t + ht, dtype=torch.float64, device="cuda"), to_dev(B))
        Lm, _ = loss(torch.tensor(t - ht, dtype=torch.float64, device="cuda"), to_dev(B))
    fdt = (float(Lp) - float(Lm)) / (2 * ht)
    assert abs(fdt - gt) <= 1e-5 * abs(fdt) + 1e-9, (fdt, gt)


def test_differentiation_workload_512(tab):
    """The differentiation workload at full size: 512 x 512 grid (n = 262144), p = 32,
    t = 1e-2, mixed precision (FP32 transforms refined to FP64, FP64 projected solves)."""
    w = inputs.WORKLOADS["cd2d-512-grad"]
    t = w["t"][0]
    torch, plan, plan_T, B, Y, loss = _loss_setup(w["sides"], w["diff"], w["vel"], t, w["p"],
                                                  w["seed"], "mixed", m=w["m"], tol=w["tol"])
    tv = torch.tensor(t, dtype=torch.float64, device="cuda", requires_grad=True)
    Bt = to_dev(B).clone().requires_grad_(True)
    L, Z = loss(tv, Bt)
    L.backward()
    G = 2.0 * (to_np(Z) - to_np(Y))
    ref = ops.exact_r_of_A_B(w["sides"], w["diff"], tuple(-v for v in w["vel"]), t, tab, G)
    assert rel(to_np(Bt.grad), ref) <= 1e-8
    # forward against the closed form too
    assert rel(to_np(Z), ops.exact_r_of_A_B(w["sides"], w["diff"], w["vel"], t, tab, B)) <= 1e-8
    ht = 1e-6 * t
    with torch.no_grad():
        Lp, _ = loss(torch.tensor(t + ht, dtype=torch.float64, device="cuda"), to_dev(B))
        Lm, _ = loss(torch.tensor(t - ht, dtype=torch.float64, device="cuda"), to_dev(B))
    fdt = (float(Lp) - float(Lm)) / (2 * ht)
    assert abs(fdt - float(tv.grad)) <= 1e-5 * abs(fdt), (fdt, float(tv.grad))
