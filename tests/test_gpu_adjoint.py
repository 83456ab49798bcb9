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
    from paper_1405_0707_gb300.autograd import expm_block
    n = int(np.prod(sides))
    B = inputs.rhs(n, p, seed)
    t0, B0 = inputs.grad_target(n, p, seed, t)
    plan = Plan(sides, diff, vel, p_max=p, m=m, tol=tol, max_cycles=400, precision=precision)
    Y, _ = plan.expm_block(t0, to_dev(B0))
    Y = Y.clone()

    def loss(tv, Bt):
        Z = expm_block(tv, Bt, plan)
        return ((Z - Y) ** 2).sum(), Z
    return torch, plan, B, Y, loss


def central_difference(loss, tv, B, D, h, Y):
    """(L(B + hD) - L(B - hD)) / 2h for L = ||Z - Y||_F^2, formed as
    <Z+ - Z-, Z+ + Z- - 2Y> / 2h: the same central difference of the computed map, without
    subtracting two nearly equal large values of L (at h = 1e-6 that subtraction alone would
    cost ~1e-5 relative)."""
    import torch
    with torch.no_grad():
        _, Zp = loss(tv, to_dev(B + h * D))
        _, Zm = loss(tv, to_dev(B - h * D))
        return float(torch.sum((Zp - Zm) * (Zp + Zm - 2.0 * Y))) / (2 * h)


@pytest.mark.parametrize("sides,diff,vel,t,p,precision", [((37, 29), 0.1, (1.0, 1.0), 0.1, 3, "fp64"),
                                                          ((40, 33), 0.1, (1.0, -0.5), 1.0, 2, "mixed"),
                                                          ((11, 9, 7), 1.0, (3.0, -2.0, 1.0), 0.3, 2, "fp64")])
def test_adjoint_matches_closed_form_and_finite_differences(tab, sides, diff, vel, t, p, precision):
    torch, plan, B, Y, loss = _loss_setup(sides, diff, vel, t, p, 17, precision)
    tv = torch.tensor(t, dtype=torch.float64, device="cuda", requires_grad=True)
    Bt = to_dev(B).clone().requires_grad_(True)
    L, Z = loss(tv, Bt)
    L.backward()
    gB, gt = to_np(Bt.grad), float(tv.grad)
    G = 2.0 * (to_np(Z) - to_np(Y))
    # dL/dB = r(tA^T) G by the closed form of A^T (velocity negated)
    ref = ops.exact_r_of_A_B(sides, diff, tuple(-v for v in vel), t, tab, G)
    assert rel(gB, ref) <= 1e-9
    # central differences along a random direction in B with the differentiation workload's
    # step h = 1e-6 (L is quadratic in B, so the difference quotient is exact up to rounding
    # and the solver's error, which it divides by 2h: FP64 solves at tol 1e-14) and in t
    rng = np.random.default_rng(3)
    D = rng.standard_normal(B.shape)
    h = 1e-6
    _, _, _, Yfd, loss_fd = _loss_setup(sides, diff, vel, t, p, 17, "fp64", tol=1e-14)
    fd = central_difference(loss_fd, tv, B, D, h, Yfd)
    assert abs(fd - np.sum(gB * D)) <= 1e-5 * abs(fd) + 1e-9, (fd, np.sum(gB * D))
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
    torch, plan, B, Y, loss = _loss_setup(w["sides"], w["diff"], w["vel"], t, w["p"],
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
    # dL/dB against central differences with h = 1e-6 along a random direction.  The two
    # perturbed losses differ by ~2h |dL/dB . D|, and each carries the solve's own error, which
    # the quotient divides by 2h: the mixed path's ~1e-12 rounding would cost ~1e-4 there, so
    # the difference quotient of the map is taken with FP64 solves converged to tol 1e-14
    # The direction is the computed gradient itself (scaled to ||B||): a random direction in
    # these 8.4e6 dimensions is nearly orthogonal to Z - Y (cosine ~ 3e-4), which would scale
    # every small difference between the two losses' solves up by ~3000 relative to the
    # directional derivative
    gB = to_np(Bt.grad)
    D = gB * (np.linalg.norm(B) / np.linalg.norm(gB))
    h = 1e-6
    _, _, _, Yfd, loss_fd = _loss_setup(w["sides"], w["diff"], w["vel"], t, w["p"], w["seed"], "fp64",
                                        m=w["m"], tol=1e-14)
    fd = central_difference(loss_fd, tv, B, D, h, Yfd)
    gD = float(np.sum(gB * D))
    assert abs(fd - gD) <= 1e-5 * abs(fd), (fd, gD)
    ht = 1e-6 * t
    with torch.no_grad():
        Lp, _ = loss(torch.tensor(t + ht, dtype=torch.float64, device="cuda"), to_dev(B))
        Lm, _ = loss(torch.tensor(t - ht, dtype=torch.float64, device="cuda"), to_dev(B))
    fdt = (float(Lp) - float(Lm)) / (2 * ht)
    assert abs(fdt - float(tv.grad)) <= 1e-5 * abs(fdt), (fdt, float(tv.grad))


def test_adjoint_entry_point_parts(tab):
    """expm_block_adjoint directly: dL/dt alone equals <G, A Z> computed on the host from the
    oracle's operator; dL/dB alone equals the closed form on A^T; both outputs together
    agree with the separate calls."""
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t, p = (33, 27), 0.1, (1.0, -1.0), 0.05, 3
    n = int(np.prod(sides))
    plan = Plan(sides, diff, vel, p_max=p, m=8, tol=1e-13)
    B = inputs.rhs(n, p, 51)
    G = inputs.rhs(n, p, 52)
    Z, _ = plan.expm_block(t, to_dev(B))
    Gd = to_dev(G)
    _, gt, _ = plan.expm_block_adjoint(t, Gd, Z, want_dB=False)
    A = ops.cd_matrix(sides, diff, vel, 1.0)
    ref_t = float(np.sum(G * (A @ to_np(Z))))
    assert abs(gt - ref_t) <= 1e-12 * abs(ref_t) + 1e-12
    dB, none, _ = plan.expm_block_adjoint(t, Gd, None, want_dt=False)
    assert none is None
    ref_B = ops.exact_r_of_A_B(sides, diff, tuple(-v for v in vel), t, tab, G)
    assert rel(to_np(dB), ref_B) <= 1e-10
    dB2, gt2, _ = plan.expm_block_adjoint(t, Gd, Z)
    assert np.array_equal(to_np(dB2), to_np(dB)) and gt2 == gt


def test_adjoint_toeplitz_is_self_adjoint(tab):
    """A symmetric Toeplitz operator is its own transpose: dL/dB = r(tT) G, checked against
    the forward call on G, and dL/dt against <G, T Z> from the oracle's product."""
    need_gpu()
    from oracle import toeplitz as TZ
    from paper_1405_0707_gb300 import Plan
    n, p, t = 3000, 2, 1.0
    a = inputs.toeplitz_column(256)
    plan = Plan.toeplitz(a, n, p_max=p, tol=1e-13)
    B, G = inputs.rhs(n, p, 53), inputs.rhs(n, p, 54)
    Z, _ = plan.expm_block(t, to_dev(B))
    dB, gt, _ = plan.expm_block_adjoint(t, to_dev(G), Z)
    ZG, _ = plan.expm_block(t, to_dev(G))
    assert np.array_equal(to_np(dB), to_np(ZG))
    col = np.zeros(n)
    col[:len(a)] = a
    ref_t = float(np.sum(G * TZ.matvec(col, to_np(Z), 1.0)))
    assert abs(gt - ref_t) <= 1e-12 * abs(ref_t)
