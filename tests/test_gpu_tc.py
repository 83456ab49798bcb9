"""The first block CGS2 pass of the mixed path on the tensor cores (tcgen05 MMAs on exact bf16
slices, accumulators in tensor memory; k_cgs_tc.cu), through the C ABI.

* The block Arnoldi relation (tA)^{-1} V_m = V_{m+1} H~_m (eq. (4.5)) holds to FP64 rounding
  with the tensor-core pass forced on, for block widths 1..16 and row counts that leave a
  ragged last 128-row tile, and H~ agrees with the CUDA-core (double-float) pass's.
* The first projection on the tensor cores (TF32 hi/lo products) keeps the relation
  FP64-exact and the basis as orthonormal as the FP32 projection kernel does.
* Converged solves with it match the closed form r(tA) B.
* Their bounded mbarrier waits: with the bound forced to zero polls every wait runs out, the
  call returns EXPM_TIMEOUT after each kernel drains its own MMAs and frees its tensor
  memory, and the device stays usable for the next call.
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


@pytest.mark.parametrize("sides,p,m", [((256, 256), 8, 6), ((130, 129), 16, 6), ((70, 66), 1, 8),
                                       ((97, 83), 12, 6), ((61, 59), 3, 10), ((33, 31, 29), 5, 6)])
def test_tc_arnoldi_relation_is_fp64_exact(sides, p, m, monkeypatch):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, t = int(np.prod(sides)), 0.05
    vel = (1.0, -0.5) if len(sides) == 2 else (1.0, -0.5, 0.3)
    V1, _ = ps.qr_positive(inputs.rhs(n, p, 8))
    out = {}
    for tc in ("1", "0"):
        monkeypatch.setenv("EXPM_CGS_TC", tc)
        plan = Plan(sides, 0.1, vel, p_max=p, m=m, precision="mixed")
        Vg, Hg = plan.arnoldi(t, to_dev(V1))
        W = np.column_stack([to_np(plan.prec_apply(t, Vg[:, j * p:(j + 1) * p])) for j in range(m)])
        Vn, Hn = to_np(Vg), to_np(Hg)
        assert np.linalg.norm(W - Vn @ Hn) <= 1e-12 * np.linalg.norm(W), (tc, np.linalg.norm(W - Vn @ Hn) / np.linalg.norm(W))
        assert np.linalg.norm(Vn.T @ Vn - np.eye((m + 1) * p)) <= 1e-5
        out[tc] = Hn
    assert np.linalg.norm(out["1"] - out["0"]) <= 1e-6 * np.linalg.norm(out["0"])


@pytest.mark.parametrize("sides,p,m", [((97, 83), 16, 10), ((61, 59), 3, 10), ((33, 31, 29), 5, 6),
                                       ((130, 129), 12, 11), ((70, 66), 1, 8)])
def test_tc_projection_keeps_the_relation_and_orthogonality(sides, p, m, monkeypatch):
    """The first projection h = V^T W on the tensor cores (TF32 hi/lo products, k_proj_tc):
    the relation stays FP64-exact (the update applies the h it records), the basis is as
    orthonormal as with the FP32 projection kernel, and H~ agrees with that kernel's to the
    second pass's FP32 level.  The cases cover one and two 128-column M tiles (cols up to 160)
    and row counts with a ragged last 256-row tile and 16-row chunk."""
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    n, t = int(np.prod(sides)), 0.05
    vel = (1.0, -0.5) if len(sides) == 2 else (1.0, -0.5, 0.3)
    V1, _ = ps.qr_positive(inputs.rhs(n, p, 9))
    out = {}
    for ptc in ("1", "0"):
        monkeypatch.setenv("EXPM_PROJ_TC", ptc)
        plan = Plan(sides, 0.1, vel, p_max=p, m=m, precision="mixed")
        Vg, Hg = plan.arnoldi(t, to_dev(V1))
        W = np.column_stack([to_np(plan.prec_apply(t, Vg[:, j * p:(j + 1) * p])) for j in range(m)])
        Vn, Hn = to_np(Vg), to_np(Hg)
        assert np.linalg.norm(W - Vn @ Hn) <= 1e-12 * np.linalg.norm(W), (ptc, np.linalg.norm(W - Vn @ Hn) / np.linalg.norm(W))
        assert np.linalg.norm(Vn.T @ Vn - np.eye((m + 1) * p)) <= 1e-5
        out[ptc] = Hn
        plan.close()
    assert np.linalg.norm(out["1"] - out["0"]) <= 1e-6 * np.linalg.norm(out["0"])


@pytest.mark.parametrize("sides,p,t", [((256, 256), 8, 0.1), ((181, 181), 16, 0.05), ((40, 37, 35), 10, 0.02)])
def test_tc_converged_matches_closed_form(tab, sides, p, t, monkeypatch):
    need_gpu()
    from paper_1405_0707_gb300 import Plan
    monkeypatch.setenv("EXPM_CGS_TC", "1")
    n = int(np.prod(sides))
    vel = (1.0, 1.0) if len(sides) == 2 else (2.0, -1.0, 1.5)
    diff = 0.1 if len(sides) == 2 else 1.0
    B = inputs.rhs(n, p, 44)
    Z, info = Plan(sides, diff, vel, p_max=p, m=10, tol=1e-11, max_cycles=400,
                   precision="mixed").expm_block(t, to_dev(B))
    assert info.converged == 1
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    assert rel(to_np(Z), ref) <= 1e-9, rel(to_np(Z), ref)


@pytest.mark.parametrize("cgs_tc,proj_tc", [("1", "0"), ("0", "1")])
def test_tc_bounded_wait_returns_timeout(cgs_tc, proj_tc, monkeypatch):
    """Each tensor-core kernel alone (the update, then the projection) with zero polls."""
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300 import _native as N
    sides, p, t = (200, 190), 8, 0.1
    n = 200 * 190
    B = to_dev(inputs.rhs(n, p, 45))
    monkeypatch.setenv("EXPM_CGS_TC", cgs_tc)
    monkeypatch.setenv("EXPM_PROJ_TC", proj_tc)
    monkeypatch.setenv("EXPM_TC_SPIN_LIMIT", "-1")      # no polls: every wait runs out
    plan = Plan(sides, 0.1, (1.0, 1.0), p_max=p, m=6, tol=1e-10, precision="mixed")
    with pytest.raises(N.ExpmError) as e:
        plan.expm_block(t, B)
    assert e.value.code == N.EXPM_TIMEOUT
    torch.cuda.synchronize()
    plan.close()
    # the device context is intact: a fresh plan with the normal bound solves
    monkeypatch.delenv("EXPM_TC_SPIN_LIMIT")
    Z, info = Plan(sides, 0.1, (1.0, 1.0), p_max=p, m=6, tol=1e-10, precision="mixed").expm_block(t, B)
    assert info.converged == 1 and np.all(np.isfinite(to_np(Z)))
