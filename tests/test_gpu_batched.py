"""expm_block_batched: independent instances of different operator family, order, width and
time in one library call, each on its own stream.  Every instance's result equals the
single-call result bit for bit (same plan, same kernels, fixed-order reductions), and each
matches its closed form or Taylor truth."""
import numpy as np
import pytest

from oracle import cf, operators as ops, toeplitz as TZ
from paper_1405_0707_gb300 import inputs
from tests.gpu_util import need_gpu, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tab():
    return cf.load_table()


def test_batched_mixed_instances(tab):
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300.api import expm_block_batched
    rng = np.random.default_rng(61)
    specs = [("cd", (41, 35), 0.1, (1.0, 1.0), 0.1, 3, "fp64"),
             ("cd", (16, 13, 11), 1.0, (2.0, -3.0, 1.5), 0.02, 5, "mixed"),
             ("cd", (300,), 1.0, (0.0,), 1.0, 1, "fp64"),
             ("toe", 2500, None, None, 1.0, 4, "fp64"),
             ("cd", (30, 29, 28), 1.0, (-4.0, 1.0, 2.0), 0.05, 8, "mixed")]
    plans, Bs, ts, refs = [], [], [], []
    for kind, shape, diff, vel, t, p, prec in specs:
        stream = torch.cuda.Stream()
        if kind == "cd":
            pl = Plan(shape, diff, vel, p_max=p, m=8, tol=1e-12, max_cycles=300, stream=stream, precision=prec)
            n = int(np.prod(shape))
        else:
            a = inputs.toeplitz_column(256)
            pl = Plan.toeplitz(a, shape, p_max=p, m=8, tol=1e-13, stream=stream, precision=prec)
            n = shape
        B = inputs.rhs(n, p, int(rng.integers(1 << 30)))
        plans.append(pl)
        Bs.append(B)
        ts.append(t)
    Bd = [to_dev(B) for B in Bs]
    torch.cuda.synchronize()
    Zs, infos = expm_block_batched(plans, ts, Bd)
    for (kind, shape, diff, vel, t, p, prec), pl, B, Bdev, Z, info in zip(specs, plans, Bs, Bd, Zs, infos):
        assert info.converged == 1
        Z1, info1 = pl.expm_block(t, Bdev)
        assert np.array_equal(to_np(Z), to_np(Z1)) and info1.cycles == info.cycles
        if kind == "cd":
            ref = ops.exact_r_of_A_B(shape, diff, vel, t, tab, B)
            assert rel(to_np(Z), ref) <= 1e-9
        else:
            col = np.zeros(shape)
            col[:257] = inputs.toeplitz_column(256)
            assert rel(to_np(Z), TZ.taylor_expm_B(col, B, t)) <= 1e-11


def test_batched_rejects_repeated_plan():
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300._native import ExpmError
    from paper_1405_0707_gb300.api import expm_block_batched
    pl = Plan((50,), 1.0, (0.0,), p_max=1)
    B = to_dev(inputs.rhs(50, 1, 1))
    with pytest.raises(ExpmError):
        expm_block_batched([pl, pl], [0.1, 0.2], [B, B])



def test_batch_graph_matches_batched_call(tab):
    """The batched solve as one CUDA graph (a device-side WHILE loop of restart cycles per
    instance, the stop test in a kernel): the same Z, bit for bit, and the same cycle counts as
    the host-driven expm_block_batched, on a mix of families, orders, widths and precisions;
    replaying the graph gives the same result again; each Z matches its closed form."""
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300.api import Batch, expm_block_batched
    rng = np.random.default_rng(62)
    specs = [("cd", (41, 35), 0.1, (1.0, 1.0), 0.1, 3, "fp64"),
             ("cd", (16, 13, 11), 1.0, (2.0, -3.0, 1.5), 0.02, 5, "mixed"),
             ("cd", (300,), 1.0, (0.0,), 1.0, 1, "fp64"),
             ("toe", 2500, None, None, 1.0, 4, "mixed"),
             ("cd", (60, 58, 57), 1.0, (-4.0, 1.0, 2.0), 0.05, 12, "mixed")]
    plans, Bs, ts = [], [], []
    for kind, shape, diff, vel, t, p, prec in specs:
        stream = torch.cuda.Stream()
        if kind == "cd":
            pl = Plan(shape, diff, vel, p_max=p, m=8, tol=1e-12, max_cycles=300, stream=stream, precision=prec)
            n = int(np.prod(shape))
        else:
            pl = Plan.toeplitz(inputs.toeplitz_column(256), shape, p_max=p, m=8, tol=1e-13, stream=stream, precision=prec)
            n = shape
        plans.append(pl)
        Bs.append(inputs.rhs(n, p, int(rng.integers(1 << 30))))
        ts.append(t)
    Bd = [to_dev(B) for B in Bs]
    torch.cuda.synchronize()
    Zr, ir = expm_block_batched(plans, ts, Bd)
    Zr = [to_np(Z) for Z in Zr]
    batch = Batch(plans, ts, Bd)
    for rep in range(2):
        Zg, ig = batch.run()
        for (kind, shape, diff, vel, t, p, prec), B, Z, Z0, i_g, i_r in zip(specs, Bs, Zg, Zr, ig, ir):
            assert i_g.converged == 1 and i_g.cycles == i_r.cycles, (rep, shape, i_g.cycles, i_r.cycles)
            assert np.array_equal(to_np(Z), Z0), (rep, shape)
            if kind == "cd":
                assert rel(Z0, ops.exact_r_of_A_B(shape, diff, vel, t, tab, B)) <= 1e-9
    batch.close()


def test_batch_graph_rejects_host_work_between_cycles():
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    from paper_1405_0707_gb300._native import ExpmError
    from paper_1405_0707_gb300.api import Batch
    B = to_dev(inputs.rhs(400, 2, 3))
    for kw in (dict(k_defl=2), dict(certify=True)):
        pl = Plan((20, 20), 0.1, (1.0, 1.0), p_max=2, m=4, stream=torch.cuda.Stream(), **kw)
        with pytest.raises(ExpmError):
            Batch([pl], [0.1], [B])


@pytest.mark.parametrize("alg", [1, 2])
def test_row_grid_share_changes_only_the_summation_order(tab, alg):
    """grid_sms sizes the grids of the row passes after the first Gram-Schmidt pass for a
    share of the SMs (fewer CTAs, more rows each).  The solve is the same up to the order of
    the per-CTA partial sums: Z agrees with the whole-device plan to rounding, takes the same
    number of cycles, and meets the closed form."""
    torch = need_gpu()
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t, p = (37, 31, 29), 1.0, (1.0, -2.0, 0.5), (0.004 if alg == 1 else 0.05), 6
    B = inputs.rhs(int(np.prod(sides)), p, 77)
    out = {}
    for share in (0, 3, 40):
        pl = Plan(sides, diff, vel, p_max=p, m=10, tol=1e-11, max_cycles=300, algorithm=alg, precision="mixed",
                  grid_sms=share, row_ctas=2)
        Z, info = pl.expm_block(t, to_dev(B))
        assert info.converged == 1 and info.algorithm == alg
        out[share] = (to_np(Z), int(info.cycles))
        pl.close()
    ref = ops.exact_r_of_A_B(sides, diff, vel, t, tab, B)
    for share in (3, 40):
        assert out[share][1] == out[0][1]
        assert rel(out[share][0], out[0][0]) <= 1e-12
        assert rel(out[share][0], ref) <= 1e-9
