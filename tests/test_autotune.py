"""The launch-shape autotuner (paper_1405_0707_gb300/autotune.py): its class keys and table
lookup on the host, and on the GPU one tuned class whose choice is a candidate and whose
tuned plan still solves to the closed form."""
import json

import numpy as np
import pytest

from paper_1405_0707_gb300 import autotune, inputs


def test_class_keys_and_lookup(tmp_path):
    k = autotune.class_key(3, 300000, 12, "mixed", 2)
    assert k == "3d/n2^18/p12/mixed/alg2"
    assert autotune.class_key(3, 2 ** 18 * 1.4, 12, "mixed", 2) == k          # within the bucket
    table = {k: {"best": [3, 6], "ms": {}}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(table))
    tab = autotune.load(str(path))
    assert autotune.options_for(tab, 3, 300000, 12, "mixed", 2) == {"row_ctas": 3, "cgs_ctas": 6}
    assert autotune.options_for(tab, 3, 300000, 13, "mixed", 2) == {"row_ctas": 0, "cgs_ctas": 0}
    assert autotune.load(str(tmp_path / "missing.json")) == {}
    assert all(1 <= r <= c <= 8 for r, c in autotune.CANDIDATES)


def test_committed_table_is_well_formed():
    """The table the bench reads (written on a GB300 by the tuner) names valid candidates."""
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1405_0707_gb300",
                        "tuning", "batched3d-64.json")
    if not os.path.exists(path):
        pytest.skip("no committed table")
    tab = autotune.load(path)
    assert tab
    for key, v in tab.items():
        assert tuple(v["best"]) in autotune.CANDIDATES + (autotune.DEFAULT,), key
        assert min(v["ms"].values()) == v["ms"]["%d,%d" % tuple(v["best"])]


@pytest.mark.gpu
def test_tuned_class_solves_to_closed_form():
    from tests.gpu_util import need_gpu, rel, to_dev, to_np
    need_gpu()
    from oracle import cf, operators as ops
    from paper_1405_0707_gb300 import Plan
    sides, diff, vel, t, p = (40, 37, 35), 1.0, (2.0, -1.0, 1.5), 0.02, 6
    res = autotune.tune_class(sides, diff, vel, t, p, 8, "mixed", 1, seed=3, reps=1)
    assert tuple(res["best"]) in autotune.CANDIDATES + (autotune.DEFAULT,)
    assert len(res["ms"]) == len(autotune.CANDIDATES) + 1 and all(v > 0 for v in res["ms"].values())
    r, c = res["best"]
    B = inputs.rhs(int(np.prod(sides)), p, 4)
    Z, info = Plan(sides, diff, vel, p_max=p, m=8, tol=1e-11, max_cycles=400, precision="mixed", row_ctas=r,
                   cgs_ctas=c).expm_block(t, to_dev(B))
    assert info.converged == 1
    assert rel(to_np(Z), ops.exact_r_of_A_B(sides, diff, vel, t, cf.load_table(), B)) <= 1e-9
