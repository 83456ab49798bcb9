"""Autotuner of the library's launch shapes (host logic; every measured step runs in the
library's kernels).

The row-parallel passes of a restart cycle (the first Gram-Schmidt pass, the Cholesky-QR
passes, the Z update, the reductions) are launched with a number of CTAs per SM that trades
latency hiding against the size of the partial-sum reductions; the best value depends on the
problem's order n and block width p.  For each problem class the tuner times one restart cycle
(opts.fixed_cycles = 1, CUDA events on the plan's stream, the median of a few repetitions) for
every candidate (row_ctas_per_sm, cgs_ctas_per_sm) and keeps the fastest.  The table is a JSON
file keyed by class, written once on the device and read by bench.py and by Plan users through
`options_for`.

A class is (number of grid dimensions, round(log2 n), p, precision, algorithm): instances of one
class share their launch geometry up to a factor below 1.5 in n.

    python -m paper_1405_0707_gb300.autotune --workload batched3d-64 --out tuning.json
"""
from __future__ import annotations

import json
import math
import os
import statistics

CANDIDATES = tuple((r, c) for r in (1, 2, 3, 4) for c in (2, 4, 6, 8) if c >= r)
DEFAULT = (0, 0)          # the library's defaults (2 and 4 CTAs per SM)


def class_key(ndim, n, p, precision, algorithm):
    """The table key of a problem class."""
    return f"{int(ndim)}d/n2^{int(round(math.log2(max(int(n), 1))))}/p{int(p)}/{precision}/alg{int(algorithm)}"


def load(path):
    """The stored table ({} when the file does not exist)."""
    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def options_for(table, ndim, n, p, precision, algorithm):
    """Plan keyword arguments (row_ctas, cgs_ctas) for a class; the library defaults when the
    class was not tuned."""
    r, c = table.get(class_key(ndim, n, p, precision, algorithm), {}).get("best", DEFAULT)
    return {"row_ctas": int(r), "cgs_ctas": int(c)}


def time_cycle(make_plan, t, B, reps=3):
    """Median event time (ms) of one restart cycle of a fresh plan from make_plan()."""
    import torch
    plan = make_plan()
    plan.expm_block(t, B)                      # warm up (and capture the cycle graph)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(plan.stream)
        plan.expm_block(t, B)
        e1.record(plan.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    plan.close()
    return statistics.median(times)


def tune_class(sides, diff, vel, t, p, m, precision, algorithm, seed=0, reps=3):
    """Time every candidate on one representative instance of a class: {"best": (r, c),
    "ms": {candidate: ms}}."""
    import numpy as np

    from . import inputs
    from .api import Plan
    n = int(np.prod(sides))
    B = inputs.to_device_colmajor(inputs.rhs(n, p, seed))
    ms = {}
    for r, c in (DEFAULT,) + CANDIDATES:
        def mk(r=r, c=c):
            return Plan(sides, diff, vel, p_max=p, m=m, fixed_cycles=1, algorithm=algorithm, precision=precision,
                        row_ctas=r, cgs_ctas=c)
        ms[f"{r},{c}"] = time_cycle(mk, t, B, reps)
    best = min(ms, key=ms.get)
    return {"best": [int(x) for x in best.split(",")], "ms": ms}


def tune_batched(instances, m, precision, auto_algorithm, reps=3, table=None):
    """Tune every class of a list of instances (dicts with sides, diff, vel, t, p, seed), the
    first instance met standing for its class."""
    import numpy as np
    table = dict(table or {})
    for d in instances:
        alg = auto_algorithm(d)
        key = class_key(len(d["sides"]), int(np.prod(d["sides"])), d["p"], precision, alg)
        if key in table:
            continue
        table[key] = tune_class(d["sides"], d["diff"], d["vel"], d["t"], d["p"], m, precision, alg, d["seed"], reps)
    return table


def main():
    import argparse
    import sys

    import numpy as np

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1405_0707_gb300 import inputs
    from paper_1405_0707_gb300 import _native as N
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="batched3d-64")
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--out", required=True)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    N.load()
    w = inputs.WORKLOADS[a.workload]
    inst = inputs.batched3d_instances(w["count"], w["seed"])
    taus, _, _, _ = N.expm_cf_coeffs(14)
    tmax = max(abs(z) for z in taus)

    def auto_alg(d):   # the library's AUTO rule: Algorithm 2 iff the Gershgorin bound >= ratio max|tau|
        bound = d["t"] * sum(4.0 * d["diff"] * (s + 1) ** 2 for s in d["sides"])
        return 2 if bound >= N.EXPM_AUTO_RATIO * tmax else 1
    table = tune_batched(inst, w["m"], a.precision, auto_alg, a.reps, load(a.out))
    with open(a.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    wins = sum(1 for v in table.values() if v["best"] != list(DEFAULT))
    print(json.dumps({"classes": len(table), "tuned_differently": wins, "out": a.out}))


if __name__ == "__main__":
    main()
