"""Host-side logic of bench.py, checked without a GPU.

- The algorithmic work model that the roofline divides by: the fused mixed path moves
  exactly one pass over the basis from the CGS class to the QR class.
- The staleness guard on the recorded ncu traffic: a record counts only while every source
  file it was taken from is unchanged.
- The host restatement of the AUTO algorithm rule, and the Toeplitz FFT length.
"""
import hashlib
import json
import os
import shutil

import pytest

import bench
from paper_1405_0707_gb300 import inputs

CD2D_CYCLES = {1e-3: 4, 1e-2: 17, 1e-1: 7}
CD2D_ALGS = {1e-3: 1, 1e-2: 1, 1e-1: 2}


def test_fused_accounting_moves_one_basis_pass():
    w = inputs.WORKLOADS["cd2d-256"]
    n, p, m = 65536, w["p"], w["m"]
    a = bench.algorithmic_work(w, p, m, CD2D_CYCLES, CD2D_ALGS)
    b = bench.algorithmic_work(w, p, m, CD2D_CYCLES, CD2D_ALGS, fused=True)
    for k in a:
        if k not in ("cgs", "qr"):
            assert a[k] == b[k]
    for i in (0, 1):                       # flops and bytes are conserved
        assert a["cgs"][i] + a["qr"][i] == pytest.approx(b["cgs"][i] + b["qr"][i], rel=1e-14)
    cycles = sum(CD2D_CYCLES.values())
    sum_cols = p * m * (m + 1) / 2          # sum over the block steps of (j + 1) p columns
    moved_bytes = cycles * 8.0 * (n * sum_cols + 2 * n * p)
    moved_flops = cycles * 2.0 * n * p * sum_cols
    assert b["qr"][1] - a["qr"][1] == pytest.approx(moved_bytes, rel=1e-14)
    assert b["qr"][0] - a["qr"][0] == pytest.approx(moved_flops, rel=1e-14)
    assert b["cgs"][0] > 0 and b["cgs"][1] > 0


def test_traffic_record_follows_its_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    key = next(iter(rec))
    sources = list(rec[key]["sources"])
    for rel in sources:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    fresh = {key: dict(rec[key])}
    fresh[key]["sources"] = {rel: hashlib.sha256((tmp_path / rel).read_bytes()).hexdigest() for rel in sources}
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(fresh))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record(key) == rec[key]["bytes_per_launch_full"]
    with open(tmp_path / sources[0], "a") as f:
        f.write("\n")
    assert bench.traffic_record(key) is None
    assert bench.traffic_record("no-such-class") is None


def test_auto_rule_on_the_workloads():
    # ||tA|| bound / max|tau| is 2.8, 28 and 280 on the 256^2 grid: only t = 0.1 passes 50
    assert [bench.auto_algorithm("cd2d-256", t) for t in sorted(CD2D_ALGS)] == [CD2D_ALGS[t] for t in sorted(CD2D_ALGS)]
    assert bench.auto_algorithm("toeplitz-1m", 1.0) == 1     # ||tT|| <= 2.36


def test_toeplitz_fft_length():
    assert bench.fft_size(inputs.WORKLOADS["toeplitz-1m"]) == 2 ** 21


def test_alu_fractions_follow_the_pipe_of_each_class():
    """A class's ALU fraction is taken against the peak of the pipe its kernels run on: FP64
    plans against the FP64 FMA peak; in mixed plans the FP32 transforms and line solves
    against the FP32 peak, and the double-float classes against none (HBM only)."""
    import bench
    g = bench.alu_fracs("gemm", "mixed", 4.025)
    assert g["pipe"] == "fp32" and abs(g["frac_fp32_alu"] - 4.025e3 / bench.FP32_PEAK_TFLOPS) < 1e-15
    for cls in ("cgs", "qr", "update", "fft", "gsf", "stencil"):
        f = bench.alu_fracs(cls, "mixed", 4.0)
        assert "frac_fp64_alu" not in f and "frac_fp32_alu" not in f, cls
    d = bench.alu_fracs("gemm", "fp64", bench.FP64_PEAK_TFLOPS / 2e3)     # half the FP64 peak
    assert d["pipe"] == "fp64" and abs(d["frac_fp64_alu"] - 0.5) < 1e-12
