"""Host-side arithmetic of bench.py's roofline record, on CPU: the compulsory bytes per
launch, the gate that drops the ncu traffic once the kernels change, and the achieved
rate, fraction and traffic scaling of the dominant kernel."""
import hashlib
import os

import numpy as np
import pytest

import bench
from paper_2410_13055_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _net(n_bus, gen_bus, n_line, bat_bus):
    return {"n_bus": n_bus, "gen_bus": np.asarray(gen_bus), "line_from": np.zeros(n_line, dtype=int),
            "bat_bus": np.asarray(bat_bus, dtype=int)}


def test_algorithmic_bytes_counts():
    # 4 buses, 3 generators (the second one variable), 5 lines, 3 batteries on 2 buses, 24 h
    T = 24
    cf = np.ones((3, T))
    cf[1, 5] = 0.5
    net = _net(4, [0, 1, 2], 5, [1, 1, 3])
    b = bench.algorithmic_bytes([net], [{"net": 0, "T": T, "cf": cf}])[0]
    # generators: x read+write 8 B each, capacity factor 4 B on the variable row only
    gen = 8 * 3 + 4 * 1
    # buses: load x r/w 8 + L 4, then u, pbar, z read+write 24; lines: delta 4 + both ends' q 8
    bus = 12 * 4 + 24 * 4
    assert b["k_bus"] == T * (gen + bus + 12 * 5 + 4 * 3)
    # line kernel: four line rows read+written (32 B), three bus rows read per bus-hour (12 B)
    assert b["k_line"] == T * (32 * 5 + 12 * 4)
    # battery kernel: 60 B per battery-hour, 8 B per distinct battery bus (2 of them)
    assert b["k_bat"] == T * (60 * 3 + 8 * 2)


def test_algorithmic_bytes_firm_rows_and_scaling():
    T = 48
    net = _net(3, [0, 2], 2, [])
    firm = bench.algorithmic_bytes([net], [{"net": 0, "T": T, "cf": np.ones((2, T))}])[0]
    var = bench.algorithmic_bytes([net], [{"net": 0, "T": T, "cf": np.full((2, T), 0.3)}])[0]
    assert var["k_bus"] - firm["k_bus"] == 4 * 2 * T
    assert var["k_line"] == firm["k_line"] and var["k_bat"] == firm["k_bat"] == 0
    # bytes scale with the horizon: the same network over twice the hours
    long = bench.algorithmic_bytes([net], [{"net": 0, "T": 2 * T, "cf": np.ones((2, 2 * T))}])[0]
    assert long == {k: 2 * v for k, v in firm.items()}


def test_algorithmic_bytes_medium_figures():
    # the per-launch figures quoted for the 100-bus, 16 x 168 h workload
    nets, scens = synth.medium(seed=1, S=16)
    per = bench.algorithmic_bytes(nets, scens)
    assert len(per) == 16
    tot = {k: sum(p[k] for p in per) for k in per[0]}
    assert tot["k_bus"] == pytest.approx(23.65e6, rel=1e-3)
    assert tot["k_line"] == pytest.approx(16.13e6, rel=1e-3)
    assert tot["k_bat"] == pytest.approx(8.95e6, rel=1e-3)


def _sha():
    src = os.path.join(ROOT, "paper_2410_13055_gb300", "csrc", "gx_kernels.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def test_profiled_traffic_gate(monkeypatch):
    cap = {"scenarios": 4, "source": "x", "traffic": {"k_bus": 100.0, "k_line": 40.0}}
    monkeypatch.setattr(bench, "PROFILED", {"sha256_prefix": _sha(), "medium": cap})
    # scaled in proportion to the scenarios
    assert bench.profiled_traffic("medium", 8, "k_bus") == pytest.approx(200.0)
    assert bench.profiled_traffic("medium", 2, "k_line") == pytest.approx(20.0)
    # a kernel or workload without a capture
    assert bench.profiled_traffic("medium", 8, "k_bat") is None
    assert bench.profiled_traffic("batching", 8, "k_bus") is None
    # the kernels changed since the capture
    monkeypatch.setattr(bench, "PROFILED", {"sha256_prefix": "0" * 16, "medium": cap})
    assert bench.profiled_traffic("medium", 8, "k_bus") is None


def test_profiled_captures_are_well_formed():
    assert len(bench.PROFILED["sha256_prefix"]) == 16
    for cfg in ("medium", "scale", "batching"):
        cap = bench.PROFILED[cfg]
        assert cap["scenarios"] > 0 and cap["source"].startswith("profiles/")
        assert os.path.exists(os.path.join(ROOT, cap["source"].split(" ")[0]))
        assert set(cap["traffic"]) <= {"k_bus", "k_line", "k_bat"}


def _roofline_inputs():
    # three scenarios; scenario 1 converged early, so it is inactive in every sampled launch
    per_scen = [{"k_bus": 1000.0, "k_line": 600.0, "k_bat": 200.0},
                {"k_bus": 3000.0, "k_line": 900.0, "k_bat": 300.0},
                {"k_bus": 2000.0, "k_line": 500.0, "k_bat": 100.0}]
    # active[s] = number of sampled launches in which scenario s still iterated
    active = [4, 0, 2]
    prof = {"k_bus": {"ms": 0.004, "samples": 4, "launches": 1000},
            "k_line": {"ms": 0.003, "samples": 4, "launches": 1000},
            "k_bat": {"ms": 0.005, "samples": 4, "launches": 500},
            "k_reduce": {"ms": 1.0, "samples": 4, "launches": 10}}
    return prof, active, per_scen


def test_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "_peaks", lambda: (1000.0, "measured"))
    monkeypatch.setattr(bench, "profiled_traffic", lambda config, n, k: None)
    prof, active, per_scen = _roofline_inputs()
    r = bench.roofline("medium", prof, active, per_scen, 3, iters_per_step=400, ms_per_step=1.0)
    k = r["kernels"]
    assert set(k) == {"k_bus", "k_line", "k_bat"}
    # bus: (4 * 1000 + 2 * 2000) / 4 samples = 2000 B per launch in 1 us
    assert k["k_bus"]["bytes_per_launch"] == pytest.approx(2000.0)
    assert k["k_bus"]["avg_launch_us"] == pytest.approx(1.0)
    assert k["k_bus"]["achieved_gbs"] == pytest.approx(2.0)
    assert k["k_line"]["bytes_per_launch"] == pytest.approx((4 * 600 + 2 * 500) / 4)
    # dominant kernel = largest total time (launches x average launch): bus 1.0 ms,
    # line 0.75 ms, battery 0.625 ms
    assert r["kernel"] == "k_bus"
    assert r["achieved"] == pytest.approx(2.0) and r["peak"] == 1000.0
    assert r["frac"] == pytest.approx(2.0 / 1000.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    # one iteration = bus + the longer of line and battery (they run side by side)
    assert r["check"]["sampled_iteration_us"] == pytest.approx(1.0 + 1.25)
    assert r["check"]["sampled_ms_per_step"] == pytest.approx(2.25 * 400 / 1e3)


def test_roofline_traffic_scaled_to_active_share(monkeypatch):
    monkeypatch.setattr(bench, "_peaks", lambda: (1000.0, "measured"))
    # capture of an all-scenario launch: 4500 B against 6000 algorithmic
    monkeypatch.setattr(bench, "profiled_traffic", lambda config, n, k: 4500.0 if k == "k_bus" else None)
    prof, active, per_scen = _roofline_inputs()
    r = bench.roofline("medium", prof, active, per_scen, 3, iters_per_step=1, ms_per_step=1.0)
    # the sampled launches average 2000 of 6000 all-scenario bytes: a third of the traffic
    assert r["traffic"] == pytest.approx(1500.0)


def test_roofline_without_samples(monkeypatch):
    monkeypatch.setattr(bench, "_peaks", lambda: (1000.0, "fallback"))
    prof = {"k_bus": {"ms": 0.0, "samples": 0, "launches": 0}}
    assert bench.roofline("medium", prof, [0], [{"k_bus": 1.0}], 1, 1, 1.0) is None
