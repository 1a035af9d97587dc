"""bench.py --counters: the algorithmic bytes of each kernel for a workload, computed on the host from
the per-unit counts (no GPU)."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_counters_follow_the_per_unit_formulas():
    out = bench.counters(argparse.Namespace(workload="elastic_vibration", batch=1))
    N, T, F = out["particles"], out["tets"], out["facets"]
    assert F == 12 * T and N > 0
    mixed, fp64 = out["mixed"], out["fp64"]
    # per facet 12R (geometry 4R, history 8R), per tetrahedron 16 B + 24R, per particle 84 / 120 B
    assert mixed["facet_pass_bytes"] == F * 48 + T * (16 + 96) + N * 84
    assert fp64["facet_pass_bytes"] == F * 96 + T * (16 + 192) + N * 120
    assert mixed["particle_pass_bytes"] == T * 4 * (4 + 24) + N * (4 + 192 + 128 + 64 + 84)
    for d in (mixed, fp64):
        assert d["step_bytes"] == d["facet_pass_bytes"] + d["particle_pass_bytes"]
        assert d["adjoint_step_bytes"] == 2 * d["step_bytes"] + d["reverse_facet_pass_bytes"] + \
            d["reverse_particle_pass_bytes"]


def test_recorded_traffic_is_tied_to_the_kernel_source(monkeypatch):
    """`traffic` in the bench line comes from profiles/traffic.json only while the kernel sources hash
    to the value the capture was taken with; any other source reads as null."""
    import json

    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    key = "facet_warp_kernel/uniaxial_tension/mixed"
    assert key in d and d[key]["bytes_per_launch"] > 0
    monkeypatch.setattr(bench, "kernel_src_hash", lambda: d[key]["kernel_src_hash"])
    assert bench.recorded_traffic("facet_warp_kernel", "uniaxial_tension", "mixed") == d[key]["bytes_per_launch"]
    assert bench.recorded_traffic("no_such_kernel", "uniaxial_tension", "mixed") is None
    monkeypatch.setattr(bench, "kernel_src_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("facet_warp_kernel", "uniaxial_tension", "mixed") is None
    assert bench.fp64_alu_roofline("uniaxial_tension", 1.5) is None


def test_fp64_alu_roofline_arithmetic(monkeypatch):
    """achieved = FP64 flops per launch / launch time, against 152 SMs x 2 DFMA x 2 flop x 2.07 GHz."""
    monkeypatch.setattr(bench, "recorded_traffic", lambda *a, **k: 9.0e8)
    r = bench.fp64_alu_roofline("uniaxial_tension", 1.5)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 9.0e8 / 1.5e-3 / 1e12) < 1e-12
    assert abs(r["peak"] - 1.25856) < 1e-9 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15


def test_cpu_all_cores_sums_concurrent_oracle_processes():
    """The all-cores oracle figure: independent oracle processes over one time window, rates summed."""
    from paper_2603_13190_gb300 import workloads

    wl = workloads.WORKLOADS["elastic_vibration"]
    spec = wl.specimen()
    r = bench.cpu_all_cores(spec, wl, workloads.workload_bc(wl.name, spec), 1e-7, budget_s=0.5, max_procs=2)
    assert r["value"] > 0 and r["kind"] == "oracle" and 1 <= r["cores"] <= 2, r
    assert "concurrent single-thread oracle processes" in r["sample"]
