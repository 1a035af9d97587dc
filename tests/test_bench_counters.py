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
    # per tetrahedron 4 shares of 24R, per particle a 160 B slot table, row pointer 4 B, state and records
    assert mixed["particle_pass_bytes"] == T * 4 * 24 + N * (160 + 4 + 192 + 128 + 64 + 84)
    assert fp64["particle_pass_bytes"] == T * 4 * 48 + N * (160 + 4 + 192 + 128 + 64)
    for d in (mixed, fp64):
        assert d["step_bytes"] == d["facet_pass_bytes"] + d["particle_pass_bytes"]
        assert d["adjoint_step_bytes"] == 2 * d["step_bytes"] + d["reverse_facet_pass_bytes"] + \
            d["reverse_particle_pass_bytes"]


def test_recorded_traffic_is_tied_to_the_kernel_source(monkeypatch):
    """`traffic` in the bench line comes from profiles/traffic.json only while the sources of the
    recorded kernel hash to the value the capture was taken with; any other source reads as null."""
    import json

    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    key = "facet_warp_kernel/uniaxial_tension/mixed"
    assert key in d and d[key]["bytes_per_launch"] > 0
    monkeypatch.setattr(bench, "kernel_src_hash", lambda kernel="": d[key]["kernel_src_hash"])
    assert bench.recorded_traffic("facet_warp_kernel", "uniaxial_tension", "mixed") == d[key]["bytes_per_launch"]
    assert bench.recorded_traffic("no_such_kernel", "uniaxial_tension", "mixed") is None
    monkeypatch.setattr(bench, "kernel_src_hash", lambda kernel="": "0" * 16)
    assert bench.recorded_traffic("facet_warp_kernel", "uniaxial_tension", "mixed") is None
    assert bench.fp64_alu_roofline("uniaxial_tension", 1.5) is None


def test_fp64_alu_roofline_arithmetic(monkeypatch):
    """achieved = FP64 flops per launch / launch time, against 152 SMs x 2 DFMA x 2 flop x 2.07 GHz."""
    monkeypatch.setattr(bench, "recorded_traffic", lambda *a, **k: 9.0e8)
    r = bench.fp64_alu_roofline("uniaxial_tension", 1.5)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 9.0e8 / 1.5e-3 / 1e12) < 1e-12
    assert abs(r["peak"] - 1.25856) < 1e-9 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15


def test_oracle_window_and_all_cores():
    """The CPU baseline: one oracle process runs the pre-roll and warm-up of the loading history and
    times the window after it; the all-cores figure starts independent oracle processes from the state
    that process reached, over one time window, and sums their rates."""
    from paper_2603_13190_gb300 import workloads

    wl = workloads.WORKLOADS["elastic_vibration"]
    spec = wl.specimen()
    w = bench.OracleWindow(spec, wl, workloads.workload_bc(wl.name, spec), preroll=3, budget_s=0.3)
    try:
        r = w.result(timeout_s=300)
        assert r["value"] > 0 and r["kind"] == "oracle" and r["cores"] == 1, r
        assert "3-step pre-roll" in r["sample"] and ("dt %.4g s" % wl.dt) in r["sample"]
        a = w.all_cores(budget_s=0.5, max_procs=2)
        assert a["value"] > 0 and a["kind"] == "oracle" and 1 <= a["cores"] <= 2, a
        assert "from the pre-rolled state" in a["sample"]
    finally:
        w.close()


def test_reference_arm_uses_the_workload_time_step_and_window():
    """Both arms step with the workload's fixed dt after the same pre-roll and warm-up."""
    from paper_2603_13190_gb300 import workloads

    wl = workloads.WORKLOADS["elastic_vibration"]
    args = type("A", (), {"workload": "elastic_vibration", "warmup": 3, "steps": 2, "preroll": None})()
    r = bench.run_reference(args, 0, 1)
    assert r["impl"] == "reference" and r["config"]["dt_s"] == wl.dt and r["value"] > 0
    assert "steps %d..%d" % (wl.preroll + 3, wl.preroll + 5) in r["config"]["timed_window"]
    for name, w in workloads.WORKLOADS.items():
        assert w.dt > 0, name


def test_fp64_alu_roofline_needs_a_count_of_the_same_workload(monkeypatch):
    """The FP64 flops of the facet pass depend on the loading state (the law's branch mix), so a
    workload without its own capture has no ALU roofline; with one, the peak takes the device's SM
    count and the sampled clock."""
    counts = {"uniaxial_tension": 1820724 * 500.0}
    monkeypatch.setattr(bench, "recorded_traffic", lambda k, w, p, f="bytes_per_launch": counts.get(w))
    assert bench.fp64_alu_roofline("confined_compression", 5.0, facets=12535080, sm_count=148, sm_mhz=2000.0) is None
    counts["confined_compression"] = 12535080 * 300.0
    r = bench.fp64_alu_roofline("confined_compression", 5.0, facets=12535080, sm_count=148, sm_mhz=2000.0)
    assert abs(r["flop_per_launch"] - 12535080 * 300.0) < 1e-3 and r["flops"] == "counted on this workload"
    assert abs(r["peak"] - 148 * 2 * 2 * 2.0e9 / 1e12) < 1e-12 and "148 SMs" in r["peak_source"]


def test_every_recorded_count_belongs_to_the_current_sources():
    """The committed DRAM traffic and FP64 flop counts were taken on the kernels as they are: each
    entry's hash is that of its kernel's current sources and build flags."""
    import json

    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert d
    for key, e in d.items():
        assert e["kernel_src_hash"] == bench.kernel_src_hash(key.split("/")[0]), key
