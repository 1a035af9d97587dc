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
