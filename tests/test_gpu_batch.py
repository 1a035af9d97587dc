"""Batched stepping: several uneven specimens in one launch per pass equal their separate runs."""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL
from parity import assert_elementwise, normwise_rel as nrel

pytestmark = pytest.mark.gpu
MAT = dict(WORKLOAD_MATERIAL)


@pytest.fixture(scope="module")
def trio():
    specs = [specimen.make_cube_specimen(L, 2.0, 4.0, n, seed=s) for L, n, s in ((9.0, 110, 31), (14.0, 420, 32),
                                                                                  (11.0, 230, 33))]
    bcs = [workloads.unconfined_compression_bc(specs[0], velocity=300.0, ramp_time=1e-5),
           workloads.uniaxial_tension_bc(specs[1], velocity=150.0, ramp_time=1e-5),
           workloads.confined_compression_bc(specs[2], velocity=300.0, ramp_time=1e-5)]
    mats = [MAT, dict(MAT, sigma_t=3.5), dict(MAT, E0=40000.0)]
    dts = [0.85 * oracle.Oracle(s, m, 1e-7, b).critical_dt() for s, m, b in zip(specs, mats, bcs)]
    return specs, bcs, mats, dts


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_single_runs_bitwise(trio, prec):
    specs, bcs, mats, dts = trio
    b = ldpm.Batch(specs, mats, prec, dts=dts, bcs=bcs)
    assert len(b) == 3
    b.step(120)
    for i, (s, m_, bc, dt) in enumerate(zip(specs, mats, bcs, dts)):
        single = ldpm.Model(s, m_, precision=prec, dt=dt, bc=bc)
        single.step(120)
        sb, ss = b.get_state(i), single.get_state()
        for x, y in zip(sb[:3], ss[:3]):
            assert np.array_equal(x, y)
        eb, rb = b.energy(i)
        es, rs = single.energy()
        assert np.array_equal(eb, es) and np.array_equal(rb, rs)
        info, dti = b.info(i)
        assert info[0] == s.n_particles and info[2] == s.n_facets and dti == dt
        single.close()


def test_batch_matches_each_oracle_fp64(trio):
    specs, bcs, mats, dts = trio
    b = ldpm.Batch(specs, mats, "fp64", dts=dts, bcs=bcs)
    b.step(80)
    for i, (s, m_, bc, dt) in enumerate(zip(specs, mats, bcs, dts)):
        o = oracle.Oracle(s, m_, dt, bc)
        o.step(80)
        qg, vg, hg, _ = b.get_state(i)
        qo, vo, ho, _ = o.get_state()
        for what, g, o_ in (("q", qg, qo), ("v", vg, vo), ("hist", hg, ho)):
            assert_elementwise(g, o_, 1e-9, "specimen %d %s" % (i, what))
        wg, eVg = b.metrics(i)
        wo, eVo = o.metrics()
        assert_elementwise(eVg, eVo, 1e-9, "specimen %d e_V" % i)


def test_autotuned_batch_stays_within_rounding(trio):
    specs, bcs, mats, dts = trio
    a = ldpm.Batch(specs, mats, "mixed", dts=dts, bcs=bcs, autotune=True)
    d = ldpm.Batch(specs, mats, "mixed", dts=dts, bcs=bcs)
    tets, lanes = a.launch_shape()
    assert tets in (8, 16, 32) and lanes in (8, 16)
    a.step(60)
    d.step(60)
    for i in range(3):
        qa, va, _, _ = a.get_state(i)
        qd, vd, _, _ = d.get_state(i)
        assert nrel(qa, qd) <= 1e-6 and nrel(va, vd) <= 1e-4


def test_batch_rejects_single_specimen_calls(trio):
    specs, bcs, mats, dts = trio
    b = ldpm.Batch(specs[:2], mats[:2], "mixed", dts=dts[:2], bcs=bcs[:2])
    with pytest.raises(ldpm.LdpmError):
        ldpm.ldpm_energy(b.h)
    with pytest.raises(ldpm.LdpmError):
        ldpm.ldpm_set_bc(b.h, bcs[0].mask, bcs[0].vel, 0.0)


def test_full_size_batch_one_step_against_oracle():
    """The benchmark's batch at full size (64 cubes, 97.7M facets) in the launch shape the autotuner
    picks for it, as the benchmark runs it: after a few steps, one more step of three sampled cubes
    against the FP64 oracle started from the batch's own state of those cubes."""
    specs = workloads.batch_specimens(64, seed=1)
    bcs = [workloads.unconfined_compression_bc(sp) for sp in specs]
    mats = [dict(MAT) for _ in specs]
    b = ldpm.Batch(specs, mats, "mixed", bcs=bcs, autotune=True)
    assert len(b) == 64 and sum(sp.n_facets for sp in specs) > 9e7
    b.step(20)
    picks = (0, 31, 63)
    before = {i: b.get_state(i) for i in picks}
    b.step(1)
    for i in picks:
        q, v, h5, st = before[i]
        dt = b.info(i)[1]
        o = oracle.Oracle(specs[i], mats[i], dt, bcs[i])
        o.set_state(q, v, h5, st)
        o.step(1)
        qo, vo, _, _ = o.get_state()
        qg, vg, _, stg = b.get_state(i)
        assert stg == st + 1
        assert nrel(qg, qo) <= 2e-5 and nrel(vg, vo) <= 2e-5, (i, nrel(qg, qo), nrel(vg, vo))
    b.close()


def test_law_constants_in_parameters_and_beyond():
    """Mixed-mode batches of up to 64 specimens take the law constants from the facet pass's kernel
    parameters (each block finds its specimen from its index), larger ones from device memory: both
    give every specimen its separate run bit for bit, at the boundary (64 and 65 specimens)."""
    specs = [specimen.make_cube_specimen(8.0, 2.0, 4.0, 80, seed=100 + i) for i in range(65)]
    bcs = [workloads.unconfined_compression_bc(s, velocity=300.0, ramp_time=1e-5) for s in specs]
    mats = [dict(MAT, sigma_t=3.0 + 0.02 * i) for i in range(65)]
    dts = [1.0e-7 * (1.0 + 0.001 * i) for i in range(65)]
    singles = {}
    for n in (64, 65):
        b = ldpm.Batch(specs[:n], mats[:n], "mixed", dts=dts[:n], bcs=bcs[:n])
        b.step(60)
        for i in (0, 31, n - 1):
            if i not in singles:
                m = ldpm.Model(specs[i], mats[i], precision="mixed", dt=dts[i], bc=bcs[i])
                m.step(60)
                singles[i] = (m.get_state(), m.energy())
                m.close()
            (ss, (es, rs)), sb = singles[i], b.get_state(i)
            for x, y in zip(sb[:3], ss[:3]):
                assert np.array_equal(x, y), (n, i)
            eb, rb = b.energy(i)
            assert np.array_equal(eb, es) and np.array_equal(rb, rs), (n, i)
        b.close()
