"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on identical seeded inputs.

Tolerances (derivation in the design notes):
  FP64 mode   per-step forces, states and tractions: per-element relative error <= 1e-10 (a floor of
              1e-4 of the tolerance times the largest element covers exact zeros; tests/parity.py);
              trajectories of tens to hundreds of steps: per element <= 1e-9.
  mixed mode  per-step node forces: normwise relative error <= 2e-5 (FP32 strains from FP64
              differences: unit roundoff 6e-8 amplified by |jump terms| / |jump| <= ~100);
              per-facet forces: all but < 0.5 % of facets within 1e-4 relative to the largest facet
              force (facets sitting on a clamp or branch threshold may resolve differently in FP32).
"""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL
from parity import assert_elementwise, normwise_rel as nrel

pytestmark = pytest.mark.gpu
MAT = dict(WORKLOAD_MATERIAL)


def loaded_state(spec, steps=400, seed=0):
    """A state with cracked, compressed and sliding facets: oracle run of fast tension plus shear."""
    bc = workloads.uniaxial_tension_bc(spec, velocity=80.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 0] = workloads.PRESCRIBED
    bc.vel[top, 0] = 40.0
    o = oracle.Oracle(spec, MAT, 1e-7, bc)
    dt = 0.9 * o.critical_dt()
    o = oracle.Oracle(spec, MAT, dt, bc)
    o.step(steps)
    return bc, dt, o


@pytest.fixture(scope="module")
def small():
    spec = specimen.shuffled(specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=5), seed=3)
    bc, dt, o = loaded_state(spec)
    return spec, bc, dt, o


def gpu_model(spec, bc, dt, prec, **kw):
    return ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc, **kw)


def compare_one_step(spec, bc, dt, o, prec):
    q, v, h5, st = o.get_state()
    m = gpu_model(spec, bc, dt, prec)
    m.set_state(q, v, h5, st)
    # forces rebuilt from the same tractions agree before stepping
    F0g, f0g = m.facet_forces()
    F0o, f0o = o.facet_forces()
    o2 = oracle.Oracle(spec, MAT, dt, bc)
    o2.set_state(q, v, h5, st)
    o2.step(1)
    m.step(1)
    qg, vg, hg, sg = m.get_state()
    qo, vo, ho, so = o2.get_state()
    Fg, fg = m.facet_forces()
    Fo, fo = o2.facet_forces()
    return dict(F0=(F0g, F0o), f0=(f0g, f0o), q=(qg, qo), v=(vg, vo), h=(hg, ho), F=(Fg, Fo), f=(fg, fo),
                step=(sg, so))


def test_one_step_parity_fp64(small):
    spec, bc, dt, o = small
    r = compare_one_step(spec, bc, dt, o, "fp64")
    assert r["step"][0] == r["step"][1]
    for k in ("F0", "f0", "q", "v", "h", "F", "f"):
        assert_elementwise(*r[k], 1e-10, k)


def test_one_step_parity_mixed(small):
    spec, bc, dt, o = small
    r = compare_one_step(spec, bc, dt, o, "mixed")
    assert nrel(*r["f0"]) <= 2e-5 and nrel(*r["f"]) <= 2e-5, (nrel(*r["f0"]), nrel(*r["f"]))
    # q_{n+1} = q_n + dt v_{n+1/2} carries the force error through dt^2 / 2 a_n: tiny but not roundoff
    assert nrel(*r["q"]) <= 1e-8 and nrel(*r["v"]) <= 2e-5
    Fg, Fo = r["F"]
    err = np.abs(Fg - Fo).max(axis=1) / np.abs(Fo).max()
    assert np.mean(err > 1e-4) < 5e-3, np.mean(err > 1e-4)


def test_trajectory_parity_fp64(small):
    """200 steps from the initial state with the same loading: FP64 states stay within 1e-9."""
    spec, bc, dt, _ = small
    o = oracle.Oracle(spec, MAT, dt, bc)
    m = gpu_model(spec, bc, dt, "fp64")
    for chunk in (1, 9, 40, 150):
        o.step(chunk)
        m.step(chunk)
        qg, vg, hg, _ = m.get_state()
        qo, vo, ho, _ = o.get_state()
        for what, g, o_ in (("q", qg, qo), ("v", vg, vo), ("hist", hg, ho)):
            assert_elementwise(g, o_, 1e-9, "%s after %d steps" % (what, chunk))
    eg, rg = m.energy()
    eo, ro = o.energy()
    assert_elementwise(eg[:3], eo[:3], 1e-9, "energies")
    assert_elementwise(rg, ro, 1e-9, "reactions")


def test_graph_and_direct_launches_agree_bitwise(small):
    spec, bc, dt, _ = small
    a = gpu_model(spec, bc, dt, "mixed", graph_chunk=8)
    b = gpu_model(spec, bc, dt, "mixed", graph_chunk=-1)
    for m in (a, b):
        m.step(37)
        m.step(5)
    sa, sb = a.get_state(), b.get_state()
    for x, y in zip(sa[:3], sb[:3]):
        assert np.array_equal(x, y)


def test_checkpoint_resume_is_bitwise(small):
    spec, bc, dt, _ = small
    m = gpu_model(spec, bc, dt, "mixed")
    m.step(20)
    ck = ldpm.ldpm_save_checkpoint(m.h)
    m.step(25)
    s1 = m.get_state()
    e1 = m.energy()
    ldpm.ldpm_load_checkpoint(m.h, ck)
    m.step(25)
    s2 = m.get_state()
    e2 = m.energy()
    for x, y in zip(s1[:3], s2[:3]):
        assert np.array_equal(x, y)
    assert s1[3] == s2[3]
    assert np.array_equal(e1[0], e2[0])


def test_single_tetrahedron_edge_case():
    spec = specimen.single_tet_specimen()
    bc = workloads.free_bc(4)
    bc.v0[:] = np.random.default_rng(0).standard_normal((4, 6))
    o = oracle.Oracle(spec, MAT, 1e-7, bc)
    dt = 0.5 * o.critical_dt()
    o = oracle.Oracle(spec, MAT, dt, bc)
    m = gpu_model(spec, bc, dt, "fp64")
    o.step(50)
    m.step(50)
    qg, vg, hg, _ = m.get_state()
    qo, vo, ho, _ = o.get_state()
    for what, g, o_ in (("q", qg, qo), ("v", vg, vo), ("hist", hg, ho)):
        assert_elementwise(g, o_, 1e-9, what)


def test_critical_step_estimate_matches_oracle(small):
    spec, bc, _, _ = small
    o = oracle.Oracle(spec, MAT, 1e-7, bc)
    dt_o = 0.9 * o.critical_dt(iters=500)
    for prec in ("fp64", "mixed"):
        m = ldpm.Model(spec, MAT, precision=prec, dt=0.0, bc=bc)
        assert abs(m.dt - dt_o) <= 0.02 * dt_o, (prec, m.dt, dt_o)


def test_elastic_vibration_energy_conservation_gpu():
    """Workload elastic_vibration on the GPU in FP64: energy error below 1 % after 2000 steps at
    0.9 dt_crit, and the energies equal the oracle's."""
    wl = workloads.WORKLOADS["elastic_vibration"]
    spec = wl.specimen()
    bc = workloads.workload_bc(wl.name, spec)
    m = ldpm.Model(spec, wl.material, precision="fp64", dt=0.0, bc=bc)
    o = oracle.Oracle(spec, wl.material, m.dt, bc)
    m.step(wl.steps)
    o.step(wl.steps)
    eg, _ = m.energy()
    eo, _ = o.energy()
    assert eg[3] < 1.0
    assert_elementwise(eg[:3], eo[:3], 1e-9, "energies")


def test_zero_steps_is_a_noop(small):
    spec, bc, dt, _ = small
    m = gpu_model(spec, bc, dt, "fp64")
    s0 = m.get_state()
    m.step(0)
    s1 = m.get_state()
    assert all(np.array_equal(a, b) for a, b in zip(s0[:3], s1[:3]))


def test_mixed_energy_sums_follow_the_fp64_path():
    """Energy sums of the mixed mode (float-float increments, FP64 accumulators) against the FP64
    mode over 1000 loaded steps of a 12 mm cube pulled at 20 mm/s (elastic and pre-peak): W_int and
    W_ext within 1e-6 relative.  The two runs differ only by the FP32 facet pass, whose rounding enters
    the work sums as unbiased per-facet errors; FP32 energy increments would add rounding of each
    particle's increment on top of that."""
    spec = specimen.make_cube_specimen(12.0, 2.0, 4.0, 320, seed=23)
    bc = workloads.uniaxial_tension_bc(spec, velocity=20.0, ramp_time=1e-5)
    dt = 0.9 * oracle.Oracle(spec, MAT, 1e-7, bc).critical_dt()
    runs = {}
    for prec in ("fp64", "mixed"):
        m = gpu_model(spec, bc, dt, prec)
        hist = []
        for _ in range(10):
            m.step(100)
            e, r = m.energy()
            hist.append(e[:3].copy())
        runs[prec] = np.array(hist)
        m.close()
    a, b = runs["mixed"], runs["fp64"]
    rel_int = np.abs(a[:, 1] - b[:, 1]) / np.abs(b[:, 1])
    rel_ext = np.abs(a[:, 0] - b[:, 0]) / np.abs(b[:, 0])
    print("mixed vs FP64 energy sums over 1000 steps: W_int %.2e, W_ext %.2e (largest relative difference)"
          % (rel_int.max(), rel_ext.max()))
    assert b[-1, 0] > 0 and b[-1, 1] > 0
    assert rel_int.max() <= 1e-6 and rel_ext.max() <= 1e-6


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_particles_beyond_the_slot_table(monkeypatch, lanes):
    """The particle pass reads a particle's first 40 (tetrahedron, vertex) slot ids from a per-particle
    table and continues a longer row through the CSR arrays.  On a cube with widely graded sizes
    (particles with up to ~74 slots, five entries past the table per lane of 8) every lane count gives
    the oracle's node forces, velocities and displacements."""
    spec = specimen.shuffled(specimen.make_cube_specimen(12.0, 0.8, 5.0, 800, seed=11), seed=2)
    cnt = np.bincount(np.asarray(spec.tets).ravel(), minlength=spec.n_particles)
    assert cnt.max() > 64 and np.sum(cnt > 40) >= 5
    bc, dt, o = loaded_state(spec, steps=150)
    monkeypatch.setenv("LDPM_GATHER_LANES", str(lanes))
    r = compare_one_step(spec, bc, dt, o, "fp64")
    for k in ("f0", "f", "v", "q"):
        assert_elementwise(*r[k], 1e-10, k)
    rm = compare_one_step(spec, bc, dt, o, "mixed")
    assert nrel(*rm["f0"]) <= 2e-5 and nrel(*rm["f"]) <= 2e-5, (nrel(*rm["f0"]), nrel(*rm["f"]))
