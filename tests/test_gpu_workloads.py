"""GPU against the FP64 oracle on workload-scale cases: metrics, boundary-condition switches, the
mixed-mode trajectory tolerances, and one-step parity at the full and maximum specimen sizes.

Mixed-mode trajectory tolerances (the precision contract of the mixed mode):
  pre-peak macroscopic stress within 1e-3 (relative to the oracle's, where above 10 % of the peak),
  energy-balance error (Sec. 4) within 1 %,
  post-peak crack openings (Sec. 4): Pearson correlation >= 0.99 and NRMSE <= 5 % (normalised by the
  oracle's largest opening).
"""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL
from parity import assert_elementwise, normwise_rel as nrel

pytestmark = pytest.mark.gpu
MAT = dict(WORKLOAD_MATERIAL)


def oracle_dt(spec, mat, bc, factor=0.9):
    return factor * oracle.Oracle(spec, mat, 1e-7, bc).critical_dt()


@pytest.fixture(scope="module")
def cracked():
    """12 mm cube pulled and sheared past its peak by the oracle."""
    spec = specimen.shuffled(specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=21), seed=5)
    bc = workloads.uniaxial_tension_bc(spec, velocity=200.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 1] = workloads.PRESCRIBED
    bc.vel[top, 1] = 60.0
    dt = oracle_dt(spec, MAT, bc)
    o = oracle.Oracle(spec, MAT, dt, bc)
    o.step(900)
    return spec, bc, dt, o


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_metrics_parity(cracked, prec, tol):
    spec, bc, dt, o = cracked
    q, v, h5, st = o.get_state()
    m = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc)
    m.set_state(q, v, h5, st)
    wg, eVg = m.metrics()
    wo, eVo = o.metrics()
    assert wo.max() > 0, "the fixture must contain cracked facets"
    assert nrel(wg, wo) <= tol and nrel(eVg, eVo) <= tol, (nrel(wg, wo), nrel(eVg, eVo))


def test_boundary_condition_switch_parity_fp64():
    """Confined compression: hydrostatic phase, then lateral faces held (ldpm_set_bc), both sides."""
    spec = specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=22)
    bc1 = workloads.confined_compression_bc(spec, velocity=400.0, phase=1, ramp_time=1e-5)
    bc2 = workloads.confined_compression_bc(spec, velocity=400.0, phase=2, ramp_time=1e-5)
    dt = oracle_dt(spec, MAT, bc1)
    o = oracle.Oracle(spec, MAT, dt, bc1)
    m = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc1)
    o.step(150)
    m.step(150)
    o.set_bc(bc2)
    m.set_bc(bc2.mask, bc2.vel, bc2.ramp_time)
    o.step(150)
    m.step(150)
    qg, vg, hg, _ = m.get_state()
    qo, vo, ho, _ = o.get_state()
    for what, g, o_ in (("q", qg, qo), ("v", vg, vo), ("hist", hg, ho)):
        assert_elementwise(g, o_, 1e-9, what)
    eg, rg = m.energy()
    eo, ro = o.energy()
    assert_elementwise(eg[:3], eo[:3], 1e-9, "energies")
    assert_elementwise(rg, ro, 1e-9, "reactions")
    assert ho[:, 0].min() < -0.5 * MAT["sigma_c0"], "compression must reach the compressive boundary"


def _mixed_tension_contract(edge, n_particles, seed, steps, every):
    """Mixed-mode GPU trajectory against the FP64 oracle through the peak and into softening."""
    spec = specimen.make_cube_specimen(edge, 2.0, 4.0, n_particles, seed=seed)
    bc = workloads.uniaxial_tension_bc(spec, velocity=50.0, ramp_time=1e-5)
    dt = oracle_dt(spec, MAT, bc)
    o = oracle.Oracle(spec, MAT, dt, bc)
    m = ldpm.Model(spec, MAT, precision="mixed", dt=dt, bc=bc)
    so, sg, eo_err, eg_err = [], [], [], []
    for _ in range(steps // every):
        o.step(every)
        m.step(every)
        eo, ro = o.energy()
        eg, rg = m.energy()
        so.append(ro[8] / spec.edge ** 2)
        sg.append(rg[8] / spec.edge ** 2)
        eo_err.append(eo[3])
        eg_err.append(eg[3])
    so, sg = np.array(so), np.array(sg)
    k = int(np.argmax(so))
    assert 0 < k < len(so) - 5 and so[-1] < 0.8 * so[k], "run must pass the peak and soften"
    pre = slice(0, k + 1)
    big = so[pre] > 0.1 * so[k]
    stress_err = np.max(np.abs(sg[pre][big] - so[pre][big]) / so[pre][big])
    wo, _ = o.metrics()
    wg, _ = m.metrics()
    corr = np.corrcoef(wo, wg)[0, 1]
    nrmse = 100.0 / wo.max() * np.sqrt(np.mean((wo - wg) ** 2))
    print("mixed tension contract, %g mm cube (%d facets): pre-peak stress %.2e, energy error %.3g %% / %.3g %%, "
          "crack opening correlation %.5f, NRMSE %.3f %%" % (edge, spec.n_facets, stress_err, max(eg_err[5:]),
                                                             max(eo_err[5:]), corr, nrmse))
    assert stress_err <= 1e-3
    assert max(eg_err[5:]) <= 1.0 and max(eo_err[5:]) <= 1.0
    assert corr >= 0.99 and nrmse <= 5.0, (corr, nrmse)
    m.close()


def test_mixed_tension_trajectory_meets_tolerances():
    """12 mm cube (~300 particles) pulled through its peak into softening."""
    _mixed_tension_contract(12.0, 320, 23, 1600, 10)


def test_mixed_tension_trajectory_meets_tolerances_25mm():
    """25 mm cube with the particle sizes (d = 2..4 mm) and density of the 1.82M-facet benchmark
    specimen (~3100 particles, ~200k facets), pulled at its 50 mm/s through the peak (about step 800)
    into softening (1200 steps)."""
    _mixed_tension_contract(25.0, int(round(25000 * (25.0 / 50.0) ** 3)), 25, 1200, 25)


@pytest.fixture(scope="module")
def hanging():
    """12 mm cube, bottom face fixed, under constant external nodal forces: a body force m g along +z
    (g = 1e8 mm/s^2, enough to crack the facets near the support) and 0.5 N along x on every top-face
    particle.  The oracle runs 300 steps."""
    spec = specimen.shuffled(specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=24), seed=6)
    bc = workloads.free_bc(spec.n_particles)
    bc.mask[spec.face_nodes(2, 0), :] = workloads.FIXED
    o = oracle.Oracle(spec, MAT, 1e-7, bc)
    f = np.zeros((spec.n_particles, 6))
    f[:, 2] = o.geometry()["mass"][:, 0] * 1e8
    f[spec.face_nodes(2, 1), 0] = 0.5
    dt = 0.9 * o.critical_dt()
    o = oracle.Oracle(spec, MAT, dt, bc, f_ext=f)
    o.step(300)
    return spec, bc, f, dt, o


def test_external_force_trajectory_fp64(hanging):
    spec, bc, f, dt, o = hanging
    h = o.get_state()[2]
    assert np.sum(h[:, 4] > 1.5 * MAT["sigma_t"] / MAT["E0"]) > 300, "facets must have cracked"
    m = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc, f_ext=f)
    m.step(300)
    qg, vg, hg, _ = m.get_state()
    qo, vo, ho, _ = o.get_state()
    assert nrel(qg, qo) <= 1e-8 and nrel(vg, vo) <= 1e-8 and nrel(hg, ho) <= 1e-7, (nrel(qg, qo), nrel(hg, ho))
    eg, rg = m.energy()
    eo, ro = o.energy()
    assert eo[0] > 0 and nrel(eg[:3], eo[:3]) <= 1e-8 and nrel(rg, ro) <= 1e-7, (eg, eo, rg, ro)
    m.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_external_force_one_step(hanging, prec, tol):
    spec, bc, f, dt, o = hanging
    q, v, h5, st = o.get_state()
    o2 = oracle.Oracle(spec, MAT, dt, bc, f_ext=f)
    o2.set_state(q, v, h5, st)
    o2.step(1)
    qo, vo, _, _ = o2.get_state()
    _, fo = o2.facet_forces()
    m = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc, f_ext=f)
    m.set_state(q, v, h5, st)
    m.step(1)
    qg, vg, _, _ = m.get_state()
    _, fg = m.facet_forces()
    if prec == "fp64":
        for what, g, o_ in (("node forces", fg, fo), ("v", vg, vo), ("q", qg, qo)):
            assert_elementwise(g, o_, tol, what)
    else:
        assert nrel(fg, fo) <= tol and nrel(vg, vo) <= tol and nrel(qg, qo) <= tol, (nrel(fg, fo), nrel(vg, vo))
    eg, _ = m.energy()
    eo, _ = o2.energy()
    assert nrel(eg[:1], eo[:1]) <= tol  # the external work of the step
    m.close()
