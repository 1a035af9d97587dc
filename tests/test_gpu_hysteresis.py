"""GPU against the FP64 oracle with the unload/reload variants of Appendix A switched on: tensile
reloading k_t = 0.5 (A.1), densified unloading stiffness E_d = 2 E0 (A.2), shear softening modulus
H_s = 0.1 E0 (A.1).  A 12 mm cube is pulled and sheared past its peak, unloaded by reversing the
loading, and reloaded; parity one step from the oracle's cycled state and over the whole cycle."""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL
from parity import assert_elementwise, normwise_rel as nrel

pytestmark = pytest.mark.gpu
VAR = dict(WORKLOAD_MATERIAL, k_t=0.5, Ed_E0=2.0, r_s=0.1)
LEGS = ((1.0, 600), (-1.0, 400), (1.0, 150))  # loading direction, steps


def _bc(spec, sign):
    bc = workloads.uniaxial_tension_bc(spec, velocity=sign * 200.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 1] = workloads.PRESCRIBED
    bc.vel[top, 1] = sign * 60.0
    return bc


@pytest.fixture(scope="module")
def cycled():
    spec = specimen.shuffled(specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=21), seed=5)
    bcs = [_bc(spec, s) for s, _ in LEGS]
    dt = 0.9 * oracle.Oracle(spec, VAR, 1e-7, bcs[0]).critical_dt()
    o = oracle.Oracle(spec, VAR, dt, bcs[0])
    for k, (_, n) in enumerate(LEGS):
        if k:
            o.set_bc(bcs[k])
        o.step(n)
    return spec, bcs, dt, o


def test_reload_rule_and_variants_change_the_cycle(cycled):
    """The variants are exercised: the same cycle with k_t = 0, E_d = E0, r_s = 0 ends elsewhere, and
    facets have cracked (e_max past the elastic limit) and sit at zero traction after unloading."""
    spec, bcs, dt, o = cycled
    base = oracle.Oracle(spec, dict(WORKLOAD_MATERIAL), dt, bcs[0])
    for k, (_, n) in enumerate(LEGS):
        if k:
            base.set_bc(bcs[k])
        base.step(n)
    h = o.get_state()[2]
    hb = base.get_state()[2]
    assert nrel(h, hb) > 1e-3
    e0 = VAR["sigma_t"] / VAR["E0"]
    assert np.sum(h[:, 4] > 2 * e0) > 50


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_one_step_from_cycled_state(cycled, prec, tol):
    spec, bcs, dt, o = cycled
    q, v, h5, st = o.get_state()
    o2 = oracle.Oracle(spec, VAR, dt, bcs[-1])
    o2.set_state(q, v, h5, st)
    o2.step(1)
    qo, vo, ho, _ = o2.get_state()
    Fo, fo = o2.facet_forces()
    m = ldpm.Model(spec, VAR, precision=prec, dt=dt, bc=bcs[-1])
    m.set_state(q, v, h5, st)
    m.step(1)
    qg, vg, hg, _ = m.get_state()
    Fg, fg = m.facet_forces()
    if prec == "fp64":
        for what, g, o_ in (("node forces", fg, fo), ("v", vg, vo), ("q", qg, qo), ("hist", hg, ho),
                            ("facet forces", Fg, Fo)):
            assert_elementwise(g, o_, tol, what)
    else:
        assert nrel(fg, fo) <= tol and nrel(vg, vo) <= tol and nrel(qg, qo) <= tol, (nrel(fg, fo), nrel(vg, vo))
    m.close()


def test_fp64_trajectory_through_the_cycle(cycled):
    spec, bcs, dt, o = cycled
    m = ldpm.Model(spec, VAR, precision="fp64", dt=dt, bc=bcs[0])
    for k, (_, n) in enumerate(LEGS):
        if k:
            m.set_bc(bcs[k].mask, bcs[k].vel, bcs[k].ramp_time)
        m.step(n)
    qg, vg, hg, _ = m.get_state()
    qo, vo, ho, _ = o.get_state()
    assert nrel(qg, qo) <= 1e-8 and nrel(hg, ho) <= 1e-7, (nrel(qg, qo), nrel(hg, ho))
    eg, rg = m.energy()
    eo, ro = o.energy()
    assert nrel(eg[:3], eo[:3]) <= 1e-8
    m.close()


def test_adjoint_with_variants_matches_oracle(cycled):
    """The gradient with H_s != 0 (softening facets) and E_d != E0, FP64, against the oracle's
    directional derivatives from the oracle's state after the first loading leg."""
    spec, bcs, dt, _ = cycled
    o = oracle.Oracle(spec, VAR, dt, bcs[0])
    o.step(200)
    q, v, h5, st = o.get_state()
    seed = np.zeros((spec.n_particles, 6))
    seed[spec.face_nodes(2, 1), 2] = 1.0
    rng = np.random.default_rng(9)
    F = spec.n_facets
    P0 = np.array([VAR["E0"], VAR["alpha"], VAR["sigma_t"]])
    D = np.array([rng.standard_normal((3, F)) * P0[:, None] for _ in range(3)])
    K = 150
    J, dJ = o.tangent(K, seed, D[:, 0], D[:, 1], D[:, 2])
    m = ldpm.Model(spec, VAR, precision="fp64", dt=dt, bc=bcs[0])
    m.set_state(q, v, h5, st)
    Jg, gE, ga, gs = m.adjoint(K, seed, ckpt_every=50)
    got = np.einsum("dpf,pf->d", D, np.array([gE, ga, gs]))
    np.testing.assert_allclose(Jg, J, rtol=1e-10)
    np.testing.assert_allclose(got, dJ, rtol=1e-7)
    m.close()
