"""GPU against the FP64 oracle with the compression and friction options of Appendix A that the
workloads leave off: beta = 0.3 in the volumetric-deviatoric strain e_DV = e_V + beta e_D (A.2),
asymptotic friction mu_inf = 0.05 (A.3), and a lower deviatoric threshold k_c1 = 0.5 (A.2).  A 10 mm
cube is compressed fast along z while its top face is sheared along y, so that a few hundred facets
harden past sigma_c0 and most of the compressed ones slide at the friction cap.  Parity of the
trajectory, of one step in each precision, and of the adjoint gradient."""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL
from parity import assert_elementwise, normwise_rel as nrel

VAR = dict(WORKLOAD_MATERIAL, beta=0.3, mu_inf=0.05, kc1=0.5)
STEPS = 300


@pytest.fixture(scope="module")
def loaded():
    spec = specimen.shuffled(specimen.make_cube_specimen(10.0, 2.0, 4.0, 220, seed=23), seed=4)
    bc = workloads.uniaxial_tension_bc(spec, velocity=-1500.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 1] = workloads.PRESCRIBED
    bc.vel[top, 1] = 600.0
    dt = 0.9 * oracle.Oracle(spec, VAR, 1e-7, bc).critical_dt()
    o = oracle.Oracle(spec, VAR, dt, bc)
    o.step(STEPS)
    return spec, bc, dt, o


def test_the_options_are_exercised(loaded):
    """Facets have hardened past sigma_c0, many compressed facets are at or near the friction cap,
    and without the three options the state differs."""
    spec, bc, dt, o = loaded
    h = o.get_state()[2]
    assert np.sum(-h[:, 0] > 1.0001 * VAR["sigma_c0"]) > 100
    base = oracle.Oracle(spec, dict(WORKLOAD_MATERIAL), dt, bc)
    base.step(STEPS)
    assert nrel(h, base.get_state()[2]) > 0.05
    # the friction return acts: the shear traction stays under the cap (which is at most
    # sigma_s + mu0 |t_N| for mu_inf <= mu0) and reaches 90 % of that bound on many facets
    tT = np.linalg.norm(h[:, 1:4], axis=1)
    tN = np.minimum(h[:, 0], 0.0)
    cap0 = VAR["r_st"] * VAR["sigma_t"] + VAR["mu0"] * -tN
    assert np.all(tT <= cap0 * (1 + 1e-12) + 1e-12)
    assert np.sum((tN < 0) & (tT > 0.9 * cap0)) > 500


@pytest.mark.gpu
def test_fp64_trajectory(loaded):
    spec, bc, dt, o = loaded
    m = ldpm.Model(spec, VAR, precision="fp64", dt=dt, bc=bc)
    m.step(STEPS)
    qg, vg, hg, _ = m.get_state()
    qo, vo, ho, _ = o.get_state()
    assert nrel(qg, qo) <= 1e-8 and nrel(hg, ho) <= 1e-7, (nrel(qg, qo), nrel(hg, ho))
    eg, _ = m.energy()
    eo, _ = o.energy()
    assert nrel(eg[:3], eo[:3]) <= 1e-8
    m.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_one_step_from_loaded_state(loaded, prec, tol):
    spec, bc, dt, o = loaded
    q, v, h5, st = o.get_state()
    o2 = oracle.Oracle(spec, VAR, dt, bc)
    o2.set_state(q, v, h5, st)
    o2.step(1)
    qo, vo, ho, _ = o2.get_state()
    Fo, fo = o2.facet_forces()
    m = ldpm.Model(spec, VAR, precision=prec, dt=dt, bc=bc)
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


@pytest.mark.gpu
def test_adjoint_matches_oracle(loaded):
    """FP64 gradient through hardening and friction sliding with beta, mu_inf != 0, against the
    oracle's directional derivatives from its state after 200 steps."""
    spec, bc, dt, _ = loaded
    o = oracle.Oracle(spec, VAR, dt, bc)
    o.step(200)
    q, v, h5, st = o.get_state()
    seed = np.zeros((spec.n_particles, 6))
    seed[spec.face_nodes(2, 1), 2] = 1.0
    seed[spec.face_nodes(2, 1), 1] = 0.5
    rng = np.random.default_rng(12)
    F = spec.n_facets
    P0 = np.array([VAR["E0"], VAR["alpha"], VAR["sigma_t"]])
    D = np.array([rng.standard_normal((3, F)) * P0[:, None] for _ in range(3)])
    K = 100
    J, dJ = o.tangent(K, seed, D[:, 0], D[:, 1], D[:, 2])
    m = ldpm.Model(spec, VAR, precision="fp64", dt=dt, bc=bc)
    m.set_state(q, v, h5, st)
    Jg, gE, ga, gs = m.adjoint(K, seed, ckpt_every=40)
    got = np.einsum("dpf,pf->d", D, np.array([gE, ga, gs]))
    np.testing.assert_allclose(Jg, J, rtol=1e-10)
    np.testing.assert_allclose(got, dJ, rtol=1e-7)
    m.close()
