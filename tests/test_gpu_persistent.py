"""Persistent launch mode: one cooperative launch per ldpm_step call with bounded grid barriers.

  * the persistent kernel is deterministic (two handles agree bit for bit) and follows the
    graph-replayed launch pairs: the same device functions in the same order, with the compiler free
    to schedule and contract multiply-adds differently in the two kernels, so the modes agree to
    rounding (FP64: per element within 1e-10, the per-step contract; mixed: within 1e-6 normwise over
    the first steps, 1e-3 after hundreds of steps of a cracking specimen), for one specimen and for a
    batch of uneven specimens;
  * its FP64 trajectory matches the oracle per element;
  * a barrier wait that runs out (one block made to skip its arrival through the fault-injection hook,
    with a short wait limit) ends the launch: ldpm_sync reports LDPM_E_TIMEOUT, the error stays until
    the state is replaced, and the handle then steps on as before.  Nothing waits without a bound.
"""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL
from parity import assert_elementwise, normwise_rel as nrel

pytestmark = pytest.mark.gpu
MAT = dict(WORKLOAD_MATERIAL)


@pytest.fixture(scope="module")
def loaded():
    spec = specimen.shuffled(specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=5), seed=3)
    bc = workloads.uniaxial_tension_bc(spec, velocity=80.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 0] = workloads.PRESCRIBED
    bc.vel[top, 0] = 40.0
    dt = 0.9 * oracle.Oracle(spec, MAT, 1e-7, bc).critical_dt()
    return spec, bc, dt


def states_equal(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])) and a[3] == b[3]


def assert_modes_agree(a, b, prec, what, mixed_tol=1e-6):
    """State b (persistent) against state a (launch pairs) of the same steps.  Mixed mode: the two
    FP32 roundings of a cracking specimen drift apart like any two mixed runs, so long windows get a
    trajectory-level tolerance."""
    assert a[3] == b[3], what
    for k, name in enumerate(("q", "v", "hist")):
        if prec == "fp64":
            assert_elementwise(b[k], a[k], 1e-10, "%s %s" % (what, name))
        else:
            assert nrel(b[k], a[k]) <= mixed_tol, (what, name, nrel(b[k], a[k]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_is_deterministic_and_follows_launch_pairs(loaded, prec):
    spec, bc, dt = loaded
    pairs = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc)
    pers = [ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc) for _ in range(2)]
    for m in pers:
        ldpm.ldpm_set_launch_mode(m.h, ldpm.LDPM_LAUNCH_PERSISTENT)
        assert ldpm.ldpm_launch_mode(m.h) == ldpm.LDPM_LAUNCH_PERSISTENT
    assert ldpm.ldpm_launch_mode(pairs.h) == ldpm.LDPM_LAUNCH_PAIRS
    for n in (1, 7, 250, 142):  # one call = one launch of n steps
        pairs.step(n)
        for m in pers:
            m.step(n)
        s0, s1, s2 = pairs.get_state(), pers[0].get_state(), pers[1].get_state()
        assert states_equal(s1, s2), n
        assert_modes_agree(s0, s1, prec, "after a call of %d steps" % n, 1e-6 if n < 100 else 1e-3)
    ea, _ = pairs.energy()
    eb, _ = pers[0].energy()
    assert nrel(eb[:3], ea[:3]) <= (1e-10 if prec == "fp64" else 1e-4)
    for m in [pairs] + pers:
        m.close()


def test_persistent_fp64_trajectory_matches_the_oracle(loaded):
    spec, bc, dt = loaded
    o = oracle.Oracle(spec, MAT, dt, bc)
    m = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc)
    ldpm.ldpm_set_launch_mode(m.h, ldpm.LDPM_LAUNCH_PERSISTENT)
    o.step(400)
    m.step(400)
    qg, vg, hg, _ = m.get_state()
    qo, vo, ho, _ = o.get_state()
    assert np.abs(ho[:, 0]).max() > 0.5 * MAT["sigma_t"]
    for what, g, r in (("q", qg, qo), ("v", vg, vo), ("hist", hg, ho)):
        assert_elementwise(g, r, 1e-9, what)
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_batch_follows_launch_pairs(prec):
    specs = [specimen.make_cube_specimen(L, 2.0, 4.0, n, seed=s) for L, n, s in ((9.0, 110, 31), (14.0, 420, 32),
                                                                                  (11.0, 230, 33))]
    bcs = [workloads.unconfined_compression_bc(specs[0], velocity=300.0, ramp_time=1e-5),
           workloads.uniaxial_tension_bc(specs[1], velocity=150.0, ramp_time=1e-5),
           workloads.confined_compression_bc(specs[2], velocity=300.0, ramp_time=1e-5)]
    mats = [MAT, dict(MAT, sigma_t=3.5), dict(MAT, E0=40000.0)]
    dts = [1.4e-7, 1.5e-7, 1.45e-7]
    a = ldpm.Batch(specs, mats, prec, dts=dts, bcs=bcs)
    b = ldpm.Batch(specs, mats, prec, dts=dts, bcs=bcs)
    ldpm.ldpm_set_launch_mode(b.h, ldpm.LDPM_LAUNCH_PERSISTENT)
    a.step(150)
    b.step(150)
    for i in range(3):
        assert_modes_agree(a.get_state(i), b.get_state(i), prec, "specimen %d" % i, 1e-3)
    a.close()
    b.close()


def test_barrier_wait_that_runs_out_reports_timeout(loaded):
    spec, bc, dt = loaded
    ref = ldpm.Model(spec, MAT, precision="mixed", dt=dt, bc=bc)
    m = ldpm.Model(spec, MAT, precision="mixed", dt=dt, bc=bc)
    for h in (ref.h, m.h):  # the reference steps persistently too, so the two agree bit for bit
        ldpm.ldpm_set_launch_mode(h, ldpm.LDPM_LAUNCH_PERSISTENT)
    m.step(20)
    ref.step(20)
    ck = ldpm.ldpm_save_checkpoint(m.h)
    # block 0 does not arrive at the first barrier; every wait gives up after 20 ms
    ldpm.ldpm_set_barrier_wait(m.h, 0.02, 0)
    m.step(5)
    with pytest.raises(ldpm.LdpmError) as ei:
        m.sync()
    assert ei.value.code == -6  # LDPM_E_TIMEOUT
    m.step(3)  # later launches return at once; the error stays
    with pytest.raises(ldpm.LdpmError) as ei:
        m.get_state()
    assert ei.value.code == -6
    # replacing the state clears it; without the hook the handle steps on as the reference does
    ldpm.ldpm_set_barrier_wait(m.h, 0.0, -1)
    ldpm.ldpm_load_checkpoint(m.h, ck)
    m.step(30)
    ref.step(30)
    assert states_equal(m.get_state(), ref.get_state())
    m.close()
    ref.close()


def test_barrier_wait_arguments_are_checked(loaded):
    spec, bc, dt = loaded
    m = ldpm.Model(spec, MAT, precision="mixed", dt=dt, bc=bc)
    for secs, skip in ((float("nan"), -1), (1e5, -1), (0.1, -2)):
        with pytest.raises(ldpm.LdpmError):
            ldpm.ldpm_set_barrier_wait(m.h, secs, skip)
    with pytest.raises(ldpm.LdpmError):
        ldpm.ldpm_set_launch_mode(m.h, 3)
    m.close()


def test_elastic_vibration_persistent_fp64_conserves_energy():
    """The 18k-facet elastic-vibration workload (launch-bound as launch pairs) in persistent launches:
    the energies of the launch pairs, error below 1 %."""
    wl = workloads.WORKLOADS["elastic_vibration"]
    spec = wl.specimen()
    bc = workloads.workload_bc(wl.name, spec)
    a = ldpm.Model(spec, wl.material, precision="fp64", dt=wl.dt, bc=bc)
    b = ldpm.Model(spec, wl.material, precision="fp64", dt=wl.dt, bc=bc)
    ldpm.ldpm_set_launch_mode(b.h, ldpm.LDPM_LAUNCH_PERSISTENT)
    a.step(wl.steps)
    b.step(wl.steps)
    ea, _ = a.energy()
    eb, _ = b.energy()
    assert nrel(eb[:3], ea[:3]) <= 1e-10 and eb[3] < 1.0
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_with_per_facet_parameters(loaded, prec):
    """The persistent kernel's per-facet parameter instantiation (E0, alpha, sigma_t per facet)."""
    spec, bc, dt = loaded
    rng = np.random.default_rng(7)
    F = spec.n_facets
    E0 = MAT["E0"] * rng.uniform(0.8, 1.2, F)
    alpha = MAT["alpha"] * rng.uniform(0.8, 1.2, F)
    sig = MAT["sigma_t"] * rng.uniform(0.7, 1.1, F)
    a = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc)
    b = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc)
    ldpm.ldpm_set_launch_mode(b.h, ldpm.LDPM_LAUNCH_PERSISTENT)
    for m in (a, b):
        m.set_facet_params(E0, alpha, sig)
        m.step(60)
    assert_modes_agree(a.get_state(), b.get_state(), prec, "per-facet parameters")
    if prec == "fp64":
        o = oracle.Oracle(spec, MAT, dt, bc)
        o.set_facet_params(E0, alpha, sig)
        o.step(60)
        qg, vg, hg, _ = b.get_state()
        qo, vo, ho, _ = o.get_state()
        for what, g, r in (("q", qg, qo), ("v", vg, vo), ("hist", hg, ho)):
            assert_elementwise(g, r, 1e-9, what)
    a.close()
    b.close()


def test_adjoint_of_a_persistent_handle(loaded):
    """ldpm_adjoint runs its own forward and reverse passes whatever the launch mode: a handle in the
    persistent mode gives the gradient of one in launch pairs, and both end in the same state."""
    spec, bc, dt = loaded
    seed = np.zeros((spec.n_particles, 6))
    seed[spec.face_nodes(2, 1), 2] = 1.0
    out = []
    for mode in (ldpm.LDPM_LAUNCH_PAIRS, ldpm.LDPM_LAUNCH_PERSISTENT):
        m = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc)
        ldpm.ldpm_set_launch_mode(m.h, mode)
        m.step(30)
        J, gE, ga, gs = m.adjoint(40, seed, ckpt_every=16)
        m.step(10)
        out.append((J, gE, ga, gs, m.get_state()))
        m.close()
    (Ja, gEa, gaa, gsa, sa), (Jb, gEb, gab, gsb, sb) = out
    assert abs(Ja - Jb) <= 1e-10 * abs(Ja)
    for x, y in ((gEa, gEb), (gaa, gab), (gsa, gsb)):
        assert nrel(y, x) <= 1e-9
    assert_modes_agree(sa, sb, "fp64", "after the adjoint and 10 more steps")
