"""GPU against the FP64 oracle on the benchmark's own specimens, loading and state.

`bench.py` times each workload after `preroll` untimed steps and 5 warm-up steps of its loading
history, with the workload's fixed time step.  Here the oracle runs exactly that history on the
full-size specimen (1.82M facets for uniaxial tension, 12.5M for confined compression), and:

  * the GPU's own FP64 trajectory to that state matches it per element (tolerance 1e-9 after ~100-200
    steps: the per-step contract 1e-10 with rounding differences that grow over the steps);
  * one GPU step from the oracle's state matches the oracle's next step per element within 1e-10
    (FP64 mode) in the node forces, the facet forces, the state and the history;
  * one mixed-mode step from the same state: node forces and velocities within 2e-5 normwise,
    per-facet forces within 1e-4 of the largest for all but 0.5 % of the facets, and the number of
    facets that took the other branch of the law is reported and bounded;
  * the mixed-mode trajectory to that state: the macroscopic response (the loaded face's reaction, or
    the external work in confined compression) within 1e-3 of the oracle's and the energy-balance
    error (Sec. 4) below 1 %.

These run before any other full-size GPU test (file name), so a failure here is the first one seen.
"""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, workloads
from parity import assert_elementwise, branch_flips, elementwise_excess, normwise_rel

pytestmark = pytest.mark.gpu
BENCH_WARMUP = 5  # bench.py's default warm-up, run after the pre-roll and before the timed steps


def macroscopic_response(name, e, r):
    """What the workload's loading measures: the top face's u_z reaction (uniaxial tension), or the
    external work of the faces moving inward (confined compression, where the opposite faces'
    reactions cancel in the per-component sums)."""
    return r[8] if name == "uniaxial_tension" else e[0]


@pytest.fixture(scope="module", params=["uniaxial_tension", "confined_compression"])
def bench_state(request):
    name = request.param
    wl = workloads.WORKLOADS[name]
    spec = wl.specimen()
    bc = workloads.workload_bc(name, spec)
    n0 = wl.preroll + BENCH_WARMUP
    o = oracle.Oracle(spec, wl.material, wl.dt, bc)
    o.step(n0)
    state = o.get_state()
    e0, r0 = o.energy()
    o.step(1)
    after = o.get_state()
    F1, f1 = o.facet_forces()
    e1, r1 = o.energy()
    del o
    return dict(name=name, wl=wl, spec=spec, bc=bc, n0=n0, state=state, e0=e0, r0=r0, after=after, F1=F1, f1=f1,
                e1=e1, r1=r1)


def test_fp64_trajectory_reaches_the_bench_state(bench_state):
    b = bench_state
    m = ldpm.Model(b["spec"], b["wl"].material, precision="fp64", dt=b["wl"].dt, bc=b["bc"])
    m.step(b["n0"])
    q, v, h5, st = m.get_state()
    qo, vo, ho, so = b["state"]
    assert st == so == b["n0"]
    for what, g, o in (("q", q, qo), ("v", v, vo), ("hist", h5, ho)):
        assert_elementwise(g, o, 1e-9, "%s %s" % (b["name"], what))
    e, r = m.energy()
    assert_elementwise(e[:3], b["e0"][:3], 1e-9, "energies")
    assert_elementwise(r, b["r0"], 1e-9, "reactions")
    # the loading wave has crossed the specimen: every facet carries traction (the timed window does
    # not run on the law's zero-strain path), both branches of the law are in use
    assert np.mean(np.abs(ho[:, 0]) > 0) > 0.99, "the loading wave must have crossed the specimen"
    assert np.any(ho[:, 0] > 0) and np.any(ho[:, 0] < 0)
    m.close()


def test_fp64_one_step_from_the_bench_state(bench_state):
    b = bench_state
    m = ldpm.Model(b["spec"], b["wl"].material, precision="fp64", dt=b["wl"].dt, bc=b["bc"])
    m.set_state(*b["state"])
    m.step(1)
    q, v, h5, _ = m.get_state()
    F, f = m.facet_forces()
    e, r = m.energy()
    qo, vo, ho, _ = b["after"]
    for what, g, o in (("node forces", f, b["f1"]), ("facet forces", F, b["F1"]), ("q", q, qo), ("v", v, vo),
                       ("hist", h5, ho), ("reactions", r, b["r1"])):
        assert_elementwise(g, o, 1e-10, "%s %s" % (b["name"], what))
    m.close()


def test_mixed_one_step_from_the_bench_state(bench_state):
    b = bench_state
    m = ldpm.Model(b["spec"], b["wl"].material, precision="mixed", dt=b["wl"].dt, bc=b["bc"])
    m.set_state(*b["state"])
    m.step(1)
    q, v, h5, _ = m.get_state()
    F, f = m.facet_forces()
    qo, vo, ho, _ = b["after"]
    Fo = b["F1"]
    err_f, err_v, err_q = normwise_rel(f, b["f1"]), normwise_rel(v, vo), normwise_rel(q, qo)
    facet_err = np.abs(F - Fo).max(axis=1) / np.abs(Fo).max()
    frac_off = float(np.mean(facet_err > 1e-4))
    flips = branch_flips(h5, ho, 1e-6 * b["wl"].material["sigma_t"])
    worst, n_bad = elementwise_excess(f, b["f1"], 2e-5)
    print("%s mixed one step: node forces %.2e, v %.2e, q %.2e normwise; facets beyond 1e-4: %.2e; branch flips "
          "%d of %d; node forces per element at 2e-5: worst %.3g x bound, %d outside" % (
              b["name"], err_f, err_v, err_q, frac_off, flips, len(F), worst, n_bad))
    assert err_f <= 2e-5 and err_v <= 2e-5 and err_q <= 1e-8
    assert frac_off < 5e-3
    assert flips <= 1e-4 * len(F)
    m.close()


def test_mixed_trajectory_to_the_bench_state(bench_state):
    b = bench_state
    m = ldpm.Model(b["spec"], b["wl"].material, precision="mixed", dt=b["wl"].dt, bc=b["bc"])
    m.step(b["n0"])
    e, r = m.energy()
    sg, so = macroscopic_response(b["name"], e, r), macroscopic_response(b["name"], b["e0"], b["r0"])
    assert abs(so) > 0
    assert abs(sg - so) <= 1e-3 * abs(so), (sg, so)
    assert e[3] <= 1.0 and b["e0"][3] <= 1.0, (e[3], b["e0"][3])
    assert normwise_rel(e[:3], b["e0"][:3]) <= 1e-3
    m.close()
