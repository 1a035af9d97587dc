"""Random-perturbation study (the paper's Sec. 5): uniform random vectors in [-eta/2, eta/2] added to
all free displacements and rotations at fixed intervals of an unconfined compression test with free
platens.  GPU parity with the oracle through perturbations, and the paper's finding on synthetic
specimens: before the peak the response is modified only slightly and returns to its course; the
differences grow after the dynamic post-peak event."""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

pytestmark = pytest.mark.gpu
MAT = dict(WORKLOAD_MATERIAL)


@pytest.fixture(scope="module")
def uc():
    spec = specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=41)
    bc = workloads.unconfined_compression_bc(spec, velocity=100.0, ramp_time=2e-5)
    dt = 0.9 * oracle.Oracle(spec, MAT, 1e-7, bc).critical_dt()
    return spec, bc, dt


def _draws(spec, eta, count, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-eta / 2, eta / 2, (spec.n_particles, 6)) for _ in range(count)]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 5e-5)])
def test_perturbed_run_matches_oracle(uc, prec, tol):
    spec, bc, dt = uc
    dqs = _draws(spec, 1e-4, 3, seed=2)
    o = oracle.Oracle(spec, MAT, dt, bc)
    m = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc)
    for dq in dqs:
        o.step(100)
        m.step(100)
        o.perturb(dq)
        m.perturb(dq)
    o.step(50)
    m.step(50)
    qo, vo, ho, _ = o.get_state()
    qg, vg, hg, _ = m.get_state()
    assert np.abs(qg - qo).max() <= tol * np.abs(qo).max()
    assert np.abs(vg - vo).max() <= 10 * tol * np.abs(vo).max()
    m.close()


def test_perturbation_study_response_returns_before_the_peak(uc):
    spec, bc, dt = uc
    every, nsteps, block = 200, 6000, 50

    def run(eta):
        m = ldpm.Model(spec, MAT, precision="mixed", dt=dt, bc=bc)
        dqs = _draws(spec, eta, nsteps // every, seed=7)
        R = []
        for n in range(nsteps // block):
            m.step(block)
            s = (n + 1) * block
            if eta > 0 and s % every == 0:
                m.perturb(dqs[s // every - 1])
            R.append(-m.energy()[1][8])
        m.close()
        return np.array(R)

    r0 = run(0.0)
    k = int(np.argmax(r0))
    assert 5 < k < len(r0) - 20, "the run must pass the peak"
    for eta in (1e-5, 1e-4):
        d = np.abs(run(eta) - r0) / r0[k]
        # before the peak: below 0.5 % of the peak load; after it: several times larger
        assert d[:k].max() <= 5e-3, (eta, d[:k].max())
        assert d[k:].max() > 3 * d[:k].max(), (eta, d[:k].max(), d[k:].max())
