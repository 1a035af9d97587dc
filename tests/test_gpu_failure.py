"""Failure detection without a GPU fault.  A step size above the stability limit of the central
difference scheme (Sec. 3: stable for dt < 2 / omega_max) makes the explicit step diverge.  The particle
pass flags the first non-finite velocity or displacement, and the library reports LDPM_E_UNSTABLE.
Non-finite numbers are ordinary data for these kernels (no kernel indexes or loops on a floating-point
value), so nothing traps and the context stays usable: a stable model on the same device runs after."""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads

pytestmark = pytest.mark.gpu
MAT = dict(workloads.WORKLOAD_MATERIAL, elastic=1)


@pytest.fixture(scope="module")
def setup():
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=1)
    bc = workloads.free_bc(spec.n_particles)
    bc.v0 = np.random.default_rng(0).standard_normal((spec.n_particles, 6))
    dt_c = oracle.Oracle(spec, MAT, 1e-7, bc).critical_dt()
    return spec, bc, dt_c


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_divergence_above_the_stability_limit_is_reported(setup, prec):
    spec, bc, dt_c = setup
    m = ldpm.Model(spec, MAT, precision=prec, dt=3.0 * dt_c, bc=bc)
    with pytest.raises(ldpm.LdpmError) as ei:
        for _ in range(40):  # the highest mode grows about 34x per step: overflow within a few hundred
            m.step(50)
            m.sync()
    assert ei.value.code == -5, str(ei.value)
    m.close()
    # the same device runs a stable model afterwards, on the oracle's trajectory
    s = ldpm.Model(spec, MAT, precision=prec, dt=0.9 * dt_c, bc=bc)
    s.step(200)
    q, v, _, _ = s.get_state(hist=False)
    s.close()
    o = oracle.Oracle(spec, MAT, 0.9 * dt_c, bc)
    o.step(200)
    qo, vo, _, _ = o.get_state()
    tol = 1e-8 if prec == "fp64" else 1e-3
    assert np.abs(q - qo).max() <= tol * np.abs(qo).max() and np.abs(v - vo).max() <= tol * np.abs(vo).max()
