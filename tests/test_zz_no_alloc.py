"""The allocation-free kinetic-energy entry point against ldpm_energy's W_kin.

Callers that may not allocate device memory (inside another component's graph capture, under a
fixed device-memory pool, in monitoring hooks) use ldpm_kinetic_energy_noalloc on their own device
arrays; its scratch is a static device array inside the library.  This file is collected last so a
run that stops at its first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2603_13190_gb300 import ldpm, specimen, workloads

pytestmark = pytest.mark.gpu


def test_noalloc_kinetic_energy_matches_ldpm_energy_twice():
    torch = pytest.importorskip("torch")
    spec = specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=8)
    rng = np.random.default_rng(4)
    mass = rng.uniform(1e-9, 3e-9, spec.n_particles)
    inertia = rng.uniform(1e-9, 3e-9, (spec.n_particles, 3))
    bc = workloads.uniaxial_tension_bc(spec, velocity=60.0, ramp_time=1e-5)
    bc.v0[:] = rng.standard_normal(bc.v0.shape)
    m = ldpm.Model(spec, workloads.WORKLOAD_MATERIAL, precision="mixed", dt=0.0, bc=bc, mass=mass,
                   inertia=inertia)
    mass6 = np.concatenate([np.repeat(mass[:, None], 3, 1), inertia], axis=1)
    stream = torch.cuda.Stream()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for n in (7, 13):  # two calls in a row, each on a new state
        m.step(n)
        e, _ = m.energy()
        _, v, _, _ = m.get_state(hist=False)
        v_d = torch.tensor(v.reshape(-1), dtype=torch.float64, device="cuda")
        m_d = torch.tensor(mass6.reshape(-1), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ldpm.ldpm_kinetic_energy_noalloc(v_d.data_ptr(), m_d.data_ptr(), v_d.numel(), out.data_ptr(), stream)
        stream.synchronize()
        got = float(out.item())
        assert abs(got - e[2]) <= 1e-12 * abs(e[2]), (got, e[2])
    m.close()


def test_noalloc_rejects_sizes_over_its_static_scratch():
    torch = pytest.importorskip("torch")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ldpm.LdpmError) as ei:
        ldpm.ldpm_kinetic_energy_noalloc(x.data_ptr(), x.data_ptr(), 4 * 1024 * 1024 + 1, x.data_ptr())
    assert ei.value.code == -1 and "static scratch limit" in str(ei.value)
