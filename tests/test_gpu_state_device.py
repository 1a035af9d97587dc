"""ldpm_get_state_device: the state of ldpm_get_state written into caller device buffers (torch
tensors), with no host copy, compared bitwise with the host read-out of the same state."""
import numpy as np
import pytest

from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_state_equals_host_state(prec):
    import torch

    spec = specimen.shuffled(specimen.make_cube_specimen(12.0, 2.0, 4.0, 300, seed=31), seed=2)
    bc = workloads.uniaxial_tension_bc(spec, velocity=300.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 0] = workloads.PRESCRIBED
    bc.vel[top, 0] = 80.0
    stream = torch.cuda.Stream()
    m = ldpm.Model(spec, dict(WORKLOAD_MATERIAL), precision=prec, dt=1.5e-7, bc=bc, stream=stream)
    m.step(137)
    qd, vd, hd, sd = m.get_state_device()
    q, v, h5, st = m.get_state()
    assert np.abs(h5).max() > 0 and np.abs(v).max() > 0
    assert np.array_equal(qd.cpu().numpy(), q) and np.array_equal(vd.cpu().numpy(), v)
    assert np.array_equal(hd.cpu().numpy(), h5) and int(sd.item()) == st == 137
    # NULL pointers are skipped
    qd2 = torch.zeros_like(qd)
    ldpm.ldpm_get_state_device(m.h, qd2.data_ptr(), 0, 0, 0)
    stream.synchronize()
    assert np.array_equal(qd2.cpu().numpy(), q)
    m.close()


def test_device_state_of_a_batch_is_concatenated():
    import torch

    specs = [specimen.make_cube_specimen(L, 2.0, 4.0, n, seed=40 + k) for k, (L, n) in enumerate([(10.0, 150), (12.0, 260)])]
    bcs = [workloads.unconfined_compression_bc(sp, velocity=300.0, ramp_time=1e-5) for sp in specs]
    stream = torch.cuda.Stream()
    b = ldpm.Batch(specs, [dict(WORKLOAD_MATERIAL)] * 2, "mixed", dts=[1.5e-7, 1.5e-7], bcs=bcs, stream=stream)
    b.step(60)
    N = sum(sp.n_particles for sp in specs)
    F = sum(sp.n_facets for sp in specs)
    q = torch.empty((N, 6), dtype=torch.float64, device="cuda")
    h5 = torch.empty((F, 5), dtype=torch.float64, device="cuda")
    ldpm.ldpm_get_state_device(b.h, q.data_ptr(), 0, h5.data_ptr(), 0)
    stream.synchronize()
    q_host = np.concatenate([b.get_state(i)[0] for i in range(2)])
    h_host = np.concatenate([b.get_state(i)[2] for i in range(2)])
    assert np.array_equal(q.cpu().numpy(), q_host) and np.array_equal(h5.cpu().numpy(), h_host)
    b.close()
