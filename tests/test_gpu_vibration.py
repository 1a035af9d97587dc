"""Free vibration on the GPU against the eigenvalues of the assembled stiffness and mass (Sec. 4.1's
free-vibration benchmark, as a spectral check): an elastic 8 mm cube starts from q = 0 with a velocity
made of three eigenmodes (K phi = w^2 M phi, K from the oracle's elastic operator, solved by LAPACK).
The FFT of each modal coordinate peaks at the scheme's discrete frequency theta_i / (2 pi dt),
cos theta_i = 1 - (w_i dt)^2 / 2, in both precisions; in FP64 every sample also follows the exact
discrete solution eta_i(n) = (dt c_i / sin theta_i) sin(n theta_i)."""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL
from test_oracle_dynamics import modal_basis

pytestmark = pytest.mark.gpu
MAT = dict(WORKLOAD_MATERIAL, elastic=1)


@pytest.fixture(scope="module")
def modes():
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=2)
    w, phi, m = modal_basis(oracle.Oracle(spec, MAT, 1e-7), spec.n_particles)
    dt = 0.9 * 2.0 / w.max()
    sel = [10, 37, len(w) - 1]
    c = np.array([1.0, -0.5, 0.2]) * 50.0
    return spec, w, phi, m, dt, sel, c


def _peak_frequency(x, dt):
    """Frequency of the largest FFT peak (Hann window, parabolic interpolation of log magnitude)."""
    X = np.abs(np.fft.rfft(x * np.hanning(len(x))))
    k = int(np.argmax(X[1:-1])) + 1
    a, b, g = np.log(X[k - 1]), np.log(X[k]), np.log(X[k + 1])
    d = 0.5 * (a - g) / (a - 2 * b + g)
    return (k + d) / (len(x) * dt)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_free_vibration_spectrum_matches_eigenvalues(modes, prec):
    spec, w, phi, m, dt, sel, c = modes
    bc = workloads.free_bc(spec.n_particles)
    bc.v0 = (phi[:, sel] @ c).reshape(-1, 6)
    g = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc, graph_chunk=-1)
    ns = 2048
    eta = np.zeros((ns, len(sel)))
    for n in range(ns):
        g.step(1)
        eta[n] = phi[:, sel].T @ (m * g.get_state(hist=False)[0].reshape(-1))
    g.close()
    theta = np.arccos(1.0 - 0.5 * (w[sel] * dt) ** 2)
    f_disc = theta / (2 * np.pi * dt)
    bin_hz = 1.0 / (ns * dt)
    for i in range(len(sel)):
        f = _peak_frequency(eta[:, i], dt)
        assert abs(f - f_disc[i]) < 0.05 * bin_hz, (i, f, f_disc[i], bin_hz)
    n = np.arange(1, ns + 1)[:, None]
    amp = dt * c / np.sin(theta)
    # FP64 to rounding; the FP32 facet pass perturbs forces by ~1e-7 relative
    tol = 1e-8 if prec == "fp64" else 1e-3
    np.testing.assert_allclose(eta, amp * np.sin(n * theta), rtol=0, atol=tol * np.abs(amp).max())
