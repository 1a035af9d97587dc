"""Pins of the oracle's unload/reload variants of Appendix A (k_t > 0, E_d != E0, r_s != 0) to closed
forms: the tensile reload rule, the densified unloading stiffness, and the shear fracture energy with
H_s = r_s E0."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

MAT = dict(WORKLOAD_MATERIAL)
L_EDGE = 3.0


def march(mat, path, eV=None):
    path = np.asarray(path, float).reshape(-1, 3)
    return oracle.facet_march(mat, L_EDGE, path, path[:, 0] if eV is None else eV)


@pytest.mark.parametrize("k_t", [0.0, 0.5, 1.0])
def test_tensile_reload_waits_for_e_tr(k_t):
    """Pure tension: soften to e_max = 3 e0, unload to zero traction (at e_u = e_max - t_top / E0) and
    on to 0.3 e_u, reload to e_max.  On reloading the traction stays zero until
    e_tr = k_t (e_max - sigma_bt / E0) = k_t e_u (or the reversal point, if later), then rises with
    slope E0 (App. A.1): t = E0 <e - max(0.3 e_u, k_t e_u)>, at most t_top."""
    mat = dict(MAT, k_t=k_t)
    E0, st = mat["E0"], mat["sigma_t"]
    e0 = st / E0
    up = np.linspace(0, 3 * e0, 3001)
    ts, _ = march(mat, [(x, 0, 0) for x in up])
    t_top = ts[-1, 0]
    e_u = 3 * e0 - t_top / E0
    down = np.linspace(3 * e0, 0.3 * e_u, 2001)[1:]
    back = np.linspace(0.3 * e_u, 3 * e0, 4001)[1:]
    path = np.concatenate([up, down, back])
    ts, em = march(mat, [(x, 0, 0) for x in path])
    t_back = ts[len(up) + len(down):, 0]
    start = max(0.3 * e_u, k_t * e_u)
    expect = np.minimum(E0 * np.maximum(back - start, 0.0), t_top)
    np.testing.assert_allclose(t_back, expect, rtol=1e-9, atol=1e-9 * st)
    assert np.all(em[len(up):] == em[len(up) - 1]), "e_max does not change below the envelope"


def test_reload_rule_only_delays_reloading():
    """On a mixed-mode cyclic path with noise, k_t > 0 can only hold the effective traction at zero
    longer than k_t = 0 (where e_tr = 0 and reloading is elastic at once): it never exceeds the
    k_t = 0 traction, and is below it somewhere."""
    rng = np.random.default_rng(4)
    e0 = MAT["sigma_t"] / MAT["E0"]
    knots = np.array([[0, 0, 0], [3, 1, 0.5], [0.5, 0.8, 0.3], [4, 0.2, -1], [1, -1, 0], [5, 2, 1]]) * e0
    path = np.concatenate([np.linspace(knots[i], knots[i + 1], 500) for i in range(len(knots) - 1)])
    path += 1e-3 * e0 * rng.standard_normal(path.shape)
    a, _ = march(dict(MAT, k_t=0.0), path)
    t_eff = np.sqrt(a[:, 0] ** 2 + (a[:, 1] ** 2 + a[:, 2] ** 2) / MAT["alpha"])
    assert np.isfinite(a).all()
    b, _ = march(dict(MAT, k_t=0.5), path)
    t_eff_b = np.sqrt(b[:, 0] ** 2 + (b[:, 1] ** 2 + b[:, 2] ** 2) / MAT["alpha"])
    assert np.all(t_eff_b <= t_eff + 1e-9 * MAT["sigma_t"])
    assert np.any(t_eff_b < t_eff - 1e-3 * MAT["sigma_t"])


def test_densified_unloading_stiffness_Ed():
    """Hydrostatic compression (e_V = e_N, so e_D = 0 and H_c = H_c0) into linear hardening, then
    unloading: the normal stiffness is E_d while -t_N,old > sigma_c0 and E0 after (App. A.2)."""
    Ed_E0 = 3.0
    mat = dict(MAT, Ed_E0=Ed_E0)
    E0, sc0 = mat["E0"], mat["sigma_c0"]
    Ed = Ed_E0 * E0
    ec0 = sc0 / E0
    Hc0 = mat["Hc0_E0"] * E0
    e_pk = -6e-3
    assert -e_pk <= mat["kc0"] * ec0  # linear hardening range
    load = np.linspace(0.0, e_pk, 6001)
    unload = np.linspace(e_pk, 0.0, 6001)[1:]
    path = np.concatenate([load, unload])
    ts, _ = march(mat, [(x, 0.0, 0.0) for x in path])
    s_pk = sc0 + (-e_pk - ec0) * Hc0
    assert abs(ts[len(load) - 1, 0] + s_pk) < 1e-9 * s_pk
    # closed form of the unloading branch
    d = unload - e_pk
    d1 = (s_pk - sc0) / Ed  # E_d until -t_N = sigma_c0 (the step that crosses uses E_d)
    t_expect = np.where(d <= d1, -s_pk + Ed * d, np.nan)
    i1 = np.flatnonzero(d <= d1)
    np.testing.assert_allclose(ts[len(load):, 0][i1], t_expect[i1], rtol=1e-10)
    # after the crossing step the slope is E0 down to zero traction, then zero
    k = i1[-1] + 1
    t_k = ts[len(load) + k - 1, 0] + Ed * (unload[k] - unload[k - 1])
    rest = ts[len(load) + k:, 0]
    expect_rest = np.minimum(t_k + E0 * (unload[k:] - unload[k]), 0.0)
    np.testing.assert_allclose(rest, expect_rest, rtol=1e-9, atol=1e-9 * sc0)


def test_shear_fracture_energy_with_H_s():
    """Shear-dominated fracture (omega -> 0, n_t = 1 so (2 omega / pi)^n_t -> 0): sigma_0 ->
    sigma_s / sqrt(alpha) and H_0 -> H_s / alpha with H_s = r_s E0 (App. A.1).  The work of the
    effective traction to full softening, sigma_0 e0 / 2 + sigma_0^2 / H_0, closed form."""
    r_s = 0.2
    mat = dict(MAT, r_s=r_s, n_t=1.0)
    E0, a = mat["E0"], mat["alpha"]
    s0 = mat["r_st"] * mat["sigma_t"] / math.sqrt(a)
    H0 = r_s * E0 / a
    e0 = s0 / E0
    e_end = e0 + 40 * s0 / H0
    eT = np.linspace(0.0, e_end / math.sqrt(a), 400001)
    path = np.stack([1e-10 * eT, eT, 0 * eT], 1)
    ts, _ = march(mat, path)
    e_eff = np.sqrt(path[:, 0] ** 2 + a * path[:, 1] ** 2)
    t_eff = np.sqrt(ts[:, 0] ** 2 + ts[:, 1] ** 2 / a)
    assert abs(t_eff.max() - s0) < 1e-3 * s0
    work = np.trapezoid(t_eff, e_eff)
    expect = s0 * e0 / 2 + s0 ** 2 / H0
    assert abs(work - expect) < 2e-3 * expect


def test_H_s_does_not_act_in_pure_tension():
    """(2 omega / pi)^n_t = 1 at omega = pi/2, so H_0 = H_t whatever r_s is."""
    e0 = MAT["sigma_t"] / MAT["E0"]
    path = [(x, 0.0, 0.0) for x in np.linspace(0, 5 * e0, 2001)]
    a, _ = march(dict(MAT, r_s=0.0), path)
    b, _ = march(dict(MAT, r_s=0.3), path)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)
