"""Pins of the oracle's facet constitutive law (paper Appendix A) to closed forms and invariants."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300.workloads import TABLE_A, WORKLOAD_MATERIAL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MAT = dict(WORKLOAD_MATERIAL)
L_EDGE = 3.0  # facet length (mm), well below l_t


def march(mat, path, eV_of=None, l=L_EDGE):
    """Drive one facet along a strain path (rows of e); returns tractions and e_max per point."""
    path = np.asarray(path, float).reshape(-1, 3)
    eV = eV_of(path.T) if eV_of else path[:, 0]
    return oracle.facet_march(mat, l, path, eV)


def test_table_a_fracture_energy_golden():
    """Appendix A prints G_t = 0.0491 N/mm next to its definition l_t sigma_t^2 / (2 E0)."""
    g = json.load(open(os.path.join(GOLDEN, "table_a.json")))
    Gt = g["l_t_mm"] * g["sigma_t_MPa"] ** 2 / (2.0 * g["E0_MPa"])
    assert abs(Gt - g["G_t_N_per_mm"]) < 5e-5
    # The parameter set the workloads build on is Table A.
    assert TABLE_A["E0"] == g["E0_MPa"] and TABLE_A["l_t"] == g["l_t_mm"] and TABLE_A["sigma_t"] == g["sigma_t_MPa"]


@pytest.mark.parametrize("e", [(1e-6, 2e-6, -1e-6), (-2e-5, 3e-6, 1e-6), (0.0, 1e-6, 0.0), (3e-6, 0.0, 0.0)])
def test_elastic_range_is_t_equals_E_e(e):
    """Sec. 2: t = E0 diag(1, alpha, alpha) e inside the elastic domain of both branches."""
    e = np.array(e)
    t, _ = oracle.facet_law(MAT, L_EDGE, e, e, e[0], np.zeros(3), 0.0)
    E = MAT["E0"] * np.array([1.0, MAT["alpha"], MAT["alpha"]])
    np.testing.assert_allclose(t, E * e, rtol=1e-13, atol=1e-300)


def test_elastic_through_sign_change():
    """An elastic path that crosses e_N = 0 stays on t = E e (both branches share the history)."""
    path = [(s, 0.3 * abs(s) + 1e-7, -0.2e-6) for s in np.linspace(2e-5, -2e-5, 41)]
    ts, _ = march(MAT, path)
    E = MAT["E0"] * np.array([1.0, MAT["alpha"], MAT["alpha"]])
    np.testing.assert_allclose(ts, E * np.array(path), rtol=1e-10, atol=1e-12)


def test_uniaxial_tension_peak_and_fracture_energy():
    """Pure tension (omega = pi/2): peak t_N = sigma_t at e_N = sigma_t / E0, and the work per unit
    area l * integral t de to full separation equals G_t = l_t sigma_t^2 / (2 E0) (App. A.1)."""
    E0, st, lt = MAT["E0"], MAT["sigma_t"], MAT["l_t"]
    e0 = st / E0
    Ht = 2 * E0 / (lt / L_EDGE - 1)
    e_end = e0 + 40 * st / Ht
    s = np.linspace(0.0, e_end, 400001)
    ts, em = march(MAT, [(x, 0.0, 0.0) for x in s])
    tN = ts[:, 0]
    assert abs(tN.max() - st) < 1e-3 * st
    assert abs(s[np.argmax(tN)] - e0) < 2 * (s[1] - s[0])
    work = L_EDGE * np.trapezoid(tN, s)
    Gt = lt * st ** 2 / (2 * E0)
    assert abs(work - Gt) < 2e-3 * Gt
    assert np.all(ts[:, 1:] == 0.0)
    np.testing.assert_allclose(em, s, rtol=0, atol=0)  # e_max tracks the monotonic effective strain


def test_unload_elastic_to_zero_and_hold():
    """After softening, unloading is elastic down to t = 0 and stays at 0 (App. A.1, k_t = 0)."""
    E0, st = MAT["E0"], MAT["sigma_t"]
    e0 = st / E0
    up = np.linspace(0, 3 * e0, 3001)
    down = np.linspace(3 * e0, 0.2 * e0, 2801)[1:]
    ts, _ = march(MAT, [(x, 0, 0) for x in np.concatenate([up, down])])
    t_top = ts[len(up) - 1, 0]
    tdown = ts[len(up):, 0]
    expect = np.maximum(t_top - E0 * (3 * e0 - down), 0.0)
    np.testing.assert_allclose(tdown, expect, rtol=1e-9, atol=1e-12)
    assert tdown[-1] == 0.0


@pytest.mark.parametrize("ratio", [0.05, 0.3, 1.0, 3.0, 20.0])
def test_peak_tractions_lie_on_tension_shear_parabola(ratio):
    """The strength limit sigma_0(omega) places the peak tractions on t_T^2 = sigma_s^2 (1 - t_N/sigma_t)
    (t_T = sqrt(t_M^2 + t_L^2), sigma_s = r_st sigma_t): an independent statement of the same envelope."""
    st, r = MAT["sigma_t"], MAT["r_st"]
    eN_end = 3e-4
    s = np.linspace(0, 1, 60001)
    path = [(x * eN_end, ratio * x * eN_end * 0.6, ratio * x * eN_end * 0.8) for x in s]
    ts, _ = march(MAT, path)
    teff = np.sqrt(ts[:, 0] ** 2 + (ts[:, 1] ** 2 + ts[:, 2] ** 2) / MAT["alpha"])
    k = int(np.argmax(teff))
    tN, tT = ts[k, 0], math.hypot(ts[k, 1], ts[k, 2])
    lhs, rhs = tT ** 2, (r * st) ** 2 * (1 - tN / st)
    assert abs(lhs - rhs) < 2e-3 * (r * st) ** 2


def test_pure_shear_peak_sigma_s_both_sides_of_zero():
    """Shear strength sigma_s = r_st sigma_t is reached both at e_N = 0+ (fracture branch, omega -> 0)
    and at e_N = 0 (friction branch, sigma_bs(0) = sigma_s): the two branches meet continuously."""
    ss = MAT["r_st"] * MAT["sigma_t"]
    s = np.linspace(0, 2e-3, 200001)
    ts_f, _ = march(MAT, [(1e-12, x, 0.0) for x in s])
    ts_c, _ = march(MAT, [(0.0, x, 0.0) for x in s])
    assert abs(ts_f[:, 1].max() - ss) < 1e-3 * ss
    assert abs(ts_c[:, 1].max() - ss) < 1e-9 * ss
    # friction branch: perfectly plastic plateau at sigma_s (r_s = 0, t_N = 0)
    assert abs(ts_c[-1, 1] - ss) < 1e-9 * ss


def test_softening_slope_scales_with_omega_power():
    """Initial post-peak slope of the effective traction is -H_0(omega); with H_s = 0 its ratio at two
    coupling angles is (omega_1 / omega_2)^n_t (App. A.1)."""
    alpha = MAT["alpha"]

    def slope(omega):
        # proportional path at fixed omega: e_N = e sin(omega), sqrt(alpha) e_M = e cos(omega)
        e_path = np.linspace(0, 4e-4, 400001)
        path = np.stack([e_path * math.sin(omega), e_path * math.cos(omega) / math.sqrt(alpha),
                         np.zeros_like(e_path)], 1)
        ts, _ = march(MAT, path)
        teff = np.sqrt(ts[:, 0] ** 2 + (ts[:, 1] ** 2 + ts[:, 2] ** 2) / alpha)
        k = int(np.argmax(teff))
        de = e_path[1] - e_path[0]
        j = k + 200
        return (teff[j + 100] - teff[j]) / (100 * de), teff[k]

    s1, _ = slope(0.3)
    s2, _ = slope(1.2)
    # slope = -H0 * exp(...) ~ -H0 (1 - H0 de / sigma0 ...) close to the peak; compare log ratio
    assert abs(math.log(s1 / s2) - MAT["n_t"] * math.log(0.3 / 1.2)) < 0.02


def test_hydrostatic_compression_plateau_hardening_exponential():
    """Hydrostatic path e_N = e_V (e_D = 0, r_DV = 0, H_c = H_c0): t_N = -E0 s until s = e_c0, then
    -(sigma_c0 + (s - e_c0) H_c0) up to e_c1 = k_c0 e_c0, then the exponential piece (App. A.2)."""
    E0, sc0, kc0 = MAT["E0"], MAT["sigma_c0"], MAT["kc0"]
    Hc0 = MAT["Hc0_E0"] * E0
    ec0 = sc0 / E0
    ec1 = kc0 * ec0
    s = np.linspace(0, 1.6 * ec1, 16001)
    ts, _ = march(MAT, [(-x, 0, 0) for x in s], eV_of=lambda e: e[0])
    tN = -ts[:, 0]
    sc1 = sc0 + (ec1 - ec0) * Hc0
    expect = np.where(s <= ec0, E0 * s,
                      np.where(s <= ec1, sc0 + (s - ec0) * Hc0, sc1 * np.exp((s - ec1) * Hc0 / sc1)))
    np.testing.assert_allclose(tN, expect, rtol=1e-9)
    # the boundary is continuous at e_c1 and the slope there is H_c0 from both sides
    k = int(np.searchsorted(s, ec1))
    dl = (tN[k - 1] - tN[k - 11]) / (s[k - 1] - s[k - 11])
    dr = (tN[k + 11] - tN[k + 1]) / (s[k + 11] - s[k + 1])
    assert abs(dl - Hc0) < 1e-6 * Hc0 and abs(dr - Hc0) < 2e-3 * Hc0


def test_deviatoric_softens_hardening_modulus():
    """Hardening slope of the compressive boundary in terms of -e_DV is H_c0 on a hydrostatic path
    (r_DV = 0 <= k_c1) and tends to H_c1 when the facet is compressed far more than its tetrahedron
    (r_DV = |e_D| / (e_V0 - e_V) >> k_c1), App. A.2."""
    E0, sc0 = MAT["E0"], MAT["sigma_c0"]
    ec0 = sc0 / E0
    Hc0, Hc1 = MAT["Hc0_E0"] * E0, MAT["Hc1_E0"] * E0

    def hardening_slope(k):
        # e_N = -k s, e_V = -s: -e_DV = s (beta = 0), deviatoric part (k - 1) s
        s = np.linspace(0, 1.5 * ec0, 15001)
        ts, _ = march(MAT, [(-k * x, 0, 0) for x in s], eV_of=lambda e: e[0] / k)
        tN = -ts[:, 0]
        return (tN[-1] - tN[-201]) / (s[-1] - s[-201]), tN

    h_hyd, _ = hardening_slope(1.0)
    assert abs(h_hyd - Hc0) < 1e-6 * Hc0
    # r_DV = 0.5 s / (e_V0 + s) stays below k_c1 = 1 on the whole path: no softening of H_c yet
    assert MAT["kc1"] == 1.0
    h_mild, _ = hardening_slope(1.5)
    assert abs(h_mild - Hc0) < 1e-6 * Hc0
    h_dev, tN = hardening_slope(200.0)
    assert Hc1 <= h_dev < 1.01 * Hc1
    # plateau sigma_c0 while -e_DV < e_c0 even though the facet strain is far beyond e_c0
    _, tN_short = hardening_slope(200.0)
    assert abs(tN_short[int(0.5 * len(tN_short))] - sc0) < 1e-9 * sc0


def test_boundary_without_compaction_stays_at_sigma_c0():
    """App. A.2: while the tetrahedron does not compact (-e_DV <= 0), sigma_bc = sigma_c0 however far
    the facet itself is compressed (no hardening branch is reached)."""
    ec0 = MAT["sigma_c0"] / MAT["E0"]
    s = np.linspace(0.0, 4.0 * ec0, 4001)
    for eV in (0.0, 2e-4):
        ts, _ = march(MAT, [(-x, 0.0, 0.0) for x in s], eV_of=lambda e: np.full_like(e[0], eV))
        tN = -ts[:, 0]
        np.testing.assert_allclose(tN, np.minimum(MAT["E0"] * s, MAT["sigma_c0"]), rtol=1e-12)


def test_beta_one_makes_the_boundary_a_function_of_e_N_alone():
    """App. A.2 with beta = 1: e_DV = e_V + (e_N - e_V) = e_N, so with the deviatoric softening of
    H_c switched off (k_c1 above any r_DV) the compressive response along e_N does not depend on the
    tetrahedron's volumetric strain: a facet compressed three times faster than its tetrahedron follows
    the hydrostatic curve point by point."""
    mat = dict(MAT, beta=1.0, kc1=1e9)
    ec1 = mat["kc0"] * mat["sigma_c0"] / mat["E0"]
    s = np.linspace(0.0, 1.5 * ec1, 15001)
    hyd, _ = march(mat, [(-x, 0.0, 0.0) for x in s], eV_of=lambda e: e[0])
    dev, _ = march(mat, [(-x, 0.0, 0.0) for x in s], eV_of=lambda e: e[0] / 3.0)
    assert -hyd[-1, 0] > mat["sigma_c0"] * 1.5  # the path went well into hardening
    np.testing.assert_allclose(dev[:, 0], hyd[:, 0], rtol=1e-12)
    # with beta = 0 the same two paths differ (e_DV = e_V), which is what makes the check bite
    h0, _ = march(dict(mat, beta=0.0), [(-x, 0.0, 0.0) for x in s], eV_of=lambda e: e[0] / 3.0)
    assert abs(h0[-1, 0] - hyd[-1, 0]) > 0.05 * abs(hyd[-1, 0])


def test_friction_cap_and_initial_slope_mu0():
    """Under fixed compression t_N the shear saturates at sigma_bs(t_N); at t_N -> 0 the cap is sigma_s
    and grows with slope mu_0 per unit compression (App. A.3)."""
    ss = MAT["r_st"] * MAT["sigma_t"]

    def plateau(eN):
        s = np.linspace(0, 6e-3, 60001)
        ts, _ = march(MAT, [(eN, x, 0.0) for x in s])
        return ts[-1, 0], ts[-1, 1]

    tN0, c0 = plateau(0.0)
    assert tN0 == 0.0 and abs(c0 - ss) < 1e-9 * ss
    d = 1e-6
    tN1, c1 = plateau(-d)
    assert abs((c1 - c0) / (-tN1) - MAT["mu0"]) < 1e-3
    tN2, c2 = plateau(-2e-3)  # deep compression (elastic: -t_N < sigma_c0)
    sN0, mu0 = MAT["sigma_N0"], MAT["mu0"]
    assert abs(c2 - (ss + mu0 * sN0 * (1 - math.exp(tN2 / sN0)))) < 1e-9 * c2


def test_friction_cap_slope_runs_from_mu0_to_mu_inf():
    """App. A.3: the friction cap sigma_bs(t_N) rises with slope mu_0 at t_N -> 0 and tends to slope
    mu_inf under deep compression.  A material with mu_inf > 0 (the workloads use 0) and a compressive
    yield stress far above the tested range, so t_N = E0 e_N stays elastic down to -12 sigma_N0.  The
    slopes are finite differences of saturated plateaus; no formula of the cap is used."""
    mat = dict(MAT, mu_inf=0.05, sigma_c0=1e6)
    E0, a, sN0 = mat["E0"], mat["alpha"], mat["sigma_N0"]

    def plateau(tN):
        eN = tN / E0
        cap = mat["r_st"] * mat["sigma_t"] + mat["mu0"] * abs(tN)  # only sizes the path
        down = [(x, 0.0, 0.0) for x in np.linspace(0.0, eN, 200)]
        side = [(eN, x, 0.0) for x in np.linspace(0.0, 3.0 * cap / (a * E0), 6001)[1:]]
        ts, _ = march(mat, down + side)
        np.testing.assert_allclose(ts[-1, 0], tN, rtol=1e-12)
        assert ts[-1, 1] == ts[-2, 1]  # sliding at the cap
        return ts[-1, 1]

    d = 1e-3
    assert abs((plateau(-d) - plateau(0.0)) / d - mat["mu0"]) < 1e-5
    assert abs((plateau(-12 * sN0) - plateau(-10 * sN0)) / (2 * sN0) - mat["mu_inf"]) < 1e-4


@pytest.mark.parametrize("eN", [1e-160, 1e-200, 5e-324])
def test_vanishing_tensile_strain_is_elastic_not_nan(eN):
    """At e_N > 0 so small that its square underflows, t / e is 0/0; the law's elastic limit t = E e
    must come out (a loading wave leaves such strains ahead of its front)."""
    e = np.array([eN, 0.0, 0.0])
    t, em = oracle.facet_law(MAT, L_EDGE, e, e, 0.0, np.zeros(3), 0.0)
    assert np.all(np.isfinite(t)) and t[0] == MAT["E0"] * eN
    assert em == math.sqrt(eN * eN)  # e_max takes the (vanishing) effective strain, |e_N| here
    # with shear strains of the same size the response is t = E0 diag(1, alpha, alpha) e
    e = np.array([eN, eN, -eN])
    t, _ = oracle.facet_law(MAT, L_EDGE, e, e, 0.0, np.zeros(3), 0.0)
    E = MAT["E0"] * np.array([1.0, MAT["alpha"], MAT["alpha"]])
    np.testing.assert_array_equal(t, E * e)
