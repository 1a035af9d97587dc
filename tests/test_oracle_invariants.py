"""Thermodynamic and monotonicity invariants of the oracle's facet law (Appendix A), on seeded random
strain cycles.

A closed strain cycle must not create energy: the work done on the facet, the sum of the tractions
times the strain increments (t is work-conjugate to e, Sec. 2), is zero for the elastic part and
positive wherever fracture, compressive hardening or friction dissipated energy.  With the
trapezoid rule the elastic part telescopes to zero exactly, so a negative total points at a branch
that returns energy it never stored (a wrong sign, a wrong unloading stiffness, a return mapping
that moves outside its surface).  The checks use no formula of the law itself:
  - the cycle's work is >= 0 (to rounding), and > 0 once the path went past every elastic limit;
  - e_max never decreases;
  - in the compression/friction branch t_N <= 0, and |t_T| <= sigma_s + mu0 |t_N| (the friction
    cap starts at sigma_s with slope mu0 and is concave);
  - every output is finite.
The material variants of App. A (k_t, E_d, r_s) are included."""
import zlib

import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

MAT = dict(WORKLOAD_MATERIAL)
L_EDGE = 3.0
VARIANTS = {
    "paper": {},
    "reload_k_t": {"k_t": 0.5},
    "densified_E_d": {"Ed_E0": 3.0},
    "shear_softening_r_s": {"r_s": 0.2},
    "all_three": {"k_t": 0.8, "Ed_E0": 2.0, "r_s": 0.1},
}


def _cycle(rng, e0, scale, knots=8, per=400):
    """A closed piecewise-linear strain path from 0 through random knots back to 0."""
    pts = [np.zeros(3)]
    for _ in range(knots):
        p = rng.uniform(-1.0, 1.0, 3) * scale * e0
        p[0] *= rng.choice([1.0, 0.3, 3.0])  # normal strain over a wider range than shear
        pts.append(p)
    pts.append(np.zeros(3))
    segs = [np.linspace(pts[k], pts[k + 1], per)[1:] for k in range(len(pts) - 1)]
    return np.concatenate([np.zeros((1, 3))] + segs)


def _work(t, path):
    dt_ = 0.5 * (t[1:] + t[:-1])
    de = np.diff(path, axis=0)
    w = np.sum(dt_ * de, axis=1)
    return w.sum(), np.abs(w).sum()


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_closed_cycles_dissipate_and_stay_admissible(variant):
    mat = dict(MAT, **VARIANTS[variant])
    e0 = mat["sigma_t"] / mat["E0"]
    rng = np.random.default_rng(zlib.crc32(variant.encode()))  # stable across processes, unlike hash()
    dissipated = 0
    for trial in range(12):
        scale = [0.5, 3.0, 12.0][trial % 3]
        path = _cycle(rng, e0, scale)
        eV = path[:, 0] * rng.uniform(0.2, 1.0)  # volumetric strain following the normal one
        t, em = oracle.facet_march(mat, L_EDGE, path, eV)
        assert np.isfinite(t).all() and np.isfinite(em).all()
        assert np.all(np.diff(em) >= 0.0), "e_max decreased"
        W, Wabs = _work(t, path)
        assert W >= -1e-6 * Wabs, (variant, trial, W, Wabs)
        # past every elastic limit: the fracture strength runs from sigma_t (pure tension) to
        # r_st sigma_t / sqrt(alpha) (pure shear)
        if em.max() > 1.5 * max(1.0, mat["r_st"] / np.sqrt(mat["alpha"])) * e0:
            assert W > 0.0
            dissipated += 1
        comp = path[:, 0] <= 0.0
        tT = np.hypot(t[:, 1], t[:, 2])
        assert np.all(t[comp, 0] <= 0.0)
        cap = mat["r_st"] * mat["sigma_t"] + mat["mu0"] * np.abs(t[comp, 0])
        assert np.all(tT[comp] <= cap * (1 + 1e-12) + 1e-12), (variant, trial)
    assert dissipated >= 2  # the larger cycles went past every elastic limit and dissipated


def test_elastic_cycle_does_no_work():
    """Inside the elastic range (|e| well below the limit) every cycle's work is zero to rounding."""
    rng = np.random.default_rng(5)
    e0 = MAT["sigma_t"] / MAT["E0"]
    for _ in range(5):
        path = _cycle(rng, e0, 0.2)
        t, _ = oracle.facet_march(MAT, L_EDGE, path, path[:, 0])
        W, Wabs = _work(t, path)
        assert abs(W) <= 1e-9 * Wabs


def test_friction_unloads_elastically_from_the_cap():
    """App. A.3 is incremental: under a constant compressive t_N, shearing past the friction cap
    slides at the cap value s, and unloading then runs elastically (slope alpha E0) from s down to the
    reverse cap -s, not back along the loading line.  s is read from the loading plateau; nothing
    of the cap formula is used.  Normal strain held in the elastic compressive range with
    e_V = e_N (no deviatoric strain)."""
    E0, a = MAT["E0"], MAT["alpha"]
    eN = -0.2 * MAT["sigma_c0"] / E0
    ramp = np.linspace(0.0, eN, 200)
    s_est = MAT["r_st"] * MAT["sigma_t"] + MAT["mu0"] * abs(E0 * eN)  # only sizes the path
    e1 = 3.0 * s_est / (a * E0)
    up = np.linspace(0.0, e1, 3001)[1:]
    down = np.linspace(e1, e1 - 4.0 * s_est / (a * E0), 4001)[1:]
    path = np.concatenate([np.stack([ramp, 0 * ramp, 0 * ramp], 1),
                           np.stack([np.full_like(up, eN), up, 0 * up], 1),
                           np.stack([np.full_like(down, eN), down, 0 * down], 1)])
    t, _ = oracle.facet_march(MAT, L_EDGE, path, path[:, 0])
    n0, n1 = len(ramp), len(ramp) + len(up)
    np.testing.assert_allclose(t[n0:, 0], E0 * eN, rtol=1e-12)
    assert np.all(t[:, 2] == 0.0)
    s = t[n1 - 1, 1]
    assert s > 0.5 * s_est
    # loading: elastic up to the cap, then sliding at it
    np.testing.assert_allclose(t[n0:n1, 1], np.minimum(a * E0 * up, s), rtol=1e-9, atol=1e-12 * s)
    # unloading: elastic from the cap down to the reverse cap
    np.testing.assert_allclose(t[n1:, 1], np.maximum(s - a * E0 * (e1 - down), -s), rtol=1e-9, atol=1e-9 * s)
