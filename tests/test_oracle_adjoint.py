"""Pins of the oracle's derivatives with respect to per-facet E0, alpha, sigma_t.

The oracle differentiates its own law and step with forward-mode dual numbers.  That derivative is
checked here against what does not depend on it:
  * central finite differences of the plain FP64 law, in every branch of App. A;
  * closed forms on two fully constrained particles: pure tension through the peak into softening
    (App. A.1 with omega = pi/2: t = E0 e, then t = sigma_t exp(-H_t (e - e0) / sigma_t)), and pure
    shear up to the friction cap (App. A.3 at t_N = 0: t_M = alpha E0 e_M, then sigma_s = r_st sigma_t);
  * central finite differences of whole trajectories of a cube (free dynamics, tension plus shear,
    before the macroscopic peak with softening facets), single-facet and dense directions;
  * the objective itself against the time mean of the reactions reported by the energy routine.
"""
import math

import numpy as np
import pytest

import oracle
from law_cases import CASES, IN_SCALE, L_FACET, case, law_point
from paper_2603_13190_gb300 import specimen, workloads
from paper_2603_13190_gb300.specimen import Specimen
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

MAT = dict(WORKLOAD_MATERIAL)
SCALE = IN_SCALE


def _sigma_bs(tN, mat=MAT):
    dmu = mat["mu0"] - mat["mu_inf"]
    return mat["r_st"] * mat["sigma_t"] + dmu * mat["sigma_N0"] - mat["mu_inf"] * tN - dmu * mat["sigma_N0"] * math.exp(
        tN / mat["sigma_N0"])


@pytest.mark.parametrize("name", sorted(CASES))
def test_law_jacobian_matches_central_differences(name):
    path, eV, i, mat = case(name)
    x = law_point(path, eV, i, mat)
    out, jac = oracle.facet_law_jacobian(mat, L_FACET, x)
    # the point lies in the intended branch
    e, t_old, em_old = x[0:3], x[7:10], x[10]
    eeff = math.sqrt(e[0] ** 2 + MAT["alpha"] * (e[1] ** 2 + e[2] ** 2))
    teff = math.sqrt(out[0] ** 2 + (out[1] ** 2 + out[2] ** 2) / MAT["alpha"])
    if name == "fracture_elastic":
        assert abs(teff - MAT["E0"] * eeff) < 1e-9 * teff
    elif name == "fracture_softening":
        assert out[3] == eeff and teff < 0.5 * MAT["E0"] * eeff
    elif name == "fracture_unloading":
        assert em_old > eeff and 0 < teff < MAT["E0"] * eeff
    elif name == "friction_return":
        assert abs(math.hypot(out[1], out[2]) - _sigma_bs(out[0])) < 1e-12 * _sigma_bs(out[0])
    elif name.startswith("hardening"):
        assert out[0] < -MAT["sigma_c0"] * 1.01
    elif name == "normal_clamped_at_zero":
        assert out[0] == 0.0 and t_old[0] < -MAT["sigma_c0"]
    elif name == "reload_crossing_e_tr":
        assert np.all(t_old == 0.0) and teff > 0 and out[3] > eeff
    elif name == "densified_unloading":
        assert -t_old[0] > MAT["sigma_c0"] and x[3] > 0
    elif name == "shear_softening_H_s":
        assert out[3] == eeff and teff < 0.5 * MAT["E0"] * eeff
    # central differences at two step sizes (both must agree with the Jacobian: no kink in between)
    for h in (1e-5, 1e-6):
        fd = np.zeros((4, 14))
        for c in range(14):
            hh = h * max(abs(x[c]), SCALE[c])
            xp, xm = x.copy(), x.copy()
            xp[c] += hh
            xm[c] -= hh
            fd[:, c] = (oracle.facet_law_jacobian(mat, L_FACET, xp)[0] - oracle.facet_law_jacobian(mat, L_FACET, xm)[0]) / (2 * hh)
        assert np.abs(fd - jac).max() <= 1e-7 * np.abs(jac).max(), (name, h, np.abs(fd - jac).max())


def test_law_jacobian_elastic_mode_and_vanishing_strain():
    el = dict(MAT, elastic=1)
    x = np.array([2e-5, -1e-5, 3e-6, 1e-6, 0, 0, 0, 0.5, 0.1, 0.0, 0.0, MAT["E0"], MAT["alpha"], MAT["sigma_t"]])
    out, jac = oracle.facet_law_jacobian(el, L_FACET, x)
    E0, a = MAT["E0"], MAT["alpha"]
    expect = np.zeros((4, 14))
    expect[0, 0], expect[1, 1], expect[2, 2] = E0, a * E0, a * E0
    expect[0, 11], expect[1, 11], expect[2, 11] = x[0], a * x[1], a * x[2]
    expect[1, 12], expect[2, 12] = E0 * x[1], E0 * x[2]
    expect[3, 10] = 1.0  # e_max passes through unchanged
    np.testing.assert_allclose(jac, expect, rtol=1e-15, atol=0)
    # vanishing effective strain in the fracture branch: t = E e and its derivative
    x = np.array([1e-200, 0, 0, 1e-200, 0, 0, 0, 0, 0, 0, 0, E0, a, MAT["sigma_t"]])
    out, jac = oracle.facet_law_jacobian(MAT, L_FACET, x)
    assert jac[0, 0] == E0 and jac[0, 11] == 1e-200 and np.all(np.isfinite(jac))


def _two_particles(dt):
    """Particles at 0 and (l, 0, 0) sharing one facet normal to x (A = h^2 / 2), no tetrahedron."""
    l, h = L_FACET, 2.0
    x = np.array([[0.0, 0.0, 0.0], [l, 0.0, 0.0]])
    vtx = np.array([[l / 2, -h / 3, -h / 3, l / 2, 2 * h / 3, -h / 3, l / 2, -h / 3, 2 * h / 3]])
    spec = Specimen(x=x, diameter=np.ones(2), tets=np.zeros((0, 4), np.int32), facet_pi=np.array([0], np.int32),
                    facet_pj=np.array([1], np.int32), facet_tet=np.array([-1], np.int32), facet_vtx=vtx, edge=l,
                    d_min=1.0, d_max=1.0)
    return spec, h * h / 2.0


def _constrained_pull(dof, speed, dt):
    spec, A = _two_particles(dt)
    bc = workloads.free_bc(2)
    bc.mask[:, :] = workloads.FIXED
    bc.mask[1, dof] = workloads.PRESCRIBED
    bc.vel[1, dof] = speed
    o = oracle.Oracle(spec, MAT, dt, bc, mass=np.full(2, 1e-6), inertia=np.full((2, 3), 1e-7))
    seed = np.zeros((2, 6))
    seed[1, dof] = 1.0
    return o, seed, A


def _unit_dirs():
    d = np.ones((1, 1))
    z = np.zeros((1, 1))
    return [(d, z, z), (z, d, z), (z, z, d)]


def test_two_particle_tension_through_softening_closed_form():
    """J = (1/K) sum_n A t_N(n) along e_N(n) = n dt v / l: elastic up to e0 = sigma_t / E0, then
    t_N = sigma_t exp(X), X = -H_t (e - e0) / sigma_t, H_t = 2 E0 / (l_t / l - 1).  Closed forms:
    dt_N/dE0 = e (elastic) or -t_N H_t e / (E0 sigma_t) (softening); dt_N/dsigma_t = 0 (elastic) or
    exp(X) (1 + H_t e / sigma_t) (softening); nothing depends on alpha (e_T = 0)."""
    dt, v, K = 1e-7, 60.0, 100
    o, seed, A = _constrained_pull(0, v, dt)
    E0, st = MAT["E0"], MAT["sigma_t"]
    Ht = 2.0 * E0 / (MAT["l_t"] / L_FACET - 1.0)
    e0 = st / E0
    J = gE = gs = 0.0
    nsoft = 0
    for n in range(1, K + 1):
        e = n * dt * v / L_FACET
        if e <= e0:
            J += A * E0 * e
            gE += A * e
        else:
            nsoft += 1
            X = -Ht * (e - e0) / st
            t = st * math.exp(X)
            J += A * t
            gE += -A * t * Ht * e / (E0 * st)
            gs += A * math.exp(X) * (1.0 + Ht * e / st)
    assert 20 < nsoft < K - 20
    got = [o.tangent(K, seed, *d) for d in _unit_dirs()]
    np.testing.assert_allclose(got[0][0], J / K, rtol=1e-9)
    np.testing.assert_allclose(got[0][1][0], gE / K, rtol=1e-8)
    np.testing.assert_allclose(got[2][1][0], gs / K, rtol=1e-8)
    assert abs(got[1][1][0]) < 1e-12 * abs(gE / K) * E0


def test_two_particle_shear_up_to_friction_cap_closed_form():
    """e_N = 0 (compression branch, t_N = 0), e_M(n) = n dt v / l: t_M = alpha E0 e_M until the cap
    sigma_bs(0) = r_st sigma_t, then the cap.  dt_M/dalpha = E0 e_M and dt_M/dE0 = alpha e_M before
    the cap; dt_M/dsigma_t = r_st at the cap."""
    dt, v, K = 1e-7, 500.0, 100
    o, seed, A = _constrained_pull(1, v, dt)
    E0, a = MAT["E0"], MAT["alpha"]
    cap = MAT["r_st"] * MAT["sigma_t"]
    J = gE = ga = gs = 0.0
    ncap = 0
    for n in range(1, K + 1):
        e = n * dt * v / L_FACET
        if a * E0 * e <= cap:
            J += A * a * E0 * e
            gE += A * a * e
            ga += A * E0 * e
        else:
            ncap += 1
            J += A * cap
            gs += A * MAT["r_st"]
    assert 20 < ncap < K - 20
    got = [o.tangent(K, seed, *d) for d in _unit_dirs()]
    np.testing.assert_allclose(got[0][0], J / K, rtol=1e-9)
    np.testing.assert_allclose([got[0][1][0], got[1][1][0], got[2][1][0]], [gE / K, ga / K, gs / K], rtol=1e-8)


@pytest.fixture(scope="module")
def cube():
    """10 mm cube pulled (top u_z at 20 mm/s) and sheared (top u_x at 8 mm/s) for 300 steps: before the
    macroscopic peak, with softening facets."""
    spec = specimen.make_cube_specimen(10.0, 2.0, 4.0, 120, seed=31)
    bc = workloads.uniaxial_tension_bc(spec, velocity=20.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 0] = workloads.PRESCRIBED
    bc.vel[top, 0] = 8.0
    dt = 0.9 * oracle.Oracle(spec, MAT, 1e-7, bc).critical_dt()
    seed = np.zeros((spec.n_particles, 6))
    seed[top, 2] = 1.0
    return spec, bc, dt, seed, 300


def test_objective_is_time_mean_of_reported_reactions_and_state_is_kept(cube):
    spec, bc, dt, seed, K = cube
    o = oracle.Oracle(spec, MAT, dt, bc)
    J, _ = o.tangent(K, seed)
    q0 = o.get_state()[0]
    assert np.array_equal(q0, np.zeros_like(q0)), "tangent must not advance the model"
    Rz = []
    for _ in range(K):
        o.step(1)
        Rz.append(o.energy()[1][8])  # prescribed DOFs, z component: the seeded top face
    np.testing.assert_allclose(J, np.mean(Rz), rtol=1e-12)


def test_objective_counts_fixed_and_prescribed_seeds(cube):
    """The objective sums seeded reactions over every constrained DOF, fixed ones included: seeds on
    the bottom face's fixed u_x, u_z and the top face's prescribed u_x, u_z give the time mean of the
    matching combination of the reported reaction sums (fixed u_x, u_z: bottom face only here)."""
    spec, bc, dt, _, K = cube
    top, bot = spec.face_nodes(2, 1), spec.face_nodes(2, 0)
    seed = np.zeros((spec.n_particles, 6))
    seed[top, 2], seed[top, 0], seed[bot, 2], seed[bot, 0] = 1.0, 0.3, -0.5, 0.25
    o = oracle.Oracle(spec, MAT, dt, bc)
    J, _ = o.tangent(K // 3, seed)
    comb = []
    for _ in range(K // 3):
        o.step(1)
        R = o.energy()[1]
        comb.append(R[8] + 0.3 * R[6] - 0.5 * R[2] + 0.25 * R[0])
    np.testing.assert_allclose(J, np.mean(comb), rtol=1e-12)
    R = o.energy()[1]
    assert abs(R[2]) > 0.1 * abs(R[8]) and abs(R[0]) > 0.0  # the fixed faces do carry load


def test_cube_tangent_matches_central_differences(cube):
    spec, bc, dt, seed, K = cube
    o = oracle.Oracle(spec, MAT, dt, bc)
    F = spec.n_facets
    probe = oracle.Oracle(spec, MAT, dt, bc)
    probe.step(K)
    w, _ = probe.metrics()
    rng = np.random.default_rng(0)
    cracked = np.flatnonzero(w > 1e-6)
    assert len(cracked) > 20
    facets = np.concatenate([rng.choice(cracked, 3, replace=False), rng.choice(F, 2, replace=False)])
    P = np.array([MAT["E0"], MAT["alpha"], MAT["sigma_t"]])
    dirs = []
    for k in facets:
        for j in range(3):
            d = np.zeros((3, F))
            d[j, k] = P[j]
            dirs.append(d)
    dirs += [rng.standard_normal((3, F)) * P[:, None] for _ in range(2)]
    D = np.array(dirs)
    _, dJ = o.tangent(K, seed, D[:, 0], D[:, 1], D[:, 2])
    h = 1e-5
    base = np.broadcast_to(P[:, None], (3, F))
    fd = []
    for d in D:
        Jpm = []
        for sgn in (1.0, -1.0):
            p = base + sgn * h * d
            o.set_facet_params(p[0], p[1], p[2])
            Jpm.append(o.tangent(K, seed)[0])
        fd.append((Jpm[0] - Jpm[1]) / (2 * h))
    o.set_facet_params()
    fd = np.array(fd)
    single, dense = slice(0, 3 * len(facets)), slice(3 * len(facets), None)
    big = np.abs(dJ[single]).max()
    assert np.count_nonzero(dJ[single][2::3]) >= 2, "softening facets must have a sigma_t derivative"
    assert np.all(np.abs(dJ[single] - fd[single]) <= 2e-3 * np.abs(fd[single]) + 1e-5 * big)
    np.testing.assert_allclose(dJ[dense], fd[dense], rtol=1e-3)


def test_law_jacobian_where_deviatoric_softening_acts():
    """App. A.2 with the facet compressed well past its tetrahedron (e_D < 0, r_DV > k_c1): H_c then
    depends on |e_D|, so the derivative passes through |x|' = sign(x) at a negative argument.  The
    point lies on the linear hardening boundary; the Jacobian matches central differences."""
    n = 40
    path = np.stack([np.linspace(0, -1.4e-2, n), np.linspace(0, 1e-4, n), np.zeros(n)], 1)
    eV = np.linspace(0, -5e-3, n)
    x = law_point(path, eV, 35, MAT)
    e_N, e_V = x[0], x[6]
    eD = e_N - e_V
    eV0 = MAT["kc3"] * MAT["sigma_c0"] / MAT["E0"]
    rDV = -abs(eD) / (e_V - eV0)
    ec0 = MAT["sigma_c0"] / MAT["E0"]
    assert eD < 0 and rDV > MAT["kc1"] + 0.3 and ec0 < -e_V < MAT["kc0"] * ec0
    out, jac = oracle.facet_law_jacobian(MAT, L_FACET, x)
    assert out[0] < -1.01 * MAT["sigma_c0"]
    for h in (1e-5, 1e-6):
        fd = np.zeros((4, 14))
        for c in range(14):
            hh = h * max(abs(x[c]), SCALE[c])
            xp, xm = x.copy(), x.copy()
            xp[c] += hh
            xm[c] -= hh
            fd[:, c] = (oracle.facet_law_jacobian(MAT, L_FACET, xp)[0] - oracle.facet_law_jacobian(MAT, L_FACET, xm)[0]) / (2 * hh)
        assert np.abs(fd - jac).max() <= 1e-7 * np.abs(jac).max(), (h, np.abs(fd - jac).max())
    # the response does depend on e_D there (the softened H_c): moving e_N alone moves t_N
    assert abs(jac[0, 0]) > 0 and abs(jac[0, 6]) > 0
