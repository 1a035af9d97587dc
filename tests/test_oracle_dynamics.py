"""Pins of the oracle's time integration (central difference, lumped mass; paper Sec. 3, Sec. 4)."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import specimen, workloads
from paper_2603_13190_gb300.specimen import Specimen
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

MAT = dict(WORKLOAD_MATERIAL)
EL = dict(WORKLOAD_MATERIAL, elastic=1)


def two_particle(l=3.0, a0=2.0):
    """Particles I at the origin and J at (l, 0, 0) sharing one square-ish facet in the mid plane."""
    x = np.array([[0.0, 0.0, 0.0], [l, 0.0, 0.0]])
    h = math.sqrt(2 * a0)  # right triangle with legs h: area a0
    vtx = np.array([[l / 2, -h / 3, -h / 3, l / 2, 2 * h / 3, -h / 3, l / 2, -h / 3, 2 * h / 3]])
    return Specimen(x=x, diameter=np.array([1.0, 1.0]), tets=np.zeros((0, 4), np.int32),
                    facet_pi=np.array([0], np.int32), facet_pj=np.array([1], np.int32),
                    facet_tet=np.array([-1], np.int32), facet_vtx=vtx, edge=l, d_min=1.0, d_max=1.0)


def test_two_particle_stiffness_and_lambda_max_closed_form():
    """One facet between two nodes, centroid on the mid plane at the axis: axial stiffness A E0 / l,
    shear stiffness A alpha E0 / l acting on g = (-1, -l/2, 1, -l/2) over (u_Iy, th_Iz, u_Jy, th_Jz).
    Largest eigenvalue of M^-1 K = max(2 k_a / m, k_s (2/m + l^2 / (2 I)))."""
    l, a0, m, I = 3.0, 2.0, 1e-6, 2e-7
    spec = two_particle(l, a0)
    o = oracle.Oracle(spec, MAT, 1e-7, mass=np.full(2, m), inertia=np.full((2, 3), I))
    A = o.geometry()["area"][0]
    assert abs(A - a0) < 1e-12
    ka, ks = A * MAT["E0"] / l, A * MAT["alpha"] * MAT["E0"] / l
    q = np.zeros((2, 6))
    q[1, 0] = 1e-3  # pull J along the axis
    f = o.elastic_force(q)
    np.testing.assert_allclose(f[:, 0], [ka * 1e-3, -ka * 1e-3], rtol=1e-12)
    q = np.zeros((2, 6))
    q[1, 1] = 1e-3  # slide J sideways: shear force and the moments of a lever l/2 on each side
    f = o.elastic_force(q)
    np.testing.assert_allclose(f[:, 1], [ks * 1e-3, -ks * 1e-3], rtol=1e-12)
    np.testing.assert_allclose(f[:, 5], [ks * 1e-3 * l / 2, ks * 1e-3 * l / 2], rtol=1e-12)
    lam = max(2 * ka / m, ks * (2 / m + l * l / (2 * I)))
    x0 = np.random.default_rng(0).standard_normal(12)
    assert abs(o.lambda_max(x0, 400) - lam) < 1e-9 * lam


def test_two_particle_axial_oscillation_period():
    """Axial vibration of the 2-node system: central difference with dt << T reproduces the period
    2 pi / omega, omega^2 = k_a (1/m_I + 1/m_J) (relative motion of two masses on a spring)."""
    l, a0, m = 3.0, 2.0, 1e-6
    spec = two_particle(l, a0)
    ka = a0 * EL["E0"] / l
    w = math.sqrt(ka * 2 / m)
    T = 2 * math.pi / w
    dt = T / 2000
    bc = workloads.free_bc(2)
    bc.v0[0, 0], bc.v0[1, 0] = -1.0, 1.0
    o = oracle.Oracle(spec, EL, dt, bc, mass=np.full(2, m), inertia=np.full((2, 3), 1e-7))
    gap = []
    for _ in range(2000):
        o.step(1)
        q, _, _, _ = o.get_state()
        gap.append(q[1, 0] - q[0, 0])
    gap = np.array(gap)
    # relative displacement 2 v0 / w sin(w t): zero crossing at half period, amplitude 2/w
    k = int(np.argmax(gap < 0))
    assert abs(k - 1000) <= 2
    assert abs(gap.max() - 2.0 / w) < 1e-5 * (2.0 / w)


def test_elastic_vibration_conserves_energy():
    """Workload 'elastic_vibration' (Sec. 4.1 stand-in): 2000 steps at 0.9 dt_crit, energy error
    below 1 % (free vibration: W_ext = 0, W_kin + W_int stays at W_kin0)."""
    wl = workloads.WORKLOADS["elastic_vibration"]
    spec = wl.specimen()
    bc = workloads.workload_bc(wl.name, spec)
    o = oracle.Oracle(spec, wl.material, 1e-7, bc)
    dt = wl.dt_factor * o.critical_dt()
    o = oracle.Oracle(spec, wl.material, dt, bc)
    o.step(wl.steps)
    (Wext, Wint, Wkin, err), _ = o.energy()
    assert Wext == 0.0
    assert err < 1.0
    assert Wint > 0.05 * Wkin  # energy really moved between kinetic and stored


def test_free_flight_conserves_momentum():
    """With no constraints the internal forces cannot change total linear or angular momentum."""
    spec = specimen.make_cube_specimen(10.0, 2.0, 4.0, 100, seed=11)
    rng = np.random.default_rng(1)
    bc = workloads.free_bc(spec.n_particles)
    bc.v0[:] = rng.standard_normal(bc.v0.shape) * 5.0
    o = oracle.Oracle(spec, MAT, 1e-7, bc)
    o = oracle.Oracle(spec, MAT, 0.9 * o.critical_dt(), bc)
    m6 = o.geometry()["mass"]

    def momenta():
        q, v, _, _ = o.get_state()
        p = (m6[:, :3] * v[:, :3]).sum(0)
        xq = spec.x + q[:, :3]
        L = (np.cross(xq, m6[:, :3] * v[:, :3]) + m6[:, 3:] * v[:, 3:]).sum(0)
        return p, L

    p0, L0 = momenta()
    o.step(300)
    p1, L1 = momenta()
    assert np.abs(p1 - p0).max() < 1e-10 * np.abs(m6[:, 0] * 5).sum()
    # small-rotation kinematics: angular momentum holds to first order in the displacements
    assert np.abs(L1 - L0).max() < 1e-2 * np.abs(L0).max()


@pytest.mark.parametrize("steps", [1500])
def test_tension_energy_balance_through_softening(steps):
    """Uniaxial tension to post-peak on a small cube: the energy balance error of Sec. 4 stays below 1 %
    and the macroscopic stress rises, peaks and softens."""
    spec = specimen.make_cube_specimen(10.0, 2.0, 4.0, 220, seed=3)
    bc = workloads.uniaxial_tension_bc(spec, velocity=50.0, ramp_time=1e-5)
    o = oracle.Oracle(spec, MAT, 1e-7, bc)
    dt = 0.9 * o.critical_dt()
    o = oracle.Oracle(spec, MAT, dt, bc)
    stress = []
    for _ in range(steps // 10):
        o.step(10)
        (Wext, Wint, Wkin, err), R = o.energy()
        stress.append(R[8] / spec.edge ** 2)  # reaction on the prescribed u_z DOFs, over the area
    stress = np.array(stress)
    k = int(np.argmax(stress))
    assert 0 < k < len(stress) - 3, "peak must lie inside the run"
    assert stress[-1] < 0.7 * stress[k]
    assert err < 1.0


def modal_basis(o, N):
    """Eigenpairs of K phi = w^2 M phi (K from the oracle's elastic operator by columns, M its lumped
    mass), phi^T M phi = 1: an independent linear-algebra route to the frequencies."""
    import scipy.linalg

    n = 6 * N
    K = np.zeros((n, n))
    for j in range(n):
        q = np.zeros(n)
        q[j] = 1.0
        K[:, j] = -o.elastic_force(q.reshape(-1, 6)).reshape(-1)
    K = 0.5 * (K + K.T)
    m = o.geometry()["mass"].reshape(-1)
    w2, phi = scipy.linalg.eigh(K, np.diag(m))
    return np.sqrt(np.maximum(w2, 0.0)), phi, m


def test_free_vibration_modes_follow_the_discrete_closed_form():
    """Elastic free vibration from q = 0 with v0 = sum c_i phi_i: central difference advances each
    mode independently, eta_i(n) = phi_i^T M q_n = (dt c_i / sin theta_i) sin(n theta_i) with
    cos theta_i = 1 - (w_i dt)^2 / 2 (the scheme's discrete frequency, Sec. 3.2)."""
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=2)
    mat = dict(WORKLOAD_MATERIAL, elastic=1)
    o0 = oracle.Oracle(spec, mat, 1e-7)
    w, phi, m = modal_basis(o0, spec.n_particles)
    dt = 0.9 * 2.0 / w.max()
    modes = [10, 37, len(w) - 1]
    c = np.array([1.0, -0.5, 0.2]) * 50.0
    v0 = (phi[:, modes] @ c).reshape(-1, 6)
    bc = workloads.free_bc(spec.n_particles)
    bc.v0 = v0
    o = oracle.Oracle(spec, mat, dt, bc)
    theta = np.arccos(1.0 - 0.5 * (w[modes] * dt) ** 2)
    for n in range(1, 301):
        o.step(1)
        if n % 50:
            continue
        q = o.get_state()[0].reshape(-1)
        eta = phi[:, modes].T @ (m * q)
        expect = dt * c / np.sin(theta) * np.sin(n * theta)
        np.testing.assert_allclose(eta, expect, rtol=0, atol=1e-9 * np.abs(dt * c / np.sin(theta)).max())


def test_rigid_perturbation_only_shifts_the_trajectory():
    """A perturbation that is a rigid translation of the whole free specimen creates no strain: the
    perturbed run equals the unperturbed one with q shifted by the translation; velocities and
    tractions are unchanged (Sec. 5's perturbations act only through strains)."""
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=2)
    rng = np.random.default_rng(1)
    bc = workloads.free_bc(spec.n_particles)
    bc.v0 = rng.standard_normal((spec.n_particles, 6)) * 20.0
    a = oracle.Oracle(spec, WORKLOAD_MATERIAL, 1e-7, bc)
    b = oracle.Oracle(spec, WORKLOAD_MATERIAL, 1e-7, bc)
    a.step(100)
    b.step(100)
    shift = np.zeros((spec.n_particles, 6))
    shift[:, :3] = [1e-3, -2e-3, 0.5e-3]
    b.perturb(shift)
    a.step(100)
    b.step(100)
    qa, va, ha, _ = a.get_state()
    qb, vb, hb, _ = b.get_state()
    np.testing.assert_allclose(qb - shift, qa, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vb, va, rtol=0, atol=1e-9 * np.abs(va).max())
    np.testing.assert_allclose(hb, ha, rtol=0, atol=1e-9 * np.abs(ha).max())


def test_perturbation_leaves_constrained_dofs_alone():
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=2)
    bc = workloads.uniaxial_tension_bc(spec, velocity=50.0, ramp_time=1e-5)
    o = oracle.Oracle(spec, WORKLOAD_MATERIAL, 1e-7, bc)
    o.step(20)
    q0 = o.get_state()[0]
    dq = np.full((spec.n_particles, 6), 1e-4)
    o.perturb(dq)
    q1 = o.get_state()[0]
    free = bc.mask == 0
    np.testing.assert_array_equal(q1[~free], q0[~free])
    np.testing.assert_allclose(q1[free] - q0[free], 1e-4, rtol=1e-9)


def test_prescribed_ramp_reaction_is_newton_on_a_rigid_body():
    """Every DOF prescribed: the translations ramp linearly to v over T, rotations held at zero.
    The body moves rigidly, so no facet strains and the reaction is the inertial force alone:
    M v / T on each translation while the ramp runs (M = rho V, the lumped masses tile the cube),
    zero once it has ended.  The work the constraint does brings the body to the kinetic energy
    M |v|^2 / 2, up to the central-difference error of the ramp's two kinks (Sec. 3, Sec. 4)."""
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=1)
    bc = workloads.free_bc(spec.n_particles)
    bc.mask[:] = workloads.PRESCRIBED
    v = np.array([30.0, -20.0, 50.0])
    bc.vel[:, :3] = v
    dt, n_ramp = 1e-7, 200
    bc.ramp_time = n_ramp * dt
    o = oracle.Oracle(spec, MAT, dt, bc)
    M = MAT["rho"] * spec.edge ** 3
    # at t = 0 the body was at rest before: the acceleration of the velocity kink is half the slope
    np.testing.assert_allclose(o.energy()[1][6:9], 0.5 * M * v / bc.ramp_time, rtol=1e-9)
    for n in (1, 57, n_ramp - 1):
        o.step(n - o.get_state()[3])
        _, R = o.energy()
        np.testing.assert_allclose(R[6:9], M * v / bc.ramp_time, rtol=1e-9)
        assert np.abs(R[9:12]).max() == 0.0 and np.abs(R[:6]).max() == 0.0
    o.step(n_ramp + 5 - o.get_state()[3])
    (Wext, Wint, Wkin, _), R = o.energy()
    assert np.abs(R).max() == 0.0 and Wint == 0.0
    Ek = 0.5 * M * float(v @ v)
    np.testing.assert_allclose(Wkin, Ek, rtol=1e-9)
    assert abs(Wext - Ek) <= Ek / n_ramp


def test_strain_perturbation_is_a_new_reference_not_an_increment():
    """Sec. 5 perturbations (reading: the perturbed state is the reference of the next strain
    increment; tractions and velocities are kept).  Two particles at rest, the facet stretched
    elastically to half its peak with the matching traction; J is then displaced along the axis by
    0.3 of the peak strain.  The next step's traction moves only by the step's own strain increment
    (dt^2 F / m, four orders below the jump), not by E0 times the perturbation.  e_max, the largest
    effective strain reached, follows the total strain to 0.8 of the peak."""
    l, m = 3.0, 1e-6
    spec = two_particle(l)
    o = oracle.Oracle(spec, MAT, 1e-7, mass=np.full(2, m), inertia=np.full((2, 3), 1e-7))
    e0 = MAT["sigma_t"] / MAT["E0"]
    q = np.zeros((2, 6))
    q[1, 0] = 0.5 * e0 * l
    t0 = MAT["E0"] * 0.5 * e0
    o.set_state(q, np.zeros((2, 6)), np.array([[t0, 0.0, 0.0, 0.0, 0.5 * e0]]))
    dq = np.zeros((2, 6))
    dq[1, 0] = 0.3 * e0 * l
    o.perturb(dq)
    o.step(1)
    _, _, h, _ = o.get_state()
    jump = MAT["E0"] * 0.3 * e0
    assert abs(h[0, 0] - t0) < 1e-2 * jump, (h[0, 0], t0, jump)
    assert abs(h[0, 4] - 0.8 * e0) < 1e-3 * e0


def test_set_bc_takes_the_constrained_velocities_at_once():
    """Switching boundary conditions mid-run: a newly prescribed DOF moves at bc_vel ramp(t) from the
    switch on (reported velocity and kinetic energy), a newly fixed one stops."""
    spec = two_particle(3.0)
    bc = workloads.free_bc(2)
    bc.v0[:, 0] = [2.0, -1.0]
    o = oracle.Oracle(spec, EL, 1e-7, bc, mass=np.full(2, 1e-6), inertia=np.full((2, 3), 1e-7))
    o.step(10)
    nb = workloads.free_bc(2)
    nb.mask[0, :] = workloads.FIXED
    nb.mask[1, 0] = workloads.PRESCRIBED
    nb.vel[1, 0] = 7.0
    nb.ramp_time = 0.0
    o.set_bc(nb)
    _, v, _, _ = o.get_state()
    assert np.all(v[0] == 0.0) and v[1, 0] == 7.0
    (_, _, Wk, _), _ = o.energy()
    np.testing.assert_allclose(Wk, 0.5 * 1e-6 * 49.0 + 0.5 * 1e-7 * float(v[1, 3:] @ v[1, 3:]) + 0.5 * 1e-6 * float(v[1, 1:3] @ v[1, 1:3]), rtol=1e-12)


def test_constant_external_force_free_flight():
    """Constant external forces f_ext, the same on both particles: the pair accelerates rigidly at
    a = f / m, which central difference integrates exactly (q_n = a (n dt)^2 / 2, v_n = a n dt), the
    facet stays unstrained, and the external work f . q equals the kinetic energy."""
    m, dt, n = 1e-6, 1e-7, 50
    spec = two_particle(3.0)
    f = np.zeros((2, 6))
    f[:, :3] = [2.0, -1.0, 0.5]
    o = oracle.Oracle(spec, MAT, dt, mass=np.full(2, m), inertia=np.full((2, 3), 1e-7), f_ext=f)
    o.step(n)
    q, v, h, _ = o.get_state()
    a = f[0, :3] / m
    np.testing.assert_allclose(q[:, :3], np.tile(0.5 * a * (n * dt) ** 2, (2, 1)), rtol=1e-12)
    np.testing.assert_allclose(v[:, :3], np.tile(a * n * dt, (2, 1)), rtol=1e-12)
    assert np.all(q[:, 3:] == 0.0) and np.all(h == 0.0)
    (Wext, Wint, Wkin, err), R = o.energy()
    np.testing.assert_allclose(Wext, float((f * q).sum()), rtol=1e-12)
    np.testing.assert_allclose(Wkin, Wext, rtol=1e-12)
    assert Wint == 0.0 and err < 1e-9 and np.all(R == 0.0)


def test_energy_balance_restarts_at_set_state():
    """set_state starts a new energy balance: W_ext = W_int = 0 and the supplied kinetic energy is
    that of the velocities just set.  A free elastic cube created with velocities v0 and then set to
    2 v0 keeps its balance (W_kin + W_int = W_kin at the set) over the following steps."""
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=1)
    bc = workloads.free_bc(spec.n_particles)
    # a smooth field (low modes, where the trapezoid energy sums are accurate)
    z, x = spec.x[:, 2] / spec.edge, spec.x[:, 0] / spec.edge
    bc.v0[:, 0] = np.sin(np.pi * z)
    bc.v0[:, 1] = 0.5 * np.cos(np.pi * x)
    o = oracle.Oracle(spec, EL, 1e-7, bc)
    dt = 0.5 * o.critical_dt()
    o = oracle.Oracle(spec, EL, dt, bc)
    o.step(40)
    q = np.zeros((spec.n_particles, 6))
    o.set_state(q, 2.0 * bc.v0, np.zeros((spec.n_facets, 5)), 0)
    (_, _, Wk0, err0), _ = o.energy()
    assert err0 == 0.0
    o.step(300)
    (Wext, Wint, Wkin, err), _ = o.energy()
    assert Wext == 0.0 and Wint > 0.05 * Wkin
    assert abs(Wkin + Wint - Wk0) < 1e-2 * Wk0 and err < 1.0
    # the error of Sec. 4 with the initial kinetic energy as the supplied energy (W_ext = 0 here)
    assert err > 0.0
    np.testing.assert_allclose(err, 100.0 * abs(Wk0 - Wint - Wkin) / Wk0, rtol=1e-9)


def test_kinetic_energy_counts_rotations():
    """W_kin = sum over DOFs of m v^2 / 2 with the rotary inertia on the rotational DOFs."""
    spec = two_particle(3.0)
    I = np.array([[1e-7, 2e-7, 3e-7], [4e-7, 5e-7, 6e-7]])
    o = oracle.Oracle(spec, EL, 1e-7, mass=np.full(2, 1e-6), inertia=I)
    v = np.zeros((2, 6))
    v[0, 3:] = [1.0, -2.0, 0.5]
    v[1, 0] = 3.0
    o.set_state(np.zeros((2, 6)), v, np.zeros((1, 5)))
    (_, _, Wkin, _), _ = o.energy()
    np.testing.assert_allclose(Wkin, 0.5 * (I[0] * v[0, 3:] ** 2).sum() + 0.5 * 1e-6 * 9.0, rtol=1e-14)


def test_external_force_with_initial_velocity_balances_energy():
    """Free pair with initial velocity v0 and constant forces f along it: the supplied energy is the
    external work plus the initial kinetic energy, so the balance of Sec. 4 holds to rounding
    (W_ext + W_kin0 = W_kin, no strain)."""
    m, dt, n = 1e-6, 1e-7, 80
    spec = two_particle(3.0)
    bc = workloads.free_bc(2)
    bc.v0[:, :3] = [5.0, 1.0, -2.0]
    f = np.zeros((2, 6))
    f[:, :3] = [0.5, 0.2, 0.1]
    o = oracle.Oracle(spec, MAT, dt, bc, mass=np.full(2, m), inertia=np.full((2, 3), 1e-7), f_ext=f)
    o.step(n)
    (Wext, Wint, Wkin, err), _ = o.energy()
    Wk0 = 0.5 * m * 2 * float(bc.v0[0, :3] @ bc.v0[0, :3])
    assert Wint == 0.0 and Wext > 0.1 * Wk0
    np.testing.assert_allclose(Wkin, Wext + Wk0, rtol=1e-12)
    assert err < 1e-9


def test_divergence_is_reported():
    """Above the stability limit (dt = 3 dt_c) the explicit step diverges; the oracle reports it
    (FloatingPointError) from a plain run and from the derivative run alike."""
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=1)
    bc = workloads.free_bc(spec.n_particles)
    bc.v0 = np.random.default_rng(0).standard_normal((spec.n_particles, 6))
    dt_c = oracle.Oracle(spec, EL, 1e-7, bc).critical_dt()
    o = oracle.Oracle(spec, EL, 3.0 * dt_c, bc)
    with pytest.raises(FloatingPointError):
        o.step(3000)
    o = oracle.Oracle(spec, EL, 3.0 * dt_c, bc)
    with pytest.raises(FloatingPointError):
        o.tangent(3000, np.zeros((spec.n_particles, 6)))


def test_constrained_dofs_start_at_their_constrained_velocity():
    """Whatever v0 says, fixed DOFs start at rest and prescribed ones at bc_vel ramp(0)."""
    spec = two_particle(3.0)
    bc = workloads.free_bc(2)
    bc.v0[:, :] = 3.0
    bc.mask[0, :] = workloads.FIXED
    bc.mask[1, 0] = workloads.PRESCRIBED
    bc.vel[1, 0] = 7.0
    bc.ramp_time = 0.0
    o = oracle.Oracle(spec, EL, 1e-7, bc, mass=np.full(2, 1e-6), inertia=np.full((2, 3), 1e-7))
    v = o.get_state()[1]
    assert np.all(v[0] == 0.0) and v[1, 0] == 7.0 and np.all(v[1, 1:] == 3.0)
