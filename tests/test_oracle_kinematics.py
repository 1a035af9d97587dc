"""Pins of the oracle's kinematics, assembly and set-up (paper Sec. 2, Eq. (1)-(2), Sec. 3.2.5)."""
import numpy as np
import pytest

import oracle
from paper_2603_13190_gb300 import specimen
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

MAT = dict(WORKLOAD_MATERIAL)


@pytest.fixture(scope="module")
def cube():
    spec = specimen.make_cube_specimen(12.0, 2.0, 4.0, 160, seed=7)
    return spec, oracle.Oracle(spec, MAT, 1e-7)


def affine_q(spec, eps, omega=None, shift=None):
    q = np.zeros((spec.n_particles, 6))
    q[:, :3] = spec.x @ np.asarray(eps).T
    if omega is not None:
        q[:, :3] += np.cross(np.broadcast_to(omega, spec.x.shape), spec.x)
        q[:, 3:] = omega
    if shift is not None:
        q[:, :3] += shift
    return q


def test_rigid_translation_gives_zero_strain_and_force(cube):
    spec, o = cube
    q = affine_q(spec, np.zeros((3, 3)), shift=np.array([0.3, -0.2, 0.7]))
    e, eV = o.strains(q)
    assert np.abs(e).max() < 1e-15 and np.abs(eV).max() < 1e-15
    assert np.abs(o.elastic_force(q)).max() < 1e-9


def test_rigid_rotation_gives_zero_strain(cube):
    """[[u]] = w x (x_J + c_J - x_I - c_I) = 0 because x_I + c_I = x_J + c_J is the facet centroid."""
    spec, o = cube
    w = np.array([1e-3, -2e-3, 0.5e-3])
    q = affine_q(spec, np.zeros((3, 3)), omega=w)
    e, eV = o.strains(q)
    assert np.abs(e).max() < 1e-14
    assert np.abs(eV).max() < 1e-14


def test_patch_test_facet_strain_is_projected_strain_tensor(cube):
    """u = eps x, theta = 0: [[u]] = l eps n, so e_N = n.eps.n and |e_T|^2 = |eps n|^2 - e_N^2 (the facet
    strains are the projection of the strain tensor, Sec. 2)."""
    spec, o = cube
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3)) * 1e-4
    eps = 0.5 * (A + A.T)
    e, eV = o.strains(affine_q(spec, eps))
    n = o.geometry()["n"]
    en = np.einsum("fi,ij,fj->f", n, eps, n)
    en_vec = n @ eps.T
    et2 = np.einsum("fi,fi->f", en_vec, en_vec) - en ** 2
    np.testing.assert_allclose(e[:, 0], en, rtol=1e-10, atol=1e-18)
    np.testing.assert_allclose(e[:, 1] ** 2 + e[:, 2] ** 2, et2, rtol=1e-8, atol=1e-20)
    # volumetric strain of every tetrahedron is tr(eps) / 3 (linearised Delta V / (3 V0))
    np.testing.assert_allclose(eV, np.trace(eps) / 3.0, rtol=1e-10)


def test_hydrostatic_has_no_deviatoric_facet_strain(cube):
    spec, o = cube
    e, eV = o.strains(affine_q(spec, 2e-4 * np.eye(3)))
    np.testing.assert_allclose(e[:, 0], 2e-4, rtol=1e-12)
    np.testing.assert_allclose(eV, 2e-4, rtol=1e-12)
    assert np.abs(e[:, 1:]).max() < 1e-17


def test_internal_forces_balance_linear_and_angular_momentum(cube):
    """Internal forces are equal and opposite on I and J and their moments about any point cancel:
    sum_p f_p = 0 and sum_p (x_p x f_p + m_p) = 0 (Eq. (2) with the arms to the common centroid)."""
    spec, o = cube
    rng = np.random.default_rng(5)
    q = rng.standard_normal((spec.n_particles, 6)) * 1e-4
    f = o.elastic_force(q)
    scale = np.abs(f).max()
    assert np.abs(f[:, :3].sum(0)).max() < 1e-12 * scale * spec.n_particles
    ang = np.cross(spec.x, f[:, :3]).sum(0) + f[:, 3:].sum(0)
    assert np.abs(ang).max() < 1e-12 * scale * spec.n_particles * spec.edge


def test_stiffness_symmetric_with_six_rigid_modes():
    """K = -df/dq (elastic) is symmetric positive semi-definite with exactly the 6 rigid-body modes
    in its null space (free specimen)."""
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 45, seed=2)
    o = oracle.Oracle(spec, MAT, 1e-7)
    n = 6 * spec.n_particles
    K = np.zeros((n, n))
    for j in range(n):
        q = np.zeros(n)
        q[j] = 1.0
        K[:, j] = -o.elastic_force(q.reshape(-1, 6)).reshape(-1)
    assert np.abs(K - K.T).max() < 1e-9 * np.abs(K).max()
    w = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert np.sum(np.abs(w) < 1e-9 * w.max()) == 6
    assert w.min() > -1e-9 * w.max()


def test_work_identity_q_dot_f_is_twice_strain_energy(cube):
    """For the linear facet law, -q . f(q) = sum_k A l e.E e (twice the stored energy)."""
    spec, o = cube
    rng = np.random.default_rng(9)
    q = rng.standard_normal((spec.n_particles, 6)) * 1e-4
    e, _ = o.strains(q)
    g = o.geometry()
    E = MAT["E0"] * np.array([1.0, MAT["alpha"], MAT["alpha"]])
    twoW = np.sum(g["area"] * g["len"] * np.einsum("fi,i,fi->f", e, E, e))
    np.testing.assert_allclose(-np.sum(q * o.elastic_force(q)), twoW, rtol=1e-10)


def test_projected_area_and_lumped_mass(cube):
    """A = A0 |n . n0| never exceeds A0; the lumped translational masses add up to rho V of the cube
    (tetrahedra tile the cube; each gives rho V_tet / 4 to its nodes, Sec. 3.2.5); rotary inertia is
    m d^2 / 10."""
    spec, o = cube
    g = o.geometry()
    v = spec.facet_vtx.reshape(-1, 3, 3)
    A0 = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)
    assert np.all(g["area"] <= A0 * (1 + 1e-12)) and np.all(g["area"] > 0)
    m = g["mass"]
    np.testing.assert_allclose(m[:, 0].sum(), MAT["rho"] * spec.edge ** 3, rtol=1e-9)
    d = np.where(spec.diameter > 0, spec.diameter, spec.diameter[spec.diameter > 0].min())
    np.testing.assert_allclose(m[:, 3], m[:, 0] * d ** 2 / 10.0, rtol=1e-14)
    # arms: x_I + c_I == x_J + c_J == facet centroid
    xc = v.mean(axis=1)
    np.testing.assert_allclose(spec.x[spec.facet_pi] + g["ci"], xc, atol=1e-12)
    np.testing.assert_allclose(spec.x[spec.facet_pj] + g["cj"], xc, atol=1e-12)


def test_frame_rotation_invariance_of_forces():
    """Relabelling I <-> J and permuting the facets (which changes every tangent frame) changes no
    force: the law is isotropic in the facet plane (Sec. 2: tangents may be chosen arbitrarily)."""
    spec = specimen.make_cube_specimen(10.0, 2.0, 4.0, 100, seed=4)
    sh = specimen.shuffled(spec, seed=1)
    rng = np.random.default_rng(2)
    q = rng.standard_normal((spec.n_particles, 6)) * 2e-4
    v = rng.standard_normal((spec.n_particles, 6)) * 1.0
    outs = []
    for s in (spec, sh):
        o = oracle.Oracle(s, MAT, 2e-7)
        o.set_state(np.zeros_like(q), v, np.zeros((s.n_facets, 5)))
        for _ in range(30):
            o.step(1)
        outs.append(o.facet_forces()[1])
    np.testing.assert_allclose(outs[0], outs[1], rtol=0, atol=1e-9 * np.abs(outs[0]).max())


def test_crack_opening_zero_while_elastic_and_equal_to_jump_when_separated():
    """w (Sec. 4) vanishes on an elastic state and equals the opening |[[u]]| of a fully separated
    facet (traction decayed to zero, App. A.1)."""
    import math
    from paper_2603_13190_gb300.specimen import Specimen
    l, h = 3.0, 2.0
    x = np.array([[0.0, 0.0, 0.0], [l, 0.0, 0.0]])
    vtx = np.array([[l / 2, -h / 3, -h / 3, l / 2, 2 * h / 3, -h / 3, l / 2, -h / 3, 2 * h / 3]])
    spec = Specimen(x=x, diameter=np.ones(2), tets=np.zeros((0, 4), np.int32), facet_pi=np.array([0], np.int32),
                    facet_pj=np.array([1], np.int32), facet_tet=np.array([-1], np.int32), facet_vtx=vtx, edge=l,
                    d_min=1.0, d_max=1.0)
    o = oracle.Oracle(spec, MAT, 1e-7, mass=np.full(2, 1e-6), inertia=np.full((2, 3), 1e-7))
    q = np.zeros((2, 6))
    q[1, 0] = 0.5 * MAT["sigma_t"] / MAT["E0"] * l  # half the peak strain: elastic
    o.set_state(q, np.zeros((2, 6)), np.zeros((1, 5)))
    o.set_state(q, np.zeros((2, 6)), np.array([[MAT["E0"] * q[1, 0] / l, 0, 0, 0, 0]]))
    w, _ = o.metrics()
    assert w[0] < 1e-12 * q[1, 0]
    # fully separated: traction zero, opening (0.02, 0.01, 0) mm
    q[1, :3] = [0.02, 0.01, 0.0]
    o.set_state(q, np.zeros((2, 6)), np.array([[0.0, 0, 0, 0, 1.0]]))
    w, _ = o.metrics()
    assert abs(w[0] - math.hypot(0.02, 0.01)) < 1e-14
    # compacted past sigma_c0: inelastic normal strain e_N - t_N / E0 = -e_c0 < 0 opens no crack
    ec0 = MAT["sigma_c0"] / MAT["E0"]
    q[1, :3] = [-2.0 * ec0 * l, 0.0, 0.0]
    o.set_state(q, np.zeros((2, 6)), np.array([[-MAT["sigma_c0"], 0, 0, 0, 0.0]]))
    w, _ = o.metrics()
    assert w[0] == 0.0


def test_volumetric_strain_metric_is_trace_over_three(cube):
    spec, o = cube
    rng = np.random.default_rng(6)
    A = rng.standard_normal((3, 3)) * 1e-4
    eps = 0.5 * (A + A.T)
    o.set_state(affine_q(spec, eps), np.zeros((spec.n_particles, 6)), np.zeros((spec.n_facets, 5)))
    _, eV = o.metrics()
    np.testing.assert_allclose(eV, np.trace(eps) / 3.0, rtol=1e-10)


def test_state_exchange_tangential_traction_in_world_frame():
    """History exchange (get_state / set_state) stores the tangential traction as a world vector
    t_M m + t_L l.  Two particles on the x axis; J is driven sideways along d = (0, 1, 2) / sqrt(5)
    (a direction with parts along both tangents of any frame) with I fixed and no rotation, an
    elastic shear of 0.2 of the cracking strain.  The stored vector is alpha E0 (delta / l) d, the
    normal traction is zero; set_state then get_state returns it unchanged, and the facet force is
    rebuilt from it as F = A (t_N n + t_T) on I with -F on J (Eq. (2a)), the lumped forces following."""
    from paper_2603_13190_gb300 import workloads
    from paper_2603_13190_gb300.specimen import Specimen
    l, h, dt, n = 3.0, 2.0, 1e-7, 40
    x = np.array([[0.0, 0.0, 0.0], [l, 0.0, 0.0]])
    vtx = np.array([[l / 2, -h / 3, -h / 3, l / 2, 2 * h / 3, -h / 3, l / 2, -h / 3, 2 * h / 3]])
    spec = Specimen(x=x, diameter=np.ones(2), tets=np.zeros((0, 4), np.int32), facet_pi=np.array([0], np.int32),
                    facet_pj=np.array([1], np.int32), facet_tet=np.array([-1], np.int32), facet_vtx=vtx, edge=l,
                    d_min=1.0, d_max=1.0)
    d = np.array([0.0, 1.0, 2.0]) / np.sqrt(5.0)
    e0 = MAT["sigma_t"] / MAT["E0"]
    delta = 0.2 * e0 * l
    bc = workloads.free_bc(2)
    bc.mask[:, :] = workloads.FIXED
    bc.mask[1, :3] = workloads.PRESCRIBED
    bc.vel[1, :3] = d * delta / (n * dt)
    kw = dict(mass=np.full(2, 1e-6), inertia=np.full((2, 3), 1e-7))
    o = oracle.Oracle(spec, MAT, dt, bc, **kw)
    o.step(n)
    q, v, h5, st = o.get_state()
    np.testing.assert_allclose(q[1, :3], delta * d, rtol=1e-12)
    tT = MAT["alpha"] * MAT["E0"] * delta / l * d
    assert abs(h5[0, 0]) < 1e-12 * np.abs(tT).max()
    np.testing.assert_allclose(h5[0, 1:4], tT, rtol=1e-10, atol=1e-14 * np.abs(tT).max())
    # round trip through a fresh model, and forces rebuilt from the history
    o2 = oracle.Oracle(spec, MAT, dt, bc, **kw)
    o2.set_state(q, v, h5, st)
    np.testing.assert_allclose(o2.get_state()[2], h5, rtol=1e-13, atol=1e-15 * np.abs(tT).max())
    A = o2.geometry()["area"][0]
    F3, f6 = o2.facet_forces()
    F = A * (h5[0, 0] * np.array([1.0, 0.0, 0.0]) + h5[0, 1:4])
    np.testing.assert_allclose(F3[0], F, rtol=1e-12, atol=1e-14 * np.abs(F).max())
    np.testing.assert_allclose(f6[0, :3], F, rtol=1e-12, atol=1e-14 * np.abs(F).max())
    np.testing.assert_allclose(f6[1, :3], -F, rtol=1e-12, atol=1e-14 * np.abs(F).max())


def test_volumetric_strain_per_tetrahedron_under_a_random_field(cube):
    """e_V of each tetrahedron is (1/3) tr of the gradient of the linear interpolant of the nodal
    displacements (App. A.2, linearised).  Independent route: solve D^T G = [u_i - u_0] for the
    gradient G of every tetrahedron (D = vertex offsets), under a random nodal field."""
    spec, o = cube
    rng = np.random.default_rng(11)
    q = np.zeros((spec.n_particles, 6))
    q[:, :3] = rng.standard_normal((spec.n_particles, 3)) * 1e-3
    o.set_state(q, np.zeros((spec.n_particles, 6)), np.zeros((spec.n_facets, 5)))
    _, eV = o.metrics()
    X, U = spec.x[spec.tets], q[spec.tets, :3]  # [T][4][3]
    D = X[:, 1:, :] - X[:, :1, :]
    dU = U[:, 1:, :] - U[:, :1, :]
    G = np.linalg.solve(D, dU)  # rows of D times G = dU: G[a, b] = d u_b / d x_a
    expect = np.trace(G, axis1=1, axis2=2) / 3.0
    assert np.std(expect) > 0.05 * np.abs(expect).max()  # the field is far from uniform
    np.testing.assert_allclose(eV, expect, rtol=1e-9, atol=1e-12 * np.abs(expect).max())
