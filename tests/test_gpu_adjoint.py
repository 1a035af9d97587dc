"""GPU adjoint against the oracle's exact derivative (forward-mode dual numbers through the oracle's
own step, pinned in test_oracle_adjoint.py).

  * the device law and its vector-Jacobian product against the oracle's law Jacobian in every branch
    of App. A (input-scaled sensitivities: FP64 within 1e-11, FP32 law within 1e-4);
  * the forward step with per-facet parameters against the oracle with the same parameters;
  * the whole reverse pass: the objective and the gradient along single-facet and dense parameter
    directions against the oracle's directional derivatives, FP64 and mixed;
  * the checkpoint interval changes nothing (FP64: bitwise) and the handle ends where ldpm_step would
    leave it;
  * the torch.autograd binding returns the reverse pass's gradient.
"""
import numpy as np
import pytest

import oracle
from law_cases import CASES, IN_SCALE, L_FACET, OUT_SCALE, case, law_point
from paper_2603_13190_gb300 import ldpm, specimen, workloads
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

pytestmark = pytest.mark.gpu
MAT = dict(WORKLOAD_MATERIAL)
P0 = np.array([MAT["E0"], MAT["alpha"], MAT["sigma_t"]])


def _law_rows(variants):
    """Rows (device layout: l, e, de, eV, t_old, e_max, E0, alpha, sigma_t, 0) at every branch point
    of the given material family and, around each, 3 random perturbations of the parameters within 1 %."""
    rng = np.random.default_rng(3)
    rows, mats = [], []
    for name in sorted(CASES):
        path, eV, i, mat = case(name)
        if (mat != MAT) != variants:
            continue
        x = law_point(path, eV, i, mat)
        for r in range(4):
            y = x.copy()
            if r:
                y[11:14] *= 1 + 0.01 * rng.uniform(-1, 1, 3)
            rows.append(np.concatenate([[L_FACET], y, [0.0]]))
            mats.append(mat)
    return np.array(rows), mats


@pytest.mark.parametrize("prec,tol", [(ldpm.LDPM_FP64, 1e-11), (ldpm.LDPM_MIXED, 1e-4)])
@pytest.mark.parametrize("variants", [False, True])
def test_law_vjp_matches_oracle_jacobian(prec, tol, variants):
    rows, mats = _law_rows(variants)
    rng = np.random.default_rng(5)
    aout = rng.standard_normal((len(rows), 4))
    out = np.zeros((len(rows), 4))
    ain = np.zeros((len(rows), 16))
    for mat in {tuple(sorted(m.items())) for m in mats}:  # one device call per material
        sel = [k for k, m in enumerate(mats) if tuple(sorted(m.items())) == mat]
        out[sel], ain[sel] = ldpm.ldpm_facet_law_vjp(prec, dict(mat), rows[sel], aout[sel])
    for k, row in enumerate(rows):
        x = row[1:15]
        mat = dict(mats[k], E0=x[11], alpha=x[12], sigma_t=x[13])
        o_ref, jac = oracle.facet_law_jacobian(mat, row[0], x)
        ref = aout[k] @ jac
        scale_o = np.abs(o_ref).max()
        assert np.abs(out[k] - o_ref).max() <= max(tol, 1e-6 if prec else 0) * scale_o + 1e-300, (k, out[k], o_ref)
        # each input's adjoint times the input's magnitude (the output change for a relative change
        # of that input), against the adjoint-weighted output magnitude
        S = np.sum(np.abs(aout[k]) * np.maximum(np.abs(o_ref), OUT_SCALE))
        err = np.abs(ain[k, 1:15] - ref) * np.maximum(np.abs(x), IN_SCALE)
        assert np.all(err <= tol * S), (k, err / S, ref)
    assert ain[:, 0].max() == 0 and ain[:, 15].max() == 0


@pytest.fixture(scope="module")
def cube():
    """The oracle pin's cube: 10 mm, top u_z at 20 mm/s and u_x at 8 mm/s, 300 steps before the
    macroscopic peak with softening facets."""
    spec = specimen.make_cube_specimen(10.0, 2.0, 4.0, 120, seed=31)
    bc = workloads.uniaxial_tension_bc(spec, velocity=20.0, ramp_time=1e-5)
    top = spec.face_nodes(2, 1)
    bc.mask[top, 0] = workloads.PRESCRIBED
    bc.vel[top, 0] = 8.0
    dt = 0.9 * oracle.Oracle(spec, MAT, 1e-7, bc).critical_dt()
    seed = np.zeros((spec.n_particles, 6))
    seed[top, 2] = 1.0
    rng = np.random.default_rng(11)
    F = spec.n_facets
    facets = rng.choice(F, 8, replace=False)
    dirs = []
    for k in facets:
        for j in range(3):
            d = np.zeros((3, F))
            d[j, k] = P0[j]
            dirs.append(d)
    dirs += [rng.standard_normal((3, F)) * P0[:, None] for _ in range(2)]
    D = np.array(dirs)
    K = 300
    o = oracle.Oracle(spec, MAT, dt, bc)
    J, dJ = o.tangent(K, seed, D[:, 0], D[:, 1], D[:, 2])
    return dict(spec=spec, bc=bc, dt=dt, seed=seed, K=K, D=D, J=J, dJ=dJ)


def _project(g, D):
    return np.einsum("dpf,pf->d", D, np.array(g))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_gradient_matches_oracle_directional_derivatives(cube, prec):
    c = cube
    m = ldpm.Model(c["spec"], MAT, precision=prec, dt=c["dt"], bc=c["bc"])
    J, gE, ga, gs = m.adjoint(c["K"], c["seed"], ckpt_every=64)
    got = _project((gE, ga, gs), c["D"])
    ref = c["dJ"]
    nd_single = len(ref) - 2
    big = np.abs(ref[:nd_single]).max()
    if prec == "fp64":
        np.testing.assert_allclose(J, c["J"], rtol=1e-11)
        assert np.all(np.abs(got[:nd_single] - ref[:nd_single]) <= 1e-8 * np.abs(ref[:nd_single]) + 1e-10 * big)
        np.testing.assert_allclose(got[nd_single:], ref[nd_single:], rtol=1e-8)
    else:
        np.testing.assert_allclose(J, c["J"], rtol=1e-5)
        assert np.all(np.abs(got[:nd_single] - ref[:nd_single]) <= 2e-3 * np.abs(ref[:nd_single]) + 1e-3 * big)
        np.testing.assert_allclose(got[nd_single:], ref[nd_single:], rtol=2e-3)
    m.close()


def test_adjoint_checkpoint_interval_changes_nothing_and_state_advances():
    spec = specimen.make_cube_specimen(8.0, 2.0, 4.0, 60, seed=2)
    bc = workloads.uniaxial_tension_bc(spec, velocity=40.0, ramp_time=1e-5)
    dt = 1.5e-7
    seed = np.zeros((spec.n_particles, 6))
    seed[spec.face_nodes(2, 1), 2] = 1.0
    seed[spec.face_nodes(2, 0), 2] = -0.5
    res = []
    for ck in (1, 7, 50, 200):
        m = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc)
        out = m.adjoint(50, seed, ckpt_every=ck)
        res.append((out, m.get_state()))
        m.close()
    ref = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc)
    ref.step(50)
    q, v, h, st = ref.get_state()
    for (J, gE, ga, gs), (q2, v2, h2, st2) in res:
        assert J == res[0][0][0]
        for a, b in zip((gE, ga, gs), res[0][0][1:]):
            assert np.array_equal(a, b)
        assert st2 == st and np.array_equal(q2, q) and np.array_equal(v2, v) and np.array_equal(h2, h)
    assert np.abs(res[0][0][1]).max() > 0


def test_forward_with_per_facet_parameters_matches_oracle():
    spec = specimen.make_cube_specimen(10.0, 2.0, 4.0, 120, seed=31)
    bc = workloads.uniaxial_tension_bc(spec, velocity=60.0, ramp_time=1e-5)
    rng = np.random.default_rng(2)
    F = spec.n_facets
    pE, pa, ps = (P0[j] * (1 + 0.2 * rng.uniform(-1, 1, F)) for j in range(3))
    dt = 1.5e-7
    o = oracle.Oracle(spec, MAT, dt, bc)
    o.set_facet_params(pE, pa, ps)
    o.step(400)
    qo, vo, ho, _ = o.get_state()
    wo, _ = o.metrics()
    for prec, tol in (("fp64", 1e-10), ("mixed", 2e-3)):
        m = ldpm.Model(spec, MAT, precision=prec, dt=dt, bc=bc)
        m.set_facet_params(pE, pa, ps)
        m.step(400)
        qg, vg, hg, _ = m.get_state()
        wg, _ = m.metrics()
        nq = np.abs(qg - qo).max() / np.abs(qo).max()
        nh = np.abs(hg - ho).max() / np.abs(ho).max()
        assert nq <= tol and nh <= 20 * tol, (prec, nq, nh)
        assert wo.max() > 0 and np.abs(wg - wo).max() <= 20 * tol * wo.max()
        m.close()
    # the material's values restored: same as a model that never had per-facet parameters
    m1 = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc)
    m1.set_facet_params(pE, pa, ps)
    m1.set_facet_params()
    m1.step(50)
    m2 = ldpm.Model(spec, MAT, precision="fp64", dt=dt, bc=bc)
    m2.step(50)
    assert np.array_equal(m1.get_state()[0], m2.get_state()[0])


def test_autograd_function_returns_the_adjoint_gradient(cube):
    torch = pytest.importorskip("torch")
    from paper_2603_13190_gb300.autograd import reaction_objective
    c = cube
    F = c["spec"].n_facets
    m = ldpm.Model(c["spec"], MAT, precision="fp64", dt=c["dt"], bc=c["bc"])
    E0 = torch.full((F,), MAT["E0"], dtype=torch.float64, requires_grad=True)
    al = torch.full((F,), MAT["alpha"], dtype=torch.float64, requires_grad=True)
    sg = torch.full((F,), MAT["sigma_t"], dtype=torch.float64, requires_grad=True)
    J = reaction_objective(E0, al, sg, m, c["K"], c["seed"], 100)
    J2 = reaction_objective(E0, al, sg, m, c["K"], c["seed"], 100)
    assert float(J) == float(J2), "keep_state: the same function at every call"
    (2.0 * J).backward()
    m2 = ldpm.Model(c["spec"], MAT, precision="fp64", dt=c["dt"], bc=c["bc"])
    m2.set_facet_params(np.full(F, MAT["E0"]), np.full(F, MAT["alpha"]), np.full(F, MAT["sigma_t"]))
    Jr, gE, ga, gs = m2.adjoint(c["K"], c["seed"], 100)
    assert float(J) == Jr
    np.testing.assert_array_equal(E0.grad.numpy(), 2.0 * gE)
    np.testing.assert_array_equal(al.grad.numpy(), 2.0 * ga)
    np.testing.assert_array_equal(sg.grad.numpy(), 2.0 * gs)
    m.close()
    m2.close()


def test_full_size_adjoint_matches_central_differences():
    """The adjoint workload at full size (50 mm cube, 1.82M facets, 5000 steps of elastic and
    pre-peak tension): the FP64 gradient of the mean top reaction along a random direction of 32
    random facets' 96 parameters, and along E0 of the 4 of them with the largest gradient, against
    central differences of the FP64 step (relative step 1e-4); the mixed-mode gradient of the same
    32 facets against the FP64 one."""
    wl = workloads.WORKLOADS["adjoint_uniaxial_tension"]
    spec = wl.specimen()
    bc = workloads.workload_bc(wl.name, spec)
    K = wl.steps
    seed = np.zeros((spec.n_particles, 6))
    seed[spec.face_nodes(2, 1), 2] = 1.0
    F = spec.n_facets
    m = ldpm.Model(spec, wl.material, precision="fp64", bc=bc)
    dt = m.dt
    start = ldpm.ldpm_save_checkpoint(m.h)
    J, gE, ga, gs = m.adjoint(K, seed, ckpt_every=250)
    rng = np.random.default_rng(7)
    fac = rng.choice(F, 32, replace=False)
    G = np.stack([gE[fac], ga[fac], gs[fac]])
    d = rng.standard_normal((3, 32)) * P0[:, None]
    h = 1e-4

    def objective(dp):
        p = np.broadcast_to(P0[:, None], (3, F)).copy()
        p[:, fac] += dp
        ldpm.ldpm_load_checkpoint(m.h, start)
        m.set_facet_params(p[0], p[1], p[2])
        return m.adjoint(K, seed, grads=False)[0]

    # the per-facet path with the material's values reproduces the uniform run
    assert abs(objective(np.zeros((3, 32))) - J) <= 1e-12 * abs(J)
    fd = (objective(h * d) - objective(-h * d)) / (2 * h)
    ad = float(np.sum(G * d))
    assert abs(fd - ad) <= 2e-3 * abs(ad), (fd, ad)
    top = np.argsort(-np.abs(G[0]))[:4]
    for i in top:
        e = np.zeros((3, 32))
        e[0, i] = P0[0]
        fdi = (objective(h * e) - objective(-h * e)) / (2 * h)
        assert abs(fdi - G[0, i] * P0[0]) <= 2e-2 * abs(G[0, i] * P0[0]), (i, fdi, G[0, i] * P0[0])
    m.close()
    mm = ldpm.Model(spec, wl.material, precision="mixed", dt=dt, bc=bc)
    Jm, gEm, gam, gsm = mm.adjoint(K, seed, ckpt_every=250)
    mm.close()
    assert abs(Jm - J) <= 1e-4 * abs(J)
    Gm = np.stack([gEm[fac], gam[fac], gsm[fac]])
    for r in range(2):  # E0 and alpha (sigma_t has no effect before any facet softens)
        assert np.abs(Gm[r] - G[r]).max() <= 2e-2 * np.abs(G[r]).max(), (r, np.abs(Gm[r] - G[r]).max(), np.abs(G[r]).max())
