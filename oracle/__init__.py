"""ctypes wrapper of the FP64 CPU oracle (ldpm_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's CPU-baseline
and reference legs.  The product path (the CUDA library and its binding) never imports this.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldpm_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

MATERIAL_FIELDS = ("rho", "E0", "alpha", "sigma_t", "l_t", "r_st", "n_t", "sigma_c0", "Hc0_E0", "Hc1_E0",
                   "kc0", "kc1", "kc2", "kc3", "mu0", "mu_inf", "sigma_N0", "Ed_E0", "beta", "k_t", "r_s")


class OrcMaterial(C.Structure):
    _fields_ = [(f, C.c_double) for f in MATERIAL_FIELDS] + [("elastic", C.c_int32), ("pad_", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P, D, I32, I64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
        L.orc_create.restype = P
        L.orc_create.argtypes = [I32, I32, I32, P, P, P, P, P, P, P, P, P, C.POINTER(OrcMaterial), D, P, P, D, P, P]
        L.orc_destroy.argtypes = [P]
        L.orc_step.argtypes = [P, I64]
        L.orc_step.restype = C.c_int
        L.orc_get_state.argtypes = [P, P, P, P, P]
        L.orc_set_state.argtypes = [P, P, P, P, I64]
        L.orc_energy.argtypes = [P, P, P]
        L.orc_facet_forces.argtypes = [P, P, P]
        L.orc_strains.argtypes = [P, P, P, P]
        L.orc_elastic_force.argtypes = [P, P, P]
        L.orc_lambda_max.argtypes = [P, P, I32]
        L.orc_lambda_max.restype = D
        L.orc_geometry.argtypes = [P, P, P, P, P, P, P]
        L.orc_facet_law.argtypes = [C.POINTER(OrcMaterial), D, P, P, D, P, D, P, P]
        L.orc_facet_march.argtypes = [C.POINTER(OrcMaterial), D, I64, P, P, P, P]
        L.orc_metrics.argtypes = [P, P, P]
        L.orc_set_bc.argtypes = [P, P, P, D]
        L.orc_set_facet_params.argtypes = [P, P, P, P]
        L.orc_perturb.argtypes = [P, P]
        L.orc_tangent.argtypes = [P, I64, P, I32, P, P, P, P, P]
        L.orc_tangent.restype = C.c_int
        L.orc_facet_law_jacobian.argtypes = [C.POINTER(OrcMaterial), D, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def material_struct(mat: dict) -> OrcMaterial:
    s = OrcMaterial()
    for f in MATERIAL_FIELDS:
        setattr(s, f, float(mat[f]))
    s.elastic = int(mat.get("elastic", 0))
    return s


def facet_law(mat: dict, l, e, de, eV, t_old, emax_old):
    """Single-facet constitutive update (App. A); returns (t_new[3], emax_new)."""
    m = material_struct(mat)
    e = np.ascontiguousarray(e, np.float64)
    de = np.ascontiguousarray(de, np.float64)
    t_old = np.ascontiguousarray(t_old, np.float64)
    t_new = np.zeros(3)
    em = C.c_double(0.0)
    lib().orc_facet_law(C.byref(m), float(l), _p(e), _p(de), float(eV), _p(t_old), float(emax_old), _p(t_new),
                        C.byref(em))
    return t_new, em.value


LAW_INPUTS = ("eN", "eM", "eL", "deN", "deM", "deL", "eV", "tN", "tM", "tL", "emax", "E0", "alpha", "sigma_t")


def facet_law_jacobian(mat: dict, l, x):
    """Constitutive update and its Jacobian at x = (e[3], de[3], eV, t_old[3], e_max_old, E0, alpha,
    sigma_t) (the order of LAW_INPUTS): returns (out[4] = t_new[3], e_max_new; jac[4, 14])."""
    m = material_struct(mat)
    x = np.ascontiguousarray(x, np.float64).reshape(14)
    out = np.zeros(4)
    jac = np.zeros((4, 14))
    lib().orc_facet_law_jacobian(C.byref(m), float(l), _p(x), _p(out), _p(jac))
    return out, jac


def facet_march(mat: dict, l, path, eV):
    """Drive one facet along a strain path (rows = total strain after each step); returns the
    tractions (n, 3) and e_max (n,) after each step."""
    m = material_struct(mat)
    path = np.ascontiguousarray(path, np.float64).reshape(-1, 3)
    eV = np.ascontiguousarray(np.broadcast_to(eV, (len(path),)), np.float64)
    t = np.zeros((len(path), 3))
    em = np.zeros(len(path))
    lib().orc_facet_march(C.byref(m), float(l), len(path), _p(path), _p(eV), _p(t), _p(em))
    return t, em


class Oracle:
    """One specimen in the oracle.  Arrays use the raw specimen ordering."""

    def __init__(self, spec, material: dict, dt: float, bc=None, mass=None, inertia=None, f_ext=None):
        self._keep = []
        N, T, F = spec.n_particles, spec.n_tets, spec.n_facets

        def arr(a, dt_):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt_)
            self._keep.append(a)
            return a

        x = arr(spec.x, np.float64)
        dia = arr(spec.diameter, np.float64)
        tets = arr(spec.tets, np.int32)
        fpi, fpj, ftet = arr(spec.facet_pi, np.int32), arr(spec.facet_pj, np.int32), arr(spec.facet_tet, np.int32)
        vtx = arr(spec.facet_vtx, np.float64)
        mask = vel = v0 = None
        ramp = 0.0
        if bc is not None:
            mask, vel, v0, ramp = arr(bc.mask, np.int32), arr(bc.vel, np.float64), arr(bc.v0, np.float64), bc.ramp_time
        self._mat = material_struct(material)
        self.material = dict(material)
        h = lib().orc_create(N, T, F, _p(x), _p(dia), _p(tets), _p(fpi), _p(fpj), _p(ftet), _p(vtx),
                             _p(arr(mass, np.float64)), _p(arr(inertia, np.float64)), C.byref(self._mat),
                             float(dt), _p(mask), _p(vel), float(ramp), _p(v0), _p(arr(f_ext, np.float64)))
        if not h:
            raise ValueError("oracle rejected the geometry")
        self.h = h
        self.N, self.T, self.F, self.dt = N, T, F, dt

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def step(self, n: int = 1) -> None:
        rc = lib().orc_step(self.h, int(n))
        if rc != 0:
            raise FloatingPointError("oracle state became non-finite")

    def get_state(self):
        q = np.zeros((self.N, 6))
        v = np.zeros((self.N, 6))
        h5 = np.zeros((self.F, 5))
        st = C.c_int64(0)
        lib().orc_get_state(self.h, _p(q), _p(v), _p(h5), C.byref(st))
        return q, v, h5, st.value

    def set_state(self, q, v, hist5, step: int = 0) -> None:
        q = np.ascontiguousarray(q, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        h5 = np.ascontiguousarray(hist5, np.float64)
        lib().orc_set_state(self.h, _p(q), _p(v), _p(h5), int(step))

    def energy(self):
        out = np.zeros(4)
        r = np.zeros(12)
        lib().orc_energy(self.h, _p(out), _p(r))
        return out, r

    def facet_forces(self):
        F3 = np.zeros((self.F, 3))
        f6 = np.zeros((self.N, 6))
        lib().orc_facet_forces(self.h, _p(F3), _p(f6))
        return F3, f6

    def strains(self, q):
        q = np.ascontiguousarray(q, np.float64)
        e = np.zeros((self.F, 3))
        eV = np.zeros(max(self.T, 1))
        lib().orc_strains(self.h, _p(q), _p(e), _p(eV))
        return e, eV[: self.T]

    def elastic_force(self, q):
        q = np.ascontiguousarray(q, np.float64)
        f = np.zeros((self.N, 6))
        lib().orc_elastic_force(self.h, _p(q), _p(f))
        return f

    def lambda_max(self, x0, iters: int = 200) -> float:
        x0 = np.ascontiguousarray(x0, np.float64)
        return float(lib().orc_lambda_max(self.h, _p(x0), int(iters)))

    def critical_dt(self, seed: int = 0, iters: int = 300) -> float:
        x0 = np.random.default_rng(seed).standard_normal(6 * self.N)
        return 2.0 / np.sqrt(self.lambda_max(x0, iters))

    def metrics(self):
        """Crack opening per facet and volumetric strain per tetrahedron of the current state."""
        w = np.zeros(self.F)
        eV = np.zeros(max(self.T, 1))
        lib().orc_metrics(self.h, _p(w), _p(eV))
        return w, eV[: self.T]

    def set_bc(self, bc) -> None:
        mask = np.ascontiguousarray(bc.mask, np.int32)
        vel = np.ascontiguousarray(bc.vel, np.float64)
        self._keep += [mask, vel]
        lib().orc_set_bc(self.h, _p(mask), _p(vel), float(bc.ramp_time))

    def perturb(self, dq) -> None:
        """q += dq [N, 6] on free DOFs; the perturbed state is the next increment's reference."""
        dq = np.ascontiguousarray(dq, np.float64).reshape(self.N, 6)
        lib().orc_perturb(self.h, _p(dq))

    def set_facet_params(self, E0=None, alpha=None, sigma_t=None) -> None:
        """Per-facet E0, alpha, sigma_t ([F] each, specimen facet order); None = material value."""
        arrs = [None if a is None else np.ascontiguousarray(np.broadcast_to(a, (self.F,)), np.float64)
                for a in (E0, alpha, sigma_t)]
        lib().orc_set_facet_params(self.h, *[_p(a) for a in arrs])

    def tangent(self, nsteps: int, seed, dE0=None, dalpha=None, dsigma_t=None):
        """J = time mean over the next `nsteps` steps of sum_i seed_i R_i (seed [N, 6], reactions on
        constrained DOFs), and its derivatives along the rows of dE0 / dalpha / dsigma_t ([nd, F] each,
        None = 0).  The model's state is left unchanged.  Returns (J, dJ[nd])."""
        seed = np.ascontiguousarray(seed, np.float64).reshape(self.N, 6)
        dirs = [None if d is None else np.ascontiguousarray(np.atleast_2d(d), np.float64) for d in (dE0, dalpha, dsigma_t)]
        nd = max([0] + [d.shape[0] for d in dirs if d is not None])
        for d in dirs:
            if d is not None and d.shape != (nd, self.F):
                raise ValueError("direction arrays must be [nd, F]")
        J = C.c_double(0.0)
        dJ = np.zeros(nd)
        rc = lib().orc_tangent(self.h, int(nsteps), _p(seed), nd, *[_p(d) for d in dirs], C.byref(J), _p(dJ))
        if rc != 0:
            raise FloatingPointError("oracle trajectory became non-finite")
        return J.value, dJ

    def geometry(self):
        n = np.zeros((self.F, 3))
        l = np.zeros(self.F)
        A = np.zeros(self.F)
        m6 = np.zeros((self.N, 6))
        ci = np.zeros((self.F, 3))
        cj = np.zeros((self.F, 3))
        lib().orc_geometry(self.h, _p(n), _p(l), _p(A), _p(m6), _p(ci), _p(cj))
        return dict(n=n, len=l, area=A, mass=m6, ci=ci, cj=cj)
