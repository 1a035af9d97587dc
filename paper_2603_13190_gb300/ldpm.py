"""Thin ctypes binding of libldpm.so (include/ldpm.h): the same entry points, argument marshalling only.

Every computation happens in the CUDA library.  If the library is missing or cannot be loaded the
import of this module's functions raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LDPM_OK = 0
ERRORS = {
    -1: "LDPM_E_INVALID_ARG",
    -2: "LDPM_E_BAD_GEOMETRY",
    -3: "LDPM_E_CUDA",
    -4: "LDPM_E_OOM",
    -5: "LDPM_E_UNSTABLE",
    -6: "LDPM_E_TIMEOUT",
    -7: "LDPM_E_UNSUPPORTED",
}
LDPM_FP64, LDPM_MIXED = 0, 1
MATERIAL_FIELDS = ("rho", "E0", "alpha", "sigma_t", "l_t", "r_st", "n_t", "sigma_c0", "Hc0_E0", "Hc1_E0",
                   "kc0", "kc1", "kc2", "kc3", "mu0", "mu_inf", "sigma_N0", "Ed_E0", "beta", "k_t", "r_s")


class LdpmError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed: %s (%s)" % (where, ERRORS.get(code, code), msg))
        self.code = code


class Geometry(C.Structure):
    _fields_ = [("n_particles", C.c_int32), ("n_tets", C.c_int32), ("n_facets", C.c_int32),
                ("x", C.c_void_p), ("diameter", C.c_void_p), ("tet", C.c_void_p), ("facet_pi", C.c_void_p),
                ("facet_pj", C.c_void_p), ("facet_tet", C.c_void_p), ("facet_vtx", C.c_void_p),
                ("mass", C.c_void_p), ("inertia", C.c_void_p)]


class Material(C.Structure):
    _fields_ = [(f, C.c_double) for f in MATERIAL_FIELDS] + [("elastic", C.c_int32), ("reserved", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("graph_chunk", C.c_int32), ("dt", C.c_double), ("dt_factor", C.c_double),
                ("cuda_stream", C.c_void_p), ("bc_mask", C.c_void_p), ("bc_vel", C.c_void_p),
                ("ramp_time", C.c_double), ("v0", C.c_void_p), ("f_ext", C.c_void_p), ("device", C.c_int32),
                ("autotune", C.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def signatures():
    """ctypes argument and result types of every entry point of include/ldpm.h (pointers and arrays
    as c_void_p)."""
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    return {
        "ldpm_create": ([P, P, P, P], C.c_int),
        "ldpm_step": ([P, I64], C.c_int),
        "ldpm_sync": ([P], C.c_int),
        "ldpm_set_launch_mode": ([P, I32], C.c_int),
        "ldpm_launch_mode": ([P], I32),
        "ldpm_set_barrier_wait": ([P, D, I32], C.c_int),
        "ldpm_get_state": ([P, P, P, P, P], C.c_int),
        "ldpm_get_state_device": ([P, P, P, P, P], C.c_int),
        "ldpm_set_state": ([P, P, P, P, I64], C.c_int),
        "ldpm_energy": ([P, P, P], C.c_int),
        "ldpm_facet_forces": ([P, P, P], C.c_int),
        "ldpm_set_bc": ([P, P, P, D], C.c_int),
        "ldpm_metrics": ([P, P, P], C.c_int),
        "ldpm_info": ([P, P, P], C.c_int),
        "ldpm_profile": ([P, I32], C.c_int),
        "ldpm_profile_read": ([P, P, P, I32], C.c_int),
        "ldpm_checkpoint_size": ([P], I64),
        "ldpm_save_checkpoint": ([P, P], C.c_int),
        "ldpm_load_checkpoint": ([P, P], C.c_int),
        "ldpm_destroy": ([P], None),
        "ldpm_last_error": ([], C.c_char_p),
        "ldpm_kinetic_energy_noalloc": ([P, P, I64, P, P], C.c_int),
        "ldpm_batch_create": ([I32, P, P, P, P], C.c_int),
        "ldpm_batch_step": ([P, I64], C.c_int),
        "ldpm_batch_size": ([P], I32),
        "ldpm_batch_get_state": ([P, I32, P, P, P, P], C.c_int),
        "ldpm_batch_energy": ([P, I32, P, P], C.c_int),
        "ldpm_batch_metrics": ([P, I32, P, P], C.c_int),
        "ldpm_batch_info": ([P, I32, P, P], C.c_int),
        "ldpm_launch_shape": ([P, P], C.c_int),
        "ldpm_set_facet_params": ([P, P, P, P], C.c_int),
        "ldpm_perturb": ([P, P], C.c_int),
        "ldpm_adjoint": ([P, I64, I32, P, P, P, P, P], C.c_int),
        "ldpm_facet_law_vjp": ([I32, P, I64, P, P, P, P], C.c_int),
    }


def lib():
    """Load libldpm.so (building it first if the sources are newer).  Raises if that fails."""
    global _lib
    if _lib is None:
        # LDPM_LIBRARY: load an already-built libldpm.so from another path (no build step)
        path = os.environ.get("LDPM_LIBRARY") or _build.build()
        if not os.path.exists(path):
            raise ImportError("libldpm.so is missing at %s" % path)
        L = C.CDLL(path)
        sig = signatures()
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != LDPM_OK:
        raise LdpmError(rc, where, lib().ldpm_last_error().decode())


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream) or None  # torch.cuda.Stream


# --------------------------------------------------------------------------------------------------
# Entry points with the C names.
# --------------------------------------------------------------------------------------------------
def _structs(spec, material: dict, precision: int, dt: float, dt_factor: float, bc, f_ext, stream, graph_chunk,
             mass, inertia, device, autotune, keep):
    def arr(a, dtp):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtp)
        keep.append(a)
        return a

    g = Geometry(spec.n_particles, spec.n_tets, spec.n_facets, _ptr(arr(spec.x, np.float64)),
                 _ptr(arr(spec.diameter, np.float64)), _ptr(arr(spec.tets, np.int32)),
                 _ptr(arr(spec.facet_pi, np.int32)), _ptr(arr(spec.facet_pj, np.int32)),
                 _ptr(arr(spec.facet_tet, np.int32)), _ptr(arr(spec.facet_vtx, np.float64)),
                 _ptr(arr(mass, np.float64)), _ptr(arr(inertia, np.float64)))
    m = Material(*[float(material[f]) for f in MATERIAL_FIELDS], int(material.get("elastic", 0)), 0)
    o = Options()
    o.precision = int(precision)
    o.graph_chunk = int(graph_chunk)
    o.dt = float(dt)
    o.dt_factor = float(dt_factor)
    o.cuda_stream = _stream_handle(stream)
    o.device = int(device)
    o.autotune = 1 if autotune else 0
    if bc is not None:
        o.bc_mask = _ptr(arr(bc.mask, np.int32))
        o.bc_vel = _ptr(arr(bc.vel, np.float64))
        o.ramp_time = float(bc.ramp_time)
        o.v0 = _ptr(arr(bc.v0, np.float64))
    o.f_ext = _ptr(arr(f_ext, np.float64))
    return g, m, o


def ldpm_create(spec, material: dict, precision: int = LDPM_MIXED, dt: float = 0.0, dt_factor: float = 0.9,
                bc=None, f_ext=None, stream=None, graph_chunk: int = 0, mass=None, inertia=None,
                device: int = -1, autotune: bool = False):
    """Create a handle from a specimen (see specimen.Specimen) and a material dict.  The caller-owned
    arrays only need to live for the duration of the call."""
    keep = []
    g, m, o = _structs(spec, material, precision, dt, dt_factor, bc, f_ext, stream, graph_chunk, mass, inertia,
                       device, autotune, keep)
    h = C.c_void_p()
    _check(lib().ldpm_create(C.byref(g), C.byref(m), C.byref(o), C.byref(h)), "ldpm_create")
    return h


def ldpm_batch_create(specs, materials, precision: int = LDPM_MIXED, dts=None, bcs=None, stream=None,
                      graph_chunk: int = 0, device: int = -1, autotune: bool = False, dt_factor: float = 0.9):
    """Create one handle stepping all specimens together (lists of equal length)."""
    n = len(specs)
    keep = []
    G, M, O = (Geometry * n)(), (Material * n)(), (Options * n)()
    for i, sp in enumerate(specs):
        g, m, o = _structs(sp, materials[i], precision, 0.0 if dts is None else dts[i], dt_factor,
                           None if bcs is None else bcs[i], None, stream, graph_chunk, None, None, device,
                           autotune, keep)
        G[i], M[i], O[i] = g, m, o
    h = C.c_void_p()
    _check(lib().ldpm_batch_create(n, G, M, O, C.byref(h)), "ldpm_batch_create")
    return h


def ldpm_batch_step(h, nsteps: int) -> None:
    _check(lib().ldpm_batch_step(h, int(nsteps)), "ldpm_batch_step")


def ldpm_batch_size(h) -> int:
    n = lib().ldpm_batch_size(h)
    if n < 0:
        _check(n, "ldpm_batch_size")
    return int(n)


def ldpm_batch_get_state(h, idx: int, N: int, F: int, hist: bool = True):
    q = np.zeros((N, 6))
    v = np.zeros((N, 6))
    h5 = np.zeros((F, 5)) if hist else None
    st = C.c_int64(0)
    _check(lib().ldpm_batch_get_state(h, int(idx), _ptr(q), _ptr(v), _ptr(h5), C.byref(st)), "ldpm_batch_get_state")
    return q, v, h5, st.value


def ldpm_batch_energy(h, idx: int):
    out = np.zeros(4)
    r = np.zeros(12)
    _check(lib().ldpm_batch_energy(h, int(idx), _ptr(out), _ptr(r)), "ldpm_batch_energy")
    return out, r


def ldpm_batch_metrics(h, idx: int, F: int, T: int):
    w = np.zeros(F)
    eV = np.zeros(T)
    _check(lib().ldpm_batch_metrics(h, int(idx), _ptr(w), _ptr(eV)), "ldpm_batch_metrics")
    return w, eV


def ldpm_batch_info(h, idx: int):
    info = np.zeros(5, np.int64)
    dt = C.c_double(0.0)
    _check(lib().ldpm_batch_info(h, int(idx), _ptr(info), C.byref(dt)), "ldpm_batch_info")
    return info, dt.value


def ldpm_launch_shape(h):
    shape = np.zeros(2, np.int32)
    _check(lib().ldpm_launch_shape(h, _ptr(shape)), "ldpm_launch_shape")
    return int(shape[0]), int(shape[1])


def ldpm_step(h, nsteps: int) -> None:
    _check(lib().ldpm_step(h, int(nsteps)), "ldpm_step")


LDPM_LAUNCH_PAIRS, LDPM_LAUNCH_PERSISTENT = 1, 2


def ldpm_set_launch_mode(h, mode: int) -> None:
    _check(lib().ldpm_set_launch_mode(h, int(mode)), "ldpm_set_launch_mode")


def ldpm_launch_mode(h) -> int:
    r = lib().ldpm_launch_mode(h)
    if r < 0:
        _check(r, "ldpm_launch_mode")
    return int(r)


def ldpm_set_barrier_wait(h, seconds: float, skip_block: int = -1) -> None:
    _check(lib().ldpm_set_barrier_wait(h, float(seconds), int(skip_block)), "ldpm_set_barrier_wait")


def ldpm_sync(h) -> None:
    _check(lib().ldpm_sync(h), "ldpm_sync")


def ldpm_get_state(h, N: int, F: int, hist: bool = True):
    q = np.zeros((N, 6))
    v = np.zeros((N, 6))
    h5 = np.zeros((F, 5)) if hist else None
    st = C.c_int64(0)
    _check(lib().ldpm_get_state(h, _ptr(q), _ptr(v), _ptr(h5), C.byref(st)), "ldpm_get_state")
    return q, v, h5, st.value


def ldpm_get_state_device(h, q_dev: int, v_dev: int, hist5_dev: int, step_dev: int) -> None:
    """Device addresses (ints, 0 = NULL) of caller-owned buffers on the handle's device."""
    _check(lib().ldpm_get_state_device(h, q_dev or None, v_dev or None, hist5_dev or None, step_dev or None),
           "ldpm_get_state_device")


def ldpm_set_state(h, q, v, hist5=None, step: int = 0) -> None:
    q = np.ascontiguousarray(q, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    h5 = None if hist5 is None else np.ascontiguousarray(hist5, np.float64)
    _check(lib().ldpm_set_state(h, _ptr(q), _ptr(v), _ptr(h5), int(step)), "ldpm_set_state")


def ldpm_energy(h):
    out = np.zeros(4)
    r = np.zeros(12)
    _check(lib().ldpm_energy(h, _ptr(out), _ptr(r)), "ldpm_energy")
    return out, r


def ldpm_facet_forces(h, N: int, F: int):
    F3 = np.zeros((F, 3))
    f6 = np.zeros((N, 6))
    _check(lib().ldpm_facet_forces(h, _ptr(F3), _ptr(f6)), "ldpm_facet_forces")
    return F3, f6


def ldpm_metrics(h, F: int, T: int):
    w = np.zeros(F)
    eV = np.zeros(T)
    _check(lib().ldpm_metrics(h, _ptr(w), _ptr(eV)), "ldpm_metrics")
    return w, eV


def ldpm_set_bc(h, mask, vel, ramp_time: float) -> None:
    mask = np.ascontiguousarray(mask, np.int32)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64)
    _check(lib().ldpm_set_bc(h, _ptr(mask), _ptr(vel), float(ramp_time)), "ldpm_set_bc")


def ldpm_info(h):
    info = np.zeros(5, np.int64)
    dt = C.c_double(0.0)
    _check(lib().ldpm_info(h, _ptr(info), C.byref(dt)), "ldpm_info")
    return info, dt.value


def ldpm_profile(h, enable: bool) -> None:
    _check(lib().ldpm_profile(h, 1 if enable else 0), "ldpm_profile")


def ldpm_profile_read(h):
    """Summed milliseconds and launch counts: kick, facet pass, particle pass, reverse facet pass,
    reverse particle pass, persistent step launch."""
    ms = np.zeros(6)
    cnt = np.zeros(6, np.int64)
    _check(lib().ldpm_profile_read(h, _ptr(ms), _ptr(cnt), 6), "ldpm_profile_read")
    return ms, cnt


def ldpm_checkpoint_size(h) -> int:
    n = lib().ldpm_checkpoint_size(h)
    if n < 0:
        _check(int(n), "ldpm_checkpoint_size")
    return int(n)


def ldpm_save_checkpoint(h) -> np.ndarray:
    buf = np.zeros(ldpm_checkpoint_size(h), np.uint8)
    _check(lib().ldpm_save_checkpoint(h, _ptr(buf)), "ldpm_save_checkpoint")
    return buf


def ldpm_load_checkpoint(h, buf) -> None:
    buf = np.ascontiguousarray(buf, np.uint8)
    _check(lib().ldpm_load_checkpoint(h, _ptr(buf)), "ldpm_load_checkpoint")


def ldpm_destroy(h) -> None:
    if h:
        lib().ldpm_destroy(h)


def ldpm_kinetic_energy_noalloc(v_dev: int, mass_dev: int, n_dof: int, out_dev: int, stream=None) -> None:
    """Device pointers in, device pointer out; enqueued on `stream`, allocates nothing."""
    _check(lib().ldpm_kinetic_energy_noalloc(C.c_void_p(v_dev), C.c_void_p(mass_dev), int(n_dof),
                                             C.c_void_p(out_dev), _stream_handle(stream)),
           "ldpm_kinetic_energy_noalloc")


def ldpm_perturb(h, dq) -> None:
    """Add dq [N, 6] to the free displacements and rotations of the current state."""
    dq = np.ascontiguousarray(dq, np.float64)
    _check(lib().ldpm_perturb(h, _ptr(dq)), "ldpm_perturb")


def ldpm_set_facet_params(h, F: int, E0=None, alpha=None, sigma_t=None) -> None:
    """Per-facet E0 / alpha / sigma_t ([F] each, facet order; None = the material's value)."""
    arrs = [None if a is None else np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (F,)))
            for a in (E0, alpha, sigma_t)]
    _check(lib().ldpm_set_facet_params(h, *[_ptr(a) for a in arrs]), "ldpm_set_facet_params")


def ldpm_adjoint(h, N: int, F: int, nsteps: int, seed, ckpt_every: int = 250, grads: bool = True):
    """Objective J (time mean of the seeded reactions over the next nsteps steps; seed [N, 6]) and its
    gradient with respect to per-facet E0, alpha, sigma_t ([F] each).  Advances the model by nsteps."""
    seed = np.ascontiguousarray(seed, np.float64).reshape(N, 6)
    J = C.c_double(0.0)
    g = [np.zeros(F) for _ in range(3)] if grads else [None, None, None]
    _check(lib().ldpm_adjoint(h, int(nsteps), int(ckpt_every), _ptr(seed), C.byref(J), *[_ptr(x) for x in g]),
           "ldpm_adjoint")
    return J.value, g[0], g[1], g[2]


def ldpm_facet_law_vjp(precision: int, material: dict, inp, adj_out):
    """Device law and its vector-Jacobian product on independent rows (layouts in include/ldpm.h):
    inp [n, 16], adj_out [n, 4] -> (out [n, 4], adj_in [n, 16])."""
    inp = np.ascontiguousarray(inp, np.float64).reshape(-1, 16)
    adj_out = np.ascontiguousarray(adj_out, np.float64).reshape(-1, 4)
    n = inp.shape[0]
    out = np.zeros((n, 4))
    adj_in = np.zeros((n, 16))
    m = Material()
    for f in MATERIAL_FIELDS:
        setattr(m, f, float(material[f]))
    m.elastic = int(material.get("elastic", 0))
    _check(lib().ldpm_facet_law_vjp(int(precision), C.byref(m), n, _ptr(inp), _ptr(adj_out), _ptr(out), _ptr(adj_in)),
           "ldpm_facet_law_vjp")
    return out, adj_in


def ldpm_last_error() -> str:
    return lib().ldpm_last_error().decode()


# --------------------------------------------------------------------------------------------------
# Convenience object (still marshalling only).
# --------------------------------------------------------------------------------------------------
class Batch:
    """Several specimens stepped together on the GPU."""

    def __init__(self, specs, materials, precision: str | int = "mixed", dts=None, bcs=None, **kw):
        prec = precision if isinstance(precision, int) else (LDPM_MIXED if precision == "mixed" else LDPM_FP64)
        self.sizes = [(s.n_particles, s.n_tets, s.n_facets) for s in specs]
        self.h = ldpm_batch_create(specs, materials, prec, dts=dts, bcs=bcs, **kw)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "h", None):
            ldpm_destroy(self.h)
            self.h = None

    def __len__(self):
        return len(self.sizes)

    def step(self, n: int = 1):
        ldpm_batch_step(self.h, n)

    def get_state(self, idx: int, hist: bool = True):
        N, _, F = self.sizes[idx]
        return ldpm_batch_get_state(self.h, idx, N, F, hist)

    def energy(self, idx: int):
        return ldpm_batch_energy(self.h, idx)

    def metrics(self, idx: int):
        _, T, F = self.sizes[idx]
        return ldpm_batch_metrics(self.h, idx, F, T)

    def info(self, idx: int):
        return ldpm_batch_info(self.h, idx)

    def launch_shape(self):
        return ldpm_launch_shape(self.h)


class Model:
    """One specimen on the GPU.  Arrays are in the specimen's own particle/facet order."""

    def __init__(self, spec, material: dict, precision: str | int = "mixed", dt: float = 0.0, bc=None, **kw):
        prec = precision if isinstance(precision, int) else (LDPM_MIXED if precision == "mixed" else LDPM_FP64)
        self.N, self.T, self.F = spec.n_particles, spec.n_tets, spec.n_facets
        self._stream = kw.get("stream")
        self.h = ldpm_create(spec, material, prec, dt=dt, bc=bc, **kw)
        info, self.dt = ldpm_info(self.h)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "h", None):
            ldpm_destroy(self.h)
            self.h = None

    def step(self, n: int = 1):
        ldpm_step(self.h, n)

    def sync(self):
        ldpm_sync(self.h)

    def get_state(self, hist: bool = True):
        return ldpm_get_state(self.h, self.N, self.F, hist)

    def get_state_device(self, hist: bool = True, device=None):
        """The state as torch tensors on the device (torch only allocates the buffers; the library's
        kernels fill them on its stream, which the caller's current stream then waits on)."""
        import torch

        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        q = torch.empty((self.N, 6), dtype=torch.float64, device=dev)
        v = torch.empty((self.N, 6), dtype=torch.float64, device=dev)
        h5 = torch.empty((self.F, 5), dtype=torch.float64, device=dev) if hist else None
        st = torch.empty((1,), dtype=torch.int64, device=dev)
        ldpm_get_state_device(self.h, q.data_ptr(), v.data_ptr(), h5.data_ptr() if hist else 0, st.data_ptr())
        if isinstance(self._stream, torch.cuda.Stream):
            torch.cuda.current_stream(dev).wait_stream(self._stream)
        else:  # a library-owned or raw stream: wait for it
            ldpm_sync(self.h)
        return q, v, h5, st

    def set_state(self, q, v, hist5=None, step: int = 0):
        ldpm_set_state(self.h, q, v, hist5, step)

    def energy(self):
        return ldpm_energy(self.h)

    def facet_forces(self):
        return ldpm_facet_forces(self.h, self.N, self.F)

    def set_bc(self, mask, vel, ramp_time):
        ldpm_set_bc(self.h, mask, vel, ramp_time)

    def metrics(self):
        return ldpm_metrics(self.h, self.F, self.T)

    def launch_shape(self):
        return ldpm_launch_shape(self.h)

    def info(self):
        return ldpm_info(self.h)

    def perturb(self, dq):
        ldpm_perturb(self.h, np.asarray(dq, np.float64).reshape(self.N, 6))

    def set_facet_params(self, E0=None, alpha=None, sigma_t=None):
        ldpm_set_facet_params(self.h, self.F, E0, alpha, sigma_t)

    def adjoint(self, nsteps: int, seed, ckpt_every: int = 250, grads: bool = True):
        """(J, dJ/dE0, dJ/dalpha, dJ/dsigma_t); the model advances by nsteps."""
        return ldpm_adjoint(self.h, self.N, self.F, nsteps, seed, ckpt_every, grads)
