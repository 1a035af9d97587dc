"""Strain-path points of the facet law in each branch of App. A (shared by the oracle's derivative
pins and the GPU parity tests of the law's vector-Jacobian product)."""
import numpy as np

import oracle
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

MAT = dict(WORKLOAD_MATERIAL)
L_FACET = 3.0
# typical magnitudes of the law's inputs (e, de, eV, t_old, e_max, E0, alpha, sigma_t) and outputs
IN_SCALE = np.array([1e-4] * 3 + [1e-6] * 3 + [1e-4] + [1.0] * 3 + [1e-4] + [MAT["E0"], MAT["alpha"], MAT["sigma_t"]])
OUT_SCALE = np.array([1.0, 1.0, 1.0, 1e-4])


def lin(a, b, n):
    return np.linspace(a, b, n)


def law_point(path, eV, i, mat=MAT):
    """Inputs of the law at step i of a strain path driven from zero (state from the steps before)."""
    t, em = oracle.facet_march(mat, L_FACET, path, eV)
    return np.concatenate([path[i], path[i] - path[i - 1], [eV[i]], t[i - 1], [em[i - 1]],
                           [mat["E0"], mat["alpha"], mat["sigma_t"]]])


def cases():
    n = 40
    z = np.zeros(n)
    c = {}
    c["fracture_elastic"] = (np.stack([lin(0, 4e-5, n), lin(0, 1e-5, n), lin(0, -4e-6, n)], 1), z, 30)
    c["fracture_softening"] = (np.stack([lin(0, 3e-4, n), lin(0, 4e-5, n), lin(0, 1e-5, n)], 1), z, 35)
    up = np.stack([lin(0, 3e-4, n), lin(0, 4e-5, n), lin(0, 1e-5, n)], 1)
    down = np.stack([lin(3e-4, 2.9e-4, n), lin(4e-5, 3.9e-5, n), lin(1e-5, 1e-5, n)], 1)
    c["fracture_unloading"] = (np.vstack([up, down]), np.zeros(2 * n), n + 10)
    c["compression_elastic"] = (np.stack([lin(0, -2e-4, n), lin(0, 3e-5, n), lin(0, -2e-5, n)], 1),
                                lin(0, -1e-4, n), 30)
    c["friction_return"] = (np.stack([lin(0, -1e-4, n), lin(0, 1.6e-3, n), lin(0, 8e-4, n)], 1),
                            lin(0, -5e-5, n), 35)
    c["hardening_linear"] = (np.stack([lin(0, -8e-3, n), lin(0, 1e-4, n), z], 1), lin(0, -5.5e-3, n), 35)
    c["hardening_exponential"] = (np.stack([lin(0, -2e-2, n), lin(0, 1e-4, n), z], 1), lin(0, -1.2e-2, n), 35)
    comp = np.stack([lin(0, -8e-3, n), lin(0, 1e-4, n), z], 1)
    back = np.array([[-2e-3, 1e-4, 0.0], [-1.9e-3, 1e-4, 0.0]])
    c["normal_clamped_at_zero"] = (np.vstack([comp, back]), np.concatenate([lin(0, -5.5e-3, n), [-3e-3, -3e-3]]), n)
    # the unload/reload variants (the material overrides are the fourth entry)
    e0 = MAT["sigma_t"] / MAT["E0"]
    soft = np.stack([lin(0, 3 * e0, n), lin(0, 0.3 * e0, n), lin(0, 0.1 * e0, n)], 1)
    unl = np.stack([lin(3 * e0, 0.2 * e0, n), lin(0.3 * e0, 0.02 * e0, n), lin(0.1 * e0, 0.007 * e0, n)], 1)
    rel = np.stack([lin(0.2 * e0, 2 * e0, n), lin(0.02 * e0, 0.2 * e0, n), lin(0.007 * e0, 0.07 * e0, n)], 1)
    c["reload_crossing_e_tr"] = (np.vstack([soft, unl, rel]), np.zeros(3 * n), None, dict(k_t=0.6))
    hyd = lin(0, -6e-3, n)
    hyd_back = lin(-6e-3, -5.5e-3, 6)[1:]
    c["densified_unloading"] = (np.stack([np.concatenate([hyd, hyd_back]), np.zeros(n + 5), np.zeros(n + 5)], 1),
                                np.concatenate([hyd, hyd_back]), n + 2, dict(Ed_E0=3.0))
    c["shear_softening_H_s"] = (np.stack([lin(0, 2 * e0, n), lin(0, 12 * e0, n), lin(0, 4 * e0, n)], 1), z, 35,
                                dict(r_s=0.2))
    return c


def case(name):
    """(path, eV, step index, material) of a named branch point; for the reload case the index is the
    step that crosses e_tr (traction zero before it, positive after it)."""
    cs = CASES[name]
    mat = dict(MAT, **(cs[3] if len(cs) > 3 else {}))
    path, eV, i = cs[0], cs[1], cs[2]
    if i is None:
        t, _ = oracle.facet_march(mat, L_FACET, path, eV)
        teff = np.sqrt(t[:, 0] ** 2 + (t[:, 1] ** 2 + t[:, 2] ** 2) / mat["alpha"])
        n = len(path) // 3
        i = 2 * n + int(np.flatnonzero(teff[2 * n:] > 0)[0])
    return path, eV, i, mat





CASES = cases()
