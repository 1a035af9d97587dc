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
    return c





CASES = cases()
