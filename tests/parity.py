"""Comparison helpers of the parity tests (GPU result against the FP64 oracle).

Per-element relative tolerance: every element of the GPU result g must satisfy

    |g - o| <= tol |o| + floor,   floor = 1e-4 tol max|o|,

so an element 10^-4 below the largest one is still held to its own relative error (the floor only
covers elements that are exact zeros or within rounding of zero in the oracle).  The FP64 mode's
per-step contract is tol = 1e-10.  The mixed mode's one-step node forces are held to a normwise
tolerance (the largest error over the largest element), because a facet computed in FP32 carries an
absolute error of the order of the unit roundoff times its own magnitude, which a small net force of
a particle (where the facet forces of ~24 tetrahedra cancel) inherits.
"""
from __future__ import annotations

import numpy as np


def elementwise_excess(g, o, tol):
    """Largest ratio |g - o| / (tol |o| + floor) over the elements (<= 1 passes) and the number of
    elements above 1."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    big = float(np.abs(o).max()) if o.size else 0.0
    bound = tol * np.abs(o) + 1e-4 * tol * big
    err = np.abs(g - o)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.where(err > 0, np.inf, 0.0))
    return (float(r.max()) if r.size else 0.0), int(np.sum(r > 1.0))


def assert_elementwise(g, o, tol, what=""):
    worst, n_bad = elementwise_excess(g, o, tol)
    assert worst <= 1.0, "%s: %d elements outside |g - o| <= %.0e |o| + floor (worst %.3g x the bound)" % (
        what, n_bad, tol, worst)


def normwise_rel(a, b):
    """max |a - b| / max |b| (the largest error relative to the largest element)."""
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a - b).max())


def branch_flips(h_gpu, h_orc, scale):
    """Facets whose normal traction has opposite signs in the two results (one took the fracture
    branch, the other compression), counting only tractions above `scale` in magnitude."""
    a, b = np.asarray(h_gpu)[:, 0], np.asarray(h_orc)[:, 0]
    return int(np.sum((np.sign(a) != np.sign(b)) & (np.maximum(np.abs(a), np.abs(b)) > scale)))
