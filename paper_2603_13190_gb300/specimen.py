"""Seeded synthetic LDPM specimens: particle placement, Delaunay mesh, 12-facet tessellation.

This module produces the raw geometry that both the CUDA library and the FP64 oracle consume.  It
holds none of the time-step arithmetic (no strains, tractions, masses or forces): only the mesh
construction that the paper delegates to a preprocessor (Sec. 3.1) and sketches in Sec. 1 and
Fig. 1 (random particle placement following a Fuller sieve curve, Delaunay tetrahedralization of the
particle centres, and a tessellation that cuts every tetrahedron into 12 triangular facets, two per
edge).

Placement.  Diameters are drawn from the number density implied by a Fuller curve with exponent
n_F (mass passing sieve d proportional to d**n_F, so the number density is proportional to
d**(n_F - 4)) between d_min and d_max, sorted largest first, and placed by random sequential
addition (RSA) inside the cube.  A particle count target fixes how many particles are drawn; the
hard-core exclusion distance between two particles is kappa * (d_i + d_j) / 2 with kappa chosen so
the excluded volume fraction stays below the RSA jamming limit.  Cube vertices, nodes along the
cube edges and RSA nodes on the cube faces carry diameter 0 (they are the zero-size surface nodes
that make the specimen faces flat, so boundary conditions act on a plane).

Tessellation (one fixed, documented choice; the paper leaves it to the preprocessor):
  * edge point E_ij: midpoint of the gap between the exclusion spheres of particles i and j on
    segment ij;
  * face point of triangle ijk: mean of its three edge points;
  * tetrahedron point C: mean of its six edge points;
  * the two facets of edge ij in a tetrahedron with other vertices k, l are the triangles
    (E_ij, F_ijk, C) and (E_ij, F_ijl, C).
Every tetrahedron therefore owns exactly 12 facets, two per edge, and facet k separates its edge's
particles I = facet_pi[k] and J = facet_pj[k].

All randomness comes from numpy's PCG64 seeded with the caller's seed, so a specimen is the same on
any machine.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # scipy is present on every machine this runs on; keep the import error readable anyway.
    from scipy.spatial import Delaunay, cKDTree
except Exception as exc:  # pragma: no cover
    raise ImportError("specimen generation needs scipy.spatial") from exc

# Local vertex pairs of the six tetrahedron edges, in the order facets are emitted.
TET_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


@dataclasses.dataclass
class Specimen:
    """Raw geometry of one specimen (mm).

    x          (N, 3) float64  particle centres
    diameter   (N,)   float64  particle diameters (0 for surface nodes)
    tets       (T, 4) int32    Delaunay tetrahedra (particle indices)
    facet_pi   (F,)   int32    particle I of each facet
    facet_pj   (F,)   int32    particle J of each facet
    facet_tet  (F,)   int32    tetrahedron owning each facet
    facet_vtx  (F, 9) float64  the facet triangle's three vertices (x0 y0 z0 x1 y1 z1 x2 y2 z2)
    edge       float            cube edge length
    d_min, d_max float          diameter range used by the placement
    """

    x: np.ndarray
    diameter: np.ndarray
    tets: np.ndarray
    facet_pi: np.ndarray
    facet_pj: np.ndarray
    facet_tet: np.ndarray
    facet_vtx: np.ndarray
    edge: float
    d_min: float
    d_max: float

    @property
    def n_particles(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_facets(self) -> int:
        return int(self.facet_pi.shape[0])

    def face_nodes(self, axis: int, side: int, tol: float | None = None) -> np.ndarray:
        """Indices of the nodes lying on the cube face x[axis] == 0 (side 0) or == edge (side 1)."""
        tol = 1e-9 * self.edge if tol is None else tol
        target = 0.0 if side == 0 else self.edge
        return np.nonzero(np.abs(self.x[:, axis] - target) <= tol)[0]


def fuller_diameters(n: int, d_min: float, d_max: float, n_f: float, rng: np.random.Generator) -> np.ndarray:
    """Draw n diameters from the Fuller-curve number density p(d) ~ d**(n_f - 4) on [d_min, d_max].

    Inverse-CDF sampling with q = 3 - n_f:  CDF(d) = (d_min**-q - d**-q) / (d_min**-q - d_max**-q).
    Returned sorted largest first (the RSA order).
    """
    q = 3.0 - n_f
    u = rng.random(n)
    a, b = d_min ** (-q), d_max ** (-q)
    d = (a - u * (a - b)) ** (-1.0 / q)
    return np.sort(d)[::-1].copy()


def _rsa_points(n_target, radii, lo, hi, rng, dim=3, max_rounds=400, batch=None):
    """Random sequential addition of len(radii) hard spheres (given exclusion radii) in a box.

    Candidates are proposed in batches; a candidate survives if it clears every placed sphere and
    every earlier surviving candidate of its batch.  Spheres that fail are retried with new random
    positions.  Returns the placed centres in the order of `radii` that were placed (may be fewer
    than requested if the box jams).
    """
    radii = np.asarray(radii, dtype=np.float64)
    n = len(radii)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    placed_pts = np.empty((0, dim))
    placed_r = np.empty((0,))
    pending = np.arange(n)
    r_max = radii.max() if n else 0.0
    batch = batch or max(256, n // 8)
    rounds = 0
    stale = 0
    while len(pending) and rounds < max_rounds and stale < 8:
        rounds += 1
        idx = pending[:batch]
        r = radii[idx]
        lo_i = lo[None, :] + r[:, None] * 0.0
        cand = lo_i + rng.random((len(idx), dim)) * (hi - lo)[None, :]
        ok = np.ones(len(idx), dtype=bool)
        if len(placed_pts):
            tree = cKDTree(placed_pts)
            # Any placed sphere within 2 r_max may conflict; check each pair exactly.
            sd = tree.sparse_distance_matrix(cKDTree(cand), 2.0 * r_max, output_type="ndarray")
            if len(sd):
                hit = sd["v"] < r[sd["j"]] + placed_r[sd["i"]]
                ok[np.unique(sd["j"][hit])] = False
        # Conflicts inside the batch: keep the earlier candidate.
        surv = np.nonzero(ok)[0]
        if len(surv) > 1:
            t2 = cKDTree(cand[surv])
            pairs = t2.query_pairs(2.0 * r_max, output_type="ndarray")
            if len(pairs):
                a, b = surv[pairs[:, 0]], surv[pairs[:, 1]]
                dd = np.linalg.norm(cand[a] - cand[b], axis=1)
                bad = dd < r[a] + r[b]
                # Of each conflicting pair the later candidate goes back to the queue.
                dead = np.zeros(len(idx), dtype=bool)
                dead[np.maximum(a[bad], b[bad])] = True
                ok &= ~dead
        acc = np.nonzero(ok)[0]
        stale = stale + 1 if len(acc) * 200 < len(idx) else 0
        placed_pts = np.vstack([placed_pts, cand[acc]])
        placed_r = np.concatenate([placed_r, r[acc]])
        rej = idx[~ok]
        pending = np.concatenate([rej, pending[batch:]])
    return placed_pts, placed_r, pending


def _surface_nodes(edge: float, h: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-size nodes on the cube surface: 8 vertices, evenly spaced edge nodes, RSA face nodes."""
    L = edge
    pts = [np.array([[i, j, k] for i in (0, L) for j in (0, L) for k in (0, L)], dtype=np.float64)]
    m = max(1, int(round(L / h)))
    s = np.arange(1, m) * (L / m)
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        for c1 in (0.0, L):
            for c2 in (0.0, L):
                p = np.zeros((len(s), 3))
                p[:, ax] = s
                p[:, o1] = c1
                p[:, o2] = c2
                pts.append(p)
    # Face interiors: 2-D RSA with exclusion diameter h, kept h/2 away from the face border.
    n_face = int(1.2 * (L / h) ** 2)
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        for c in (0.0, L):
            p2, _, _ = _rsa_points(n_face, np.full(n_face, 0.5 * h), [0.5 * h] * 2, [L - 0.5 * h] * 2, rng, dim=2,
                                   max_rounds=30)
            p = np.zeros((len(p2), 3))
            p[:, ax] = c
            p[:, o1] = p2[:, 0]
            p[:, o2] = p2[:, 1]
            pts.append(p)
    return np.vstack(pts)


def tessellate(x: np.ndarray, radius: np.ndarray, tets: np.ndarray):
    """Cut every tetrahedron into 12 facets (two per edge); see the module docstring for the points.

    Returns facet_pi, facet_pj, facet_tet (int32) and facet_vtx (F, 9) in tetrahedron-major,
    edge-major order (facet 12*t + 2*e + s is side s of edge e of tetrahedron t).
    """
    T = tets.shape[0]
    P = x[tets]  # (T, 4, 3)
    R = radius[tets]  # (T, 4)
    E = np.empty((T, 6, 3))
    for e, (a, b) in enumerate(TET_EDGES):
        d = P[:, b] - P[:, a]
        L = np.linalg.norm(d, axis=1)
        gap = np.maximum(L - R[:, a] - R[:, b], 0.0)
        s = np.where(L > 0, (np.minimum(R[:, a], L) + 0.5 * gap) / np.where(L > 0, L, 1.0), 0.5)
        s = np.clip(s, 0.0, 1.0)
        E[:, e] = P[:, a] + s[:, None] * d
    edge_id = {}
    for e, (a, b) in enumerate(TET_EDGES):
        edge_id[(a, b)] = e
        edge_id[(b, a)] = e
    faces = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
    Fp = {}
    for f in faces:
        i, j, k = f
        Fp[f] = (E[:, edge_id[(i, j)]] + E[:, edge_id[(j, k)]] + E[:, edge_id[(i, k)]]) / 3.0
    C = E.mean(axis=1)
    fpi = np.empty((T, 12), dtype=np.int32)
    fpj = np.empty((T, 12), dtype=np.int32)
    vtx = np.empty((T, 12, 9))
    for e, (a, b) in enumerate(TET_EDGES):
        others = [v for v in range(4) if v not in (a, b)]
        for s, o in enumerate(others):
            face = tuple(sorted((a, b, o)))
            slot = 2 * e + s
            fpi[:, slot] = tets[:, a]
            fpj[:, slot] = tets[:, b]
            vtx[:, slot, 0:3] = E[:, e]
            vtx[:, slot, 3:6] = Fp[face]
            vtx[:, slot, 6:9] = C
    ftet = np.repeat(np.arange(T, dtype=np.int32), 12)
    return fpi.reshape(-1), fpj.reshape(-1), ftet, vtx.reshape(-1, 9)


def make_cube_specimen(edge: float, d_min: float, d_max: float, n_particles: int, seed: int,
                       fuller_exponent: float = 0.4, phi_excluded: float = 0.25) -> Specimen:
    """Generate a cube specimen [0, edge]^3 with about n_particles nodes (interior + surface).

    phi_excluded: volume fraction of the hard-core exclusion spheres (kept below RSA jamming).
    """
    rng = np.random.default_rng(seed)
    L = float(edge)
    V = L ** 3
    h = (V / n_particles) ** (1.0 / 3.0)  # mean node spacing; also the surface-node spacing
    surf = _surface_nodes(L, h, rng)
    n_int = max(1, n_particles - len(surf))
    d = fuller_diameters(n_int, d_min, d_max, fuller_exponent, rng)
    vol = float(np.sum(np.pi * d ** 3 / 6.0))
    kappa = (phi_excluded * V / vol) ** (1.0 / 3.0)
    r_ex = 0.5 * kappa * d
    margin = np.maximum(r_ex, 0.5 * h)
    # Place inside the shrunken box; per-particle margins are handled by clipping the box to the
    # largest margin (conservative and simple).
    m = float(margin.max())
    pts, r_pl, _ = _rsa_points(n_int, r_ex, [m] * 3, [L - m] * 3, rng, dim=3)
    order = np.argsort(-r_pl, kind="stable")
    pts, r_pl = pts[order], r_pl[order]
    d_pl = 2.0 * r_pl / kappa
    x = np.vstack([pts, surf])
    diameter = np.concatenate([d_pl, np.zeros(len(surf))])
    radius = np.concatenate([r_pl, np.zeros(len(surf))])

    tri = Delaunay(x)
    tets = tri.simplices.astype(np.int64)
    P = x[tets]
    vol6 = np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))
    keep = np.abs(vol6) > 1e-6 * np.median(np.abs(vol6))
    tets = tets[keep]
    # Drop nodes no kept tetrahedron uses, then renumber.
    used = np.zeros(len(x), dtype=bool)
    used[tets.reshape(-1)] = True
    remap = -np.ones(len(x), dtype=np.int64)
    remap[used] = np.arange(int(used.sum()))
    x, diameter, radius = x[used], diameter[used], radius[used]
    tets = remap[tets].astype(np.int32)
    fpi, fpj, ftet, vtx = tessellate(x, radius, tets)
    return Specimen(x=np.ascontiguousarray(x), diameter=np.ascontiguousarray(diameter), tets=tets,
                    facet_pi=fpi, facet_pj=fpj, facet_tet=ftet, facet_vtx=np.ascontiguousarray(vtx),
                    edge=L, d_min=float(d_min), d_max=float(d_max))


def single_tet_specimen(scale: float = 2.0, seed: int = 0) -> Specimen:
    """Four particles forming one (slightly irregular) tetrahedron, 12 facets.  Edge case input."""
    rng = np.random.default_rng(seed)
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64) * scale
    x += 0.1 * scale * rng.standard_normal(x.shape)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    P = x[tets]
    v6 = np.dot(P[0, 1] - P[0, 0], np.cross(P[0, 2] - P[0, 0], P[0, 3] - P[0, 0]))
    if v6 < 0:
        tets = np.array([[0, 2, 1, 3]], dtype=np.int32)
    diameter = np.full(4, 0.5 * scale)
    radius = 0.2 * diameter
    fpi, fpj, ftet, vtx = tessellate(x, radius, tets)
    return Specimen(x=x, diameter=diameter, tets=tets, facet_pi=fpi, facet_pj=fpj, facet_tet=ftet,
                    facet_vtx=vtx, edge=scale, d_min=0.5 * scale, d_max=0.5 * scale)


def shuffled(spec: Specimen, seed: int, swap_ij: bool = True) -> Specimen:
    """The same specimen with facets in random order and, optionally, I/J swapped at random.

    Physically identical; used to check that consumers do not depend on input ordering.
    """
    rng = np.random.default_rng(seed)
    perm = rng.permutation(spec.n_facets)
    fpi, fpj = spec.facet_pi[perm].copy(), spec.facet_pj[perm].copy()
    if swap_ij:
        sw = rng.random(spec.n_facets) < 0.5
        fpi[sw], fpj[sw] = spec.facet_pj[perm][sw], spec.facet_pi[perm][sw]
    return dataclasses.replace(spec, facet_pi=fpi, facet_pj=fpj, facet_tet=spec.facet_tet[perm].copy(),
                               facet_vtx=spec.facet_vtx[perm].copy())
