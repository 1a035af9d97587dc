"""The seeded input generator (paper Sec. 3.1 geometry: particles, Delaunay tetrahedra, 12 facets per
tetrahedron): the workload sizes it produces, the mesh rules every consumer relies on, determinism,
and the facet shuffle used by the order-independence tests.  The generator holds none of the
method's arithmetic; both the oracle and the library consume what it writes."""
import numpy as np
import pytest

from paper_2603_13190_gb300 import specimen, workloads


@pytest.mark.parametrize("name,N,T,F", [("elastic_vibration", 388, 1534, 18408),
                                        ("uniaxial_tension", 24925, 151727, 1820724)])
def test_workload_sizes(name, N, T, F):
    """The sizes the design and the bench lines quote for these workloads (seeded, so exact)."""
    s = workloads.WORKLOADS[name].specimen()
    assert (s.n_particles, s.n_tets, s.n_facets) == (N, T, F)


@pytest.fixture(scope="module")
def cube():
    return specimen.make_cube_specimen(12.0, 2.0, 4.0, 200, seed=5)


def test_mesh_rules(cube):
    """12 facets per tetrahedron, two on each of its 6 edges, each joining two of its vertices; the
    tetrahedra tile the cube (their volumes add up to edge^3)."""
    s = cube
    assert s.n_facets == 12 * s.n_tets
    for t in range(s.n_tets):
        ks = np.flatnonzero(s.facet_tet == t)
        assert len(ks) == 12
        verts = set(s.tets[t].tolist())
        edges = {}
        for k in ks:
            i, j = int(s.facet_pi[k]), int(s.facet_pj[k])
            assert i != j and {i, j} <= verts
            edges[frozenset((i, j))] = edges.get(frozenset((i, j)), 0) + 1
        assert len(edges) == 6 and set(edges.values()) == {2}
    X = s.x[s.tets]
    vol = np.abs(np.einsum("ti,ti->t", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))) / 6.0
    assert np.all(vol > 0)
    np.testing.assert_allclose(vol.sum(), s.edge ** 3, rtol=1e-9)


def test_diameters_and_surface_nodes(cube):
    """Interior particles carry diameters in [d_min, d_max]; the zero-size nodes sit on the cube's
    faces; every particle lies in the cube."""
    s = cube
    assert np.all(s.x >= -1e-9) and np.all(s.x <= s.edge + 1e-9)
    zero = s.diameter == 0.0
    inner = ~zero
    assert np.all((s.diameter[inner] >= s.d_min - 1e-12) & (s.diameter[inner] <= s.d_max + 1e-12))
    on_face = np.any((np.abs(s.x) < 1e-9) | (np.abs(s.x - s.edge) < 1e-9), axis=1)
    assert np.all(on_face[zero]) and zero.sum() > 0


def test_seeded_and_deterministic():
    a = specimen.make_cube_specimen(10.0, 2.0, 4.0, 120, seed=3)
    b = specimen.make_cube_specimen(10.0, 2.0, 4.0, 120, seed=3)
    c = specimen.make_cube_specimen(10.0, 2.0, 4.0, 120, seed=4)
    for f in ("x", "diameter", "tets", "facet_pi", "facet_pj", "facet_tet", "facet_vtx"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert a.x.shape != c.x.shape or not np.array_equal(a.x, c.x)


def test_shuffle_is_a_relabelling(cube):
    """The shuffled specimen holds the same facets (triangle, tetrahedron, unordered particle pair),
    in another order and with I and J swapped on about half of them."""
    s, r = cube, specimen.shuffled(cube, seed=9)

    def keyset(sp):
        return sorted((int(sp.facet_tet[k]), min(int(sp.facet_pi[k]), int(sp.facet_pj[k])),
                       max(int(sp.facet_pi[k]), int(sp.facet_pj[k])), tuple(np.round(sp.facet_vtx[k], 12)))
                      for k in range(sp.n_facets))

    assert keyset(s) == keyset(r)
    assert not np.array_equal(s.facet_tet, r.facet_tet)
    flipped = np.mean(r.facet_pi > r.facet_pj) - np.mean(s.facet_pi > s.facet_pj)
    assert abs(flipped) < 0.5 and 0 < np.mean(r.facet_pi > r.facet_pj) < 1
