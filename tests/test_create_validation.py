"""Host-side geometry checks of ldpm_create, which run before any CUDA call.

Each bad input is rejected with LDPM_E_BAD_GEOMETRY, and the message names the first offending facet
(or its tetrahedron) in the caller's order.  The facet checks run on several host threads once a
specimen has more than 65536 facets.  The specimen here has 88k facets, so errors are planted in
different threads' ranges, and errors of different kinds are ordered against each other."""
import dataclasses

import numpy as np
import pytest

from paper_2603_13190_gb300 import ldpm, specimen
from paper_2603_13190_gb300.workloads import WORKLOAD_MATERIAL

MAT = dict(WORKLOAD_MATERIAL)


@pytest.fixture(scope="module")
def big():
    s = specimen.make_cube_specimen(20.0, 2.0, 4.0, 1500, seed=7)
    assert s.n_facets > 65536
    return s


def _msg(s, mat=MAT):
    with pytest.raises(ldpm.LdpmError) as ei:
        ldpm.ldpm_create(s, mat)
    assert ei.value.code == -2, str(ei.value)
    return str(ei.value)


def _zero_area(fv, k):
    fv = fv.copy()
    fv[k, 3:6] = fv[k, 0:3]
    fv[k, 6:9] = fv[k, 0:3]
    return fv


def _stranger(s, k):
    """A particle that is not a vertex of facet k's tetrahedron."""
    own = set(s.tets[s.facet_tet[k]].tolist())
    return next(p for p in range(s.n_particles) if p not in own)


def test_valid_specimen_passes_the_checks(big):
    """The unmodified specimen gets past validation: on a machine without a GPU the next step, device
    selection, fails with LDPM_E_CUDA; with a GPU the handle is created."""
    try:
        h = ldpm.ldpm_create(big, MAT)
    except ldpm.LdpmError as e:
        assert e.code == -3, str(e)
    else:
        ldpm.ldpm_destroy(h)


@pytest.mark.parametrize("first,second", [("area", "tet"), ("tet", "area"), ("vertex", "area"), ("area", "vertex")])
def test_first_failure_in_callers_order_across_kinds(big, first, second):
    F = big.n_facets
    k_early, k_late = F // 3 + 5, F - 3  # in different threads' ranges
    ft, fv, fpi = big.facet_tet.copy(), big.facet_vtx, big.facet_pi.copy()
    for kind, k in ((first, k_early), (second, k_late)):
        if kind == "area":
            fv = _zero_area(fv, k)
        elif kind == "tet":
            ft[k] = big.n_tets
        else:
            fpi[k] = _stranger(big, k)
    msg = _msg(dataclasses.replace(big, facet_tet=ft, facet_vtx=fv, facet_pi=fpi))
    expect = {"area": "facet %d: zero edge length or facet area",
              "tet": "facet %d: tetrahedron index out of range",
              "vertex": "facet %d: I and J must be two vertices of its tetrahedron"}[first] % k_early
    assert expect in msg, msg


def test_same_kind_reports_the_earliest(big):
    F = big.n_facets
    fpi = big.facet_pi.copy()
    for k in (F - 10, F // 2, 7):
        fpi[k] = _stranger(big, k)
    assert "facet 7: I and J" in _msg(dataclasses.replace(big, facet_pi=fpi))


def test_three_facets_on_one_edge(big):
    """Facet k moved onto another edge of its tetrahedron: that edge now has three facets, and the
    tetrahedron is named."""
    F = big.n_facets
    k = F - 100
    t = int(big.facet_tet[k])
    pair = {int(big.facet_pi[k]), int(big.facet_pj[k])}
    others = [j for j in np.flatnonzero(big.facet_tet == t) if {int(big.facet_pi[j]), int(big.facet_pj[j])} != pair]
    j = int(others[0])
    fpi, fpj = big.facet_pi.copy(), big.facet_pj.copy()
    fpi[k], fpj[k] = big.facet_pi[j], big.facet_pj[j]
    msg = _msg(dataclasses.replace(big, facet_pi=fpi, facet_pj=fpj))
    assert "tetrahedron %d: more than 2 facets on one edge" % t in msg, msg


def test_edge_longer_than_l_t(big):
    """The first facet (caller's order) whose edge is at least l_t is named, with its length."""
    d = big.x[big.facet_pj] - big.x[big.facet_pi]
    length = np.sqrt((d * d).sum(1))
    l_t = float(np.sort(length)[-40])
    k = int(np.flatnonzero(length >= l_t)[0])
    msg = _msg(big, dict(MAT, l_t=l_t))
    assert "facet %d: edge length" % k in msg and ">= l_t" in msg, msg


def test_tetrahedron_checks(big):
    tets = big.tets.copy()
    tets[5000, 2] = big.n_particles
    assert "tet 5000: particle index out of range" in _msg(dataclasses.replace(big, tets=tets))
    tets = big.tets.copy()
    tets[6000, 3] = tets[6000, 1]
    assert "tet 6000: repeated particle" in _msg(dataclasses.replace(big, tets=tets))


def test_empty_specimen_and_empty_batch_are_rejected():
    """The smallest specimen the step accepts is one tetrahedron with its 12 facets; an empty one is
    rejected with LDPM_E_BAD_GEOMETRY before any CUDA call, and a batch of no specimens with
    LDPM_E_INVALID_ARG."""
    one = specimen.single_tet_specimen()
    empty = dataclasses.replace(one, tets=np.zeros((0, 4), np.int32), facet_pi=np.zeros(0, np.int32),
                                facet_pj=np.zeros(0, np.int32), facet_tet=np.zeros(0, np.int32),
                                facet_vtx=np.zeros((0, 9)))
    assert "need N >= 4, T >= 1 and F == 12 T" in _msg(empty)
    with pytest.raises(ldpm.LdpmError) as ei:
        ldpm.ldpm_batch_create([], [])
    assert ei.value.code == -1, str(ei.value)
