"""CPU checks of the C-ABI library: it loads, exports every symbol include/ldpm.h declares, and rejects
bad input on the host before touching CUDA."""
import dataclasses
import os
import re

import numpy as np
import pytest

from paper_2603_13190_gb300 import ldpm, specimen, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ldpm_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ldpm_create", "ldpm_step", "ldpm_get_state", "ldpm_set_state", "ldpm_energy",
                     "ldpm_facet_forces", "ldpm_destroy", "ldpm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = ldpm.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def _expect(code, fn):
    with pytest.raises(ldpm.LdpmError) as ei:
        fn()
    assert ei.value.code == code, str(ei.value)
    return str(ei.value)


@pytest.fixture(scope="module")
def tet():
    return specimen.single_tet_specimen()


MAT = workloads.WORKLOAD_MATERIAL


def test_rejects_facet_not_on_its_tetrahedron(tet):
    bad = dataclasses.replace(tet, facet_pj=tet.facet_pi.copy())
    _expect(-2, lambda: ldpm.ldpm_create(bad, MAT))


def test_rejects_wrong_facet_count(tet):
    bad = dataclasses.replace(tet, facet_pi=tet.facet_pi[:11], facet_pj=tet.facet_pj[:11],
                              facet_tet=tet.facet_tet[:11], facet_vtx=tet.facet_vtx[:11])
    _expect(-2, lambda: ldpm.ldpm_create(bad, MAT))


def test_rejects_three_facets_on_one_edge(tet):
    fpi, fpj = tet.facet_pi.copy(), tet.facet_pj.copy()
    fpi[2], fpj[2] = fpi[0], fpj[0]
    bad = dataclasses.replace(tet, facet_pi=fpi, facet_pj=fpj)
    _expect(-2, lambda: ldpm.ldpm_create(bad, MAT))


def test_rejects_flat_tetrahedron(tet):
    x = tet.x.copy()
    x[:, 2] = 0.0  # all four vertices in one plane
    _expect(-2, lambda: ldpm.ldpm_create(dataclasses.replace(tet, x=x), MAT))


def test_rejects_out_of_range_index(tet):
    tets = tet.tets.copy()
    tets[0, 0] = 99
    _expect(-2, lambda: ldpm.ldpm_create(dataclasses.replace(tet, tets=tets), MAT))


def test_rejects_edge_longer_than_l_t(tet):
    _expect(-2, lambda: ldpm.ldpm_create(tet, dict(MAT, l_t=0.5)))


@pytest.mark.parametrize("field,value,code", [("k_t", -0.5, -1), ("r_s", -0.1, -1), ("Ed_E0", 0.0, -1),
                                              ("E0", -1.0, -1), ("alpha", float("nan"), -1)])
def test_rejects_invalid_material(tet, field, value, code):
    _expect(code, lambda: ldpm.ldpm_create(tet, dict(MAT, **{field: value})))


def test_rejects_bad_bc_code(tet):
    bc = workloads.free_bc(4)
    bc.mask[0, 0] = 7
    _expect(-1, lambda: ldpm.ldpm_create(tet, MAT, bc=bc))


def test_null_handle_calls_fail_cleanly():
    L = ldpm.lib()
    assert L.ldpm_step(None, 1) == -1
    assert L.ldpm_energy(None, None, None) == -1
    assert L.ldpm_sync(None) == -1
    assert L.ldpm_adjoint(None, 10, 5, None, None, None, None, None) == -1
    assert L.ldpm_set_facet_params(None, None, None, None) == -1
    L.ldpm_destroy(None)
    assert ldpm.ldpm_last_error() != ""


def test_law_vjp_hook_rejects_bad_arguments():
    rows, aout = np.zeros((1, 16)), np.zeros((1, 4))
    _expect(-1, lambda: ldpm.ldpm_facet_law_vjp(5, MAT, rows, aout))
    _expect(-1, lambda: ldpm.ldpm_facet_law_vjp(ldpm.LDPM_FP64, dict(MAT, E0=-1.0), rows, aout))


def test_no_cpu_fallback_in_product_path():
    """The binding and package never import the oracle."""
    for fn in ("ldpm.py", "__init__.py", "build.py", "specimen.py", "workloads.py", "autograd.py"):
        src = open(os.path.join(ROOT, "paper_2603_13190_gb300", fn)).read()
        assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), fn


def declared_prototypes():
    """{name: (return type, [parameter types])} of the header's ldpm_* functions, comments removed."""
    src = ""
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src += open(os.path.join(ROOT, "include", fn)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for ret, name, params in re.findall(r"^\s*((?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**)\s*(ldpm_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;",
                                        src, re.M | re.S):
        ps = [p.strip() for p in params.replace("\n", " ").split(",") if p.strip() and p.strip() != "void"]
        out[name] = (ret.strip(), ps)
    return out


def _ctype_of(decl: str):
    import ctypes as C

    if "*" in decl or "[" in decl or decl.split()[0] == "ldpm_t":
        return C.c_void_p
    base = decl.replace("const ", "").split()[0]
    return {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double, "int": C.c_int}[base]


def test_binding_signatures_match_the_header():
    """The ctypes table of the binding agrees with every prototype of include/ldpm.h, argument by
    argument (a drift here would pass wrong-width values across the ABI)."""
    import ctypes as C

    protos = declared_prototypes()
    sig = ldpm.signatures()
    assert sorted(protos) == sorted(sig)
    rets = {"int": C.c_int, "int64_t": C.c_int64, "int32_t": C.c_int32, "void": None, "const char *": C.c_char_p,
            "const char*": C.c_char_p}
    for name, (ret, params) in protos.items():
        args, res = sig[name]
        assert [_ctype_of(p) for p in params] == list(args), (name, params, args)
        assert rets[" ".join(ret.split())] == res, (name, ret, res)


def header_struct(name):
    """[(field, C type)] of `typedef struct { ... } name;` in include/ldpm.h, comments removed."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ldpm.h")).read(), flags=re.S)
    body = re.search(r"typedef struct\s*\{([^{}]*)\}\s*%s\s*;" % name, src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.match(r"(?:const\s+)?([A-Za-z_][A-Za-z0-9_]*)\s+(.*)", decl)
        base, names = m.group(1), m.group(2)
        for n in names.split(","):
            n = n.strip()
            fields.append((n.lstrip("*").strip(), "ptr" if n.startswith("*") or base == "void" else base))
    return fields


@pytest.mark.parametrize("cname,pyname", [("ldpm_geometry", "Geometry"), ("ldpm_material", "Material"),
                                          ("ldpm_options", "Options")])
def test_binding_structs_match_the_header(cname, pyname):
    """Field names, order and C types of the ABI structs agree with their ctypes mirrors."""
    import ctypes as C

    want = {"ptr": C.c_void_p, "int32_t": C.c_int32, "double": C.c_double}
    got = [(f, t) for f, t in getattr(ldpm, pyname)._fields_]
    hdr = header_struct(cname)
    assert [f for f, _ in hdr] == [f for f, _ in got], (cname, hdr, got)
    assert [want[t] for _, t in hdr] == [t for _, t in got], cname


def test_error_codes_documented_as_returned_are_returned():
    """Every LDPM_E_* code of the header is produced somewhere in the library's sources, except the
    ones the header marks reserved, which none produces; the binding names every code."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ldpm.h")).read(), flags=re.S)
    raw = open(os.path.join(ROOT, "include", "ldpm.h")).read()
    codes = dict(re.findall(r"#define (LDPM_E_[A-Z_]+) \((-\d+)\)", src))
    reserved = set(re.findall(r"#define (LDPM_E_[A-Z_]+) \(-\d+\)\s*/\*\s*reserved", raw))
    csrc = os.path.join(ROOT, "paper_2603_13190_gb300", "csrc")
    used = set()
    for f in os.listdir(csrc):
        used |= set(re.findall(r"LDPM_E_[A-Z_]+", open(os.path.join(csrc, f)).read()))
    assert reserved <= set(codes)
    for c in codes:
        assert (c in used) != (c in reserved), c
        assert ldpm.ERRORS[int(codes[c])] == c
