"""The oracle's ctypes binding agrees with the C prototypes in ldpm_oracle.cpp, argument by argument
(a width or order mismatch would feed the oracle wrong inputs and every pin built on it)."""
import ctypes as C
import os
import re

import oracle


def oracle_prototypes():
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ldpm_oracle.cpp")).read()
    block = src[src.index('extern "C" {'):]
    block = block[:block.index("\n}\n")]
    out = {}
    for ret, name, params in re.findall(r"^\s*([A-Za-z_][A-Za-z0-9_]*\s*\**)\s*(orc_[a-z_]+)\s*\(([^;]*?)\)\s*;",
                                        block, re.M | re.S):
        out[name] = (ret.strip(), [p.strip() for p in params.replace("\n", " ").split(",") if p.strip()])
    return out


def _matches(decl, ct):
    if "*" in decl or "[" in decl:
        return ct is C.c_void_p or (isinstance(ct, type) and issubclass(ct, C._Pointer))
    base = decl.replace("const ", "").split()[0]
    return ct is {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double}[base]


def test_oracle_binding_matches_its_prototypes():
    L = oracle.lib()
    protos = oracle_prototypes()
    assert len(protos) >= 20
    configured = 0
    for name, (ret, params) in protos.items():
        fn = getattr(L, name)
        if fn.argtypes is None:  # not used by the binding
            continue
        configured += 1
        assert len(fn.argtypes) == len(params), (name, params, fn.argtypes)
        for p, ct in zip(params, fn.argtypes):
            assert _matches(p, ct), (name, p, ct)
        if ret in ("double", "int", "int32_t", "int64_t") or ret.endswith("*"):
            want = {"double": C.c_double, "int": C.c_int, "int32_t": C.c_int32, "int64_t": C.c_int64}.get(ret, C.c_void_p)
            assert fn.restype is want, (name, ret, fn.restype)
    assert configured == len(protos) - 1  # orc_sizes is not used
