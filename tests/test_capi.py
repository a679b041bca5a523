"""The C-ABI library builds, loads, and exports every function that
include/svn.h declares (no GPU needed: nothing is called but
svn_default_params and argument validation that fails before any CUDA call).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "svn.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*|unsigned long long|long long|svn_handle\s*\*)\s*(svn_\w+)\s*\(", hdr,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_10822_gb300 import build, capi
    build.build()
    return capi.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("svn_create", "svn_set_forcing", "svn_step", "svn_destroy", "svn_last_error",
              "svn_residual", "svn_energy", "svn_linearize", "svn_apply", "svn_precondition",
              "svn_krylov_solve", "svn_dual_update", "svn_get_state", "svn_set_state"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2204_10822_gb300 import capi
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(capi.exported_symbols())


def test_default_params_and_argument_checks(lib):
    from paper_2204_10822_gb300 import capi
    p = capi.SvnParams()
    assert lib.svn_default_params(ctypes.byref(p)) == 0
    assert p.Pstar == 27500.0 and p.e == 2.0 and p.delta_min == 2e-9 and p.max_newton == 200
    assert lib.svn_default_params(None) == -1
    h = ctypes.c_void_p()
    g = capi.SvnGrid(15, 512e3)           # odd N is rejected before any device work
    rc = lib.svn_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h))
    assert rc == -1
    assert b"even" in lib.svn_last_error(h)
    lib.svn_destroy(h)
    assert lib.svn_destroy(None) == -1


def _struct_fields(name):
    hdr = open(os.path.join(ROOT, "include", "svn.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), hdr, flags=re.S).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"^(int|double|const\s+\w+\s*\*)\s+", "", decl)
        for part in decl.split(","):
            names.append(re.sub(r"\[.*\]", "", part).strip())
    return names


@pytest.mark.parametrize("cname,pyname", [("svn_params", "SvnParams"), ("svn_stats", "SvnStats"),
                                          ("svn_grid", "SvnGrid")])
def test_ctypes_structs_match_header(cname, pyname):
    from paper_2204_10822_gb300 import capi
    assert _struct_fields(cname) == [f[0] for f in getattr(capi, pyname)._fields_]
