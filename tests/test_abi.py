"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; the ctypes binding declares exactly those names."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(sbm_[A-Za-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2212_02362_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(libpath):
    from paper_2212_02362_gb300 import _capi
    assert set(_capi.EXPORTED) == _declared()
    _capi.load(libpath)


def test_library_has_no_dynamic_cudart(libpath):
    # statically linked runtime: the library loads on hosts without libcudart
    ctypes.CDLL(libpath)


def test_status_strings_and_null_handles(libpath):
    from paper_2212_02362_gb300 import _capi
    lib = _capi.load(libpath)
    assert lib.sbm_status_string(0) == b"SBM_OK"
    assert lib.sbm_status_string(6) == b"SBM_ERR_DIVERGED"
    # null handles are rejected on the host without touching a device
    assert lib.sbm_set_bc(None, 0, 0, 1, 0.0) == _capi.SBM_ERR_ARG
    assert lib.sbm_solve(None, None, None, None) == _capi.SBM_ERR_ARG
    o = _capi.sbm_opts()
    lib.sbm_default_opts(ctypes.byref(o))
    assert o.tol == 1e-10 and o.max_cycles == 500 and o.nu1 == 2 and o.nu2 == 2
    assert abs(o.omega - 2.0 / 3.0) < 1e-15


def test_noalloc_argument_checks_run_on_the_host(libpath):
    # sbm_residual_noalloc validates sizes and moduli before any CUDA call, with the
    # same moduli rule as sbm_set_moduli (3D bulk mode: C11 + 2 C12 > 0; finite)
    import numpy as np
    from paper_2212_02362_gb300 import _capi
    lib = _capi.load(libpath)
    buf = np.zeros(8)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    bits = (ctypes.c_uint * 3)(0, 0, 0)
    nrm = ctypes.c_double()

    def call(dim, n, h, mod):
        return lib.sbm_residual_noalloc(dim, (ctypes.c_int * 3)(*n), h, (ctypes.c_double * 3)(*mod), bits,
                                        p, p, p, p, ctypes.byref(nrm), None)

    for mod in [(1.0, -0.6, 0.5), (float("inf"), 0.6, 0.5), (1.0, 0.6, 0.0), (0.5, 0.6, 0.5)]:
        assert call(3, (9, 9, 9), 0.125, mod) == _capi.SBM_ERR_ARG, mod
        assert b"positive definite" in lib.sbm_last_error(None)
    # the same cubic moduli are definite in plane strain (no bulk condition in 2D)
    assert call(2, (9, 9, 1), 0.125, (1.0, -0.6, 0.5)) != _capi.SBM_ERR_ARG or \
        b"positive definite" not in lib.sbm_last_error(None)
    assert call(3, (1, 9, 9), 0.125, (1.0, 0.6, 0.5)) == _capi.SBM_ERR_ARG
    assert call(3, (9, 9, 9), 0.0, (1.0, 0.6, 0.5)) == _capi.SBM_ERR_ARG
    assert call(4, (9, 9, 9), 0.125, (1.0, 0.6, 0.5)) == _capi.SBM_ERR_ARG
    # beyond the fixed scratch: rejected before the device is touched
    assert call(2, (4097, 4097, 1), 1.0 / 4096, (1.0, 0.6, 0.5)) == _capi.SBM_ERR_ARG
    assert b"fixed scratch" in lib.sbm_last_error(None)


def test_enum_constants_match_header():
    """Every `NAME = value` of the header's enums has the same value in the binding."""
    from paper_2212_02362_gb300 import _capi
    consts = {}
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
        for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", text, flags=re.S):
            for name, val in re.findall(r"\b(SBM_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
                consts[name] = int(val)
    assert "SBM_K_GS" in consts
    for name, val in consts.items():
        if hasattr(_capi, name):
            assert getattr(_capi, name) == val, name
    assert all(hasattr(_capi, n) for n in consts if n.startswith("SBM_K_")), consts
