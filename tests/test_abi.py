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
