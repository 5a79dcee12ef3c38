"""The C-ABI library builds for sm_103a, loads on a machine without a GPU, and exports every
entry point that include/shbim.h declares (CPU only: no compute call is made)."""
import os
import re

import pytest

import paper_1811_10270_gb300 as S
from paper_1811_10270_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(S.LIB_PATH):
        B.build()
    return S.lib()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "shbim.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(shbim_[A-Za-z0-9_]+)\s*\(", hdr)))


def test_header_declares_the_binding_exports():
    assert set(declared_symbols()) == set(S.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_context_create_destroy_and_option_validation(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.shbim_create(None, ctypes.byref(h)) == 0
    a = ctypes.c_int64(-1)
    assert lib.shbim_sizes(h, ctypes.byref(a), None, None) == 0 and a.value == 0
    assert lib.shbim_set_precision(h, 7) == -1
    assert b"precision" in lib.shbim_last_error(h)
    assert lib.shbim_set_R(h, -1.0) == -1
    # calls that need drops fail cleanly before any device work
    assert lib.shbim_eval_electric(h, 0, None, None, 1, None) == -1
    assert lib.shbim_gmres_step(h, None, None) == -1
    assert lib.shbim_destroy(h) == 0
    bad = S.Opts(5, 50, 1e-8, 100, 1.0)
    h2 = ctypes.c_void_p()
    assert lib.shbim_create(ctypes.byref(bad), ctypes.byref(h2)) == -1
    bad = S.Opts(0, 50, 1e-8, 100, -2.0)
    assert lib.shbim_create(ctypes.byref(bad), ctypes.byref(h2)) == -1


def test_set_drops_rejects_bad_degrees(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.shbim_create(None, ctypes.byref(h)) == 0
    for p in (0, 65):
        P = (ctypes.c_int32 * 1)(p)
        assert lib.shbim_set_drops(h, 1, P, None, ctypes.c_void_p(16), None) == -1
    assert lib.shbim_set_drops(h, 0, None, None, None, None) == -1
    lib.shbim_destroy(h)


def test_header_error_codes_match_the_binding():
    hdr = open(os.path.join(ROOT, "include", "shbim.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"#define SHBIM_(ERR_[A-Z_]+) \((-?\d+)\)", hdr))
    assert codes["ERR_TIMEOUT"] == S.ERR_TIMEOUT == -5
    assert codes["ERR_ARG"] == S.ERR_ARG and codes["ERR_CUDA"] == S.ERR_CUDA


def test_host_side_argument_checks(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.shbim_create(None, ctypes.byref(h)) == 0
    assert lib.shbim_set_wait_limit(h, 0.0) == -1 and b"wait limit" in lib.shbim_last_error(h)
    assert lib.shbim_set_wait_limit(h, 1e9) == -1
    assert lib.shbim_set_wait_limit(h, 0.5) == 0
    fd = (ctypes.c_int32 * 1)(0)
    assert lib.shbim_sht(h, 0, 0, 1, fd, None, None, None) == -1   # no drops set
    d, r = ctypes.c_double(), ctypes.c_double()
    assert lib.shbim_near_min_distance(h, ctypes.byref(d), ctypes.byref(r)) == 0
    assert d.value == float("inf") and r.value == float("inf")
    lib.shbim_destroy(h)
