"""The C-ABI library builds, loads and exports every function include/demag.h
declares; argument validation rejects bad input before any launch (no GPU
needed: these paths return before touching the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "demag.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(demag_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("demag_build_factors", "demag_apply_full", "demag_apply_cp", "demag_apply_tucker",
                     "demag_apply_tt", "demag_apply_adjoint", "demag_plan_destroy", "demag_num_terms",
                     "demag_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol(lib):
    from paper_1212_3509_gb300 import _abi
    assert set(declared_functions()) <= set(_abi._SIGS)


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3), ("R", ctypes.c_int), ("c0", ctypes.c_double)]


@pytest.mark.parametrize("n,h,R,c0,code", [
    ((0, 4, 4), (1, 1, 1), 41, 2.15, 1),       # empty grid
    ((4, 4, 4), (1, -1, 1), 41, 2.15, 1),      # negative spacing
    ((4, 4, 4), (1, 1, 1), 40, 2.15, 1),       # even R
    ((4, 4, 4), (1, 1, 1), 3, 2.15, 1),        # R < 5
    ((4, 4, 4), (1, 1, 1), 41, 0.0, 1),        # c0 <= 0
    ((4, 4, 4), (1, 1, 1), 2 * 257 + 1, 2.15, 5),  # too many terms (M <= 256)
])
def test_build_factors_rejects_bad_grids(lib, n, h, R, c0, code):
    lib.demag_build_factors.restype = ctypes.c_int
    lib.demag_build_factors.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    lib.demag_last_error.restype = ctypes.c_char_p
    lib.demag_last_error.argtypes = [ctypes.c_void_p]
    d = Desc((ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*h), R, c0)
    out = ctypes.c_void_p(1234)
    st = lib.demag_build_factors(ctypes.byref(d), ctypes.byref(out), None)
    assert st == code
    assert out.value is None
    assert len(lib.demag_last_error(None)) > 0


def test_null_arguments_are_rejected(lib):
    lib.demag_build_factors.restype = ctypes.c_int
    assert lib.demag_build_factors(None, None, None) == 1
    lib.demag_apply_full.restype = ctypes.c_int
    lib.demag_apply_full.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.demag_apply_full(None, None, None, 1, None) == 1
    lib.demag_num_terms.restype = ctypes.c_int
    lib.demag_num_terms.argtypes = [ctypes.c_void_p]
    assert lib.demag_num_terms(None) == -1
    lib.demag_set_fused.restype = ctypes.c_int
    lib.demag_set_fused.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.demag_set_fused(None, 1) == 1
    lib.demag_forward_schedule.restype = ctypes.c_int
    lib.demag_forward_schedule.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.demag_forward_schedule(None, 3) == -1
    lib.demag_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.demag_plan_destroy(None)
