"""Host-side checks of the C-ABI library that need no GPU.

The library must load, export every entry point include/etc.h declares, and
reject bad arguments on the host (before any CUDA call) with ETC_EINVAL.
"""
import ctypes
import os
import re

import pytest

from paper_2404_02433_b300 import binding as B
from paper_2404_02433_b300 import build as BUILD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "etc.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:etc_status|const char\*|unsigned long long)\s+(etc_\w+)\s*\(",
                                 text, re.M)))


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("etc_create_rve", "etc_set_reference_params", "etc_solve_direction",
                     "etc_effective_tensor", "etc_destroy_rve", "etc_get_solution"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(B.EXPORTED) | set(declared_functions())


def test_binding_names_match_header():
    assert set(B.EXPORTED) >= set(declared_functions())


def test_default_opts(lib):
    o = B.EtcOpts()
    assert lib.etc_default_opts(ctypes.byref(o)) == B.ETC_OK
    assert o.rtol == 1e-8 and o.maxit == 5000 and o.precision == B.ETC_PREC_FP64
    assert lib.etc_default_opts(None) == B.ETC_EINVAL


@pytest.mark.parametrize("dims,lens", [((0, 4, 4), (1, 1, 1)), ((4, -1, 4), (1, 1, 1)),
                                        ((4, 4, 9000), (1, 1, 1)), ((4, 4, 4), (0, 1, 1)),
                                        ((4, 4, 4), (1, float("nan"), 1)),
                                        ((4, 4, 4), (1, 1, -2))])
def test_create_rejects_bad_sizes_on_host(lib, dims, lens):
    h = ctypes.c_void_p()
    dummy = (ctypes.c_double * 1)(1.0)
    st = lib.etc_create_rve(*dims, *lens, ctypes.cast(dummy, ctypes.c_void_p), None, None, None,
                            ctypes.byref(h))
    assert st == B.ETC_EINVAL
    assert not h.value


def test_create_rejects_null_kappa_and_out(lib):
    h = ctypes.c_void_p()
    assert lib.etc_create_rve(2, 2, 2, 1.0, 1.0, 1.0, None, None, None, None,
                              ctypes.byref(h)) == B.ETC_EINVAL
    dummy = (ctypes.c_double * 8)(*([1.0] * 8))
    assert lib.etc_create_rve(2, 2, 2, 1.0, 1.0, 1.0, ctypes.cast(dummy, ctypes.c_void_p), None,
                              None, None, None) == B.ETC_EINVAL


def test_null_handle_calls_are_rejected(lib):
    k = ctypes.c_double()
    assert lib.etc_solve_direction(None, 0, 1.0, 0.0, None, ctypes.byref(k), None) == B.ETC_EINVAL
    assert lib.etc_get_solution(None, 0, None) == B.ETC_EINVAL
    assert lib.etc_effective_tensor(None, None, None, None) == B.ETC_EINVAL
    assert lib.etc_destroy_rve(None) == B.ETC_OK
    d = (ctypes.c_int * 3)()
    assert lib.etc_loading_dims(None, 0, d) == B.ETC_EINVAL


def test_handle_less_calls_give_a_reason(lib):
    # calls without a handle report why they were refused through etc_last_error(NULL)
    lib.etc_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    dummy = (ctypes.c_double * 8)(*([1.0] * 8))
    assert lib.etc_create_rve(0, 2, 2, 1.0, 1.0, 1.0, ctypes.cast(dummy, ctypes.c_void_p), None,
                              None, None, ctypes.byref(h)) == B.ETC_EINVAL
    assert b"1..8192" in lib.etc_last_error(None)
    assert lib.etc_create_rve(2, 2, 2, 1.0, 0.0, 1.0, ctypes.cast(dummy, ctypes.c_void_p), None,
                              None, None, ctypes.byref(h)) == B.ETC_EINVAL
    assert b"lx, ly, lz" in lib.etc_last_error(None)


@pytest.mark.parametrize("dims", [(4096, 2, 2), (2, 4096, 2), (1024, 1024, 2)])
def test_static_apply_refuses_sizes_beyond_its_scratch(lib, dims):
    # the allocation-free apply checks its fixed limits before any CUDA call
    lib.etc_last_error.restype = ctypes.c_char_p
    kref = (ctypes.c_double * 5)(*([1.0] * 5))
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert B.load_library().etc_apply_reference_inverse_static(
        *dims, kref, p, p, None) == B.ETC_EINVAL
    msg = lib.etc_last_error(None)
    assert b"n0, n1 <= 2048" in msg and b"2^20" in msg


def test_status_strings(lib):
    for s in range(7):
        assert lib.etc_status_string(s)
    assert lib.etc_status_string(99) == b"unknown status"
