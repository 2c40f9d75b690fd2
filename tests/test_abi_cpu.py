"""Host-only checks of the C ABI: the library builds and loads without a
GPU, exports every function that include/*.h declares, and rejects bad
arguments before touching the device."""
import ctypes
import glob
import os
import re

import pytest

from paper_1909_04539_gb300 import build as libbuild
from paper_1909_04539_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return _lib.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(bs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(L, n), n
    # and the binding covers the same set
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_lhs_bytes_matches_paper_storage(L):
    # Sec. 3.1: one shared copy of 3N coefficients (tri); Sec. 4.1: 5N (penta)
    assert L.bs_lhs_bytes(3, 1024, 8) == 3 * 1024 * 8
    assert L.bs_lhs_bytes(5, 512, 8) == 5 * 512 * 8
    assert L.bs_lhs_bytes(4, 10, 8) == -1


def test_factor_argument_errors(L):
    h = ctypes.c_void_p()
    bands = (ctypes.c_double * 15)()
    assert L.bs_factor(None, 3, 5, ctypes.byref(h)) == 1
    assert L.bs_factor(bands, 4, 3, ctypes.byref(h)) == 1
    assert L.bs_factor(bands, 3, 1, ctypes.byref(h)) == 1
    assert L.bs_factor(bands, 5, 3, ctypes.byref(h)) == 1
    assert L.bs_factor(bands, 3, 5, None) == 1
    assert b"width" in L.bs_last_error() or b"N must" in L.bs_last_error() or b"NULL" in L.bs_last_error()


def test_solve_rejects_unknown_handle(L):
    bogus = ctypes.c_void_p(0x1234)
    assert L.bs_solve(bogus, ctypes.c_void_p(0x1000), 0, 0, 4, None) == 1
    assert L.bs_solve(None, ctypes.c_void_p(0x1000), 0, 0, 4, None) == 1
    assert L.bs_solve_adjoint(None, ctypes.c_void_p(0x1000), 0, 0, 4, None, None, None) == 1
    assert L.bs_destroy(bogus) == 1
    assert L.bs_destroy(None) == 0
    assert L.bs_strerror(2).startswith(b"zero or non-finite pivot")


def test_set_option(L):
    assert L.bs_set_option(0, 0) == 0
    assert L.bs_set_option(99, 1) == 1
    assert L.bs_set_option(0, -5) == 1
    # BS_OPT_CTA_THREADS takes 0, 32 or a multiple of 64 up to 512
    for v in (32, 64, 128, 192, 448, 512, 0):
        assert L.bs_set_option(7, v) == 0
    for v in (1, 48, 96, 576):
        assert L.bs_set_option(7, v) == 1
    assert L.bs_set_option(7, 0) == 0
    # BS_OPT_F64_PAIRS 0..3, BS_OPT_WINDOW 0..2
    for opt, good, bad in ((8, (0, 1, 2, 3), (4,)), (9, (0, 1, 2), (3,))):
        for v in good:
            assert L.bs_set_option(opt, v) == 0
        for v in bad:
            assert L.bs_set_option(opt, v) == 1
        assert L.bs_set_option(opt, 0) == 0


def test_option_constants_match_header():
    """The binding's OPT_* values are the header's bs_option values."""
    import re

    import paper_1909_04539_gb300 as bs

    hdr = open(os.path.join(ROOT, "include", "bsolve.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"BS_OPT_(\w+)\s*=\s*(\d+)", hdr))
    for name, val in enum.items():
        if name == "COUNT":
            continue
        assert getattr(bs, "OPT_" + name) == val, name


def test_newer_entry_points_reject_bad_arguments(L):
    """Argument errors of the periodic factorisation and of the entry points
    that take a handle are reported before any device work."""
    h = ctypes.c_void_p()
    bands = (ctypes.c_double * 9)()
    assert L.bs_factor_periodic(None, 3, ctypes.byref(h)) == 1
    assert L.bs_factor_periodic(bands, 2, ctypes.byref(h)) == 1
    assert b"N must be" in L.bs_last_error()
    assert L.bs_factor_periodic(bands, 3, None) == 1
    bogus = ctypes.c_void_p(0x1234)
    p = ctypes.c_void_p(0x1000)
    assert L.bs_cn_steps(bogus, p, 0, 0, 4, 1, None) == 1
    assert L.bs_adi_halfstep(bogus, p, p, 0, 8, 8, ctypes.c_double(0.5), 0, 0, None) == 1
    assert L.bs_solve_refine(bogus, p, 1, p, 0, 4, 1, 0, None) == 1
    assert L.bs_band_grad(bogus, p, p, 0, 0, 4, p, None) == 1
    assert L.bs_band_grad_noalloc(bogus, p, p, 0, 0, 4, p, None) == 1
    assert L.bs_solve_bf16(bogus, p, p, 0, 4, None) == 1
    assert b"unknown handle" in L.bs_last_error()
