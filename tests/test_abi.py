"""The C-ABI library builds, loads and exports every symbol include/w2.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2511_11354_gb300 import build as w2build
from paper_2511_11354_gb300 import w2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(w2_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    path = w2build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("w2_create", "w2_set_potentials", "w2_step", "w2_observables", "w2_set_state",
              "w2_get_state", "w2_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(w2.EXPORTS) <= _declared()


def test_status_strings_without_gpu(lib):
    lib.w2_status_string.restype = ctypes.c_char_p
    lib.w2_status_string.argtypes = [ctypes.c_int]
    assert lib.w2_status_string(0) == b"ok"
    assert lib.w2_status_string(-5).startswith(b"time step unstable")


def test_create_rejects_bad_config_without_touching_the_device(lib):
    lib.w2_create.argtypes = [ctypes.POINTER(w2.Config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p(1)
    bad = w2.Config(2, 8, 1.0, 0.01, 1.0, 1.0, 0, 0)          # nx < 4
    assert lib.w2_create(ctypes.byref(bad), None, ctypes.byref(out)) == -1
    assert out.value is None
    odd = w2.Config(8, 7, 1.0, 0.01, 1.0, 1.0, 0, 0)          # odd nk
    assert lib.w2_create(ctypes.byref(odd), None, ctypes.byref(out)) == -1
    prec = w2.Config(8, 8, 1.0, 0.01, 1.0, 1.0, 9, 0)         # unknown precision
    assert lib.w2_create(ctypes.byref(prec), None, ctypes.byref(out)) == -8
    assert lib.w2_create(None, None, ctypes.byref(out)) == -1
