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


def test_sem_create_rejects_bad_config_without_touching_the_device(lib):
    lib.w2_sem_create.argtypes = [ctypes.POINTER(w2.SemConfig), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p(1)
    good = dict(nx=17, ncell=2, nq=6, L=12.0, Lp=10.0, dt=0.01, hbar=1.0, mass=1.0, xc_kind=0, precision=0)
    for change in (dict(nx=7), dict(nq=1), dict(nq=33), dict(ncell=9, nq=32), dict(L=0.0), dict(dt=-1.0),
                   dict(xc_kind=3), dict(precision=1), dict(nx=257, precision=3), dict(Lp=1e4)):
        cfg = w2.SemConfig(**{**good, **change})
        assert lib.w2_sem_create(ctypes.byref(cfg), None, ctypes.byref(out)) == -1, change
        assert out.value is None


def test_argument_errors_of_the_eigensolver_and_staging_without_a_device(lib):
    lib.w2_hermitian_eigvals.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p]
    buf = ctypes.create_string_buffer(64)
    assert lib.w2_hermitian_eigvals(None, 4, 1, ctypes.addressof(buf), None) == -1
    assert lib.w2_hermitian_eigvals(ctypes.addressof(buf), 0, 1, ctypes.addressof(buf), None) == -1
    assert lib.w2_hermitian_eigvals(ctypes.addressof(buf), 4097, 1, ctypes.addressof(buf), None) == -1
    assert lib.w2_hermitian_eigvals(ctypes.addressof(buf), 4, 0, ctypes.addressof(buf), None) == -1
    lib.w2_stage_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.w2_use_staged_state.argtypes = [ctypes.c_void_p]
    assert lib.w2_stage_state(None, ctypes.addressof(buf)) == -1
    assert lib.w2_use_staged_state(None) == -1
