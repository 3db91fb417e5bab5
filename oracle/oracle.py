"""ctypes wrapper around ``w2_oracle.c`` (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "w2_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libw2_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)
_dp = ctypes.POINTER(ctypes.c_double)


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp); returns the library path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the argument types of the oracle's entry points on ``lib``."""
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 7 + [
        ctypes.c_int, ORC_FN, ctypes.c_void_p, ORC_FN, ctypes.c_void_p]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    for name in ("orc_marginals",):
        getattr(lib, name).argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.orc_potential_fine.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.orc_theta_with.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_int, _dp]
    lib.orc_theta.argtypes = [ctypes.c_void_p, _dp, _dp]
    _ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_theta_with_sample.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_int, _ip, ctypes.c_int, _dp]
    lib.orc_advect_sample.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _ip, ctypes.c_int, _dp]
    lib.orc_shift_line.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp]
    lib.orc_advect.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp]
    lib.orc_step.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int]
    lib.orc_step.restype = ctypes.c_int
    lib.orc_observables.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_set_hartree_poisson.argtypes = [ctypes.c_void_p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


_variants = {}


def variant(name: str, replacements) -> ctypes.CDLL:
    """A copy of the oracle with a planted mistake, for tests that show a pin
    catches it: each (old, new) pair of ``replacements`` must occur exactly
    once in ``w2_oracle.c``.  Compiled into ``_build/variants/<name>.so``."""
    with _lock:
        if name in _variants:
            return _variants[name]
        src = open(_SRC).read()
        for old, new in replacements:
            if src.count(old) != 1:
                raise ValueError(f"variant {name}: {old!r} occurs {src.count(old)} times")
            src = src.replace(old, new)
        d = os.path.join(_HERE, "_build", "variants")
        os.makedirs(d, exist_ok=True)
        c_path = os.path.join(d, f"{name}.{os.getpid()}.c")
        so = os.path.join(d, f"{name}.{os.getpid()}.so")
        with open(c_path, "w") as fh:
            fh.write(src)
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", c_path, "-o", so, "-lm"],
                       check=True)
        lib = _configure(ctypes.CDLL(so))
        os.remove(c_path)
        _variants[name] = lib
        return lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Oracle:
    """One problem instance: grid, potentials (sampled once), time step."""

    def __init__(self, prob, lib=None):
        self.lib = _load() if lib is None else lib
        self.prob = prob
        self._cb_ext = ORC_FN(lambda x, _u: float(prob.vext(x)))
        self._cb_ee = ORC_FN(lambda r, _u: float(prob.vee(r)))
        h = self.lib.orc_create(prob.nx, prob.nk, prob.L, prob.dt, prob.hbar, prob.mass, prob.gamma,
                                prob.c_hartree, prob.c_xc, prob.xc_kind, self._cb_ext, None,
                                self._cb_ee, None)
        if not h:
            raise ValueError("oracle rejected the problem description")
        self.h = ctypes.c_void_p(h)
        self.shape = (prob.nx, prob.nx, prob.nk, prob.nk)
        if getattr(prob, "hartree", "pair") == "poisson":
            self.lib.orc_set_hartree_poisson(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.orc_destroy(h)
            self.h = None

    @staticmethod
    def threads() -> int:
        return int(_load().orc_threads())

    def _f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == self.shape, (f.shape, self.shape)
        return f

    def marginals(self, f):
        f = self._f(f)
        n1 = np.zeros(self.prob.nx)
        n2 = np.zeros(self.prob.nx)
        self.lib.orc_marginals(self.h, _ptr(f), _ptr(n1), _ptr(n2))
        return n1, n2

    def potential_fine(self, n):
        """U(x_i + l h') on [nx][2 nk] for a particle with density n (or None)."""
        out = np.zeros((self.prob.nx, 2 * self.prob.nk))
        nn = None if n is None else np.ascontiguousarray(n, dtype=np.float64)
        self.lib.orc_potential_fine(self.h, _ptr(nn), _ptr(out))
        return out

    def theta(self, f):
        f = self._f(f)
        out = np.empty_like(f)
        self.lib.orc_theta(self.h, _ptr(f), _ptr(out))
        return out

    def theta_with(self, f, U1, U2, terms=7):
        f = self._f(f)
        out = np.empty_like(f)
        U1 = np.ascontiguousarray(U1, dtype=np.float64)
        U2 = np.ascontiguousarray(U2, dtype=np.float64)
        self.lib.orc_theta_with(self.h, _ptr(f), _ptr(U1), _ptr(U2), int(terms), _ptr(out))
        return out

    def theta_sample(self, f, xs, U1=None, U2=None, terms=7):
        """Theta f at the listed spatial points only (X = i1*nx + i2); the
        one-body potentials default to those of f's own densities."""
        f = self._f(f)
        if U1 is None or U2 is None:
            n1, n2 = self.marginals(f)
            U1, U2 = self.potential_fine(n1), self.potential_fine(n2)
        xs = np.ascontiguousarray(xs, dtype=np.intc)
        out = np.empty((xs.size, self.prob.nk, self.prob.nk))
        self.lib.orc_theta_with_sample(self.h, _ptr(f), _ptr(np.ascontiguousarray(U1)),
                                       _ptr(np.ascontiguousarray(U2)), int(terms),
                                       xs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(xs.size), _ptr(out))
        return out

    def advect_sample(self, f, planes, tau=None):
        """The characteristic shift of the listed momentum planes (n1*nk + n2)."""
        f = self._f(f)
        planes = np.ascontiguousarray(planes, dtype=np.intc)
        out = np.empty((planes.size, self.prob.nx, self.prob.nx))
        self.lib.orc_advect_sample(self.h, _ptr(f), float(self.prob.dt if tau is None else tau),
                                   planes.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(planes.size), _ptr(out))
        return out

    def shift_line(self, line, shift):
        line = np.ascontiguousarray(line, dtype=np.float64)
        assert line.shape == (self.prob.nx,)
        out = np.empty_like(line)
        self.lib.orc_shift_line(self.h, _ptr(line), float(shift), _ptr(out))
        return out

    def advect(self, f, tau=None):
        f = self._f(f)
        out = np.empty_like(f)
        self.lib.orc_advect(self.h, _ptr(f), float(self.prob.dt if tau is None else tau), _ptr(out))
        return out

    def step(self, f, nsteps=1):
        f = self._f(f).copy()
        rc = self.lib.orc_step(self.h, _ptr(f), int(nsteps))
        if rc:
            raise MemoryError("oracle step failed")
        return f

    def observables(self, f):
        f = self._f(f)
        obs = np.zeros(5)
        n1 = np.zeros(self.prob.nx)
        n12 = np.zeros((self.prob.nx, self.prob.nx))
        self.lib.orc_observables(self.h, _ptr(f), _ptr(obs), _ptr(n1), _ptr(n12))
        return {"mass": obs[0], "energy": obs[1], "purity": obs[2], "entropy_lin": obs[3],
                "l2norm": obs[4], "n1": n1, "n12": n12}
