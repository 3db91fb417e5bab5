"""Thin ctypes binding of the w2 C ABI (include/w2.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libw2.so``.  There is no CPU fallback; if the library is
missing or no sm_103a device is usable, the calls raise.

Device arrays are torch CUDA tensors (float64, contiguous, layout
[nx][nx][nk][nk]); the context runs on torch's current stream unless a stream
is given.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libw2.so")

W2_F64 = 0

STATUS = {0: "W2_OK", -1: "W2_ERR_ARG", -2: "W2_ERR_CUDA", -3: "W2_ERR_OOM", -4: "W2_ERR_STATE",
          -5: "W2_ERR_UNSTABLE", -6: "W2_ERR_NONFINITE", -7: "W2_ERR_TIMEOUT", -8: "W2_ERR_UNSUPPORTED"}

EXPORTS = ("w2_create", "w2_set_potentials", "w2_set_state", "w2_get_state", "w2_step",
           "w2_step_profile", "w2_observables", "w2_theta", "w2_advect", "w2_destroy", "w2_status_string")
STEP_KERNELS = ("xsum_f", "tables_f", "theta_predictor", "shift_x2", "shift_x1_lawson", "xsum_ftilde",
                "tables_ftilde", "theta_corrector")


class W2Error(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nk", ctypes.c_int32), ("L", ctypes.c_double),
                ("dt", ctypes.c_double), ("hbar", ctypes.c_double), ("mass", ctypes.c_double),
                ("precision", ctypes.c_int32), ("xc_kind", ctypes.c_int32)]


class Obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("energy", ctypes.c_double), ("purity", ctypes.c_double),
                ("entropy_lin", ctypes.c_double), ("l2norm", ctypes.c_double), ("step", ctypes.c_int64)]


W2_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)
_lib = None


def load(path: str = LIB_PATH):
    """Load the library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"w2 CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    lib.w2_create.argtypes = [ctypes.POINTER(Config), vp, ctypes.POINTER(vp)]
    lib.w2_set_potentials.argtypes = [vp, W2_FN, vp, W2_FN, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.w2_set_state.argtypes = [vp, vp, ctypes.c_int32]
    lib.w2_get_state.argtypes = [vp, vp, ctypes.c_int32]
    lib.w2_step.argtypes = [vp, ctypes.c_int32]
    lib.w2_step_profile.argtypes = [vp, ctypes.c_int32, dp]
    lib.w2_observables.argtypes = [vp, ctypes.POINTER(Obs), dp, dp]
    lib.w2_theta.argtypes = [vp, vp, vp]
    lib.w2_advect.argtypes = [vp, vp, vp]
    lib.w2_destroy.argtypes = [vp]
    lib.w2_destroy.restype = None
    lib.w2_status_string.argtypes = [ctypes.c_int]
    lib.w2_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("w2_destroy", "w2_status_string"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int, what: str):
    if code != 0:
        raise W2Error(code, what)


def _dev_ptr(t, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"shape {tuple(t.shape)} != {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Observables:
    mass: float
    energy: float
    purity: float
    entropy_lin: float
    l2norm: float
    step: int
    n1: np.ndarray
    n12: np.ndarray
    status: str


class Context:
    """A w2_ctx: one problem on the current CUDA device."""

    def __init__(self, nx, nk, L, dt, hbar=1.0, mass=1.0, xc_kind=0, stream=None):
        import torch
        self.lib = load()
        self.shape = (nx, nx, nk, nk)
        self.nx, self.nk = nx, nk
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        cfg = Config(nx, nk, L, dt, hbar, mass, W2_F64, xc_kind)
        h = ctypes.c_void_p()
        _check(self.lib.w2_create(ctypes.byref(cfg), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)),
               "w2_create")
        self.h = h
        self._keep = []

    @classmethod
    def from_problem(cls, prob, stream=None):
        ctx = cls(prob.nx, prob.nk, prob.L, prob.dt, prob.hbar, prob.mass, prob.xc_kind, stream)
        ctx.set_potentials(prob.vext, prob.vee, prob.gamma, prob.c_hartree, prob.c_xc)
        return ctx

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.w2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_potentials(self, vext, vee, gamma=1.0, c_hartree=1.0, c_xc=0.0):
        ce = W2_FN(lambda x, _u: float(vext(x))) if vext is not None else ctypes.cast(None, W2_FN)
        cw = W2_FN(lambda r, _u: float(vee(r))) if vee is not None else ctypes.cast(None, W2_FN)
        self._keep = [ce, cw]
        _check(self.lib.w2_set_potentials(self.h, ce, None, cw, None, gamma, c_hartree, c_xc), "w2_set_potentials")

    def set_state(self, f):
        """f: float64 CUDA tensor (device copy) or numpy array (host copy)."""
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
            assert f.shape == self.shape
            _check(self.lib.w2_set_state(self.h, ctypes.c_void_p(f.ctypes.data), 0), "w2_set_state")
        else:
            _check(self.lib.w2_set_state(self.h, _dev_ptr(f, self.shape), 1), "w2_set_state")

    def get_state(self, out=None):
        import torch
        if out is None:
            out = np.empty(self.shape)
        if isinstance(out, np.ndarray):
            _check(self.lib.w2_get_state(self.h, ctypes.c_void_p(out.ctypes.data), 0), "w2_get_state")
        elif isinstance(out, torch.Tensor) and not out.is_cuda:
            _check(self.lib.w2_get_state(self.h, ctypes.c_void_p(out.data_ptr()), 0), "w2_get_state")
        else:
            _check(self.lib.w2_get_state(self.h, _dev_ptr(out, self.shape), 1), "w2_get_state")
        return out

    def step(self, nsteps=1):
        _check(self.lib.w2_step(self.h, int(nsteps)), "w2_step")

    def step_profile(self, nsteps):
        """Advance nsteps steps with CUDA events around each kernel; returns the
        mean milliseconds per kernel of a step (see STEP_KERNELS)."""
        ms = np.zeros(len(STEP_KERNELS))
        _check(self.lib.w2_step_profile(self.h, int(nsteps), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "w2_step_profile")
        return ms

    def observables(self, raise_nonfinite=False) -> Observables:
        o = Obs()
        n1 = np.zeros(self.nx)
        n12 = np.zeros((self.nx, self.nx))
        dp = ctypes.POINTER(ctypes.c_double)
        code = self.lib.w2_observables(self.h, ctypes.byref(o), n1.ctypes.data_as(dp), n12.ctypes.data_as(dp))
        if code not in (0, -6) or (code == -6 and raise_nonfinite):
            _check(code, "w2_observables")
        return Observables(o.mass, o.energy, o.purity, o.entropy_lin, o.l2norm, o.step, n1, n12, STATUS[code])

    def theta(self, f, out):
        _check(self.lib.w2_theta(self.h, _dev_ptr(f, self.shape), _dev_ptr(out, self.shape)), "w2_theta")
        return out

    def advect(self, f, out):
        _check(self.lib.w2_advect(self.h, _dev_ptr(f, self.shape), _dev_ptr(out, self.shape)), "w2_advect")
        return out
