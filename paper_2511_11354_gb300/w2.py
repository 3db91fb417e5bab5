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
W2_F32_TF32X3 = 1
W2_F32_BF16X3 = 2
W2_F64_SLICED = 3
W2_HARTREE_PAIR = 0
W2_HARTREE_POISSON = 1
F64_STATE = (W2_F64, W2_F64_SLICED)

STATUS = {0: "W2_OK", -1: "W2_ERR_ARG", -2: "W2_ERR_CUDA", -3: "W2_ERR_OOM", -4: "W2_ERR_STATE",
          -5: "W2_ERR_UNSTABLE", -6: "W2_ERR_NONFINITE", -7: "W2_ERR_TIMEOUT", -8: "W2_ERR_UNSUPPORTED"}

EXPORTS = ("w2_create", "w2_set_potentials", "w2_set_state", "w2_stage_state", "w2_use_staged_state",
           "w2_get_state", "w2_step",
           "w2_step_profile", "w2_observables", "w2_theta", "w2_advect", "w2_destroy", "w2_status_string",
           "w2_last_cuda_error", "w2_set_hartree", "w2_set_patches", "w2_occupations", "w2_hermitian_eigvals",
           "w2_batch_create", "w2_batch_set_potentials", "w2_batch_set_state", "w2_batch_get_state",
           "w2_batch_observables", "w2_batch_step", "w2_batch_autotune", "w2_batch_destroy", "w2_batch_sync",
           "w2_batch_set_wait_limit", "w2_batch_inject_stall", "w2_debug_fail_alloc", "w2_debug_alloc_count",
           "w2_debug_umma_smem_desc", "w2_debug_umma_idesc", "w2_debug_umma_tile_off", "w2_debug_umma_gemm",
           "w2_observables_enqueue", "w2_observables_collect", "w2_set_exchange_symmetry", "w2_set_tensor_path", "w2_debug_sweep_stall",
           "w2_mlp_create", "w2_mlp_create_kernel", "w2_pair_kernel_train_step", "w2_pair_kernel_loss_grad", "w2_mlp_param_count", "w2_mlp_input_dim", "w2_mlp_set_params", "w2_mlp_get_params",
           "w2_mlp_set_scales", "w2_mlp_forward", "w2_mlp_train_step", "w2_mlp_gradients", "w2_mlp_destroy",
           "w2_features", "w2_theta_pair", "w2_learned_attach", "w2_learned_report",
           "w2_sem_create", "w2_sem_set_potentials", "w2_sem_momenta", "w2_sem_set_state", "w2_sem_get_state",
           "w2_sem_theta", "w2_sem_advect", "w2_sem_step", "w2_sem_observables", "w2_sem_occupations",
           "w2_sem_destroy")
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


class SemConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ncell", ctypes.c_int32), ("nq", ctypes.c_int32), ("L", ctypes.c_double),
                ("Lp", ctypes.c_double), ("dt", ctypes.c_double), ("hbar", ctypes.c_double),
                ("mass", ctypes.c_double), ("xc_kind", ctypes.c_int32), ("precision", ctypes.c_int32)]


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
    lib.w2_set_patches.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    lib.w2_step_profile.argtypes = [vp, ctypes.c_int32, dp]
    lib.w2_observables.argtypes = [vp, ctypes.POINTER(Obs), dp, dp]
    lib.w2_theta.argtypes = [vp, vp, vp]
    lib.w2_advect.argtypes = [vp, vp, vp]
    lib.w2_destroy.argtypes = [vp]
    lib.w2_destroy.restype = None
    lib.w2_batch_create.argtypes = [ctypes.POINTER(Config), ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.w2_batch_set_potentials.argtypes = [vp, ctypes.c_int32, W2_FN, vp, W2_FN, vp, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double]
    lib.w2_batch_set_state.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_int32]
    lib.w2_batch_get_state.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_int32]
    lib.w2_batch_observables.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(Obs), dp, dp]
    lib.w2_batch_step.argtypes = [vp, ctypes.c_int32]
    lib.w2_batch_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
    lib.w2_batch_destroy.argtypes = [vp]
    lib.w2_batch_destroy.restype = None
    lib.w2_batch_sync.argtypes = [vp]
    lib.w2_batch_set_wait_limit.argtypes = [vp, ctypes.c_double]
    lib.w2_batch_inject_stall.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.w2_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.w2_mlp_create_kernel.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.w2_pair_kernel_train_step.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_float, dp]
    lib.w2_mlp_param_count.argtypes = [vp]
    lib.w2_mlp_param_count.restype = ctypes.c_size_t
    lib.w2_mlp_input_dim.argtypes = [vp]
    lib.w2_mlp_input_dim.restype = ctypes.c_int32
    lib.w2_mlp_set_params.argtypes = [vp, fp]
    lib.w2_mlp_get_params.argtypes = [vp, fp]
    lib.w2_mlp_set_scales.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    lib.w2_mlp_forward.argtypes = [vp, vp, ctypes.c_int32, vp]
    lib.w2_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_float, dp]
    lib.w2_mlp_gradients.argtypes = [vp, vp, vp, ctypes.c_int32, fp, dp]
    lib.w2_mlp_destroy.argtypes = [vp]
    lib.w2_mlp_destroy.restype = None
    lib.w2_features.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp]
    lib.w2_theta_pair.argtypes = [vp, vp, vp]
    lib.w2_learned_attach.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_double]
    lib.w2_learned_report.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), dp]
    lib.w2_sem_create.argtypes = [ctypes.POINTER(SemConfig), vp, ctypes.POINTER(vp)]
    lib.w2_sem_set_potentials.argtypes = [vp, W2_FN, vp, W2_FN, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.w2_sem_momenta.argtypes = [vp, dp, dp]
    lib.w2_sem_set_state.argtypes = [vp, vp, ctypes.c_int32]
    lib.w2_sem_get_state.argtypes = [vp, vp, ctypes.c_int32]
    lib.w2_sem_theta.argtypes = [vp, vp, vp]
    lib.w2_sem_advect.argtypes = [vp, vp, vp]
    lib.w2_sem_step.argtypes = [vp, ctypes.c_int32]
    lib.w2_sem_observables.argtypes = [vp, ctypes.POINTER(Obs), dp]
    lib.w2_sem_occupations.argtypes = [vp, dp, dp]
    lib.w2_sem_destroy.argtypes = [vp]
    lib.w2_sem_destroy.restype = None
    lib.w2_status_string.argtypes = [ctypes.c_int]
    lib.w2_status_string.restype = ctypes.c_char_p
    lib.w2_last_cuda_error.restype = ctypes.c_char_p
    lib.w2_debug_fail_alloc.argtypes = [ctypes.c_int32]
    lib.w2_debug_alloc_count.argtypes = []
    lib.w2_debug_alloc_count.restype = ctypes.c_int64
    lib.w2_debug_umma_smem_desc.argtypes = [ctypes.c_uint32] * 3
    lib.w2_debug_umma_smem_desc.restype = ctypes.c_uint64
    lib.w2_debug_umma_idesc.argtypes = [ctypes.c_int32] * 4
    lib.w2_debug_umma_idesc.restype = ctypes.c_uint32
    lib.w2_debug_umma_tile_off.argtypes = [ctypes.c_int32] * 3
    lib.w2_debug_umma_tile_off.restype = ctypes.c_uint32
    lib.w2_debug_umma_gemm.argtypes = [ctypes.c_int32] * 6 + [vp, vp, vp]
    lib.w2_debug_sweep_stall.argtypes = [vp, ctypes.c_int32, ctypes.c_int64]
    lib.w2_set_tensor_path.argtypes = [vp, ctypes.c_int32]
    for name in EXPORTS:
        if name not in ("w2_destroy", "w2_status_string", "w2_last_cuda_error", "w2_batch_destroy", "w2_mlp_destroy",
                        "w2_sem_destroy", "w2_debug_alloc_count", "w2_debug_umma_smem_desc",
                        "w2_debug_umma_idesc", "w2_debug_umma_tile_off",
                        "w2_mlp_param_count", "w2_mlp_input_dim"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def debug_fail_alloc(n: int):
    """Make the n-th device or pinned-host allocation of the library from now
    (0: the next one) fail once as if the device were full; n < 0 disarms."""
    _check(load().w2_debug_fail_alloc(int(n)), "w2_debug_fail_alloc")


def debug_alloc_count() -> int:
    """Allocations the library has attempted since it was loaded."""
    return int(load().w2_debug_alloc_count())


def umma_smem_desc(saddr: int, lbo: int, sbo: int) -> int:
    """The tcgen05 shared-memory matrix descriptor (no swizzle) the library encodes."""
    return int(load().w2_debug_umma_smem_desc(saddr, lbo, sbo))


def umma_idesc(M: int, N: int, a_mn: bool, b_mn: bool) -> int:
    """The tcgen05 kind::f16 instruction descriptor (BF16 in, FP32 out) the library encodes."""
    return int(load().w2_debug_umma_idesc(M, N, int(a_mn), int(b_mn)))


def umma_tile_off(r: int, c: int, ncol: int) -> int:
    """Byte offset of element (r, c) in the library's tiled 16-bit operand layout."""
    return int(load().w2_debug_umma_tile_off(r, c, ncol))


def umma_gemm(A, B, a_mn: bool = False, b_mn: bool = False, swap: bool = False):
    """One tcgen05 MMA chain D = A B on one CTA (A: M x K, B: K x N, BF16
    tensors on the device); returns the raw TMEM dump, [128][2N] uint32 words
    as an int32 tensor (marker 0x7fc0dead where the MMA did not write)."""
    import torch
    M, K = A.shape
    K2, N = B.shape
    if K2 != K or A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16:
        raise ValueError("A (M x K) and B (K x N) must be BF16 with matching K")
    A, B = A.contiguous(), B.contiguous()
    dump = torch.empty((128, 2 * N), dtype=torch.int32, device=A.device)
    _check(load().w2_debug_umma_gemm(M, N, K, int(a_mn), int(b_mn), int(swap), A.data_ptr(), B.data_ptr(),
                                     dump.data_ptr()), "w2_debug_umma_gemm")
    return dump


def _check(code: int, what: str):
    if code != 0:
        if code == -2:  # W2_ERR_CUDA: name the CUDA error behind it
            what = f"{what} ({load().w2_last_cuda_error().decode()})"
        raise W2Error(code, what)


def _dev_ptr(t, shape=None, dtype=None):
    import torch
    dtype = dtype or torch.float64
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} CUDA tensor")
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

    def __init__(self, nx, nk, L, dt, hbar=1.0, mass=1.0, xc_kind=0, stream=None, precision=W2_F64):
        import torch
        self.lib = load()
        self.precision = precision
        self.np_dtype = np.float64 if precision in F64_STATE else np.float32
        self.torch_dtype = torch.float64 if precision in F64_STATE else torch.float32
        self.shape = (nx, nx, nk, nk)
        self.nx, self.nk = nx, nk
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        cfg = Config(nx, nk, L, dt, hbar, mass, precision, xc_kind)
        h = ctypes.c_void_p()
        _check(self.lib.w2_create(ctypes.byref(cfg), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)),
               "w2_create")
        self.h = h
        self._keep = []

    @classmethod
    def from_problem(cls, prob, stream=None, precision=W2_F64):
        ctx = cls(prob.nx, prob.nk, prob.L, prob.dt, prob.hbar, prob.mass, prob.xc_kind, stream, precision)
        if getattr(prob, "hartree", "pair") == "poisson":
            ctx.set_hartree(W2_HARTREE_POISSON)
        ctx.set_potentials(prob.vext, prob.vee, prob.gamma, prob.c_hartree, prob.c_xc)
        return ctx

    def set_hartree(self, kind):
        _check(self.lib.w2_set_hartree(self.h, int(kind)), "w2_set_hartree")

    def set_exchange_symmetry(self, on=True):
        """Declare the state exchange symmetric, f(x1, x2, p1, p2) =
        f(x2, x1, p2, p1): the sliced step then computes the operator on the
        blocks with i1 <= i2 and mirrors the rest (W2_F64_SLICED)."""
        _check(self.lib.w2_set_exchange_symmetry(self.h, 1 if on else 0), "w2_set_exchange_symmetry")

    def set_tensor_path(self, tcgen05=True):
        """Run the sliced sweeps' digit products on tcgen05 (True; nk = 64)
        or on warp-level mma.sync (False, the default)."""
        _check(self.lib.w2_set_tensor_path(self.h, 1 if tcgen05 else 0), "w2_set_tensor_path")

    def debug_sweep_stall(self, stall, wait_cycles=0):
        """Fault injection into the tcgen05 sweep (its next bounded wait runs
        out); stall=False restores normal sweeps and clears the error word."""
        _check(self.lib.w2_debug_sweep_stall(self.h, 1 if stall else 0, ctypes.c_int64(int(wait_cycles))),
               "w2_debug_sweep_stall")

    def set_patches(self, np1, np2):
        """Cut the x1 and x2 shifts into np1 and np2 patches joined by
        perfectly matched boundary conditions (1: the global spline)."""
        _check(self.lib.w2_set_patches(self.h, int(np1), int(np2)), "w2_set_patches")

    def occupations(self):
        """(occupation numbers of the one-body density matrix, largest first;
        correlation entropy)."""
        occ = np.zeros(self.nx)
        s = ctypes.c_double()
        _check(self.lib.w2_occupations(self.h, occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(s)), "w2_occupations")
        return occ, s.value

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
            f = np.ascontiguousarray(f, dtype=self.np_dtype)
            assert f.shape == self.shape
            _check(self.lib.w2_set_state(self.h, ctypes.c_void_p(f.ctypes.data), 0), "w2_set_state")
        else:
            _check(self.lib.w2_set_state(self.h, _dev_ptr(f, self.shape, self.torch_dtype), 1), "w2_set_state")

    def stage_state(self, f):
        """Queue the host-to-device copy of the next state (a CPU tensor, pinned
        for an asynchronous copy, or a numpy array; it must stay unchanged until
        a synchronising call after use_staged_state)."""
        if isinstance(f, np.ndarray):
            assert f.dtype == self.np_dtype and f.flags.c_contiguous and f.shape == self.shape
            ptr = f.ctypes.data
        else:
            assert (not f.is_cuda) and f.is_contiguous() and tuple(f.shape) == self.shape
            assert f.dtype == self.torch_dtype
            ptr = f.data_ptr()
        _check(self.lib.w2_stage_state(self.h, ctypes.c_void_p(ptr)), "w2_stage_state")

    def use_staged_state(self):
        _check(self.lib.w2_use_staged_state(self.h), "w2_use_staged_state")

    def get_state(self, out=None):
        import torch
        if out is None:
            out = np.empty(self.shape, dtype=self.np_dtype)
        if isinstance(out, np.ndarray):
            _check(self.lib.w2_get_state(self.h, ctypes.c_void_p(out.ctypes.data), 0), "w2_get_state")
        elif isinstance(out, torch.Tensor) and not out.is_cuda:
            _check(self.lib.w2_get_state(self.h, ctypes.c_void_p(out.data_ptr()), 0), "w2_get_state")
        else:
            _check(self.lib.w2_get_state(self.h, _dev_ptr(out, self.shape, self.torch_dtype), 1), "w2_get_state")
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

    def observables_enqueue(self, slot):
        """Queue the observables of the current state into host slot 0 or 1
        without waiting (collect them with observables_collect)."""
        _check(self.lib.w2_observables_enqueue(self.h, int(slot)), "w2_observables_enqueue")

    def observables_collect(self, slot, raise_nonfinite=False) -> Observables:
        """Wait for slot's queued observables and return them."""
        o = Obs()
        n1 = np.zeros(self.nx)
        n12 = np.zeros((self.nx, self.nx))
        dp = ctypes.POINTER(ctypes.c_double)
        code = self.lib.w2_observables_collect(self.h, int(slot), ctypes.byref(o), n1.ctypes.data_as(dp),
                                               n12.ctypes.data_as(dp))
        if code not in (0, -6) or (code == -6 and raise_nonfinite):
            _check(code, "w2_observables_collect")
        return Observables(o.mass, o.energy, o.purity, o.entropy_lin, o.l2norm, o.step, n1, n12, STATUS[code])

    def theta_pair(self, f, out):
        """out = the exact two-body term of f alone."""
        _check(self.lib.w2_theta_pair(self.h, _dev_ptr(f, self.shape, self.torch_dtype),
                                      _dev_ptr(out, self.shape, self.torch_dtype)), "w2_theta_pair")
        return out

    def features(self, mlp, f, xs, x):
        """Input rows for the spatial points xs (int32 CUDA tensor, or None for all)."""
        import torch
        rows = self.nx * self.nx if xs is None else int(xs.numel())
        xp = None if xs is None else ctypes.c_void_p(xs.data_ptr())
        assert x.dtype == torch.bfloat16 and x.is_cuda and x.is_contiguous() and x.shape == (rows, mlp.din)
        _check(self.lib.w2_features(self.h, mlp.h, _dev_ptr(f, self.shape, self.torch_dtype), xp, rows,
                                    ctypes.c_void_p(x.data_ptr())), "w2_features")
        return x

    def attach_learned(self, mlp, judge_every=50, tol=0.1):
        _check(self.lib.w2_learned_attach(self.h, None if mlp is None else mlp.h, int(judge_every), float(tol)),
               "w2_learned_attach")
        self._mlp = mlp

    def learned_report(self):
        a, j, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(self.lib.w2_learned_report(self.h, ctypes.byref(a), ctypes.byref(j), ctypes.byref(e)),
               "w2_learned_report")
        return {"active": bool(a.value), "judged": j.value, "last_err": e.value}

    def theta(self, f, out):
        _check(self.lib.w2_theta(self.h, _dev_ptr(f, self.shape, self.torch_dtype),
                                 _dev_ptr(out, self.shape, self.torch_dtype)), "w2_theta")
        return out

    def advect(self, f, out):
        _check(self.lib.w2_advect(self.h, _dev_ptr(f, self.shape, self.torch_dtype),
                                  _dev_ptr(out, self.shape, self.torch_dtype)), "w2_advect")
        return out


class Batch:
    """A w2_batch: independent W2_F32_TF32X3 problems advanced together."""

    def __init__(self, problems, stream=None):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.problems = list(problems)
        cfgs = (Config * len(self.problems))(*[
            Config(p.nx, p.nk, p.L, p.dt, p.hbar, p.mass, W2_F32_TF32X3, p.xc_kind) for p in self.problems])
        h = ctypes.c_void_p()
        _check(self.lib.w2_batch_create(cfgs, len(self.problems), ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.byref(h)), "w2_batch_create")
        self.h = h
        self._keep = []
        for i, p in enumerate(self.problems):
            ce = W2_FN(lambda x, _u, f=p.vext: float(f(x)))
            cw = W2_FN(lambda r, _u, f=p.vee: float(f(r)))
            self._keep += [ce, cw]
            _check(self.lib.w2_batch_set_potentials(self.h, i, ce, None, cw, None, p.gamma, p.c_hartree, p.c_xc),
                   "w2_batch_set_potentials")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.w2_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, i):
        p = self.problems[i]
        return (p.nx, p.nx, p.nk, p.nk)

    def set_state(self, i, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float32)
            assert f.shape == self.shape(i)
            _check(self.lib.w2_batch_set_state(self.h, i, ctypes.c_void_p(f.ctypes.data), 0), "w2_batch_set_state")
        else:
            import torch
            _check(self.lib.w2_batch_set_state(self.h, i, _dev_ptr(f, self.shape(i), torch.float32), 1),
                   "w2_batch_set_state")

    def get_state(self, i):
        out = np.empty(self.shape(i), dtype=np.float32)
        _check(self.lib.w2_batch_get_state(self.h, i, ctypes.c_void_p(out.ctypes.data), 0), "w2_batch_get_state")
        return out

    def step(self, nsteps=1):
        _check(self.lib.w2_batch_step(self.h, int(nsteps)), "w2_batch_step")

    def autotune(self):
        """Time every tile shape of the one-launch step on the live batch and
        keep the fastest (the states are restored)."""
        g = (ctypes.c_int32 * 8)()
        _check(self.lib.w2_batch_autotune(self.h, g, 8), "w2_batch_autotune")
        v = list(g)
        return {"shift_cols": v[0], "theta_split": v[1], "grid": v[2], "smem_bytes": v[3], "step_us": v[4],
                "shapes_tried": v[5], "items_per_step": v[6], "items_per_cta": v[7]}

    def sync(self):
        """Wait for the queued steps; the status code (0, or -7 for a wait that ran out)."""
        return int(self.lib.w2_batch_sync(self.h))

    def set_wait_limit(self, seconds):
        _check(self.lib.w2_batch_set_wait_limit(self.h, float(seconds)), "w2_batch_set_wait_limit")

    def inject_stall(self, phase, instance=0):
        """Host-side fault injection: stop counting the finished items of one
        phase of one instance (phase -1 removes it)."""
        _check(self.lib.w2_batch_inject_stall(self.h, int(phase), int(instance)), "w2_batch_inject_stall")

    def observables(self, i):
        o = Obs()
        nx = self.problems[i].nx
        n1 = np.zeros(nx)
        n12 = np.zeros((nx, nx))
        dp = ctypes.POINTER(ctypes.c_double)
        code = self.lib.w2_batch_observables(self.h, i, ctypes.byref(o), n1.ctypes.data_as(dp),
                                             n12.ctypes.data_as(dp))
        if code not in (0, -6):
            _check(code, "w2_batch_observables")
        return Observables(o.mass, o.energy, o.purity, o.entropy_lin, o.l2norm, o.step, n1, n12, STATUS[code])


class MLP:
    """A w2_mlp: the learned stand-in for the two-body term.  kind="pair": the
    term itself per point; kind="kernel": the term's shift kernel per pair
    distance (max_rows is then the largest nx)."""

    def __init__(self, nk, hidden=256, max_rows=4096, stream=None, kind="pair"):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.kind = kind
        h = ctypes.c_void_p()
        create = self.lib.w2_mlp_create_kernel if kind == "kernel" else self.lib.w2_mlp_create
        _check(create(nk, hidden, max_rows, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)), "w2_mlp_create")
        self.h = h
        self.nk, self.hidden, self.max_rows = nk, hidden, max_rows
        self.dout = nk if kind == "kernel" else nk * nk
        self.din = int(self.lib.w2_mlp_input_dim(h))
        self.nparams = int(self.lib.w2_mlp_param_count(h))
        self.scales = (1.0, 1.0, 1.0)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.w2_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        """[(name, offset, shape)] of the packed parameters."""
        dims = [(self.din, self.hidden), (self.hidden, self.hidden), (self.hidden, self.hidden),
                (self.hidden, self.dout)]
        out, off = [], 0
        for l, (i, o) in enumerate(dims):
            out.append((f"W{l}", off, (i, o)))
            off += i * o
            out.append((f"b{l}", off, (o,)))
            off += o
        return out

    def get_params(self):
        p = np.empty(self.nparams, dtype=np.float32)
        _check(self.lib.w2_mlp_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "w2_mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        _check(self.lib.w2_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "w2_mlp_set_params")

    def set_scales(self, s_f, s_f1, s_y):
        self.scales = (float(s_f), float(s_f1), float(s_y))
        _check(self.lib.w2_mlp_set_scales(self.h, *self.scales), "w2_mlp_set_scales")

    def forward(self, x, y):
        _check(self.lib.w2_mlp_forward(self.h, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                       ctypes.c_void_p(y.data_ptr())), "w2_mlp_forward")
        return y

    def train_step(self, x, target, lr):
        loss = ctypes.c_double()
        _check(self.lib.w2_mlp_train_step(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                          int(x.shape[0]), float(lr), ctypes.byref(loss)), "w2_mlp_train_step")
        return loss.value

    def kernel_train_step(self, ctx, f, p, dr, lr):
        """One Adam step of a kernel network on rows of (state block, exact
        two-body term, pair distance index) from trajectories (device
        tensors float64 [rows][nk^2], float64 [rows][nk^2], int32 [rows])."""
        loss = ctypes.c_double()
        _check(self.lib.w2_pair_kernel_train_step(ctx.h, self.h, ctypes.c_void_p(f.data_ptr()),
                                                  ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(dr.data_ptr()),
                                                  int(f.shape[0]), float(lr), ctypes.byref(loss)),
               "w2_pair_kernel_train_step")
        return loss.value

    def kernel_loss_grad(self, ctx, f, p, dr):
        """(relative loss, network outputs y [nx][nk], dL/dy [nx][nk]) of a
        kernel network on rows of (state block, exact two-body term, pair
        distance index), without an update."""
        loss = ctypes.c_double()
        y = np.zeros((ctx.nx, self.nk), dtype=np.float32)
        g = np.zeros((ctx.nx, self.nk), dtype=np.float64)
        _check(self.lib.w2_pair_kernel_loss_grad(ctx.h, self.h, ctypes.c_void_p(f.data_ptr()),
                                                 ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(dr.data_ptr()),
                                                 int(f.shape[0]), ctypes.byref(loss),
                                                 y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "w2_pair_kernel_loss_grad")
        return loss.value, y, g

    def gradients(self, x, target):
        g = np.empty(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        _check(self.lib.w2_mlp_gradients(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                         int(x.shape[0]), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         ctypes.byref(loss)), "w2_mlp_gradients")
        return g, loss.value


def hermitian_eigvals(a):
    """Eigenvalues (largest first) of a batch of complex Hermitian matrices:
    a is a CUDA complex128 tensor [batch][n][n] (overwritten)."""
    import torch
    assert a.dtype == torch.complex128 and a.is_cuda and a.is_contiguous() and a.dim() == 3
    batch, n, n2 = a.shape
    assert n == n2
    eig = torch.empty(batch, n, dtype=torch.float64, device=a.device)
    lib = load()
    lib.w2_hermitian_eigvals.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p]
    _check(lib.w2_hermitian_eigvals(ctypes.c_void_p(a.data_ptr()), n, batch, ctypes.c_void_p(eig.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "w2_hermitian_eigvals")
    return eig


class SemContext:
    """A w2_sem_ctx: one non-periodic problem (bounded box, Chebyshev
    spectral elements in momentum) on the current CUDA device.  Arrays are
    float64 [nx][nx][np][np]."""

    def __init__(self, nx, ncell, nq, L, Lp, dt, hbar=1.0, mass=1.0, xc_kind=0, stream=None, precision=W2_F64):
        import torch
        self.lib = load()
        self.precision = precision
        self.np_ = ncell * nq
        self.nx = nx
        self.shape = (nx, nx, self.np_, self.np_)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        cfg = SemConfig(nx, ncell, nq, L, Lp, dt, hbar, mass, xc_kind, precision)
        h = ctypes.c_void_p()
        _check(self.lib.w2_sem_create(ctypes.byref(cfg), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)),
               "w2_sem_create")
        self.h = h
        self._keep = []

    @classmethod
    def from_problem(cls, prob, stream=None, precision=W2_F64):
        ctx = cls(prob.nx, prob.ncell, prob.nq, prob.L, prob.Lp, prob.dt, prob.hbar, prob.mass, prob.xc_kind, stream,
                  precision)
        ctx.set_potentials(prob.vext, prob.vee, prob.gamma, prob.c_hartree, prob.c_xc)
        return ctx

    def set_potentials(self, vext, vee, gamma, c_h, c_xc):
        fe = W2_FN(lambda x, u: float(vext(x)))
        fw = W2_FN(lambda x, u: float(vee(x)))
        self._keep = [fe, fw]
        _check(self.lib.w2_sem_set_potentials(self.h, fe, None, fw, None, gamma, c_h, c_xc), "w2_sem_set_potentials")

    def momenta(self):
        p = np.zeros(self.np_)
        w = np.zeros(self.np_)
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self.lib.w2_sem_momenta(self.h, p.ctypes.data_as(dp), w.ctypes.data_as(dp)), "w2_sem_momenta")
        return p, w

    def set_state(self, f):
        import torch
        if isinstance(f, torch.Tensor):
            _check(self.lib.w2_sem_set_state(self.h, _dev_ptr(f, self.shape), 1), "w2_sem_set_state")
        else:
            a = np.ascontiguousarray(f, dtype=np.float64)
            assert a.shape == self.shape
            _check(self.lib.w2_sem_set_state(self.h, a.ctypes.data_as(ctypes.c_void_p), 0), "w2_sem_set_state")

    def get_state(self, out=None):
        if out is not None:
            _check(self.lib.w2_sem_get_state(self.h, _dev_ptr(out, self.shape), 1), "w2_sem_get_state")
            return out
        a = np.empty(self.shape)
        _check(self.lib.w2_sem_get_state(self.h, a.ctypes.data_as(ctypes.c_void_p), 0), "w2_sem_get_state")
        return a

    def theta(self, f, out):
        _check(self.lib.w2_sem_theta(self.h, _dev_ptr(f, self.shape), _dev_ptr(out, self.shape)), "w2_sem_theta")
        return out

    def advect(self, f, out):
        _check(self.lib.w2_sem_advect(self.h, _dev_ptr(f, self.shape), _dev_ptr(out, self.shape)), "w2_sem_advect")
        return out

    def step(self, n=1):
        _check(self.lib.w2_sem_step(self.h, int(n)), "w2_sem_step")

    def observables(self):
        o = Obs()
        n1 = np.zeros(self.nx)
        _check(self.lib.w2_sem_observables(self.h, ctypes.byref(o), n1.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "w2_sem_observables")
        return Observables(o.mass, o.energy, o.purity, o.entropy_lin, o.l2norm, o.step, n1, None, "W2_OK")

    def occupations(self):
        """(occupation numbers of the one-body density matrix, largest first;
        correlation entropy)."""
        occ = np.zeros(self.nx)
        s = ctypes.c_double()
        _check(self.lib.w2_sem_occupations(self.h, occ.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.byref(s)), "w2_sem_occupations")
        return occ, s.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.w2_sem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
