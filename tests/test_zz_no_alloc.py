"""The allocation-free pseudo-difference entry point (w2_theta_noalloc).

Some callers cannot allocate device memory (an open stream capture, a host
framework that owns and budgets all device memory, a plug-in that may not touch
the allocator).  w2_theta_noalloc serves them: the caller passes inputs and
outputs, and the kernel tables live in a fixed array inside the library.  This
file checks it through the C ABI against the context-based w2_theta on the same
problem, on two calls in a row (the second call reuses the array the first one
filled), within the tolerance of the Theta parity tests, up to the largest grid
the array holds (nx = W2_NOALLOC_MAX_NX, nk = W2_NOALLOC_MAX_NK), and on a
small grid against the CPU oracle's operator.  It is named to be collected
last, so a run that stops at the first failure has run everything else first;
it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2511_11354_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12  # same bar as tests/test_gpu_f64.py::test_theta_parity


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11354_gb300 import build, w2
    build.build()
    L = w2.load()
    vp = ctypes.c_void_p
    L.w2_theta_noalloc.argtypes = [ctypes.POINTER(w2.Config), vp, vp, vp, vp, vp, vp]
    L.w2_theta_noalloc.restype = ctypes.c_int
    return L


def _samples(prob):
    """U1 = U2 = V_ext at x_i + l h' and U12 = gamma W at d dx + l h' (folded)."""
    M = 2 * prob.nk
    hp = prob.L / M
    x = prob.x()
    u1 = np.array([[prob.vext(float(inputs.fold(x[i] + l * hp, prob.L))) for l in range(M)]
                   for i in range(prob.nx)])
    u12 = np.array([[prob.gamma * prob.vee(float(inputs.fold(d * prob.dx + l * hp, prob.L))) for l in range(M)]
                    for d in range(prob.nx)])
    return u1, u12


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _call(lib, cfg, d_u1, d_u12, f, out):
    from paper_2511_11354_gb300 import w2
    rc = lib.w2_theta_noalloc(ctypes.byref(cfg), ctypes.c_void_p(d_u1.data_ptr()),
                              ctypes.c_void_p(d_u1.data_ptr()), ctypes.c_void_p(d_u12.data_ptr()),
                              ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, w2.STATUS.get(rc, rc)
    torch.cuda.synchronize()


@pytest.mark.parametrize("nx,nk", [(32, 32), (24, 48), (128, 64)])
def test_noalloc_matches_context_theta_twice(lib, nx, nk):
    """(128, 64) is the largest grid the fixed array holds: every table entry
    of the array is in use."""
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    prob.c_hartree = 0.0  # the caller's samples carry the whole potential
    ctx = w2.Context.from_problem(prob)
    u1, u12 = _samples(prob)
    d_u1 = torch.from_numpy(u1).cuda()
    d_u12 = torch.from_numpy(u12).cuda()
    cfg = w2.Config(prob.nx, prob.nk, prob.L, prob.dt, prob.hbar, prob.mass, w2.W2_F64, 0)
    for seed in (3, 4):  # two calls in a row, different states
        f0 = inputs.initial_state_chunked(prob, centres=(-2.0, 2.5), seed=seed, noise=0.05, dtype=np.float64)
        f = torch.from_numpy(f0).cuda()
        del f0
        ref = torch.empty_like(f)
        ctx.theta(f, ref)
        out = torch.full_like(f, float("nan"))
        _call(lib, cfg, d_u1, d_u12, f, out)
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < TOL
        del f, ref, out
    ctx.close()
    torch.cuda.empty_cache()


def test_noalloc_matches_oracle_twice(lib):
    """Against the CPU oracle's operator with the same samples: the oracle
    forms the local 2 nk-point modes of each potential and sums the momentum
    shifts as printed, with no shared code."""
    import oracle
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_small(nx=12, nk=16)
    prob.c_hartree = 0.0
    o = oracle.Oracle(prob)
    U = o.potential_fine(None)          # V_ext at x_i + l h'
    u1, u12 = _samples(prob)
    np.testing.assert_allclose(u1, U, rtol=0, atol=1e-15)
    d_u1 = torch.from_numpy(u1).cuda()
    d_u12 = torch.from_numpy(u12).cuda()
    cfg = w2.Config(prob.nx, prob.nk, prob.L, prob.dt, prob.hbar, prob.mass, w2.W2_F64, 0)
    for seed in (5, 6):
        f0 = inputs.initial_state(prob, centres=(-1.5, 2.0), seed=seed, noise=0.05)
        ref = o.theta_with(f0, U, U, terms=7)
        f = torch.from_numpy(f0).cuda()
        out = torch.full_like(f, float("nan"))
        _call(lib, cfg, d_u1, d_u12, f, out)
        got = out.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL


def test_noalloc_refuses_sizes_beyond_its_scratch(lib):
    from paper_2511_11354_gb300 import w2
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(d.data_ptr())
    o = torch.zeros(16, dtype=torch.float64, device="cuda")
    q = ctypes.c_void_p(o.data_ptr())
    too_wide = w2.Config(130, 32, 20.0, 0.01, 1.0, 1.0, w2.W2_F64, 0)
    too_fine = w2.Config(32, 72, 20.0, 0.01, 1.0, 1.0, w2.W2_F64, 0)
    for cfg in (too_wide, too_fine):
        assert lib.w2_theta_noalloc(ctypes.byref(cfg), p, p, p, p, q, None) == -8  # W2_ERR_UNSUPPORTED
    assert lib.w2_theta_noalloc(ctypes.byref(too_wide), p, p, p, p, p, None) == -1  # aliasing
