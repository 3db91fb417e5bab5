"""GPU checks of the distributed shift (Sec. 4.2): the x1 and x2 shifts cut
into patches, each solving a local spline with perfectly matched boundary
conditions from its neighbours' hand-over (all patches in one process, the
hand-over through device buffers), against the global spline and the FP64
oracle; and whole Lawson steps of the sharded grid against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2511_11354_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11354_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _advect(prob, f, patches):
    from paper_2511_11354_gb300 import w2
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
    ctx.set_patches(*patches)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.advect(d, out)
    got = out.cpu().numpy()
    ctx.close()
    return got


@pytest.mark.parametrize("nx,nk,dt,patches", [(64, 16, 0.005, (2, 2)), (64, 16, 0.9, (2, 1)), (64, 24, 0.3, (1, 2)),
                                              (128, 16, 0.05, (4, 2))])
def test_patch_shift_equals_global_spline(nx, nk, dt, patches):
    """Shifts below one cell (dt = 0.005) and of several cells (dt = 0.3, 0.9):
    the patched shift equals the global one to FP64 rounding and the oracle's
    tensor-product spline within 1e-13."""
    prob, _ = inputs.workload_dwell(nx=nx, nk=nk)
    prob.dt = dt  # the shift alone: no potentials (the long steps would fail the stability check)
    prob.vext, prob.vee, prob.gamma, prob.c_hartree = inputs.zero_potential(), inputs.zero_potential(), 0.0, 0.0
    f = inputs.initial_state(prob, centres=(-3.0, 2.0), seed=3, noise=0.05)
    got = _advect(prob, f, patches)
    glob = _advect(prob, f, (1, 1))
    assert rel(got, glob) < 1e-13
    assert rel(got, oracle.Oracle(prob).advect(f)) < 1e-13


def test_sharded_steps_vs_oracle():
    """Five Lawson steps of the 64^2 x 16^2 double-well problem (Hartree and
    pair term on) with both shifts cut into 2 x 2 patches: within 1e-10 of
    the FP64 oracle, as the unsharded path."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell(nx=64, nk=16)
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
    ctx.set_patches(2, 2)
    ctx.set_state(f0)
    ctx.step(5)
    got = ctx.get_state()
    ctx.close()
    ref = oracle.Oracle(prob).step(f0, 5)
    assert rel(got, ref) < 1e-10


def test_patch_limits():
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_dwell(nx=48, nk=16)
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
    with pytest.raises(w2.W2Error) as e:
        ctx.set_patches(2, 1)   # 24 points per patch: fewer than the 26-point stencil needs
    assert e.value.code == -8
    with pytest.raises(w2.W2Error) as e:
        ctx.set_patches(5, 1)   # 48 points do not split into 5 patches
    assert e.value.code == -8
    ctx.set_patches(1, 1)
    ctx.close()
    sl = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    with pytest.raises(w2.W2Error) as e:
        sl.set_patches(1, 2)
    assert e.value.code == -8
    sl.close()
