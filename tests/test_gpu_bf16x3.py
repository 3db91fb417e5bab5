"""GPU checks of the precision form's BF16 variant (W2_F32_BF16X3: FP32
state, the contractions with the state in three BF16 parts and the kernel in
four on mma.sync m16n8k16, FP32 accumulation; the shift and the reductions as
in W2_F32_TF32X3).

Bars as for the TF32 variant: the operator within 2e-6 relative L2 of the
FP64 oracle on the same FP32 input (every supported nk, ragged nx), the
corrector and its per-X sums through whole steps within 1e-6 of the oracle
(20 steps) and of the sliced FP64 path (500 steps of the 64^4 double-well
workload, observables every 50 steps), and the timed 128^4 workload on
sampled outputs.
"""
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ctx(prob, precision=None):
    from paper_2511_11354_gb300 import w2
    return w2.Context.from_problem(prob, precision=w2.W2_F32_BF16X3 if precision is None else precision)


@pytest.mark.parametrize("nx,nk", [(8, 16), (12, 32), (20, 48), (16, 64), (5, 80), (7, 96), (4, 112), (6, 128)])
def test_theta_bf16x3_parity(nx, nk):
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=11, noise=0.05).astype(np.float32)
    ctx = _ctx(prob)
    out = torch.empty(*f.shape, dtype=torch.float32, device="cuda")
    ctx.theta(torch.from_numpy(f).cuda(), out)
    ref = oracle.Oracle(prob).theta(f.astype(np.float64))
    err = rel(out.cpu().numpy(), ref)
    assert err < 2e-6, err


def test_theta_bf16x3_and_tf32x3_agree():
    """The two splittings of the same contraction on the same FP32 input:
    both are within their bar of the oracle, hence of each other."""
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_dwell(nx=24, nk=64)
    f = inputs.initial_state(prob, centres=(-3.0, 2.0), seed=4, noise=0.05).astype(np.float32)
    d = torch.from_numpy(f).cuda()
    outs = []
    for p in (w2.W2_F32_BF16X3, w2.W2_F32_TF32X3):
        c = _ctx(prob, p)
        o = torch.empty_like(d)
        c.theta(d, o)
        outs.append(o.cpu().numpy())
        c.close()
    assert rel(outs[0], outs[1]) < 4e-6


def test_step_bf16x3_small_workload_vs_oracle():
    prob, f0 = inputs.workload_small(nx=32, nk=32)
    ctx = _ctx(prob)
    ctx.set_state(f0.astype(np.float32))
    ctx.step(20)
    ref = oracle.Oracle(prob).step(f0, 20)
    assert rel(ctx.get_state(), ref) < 1e-6


def test_step_bf16x3_dwell_64_500_steps_vs_sliced_f64():
    """500 steps of the 64^4 double-well workload against the sliced FP64
    path (held to the oracle at 1e-10), state and observables every 50 steps
    within 1e-6."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell()
    a = _ctx(prob, w2.W2_F64_SLICED)
    a.set_state(f0)
    b = _ctx(prob)
    b.set_state(f0.astype(np.float32))
    for _ in range(10):
        a.step(50)
        b.step(50)
        x, y = a.observables(), b.observables()
        assert abs(y.mass - x.mass) < 1e-6 * abs(x.mass)
        assert abs(y.energy - x.energy) < 1e-6 * abs(x.energy)
        assert abs(y.entropy_lin - x.entropy_lin) < 1e-6
        assert np.abs(y.n1 - x.n1).max() < 1e-6 * np.abs(x.n1).max()
        assert np.abs(y.n12 - x.n12).max() < 1e-6 * np.abs(x.n12).max()
    err = rel(b.get_state(), a.get_state())
    assert err < 1e-6, err
    a.close()
    b.close()


def test_step_bf16x3_exchange_symmetry_and_determinism():
    prob, f0 = inputs.workload_small(nx=16, nk=32)
    outs = []
    for _ in range(2):
        c = _ctx(prob)
        c.set_state(f0.astype(np.float32))
        c.step(10)
        outs.append(c.get_state())
        c.close()
    assert np.array_equal(outs[0], outs[1])
    g = outs[0].astype(np.float64)
    assert np.abs(g - g.transpose(1, 0, 3, 2)).max() < 1e-5 * np.abs(g).max()


def test_bf16x3_full_size_128_sampled_outputs():
    """The timed 128^4 workload: the operator at 24 sampled spatial points
    against the oracle, then one step that stays finite and exchange
    symmetric."""
    prob, _ = inputs.workload_dwell(nx=128, nk=128)
    f = inputs.initial_state_chunked(prob, centres=inputs.draw_centres(2), seed=2)
    ctx = _ctx(prob)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    rng = np.random.default_rng(0)
    o = oracle.Oracle(prob)
    f64 = f.astype(np.float64)
    del f
    xs = rng.choice(prob.nx * prob.nx, 24, replace=False)
    ctx.theta(d, out)
    got = out.view(prob.nx * prob.nx, prob.nk, prob.nk)[torch.from_numpy(xs).cuda()].cpu().numpy()
    assert rel(got, o.theta_sample(f64, xs)) < 2e-6
    del f64
    ctx.set_state(d)
    ctx.step(1)
    ctx.get_state(out)
    assert bool(torch.isfinite(out).all())
    sym = out.permute(1, 0, 3, 2)
    assert float((out - sym).abs().max()) < 1e-5 * float(out.abs().max())
    ctx.close()
