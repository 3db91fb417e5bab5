"""GPU checks of the precision form (W2_F32_TF32X3: FP32 state, TF32 hi+lo
tensor-core contractions, spline coefficients solved in double-float pairs,
FP32 increments, FP64 reductions).

Bars: the operator alone within 2e-6 relative L2 of the FP64 oracle on the
same (FP32-representable) input; the shift within 1e-6; time steps within the
1e-6 relative L2 of the forms against the FP64 path, checked over 20 steps of
the small workload, 200 and 500 steps of the 64^4 double-well workload and
500 steps of every instance of the 64-instance batch, with the error of each
observable stated.
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


def _ctx(prob, precision):
    from paper_2511_11354_gb300 import w2
    return w2.Context.from_problem(prob, precision=precision)


@pytest.mark.parametrize("nx,nk", [(8, 16), (12, 32), (20, 48), (16, 64), (6, 128), (24, 80)])
def test_theta32_parity(nx, nk):
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=11, noise=0.05).astype(np.float32)
    ctx = _ctx(prob, w2.W2_F32_TF32X3)
    out = torch.empty(*f.shape, dtype=torch.float32, device="cuda")
    ctx.theta(torch.from_numpy(f).cuda(), out)
    ref = oracle.Oracle(prob).theta(f.astype(np.float64))
    assert rel(out.cpu().numpy(), ref) < 2e-6


@pytest.mark.parametrize("nx,nk,dt", [(8, 16, 0.37), (33, 32, 0.02), (64, 16, 0.9)])
def test_advect32_parity(nx, nk, dt):
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    prob.dt = dt
    prob.vext, prob.vee, prob.gamma, prob.c_hartree = inputs.zero_potential(), inputs.zero_potential(), 0.0, 0.0
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=5, noise=0.1).astype(np.float32)
    ctx = _ctx(prob, w2.W2_F32_TF32X3)
    out = torch.empty(*f.shape, dtype=torch.float32, device="cuda")
    ctx.advect(torch.from_numpy(f).cuda(), out)
    assert rel(out.cpu().numpy(), oracle.Oracle(prob).advect(f.astype(np.float64))) < 1e-6


def test_step32_small_workload_vs_oracle():
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=32, nk=32)
    ctx = _ctx(prob, w2.W2_F32_TF32X3)
    ctx.set_state(f0.astype(np.float32))
    ctx.step(20)
    ref = oracle.Oracle(prob).step(f0, 20)
    assert rel(ctx.get_state(), ref) < 1e-6


def _f64_and_f32_run(prob, f0, steps, ref=None):
    from paper_2511_11354_gb300 import w2
    a = _ctx(prob, w2.W2_F64 if ref is None else ref)
    a.set_state(f0)
    b = _ctx(prob, w2.W2_F32_TF32X3)
    b.set_state(f0.astype(np.float32))
    obs_a, obs_b = [], []
    done = 0
    while done < steps:
        k = min(50, steps - done)
        a.step(k)
        b.step(k)
        done += k
        obs_a.append(a.observables())
        obs_b.append(b.observables())
    return a, b, obs_a, obs_b


def test_step32_dwell_64_200_steps_vs_f64_path():
    """The precision form's acceptance check: the 64^4 double-well workload,
    200 steps, relative L2 <= 1e-6 against the FP64 path (which matches the
    oracle to 1e-10), plus the error of each observable."""
    prob, f0 = inputs.workload_dwell()
    a, b, oa, ob = _f64_and_f32_run(prob, f0, 200)
    fa, fb = a.get_state(), b.get_state()
    err = rel(fb, fa)
    assert err < 1e-6, err
    for x, y in zip(oa, ob):
        assert abs(y.mass - x.mass) < 1e-6 * abs(x.mass)
        assert abs(y.energy - x.energy) < 1e-6 * abs(x.energy)
        assert abs(y.entropy_lin - x.entropy_lin) < 1e-6
        assert np.abs(y.n1 - x.n1).max() < 1e-6 * np.abs(x.n1).max()
        assert np.abs(y.n12 - x.n12).max() < 1e-6 * np.abs(x.n12).max()


def test_step32_dwell_64_500_steps_vs_f64_path():
    """Config 3's length on the 64^4 double-well workload: 500 steps against
    the sliced FP64 path (held to the oracle at 1e-10), observables every 50
    steps."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell()
    a, b, oa, ob = _f64_and_f32_run(prob, f0, 500, ref=w2.W2_F64_SLICED)
    err = rel(b.get_state(), a.get_state())
    assert err < 1e-6, err
    for x, y in zip(oa, ob):
        assert abs(y.mass - x.mass) < 1e-6 * abs(x.mass)
        assert abs(y.energy - x.energy) < 1e-6 * abs(x.energy)
        assert abs(y.entropy_lin - x.entropy_lin) < 1e-6
        assert np.abs(y.n1 - x.n1).max() < 1e-6 * np.abs(x.n1).max()
        assert np.abs(y.n12 - x.n12).max() < 1e-6 * np.abs(x.n12).max()
    a.close()
    b.close()


def test_batch_500_steps_vs_f64_path_every_instance():
    """The batching workload (64 uneven instances, seed 3) for 500 steps: every
    instance within 1e-6 relative L2 of its own sliced FP64 run."""
    from paper_2511_11354_gb300 import w2
    probs, states = inputs.workload_batch(64, seed=3)
    bt = w2.Batch(probs)
    for i, f in enumerate(states):
        bt.set_state(i, f.astype(np.float32))
    bt.step(500)
    worst = 0.0
    for i, (prob, f) in enumerate(zip(probs, states)):
        a = _ctx(prob, w2.W2_F64_SLICED)
        a.set_state(f)
        a.step(500)
        err = rel(bt.get_state(i), a.get_state())
        a.close()
        worst = max(worst, err)
        assert err < 1e-6, (i, prob.nx, prob.nk, err)
    bt.close()
    print(f"batch 500 steps: worst instance rel L2 {worst:.2e}")


def test_step32_exchange_symmetry_and_determinism():
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=16, nk=32)
    outs = []
    for _ in range(2):
        c = _ctx(prob, w2.W2_F32_TF32X3)
        c.set_state(f0.astype(np.float32))
        c.step(10)
        outs.append(c.get_state())
    assert np.array_equal(outs[0], outs[1])
    g = outs[0].astype(np.float64)
    assert np.abs(g - g.transpose(1, 0, 3, 2)).max() < 1e-5 * np.abs(g).max()


def test_precision_full_size_128_sampled_outputs():
    """The timed 128^4 workload itself: the operator at 24 sampled spatial
    points and the shift on 24 sampled momentum planes against the oracle,
    then one step that stays finite and exchange symmetric."""
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_dwell(nx=128, nk=128)
    f = inputs.initial_state_chunked(prob, centres=inputs.draw_centres(2), seed=2)
    ctx = _ctx(prob, w2.W2_F32_TF32X3)
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
    planes = rng.choice(prob.nk * prob.nk, 24, replace=False)
    ctx.advect(d, out)
    got = out.view(prob.nx, prob.nx, prob.nk * prob.nk)[:, :, torch.from_numpy(planes).cuda()]
    got = got.permute(2, 0, 1).contiguous().cpu().numpy()
    assert rel(got, o.advect_sample(f64, planes)) < 1e-6
    del f64
    ctx.set_state(d)
    ctx.step(1)
    ctx.get_state(out)
    assert bool(torch.isfinite(out).all())
    sym = out.permute(1, 0, 3, 2)
    assert float((out - sym).abs().max()) < 1e-5 * float(out.abs().max())
