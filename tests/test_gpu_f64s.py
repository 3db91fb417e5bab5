"""GPU parity of the sliced FP64 path (W2_F64_SLICED: the pseudo-difference
contractions as exact products of six 8-bit slices on the BF16 tensor cores,
the spline shift in double-float pairs) against the FP64 oracle, through the
C ABI.

Bars: the operator alone within 2e-12 relative L2 of the oracle (the slices
keep 48 bits of each operand relative to its block maximum; the difference
operator's cancellation costs about two decimal digits of that); the shift
within 1e-13 (pairs keep about 47 bits per operation); whole time steps within
1e-10 relative L2, the FP64 bar of the plain path.
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ctx(prob):
    from paper_2511_11354_gb300 import w2
    return w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nx,nk", [(8, 16), (12, 32), (20, 48), (16, 64), (7, 32), (33, 64)])
def test_sliced_theta_parity(nx, nk):
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=11, noise=0.05)
    ctx = _ctx(prob)
    out = torch.empty(prob.nx, prob.nx, prob.nk, prob.nk, dtype=torch.float64, device="cuda")
    ctx.theta(_dev(f), out)
    assert rel(out.cpu().numpy(), oracle.Oracle(prob).theta(f)) < 2e-12


def test_sliced_theta_parity_xc_hartree_and_signs():
    """H-L exchange-correlation on, and a state of both signs with a wide
    dynamic range inside each block (exercises the balanced digits and the
    per-block exponents)."""
    prob, f = inputs.workload_small(nx=16, nk=32)
    prob.c_xc, prob.xc_kind = -0.7, 2
    rng = np.random.default_rng(3)
    f = f * (1.0 + 0.5 * rng.standard_normal(f.shape)) - 0.3 * f.mean()
    f[3, 5] *= 1e-9  # one block many binades below the others
    ctx = _ctx(prob)
    out = torch.empty(*f.shape, dtype=torch.float64, device="cuda")
    ctx.theta(_dev(f), out)
    ref = oracle.Oracle(prob).theta(f)
    got = out.cpu().numpy()
    assert rel(got, ref) < 2e-12
    assert rel(got[3, 5], ref[3, 5]) < 2e-12  # the per-block scale keeps the small block's digits


@pytest.mark.parametrize("nx,nk,dt", [(8, 16, 0.37), (12, 32, 0.37), (33, 48, 0.05), (64, 64, 0.9), (20, 64, 0.005)])
def test_sliced_advect_parity(nx, nk, dt):
    """The double-float spline shift of the sliced path (shifts of many cells
    down to a small fraction of one) against the oracle's FP64 shift."""
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    prob.dt = dt
    prob.vext, prob.vee, prob.gamma, prob.c_hartree = inputs.zero_potential(), inputs.zero_potential(), 0.0, 0.0
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=5, noise=0.1)
    ctx = _ctx(prob)
    out = torch.empty(*f.shape, dtype=torch.float64, device="cuda")
    ctx.advect(_dev(f), out)
    assert rel(out.cpu().numpy(), oracle.Oracle(prob).advect(f)) < 1e-13


def test_sliced_step_parity_small_workload():
    prob, f0 = inputs.workload_small()
    ctx = _ctx(prob)
    ctx.set_state(f0)
    ctx.step(20)
    assert rel(ctx.get_state(), oracle.Oracle(prob).step(f0, 20)) < 1e-10


@pytest.mark.parametrize("nx,nk,steps", [(16, 16, 10), (20, 32, 5), (24, 48, 3)])
def test_sliced_step_parity_dwell_shapes(nx, nk, steps):
    prob, f0 = inputs.workload_dwell(nx=nx, nk=nk)
    ctx = _ctx(prob)
    ctx.set_state(_dev(f0))
    ctx.step(steps)
    assert rel(ctx.get_state(), oracle.Oracle(prob).step(f0, steps)) < 1e-10


def test_sliced_step_parity_full_size_workload():
    """64^4 double well (the benchmark workload, in its timed launch
    configuration), 2 steps, every element compared."""
    prob, f0 = inputs.workload_dwell()
    ctx = _ctx(prob)
    ctx.set_state(_dev(f0))
    ctx.step(2)
    got = ctx.get_state()
    assert rel(got, oracle.Oracle(prob).step(f0, 2)) < 1e-10
    assert np.abs(got - got.transpose(1, 0, 3, 2)).max() < 1e-13 * np.abs(got).max()


@pytest.mark.parametrize("prec", ["W2_F64_SLICED", "W2_F64"])
def test_largest_fp64_grid_sampled(prec):
    """The largest grid of the FP64 paths (nx = 128, nk = 64: 67M points,
    537 MB per array).  The operator at 16 sampled spatial points and the
    shift of 8 sampled momentum planes (lines of 128 points) against the
    oracle, then one step that stays finite and exchange symmetric."""
    from paper_2511_11354_gb300 import w2
    prob = inputs.Problem(nx=128, nk=64, L=24.0, dt=0.005, vext=inputs.double_well(20.0),
                          vee=inputs.soft_coulomb(1.0), gamma=1.0, c_hartree=1.0)
    f = inputs.initial_state_chunked(prob, centres=inputs.draw_centres(5), seed=5, dtype=np.float64)
    ctx = w2.Context.from_problem(prob, precision=getattr(w2, prec))
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    rng = np.random.default_rng(3)
    o = oracle.Oracle(prob)
    xs = rng.choice(prob.nx * prob.nx, 16, replace=False)
    ctx.theta(d, out)
    got = out.view(prob.nx * prob.nx, prob.nk, prob.nk)[torch.from_numpy(xs).cuda()].cpu().numpy()
    assert rel(got, o.theta_sample(f, xs)) < 2e-12
    planes = rng.choice(prob.nk * prob.nk, 8, replace=False)
    ctx.advect(d, out)
    got = out.view(prob.nx, prob.nx, prob.nk * prob.nk)[:, :, torch.from_numpy(planes).cuda()]
    got = got.permute(2, 0, 1).contiguous().cpu().numpy()
    assert rel(got, o.advect_sample(f, planes)) < 1e-13
    del f
    ctx.set_state(d)
    ctx.step(1)
    ctx.get_state(out)
    assert bool(torch.isfinite(out).all())
    g = out.view(prob.nx, prob.nx, prob.nk, prob.nk)
    assert (g - g.permute(1, 0, 3, 2)).abs().max().item() < 1e-13 * g.abs().max().item()


def test_sliced_and_fp64_pipe_paths_agree_over_200_steps():
    """The two FP64 paths on the 64^4 workload over 200 steps (the FP64-pipe
    path is itself held to the oracle by test_gpu_f64.py)."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell()
    a = w2.Context.from_problem(prob)
    b = _ctx(prob)
    d = _dev(f0)
    a.set_state(d)
    b.set_state(d)
    a.step(200)
    b.step(200)
    assert rel(b.get_state(), a.get_state()) < 1e-10
    oa, ob = a.observables(), b.observables()
    for k in ("mass", "energy", "entropy_lin"):
        assert abs(getattr(ob, k) - getattr(oa, k)) < 1e-11 * max(1.0, abs(getattr(oa, k))), k


def test_sliced_and_fp64_pipe_paths_agree_over_1000_steps_logged_every_10():
    """The headline workload at its full length: 1000 steps of the 64^4
    double well with mass, energy and linear entropy logged every 10 steps
    (through the asynchronous read-back), the sliced path against the
    FP64-pipe path at every log point and in the final state."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell()
    a = w2.Context.from_problem(prob)
    b = _ctx(prob)
    d = _dev(f0)
    a.set_state(d)
    b.set_state(d)
    worst = 0.0
    for k in range(100):
        a.step(10)
        b.step(10)
        a.observables_enqueue(0)
        b.observables_enqueue(0)
        oa, ob = a.observables_collect(0), b.observables_collect(0)
        assert ob.step == oa.step == 10 * (k + 1)
        for name in ("mass", "energy", "entropy_lin"):
            dv = abs(getattr(ob, name) - getattr(oa, name)) / max(1.0, abs(getattr(oa, name)))
            worst = max(worst, dv)
    err = rel(b.get_state(), a.get_state())
    print(f"1000 steps: state rel L2 {err:.2e}, worst logged observable {worst:.2e}")
    assert err < 1e-11, err        # measured 1.8e-13
    assert worst < 1e-11, worst    # measured 3.6e-13
    a.close()
    b.close()


@pytest.mark.parametrize("nx,nk,steps", [(8, 16, 4), (5, 32, 3), (12, 48, 3), (64, 64, 5)])
def test_exchange_symmetric_sweep(nx, nk, steps):
    """w2_set_exchange_symmetry: on an exchange-symmetric state the sweeps
    over the blocks with i1 <= i2 plus their transposed mirrors give the
    steps of the full sweep to rounding (1e-13) and the oracle within 1e-10;
    the state stays symmetric; the other precisions refuse the mode."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell(nx=nx, nk=nk)
    assert np.array_equal(f0, f0.transpose(1, 0, 3, 2))
    full = _ctx(prob)
    sym = _ctx(prob)
    sym.set_exchange_symmetry(True)
    d = _dev(f0)
    full.set_state(d)
    sym.set_state(d)
    full.step(steps)
    sym.step(steps)
    a, b = full.get_state(), sym.get_state()
    assert rel(b, a) < 1e-13, rel(b, a)
    assert rel(b, oracle.Oracle(prob).step(f0, steps)) < 1e-10
    assert np.abs(b - b.transpose(1, 0, 3, 2)).max() < 1e-13 * np.abs(b).max()
    oa, ob = full.observables(), sym.observables()
    for k in ("mass", "energy", "entropy_lin"):
        assert abs(getattr(ob, k) - getattr(oa, k)) < 1e-13 * max(1.0, abs(getattr(oa, k))), k
    sym.set_exchange_symmetry(False)  # and back: the full sweep again
    sym.set_state(d)
    sym.step(steps)
    assert np.array_equal(sym.get_state(), a)
    full.close()
    sym.close()
    for p in (w2.W2_F64, w2.W2_F32_TF32X3):
        c = w2.Context.from_problem(prob, precision=p)
        with pytest.raises(w2.W2Error) as e:
            c.set_exchange_symmetry(True)
        assert e.value.name == "W2_ERR_UNSUPPORTED"
        c.close()


def test_sliced_determinism_and_resume():
    prob, f0 = inputs.workload_small(nx=16, nk=16)
    a = _ctx(prob)
    a.set_state(f0)
    a.step(12)
    b = _ctx(prob)
    b.set_state(f0)
    b.step(6)
    c = _ctx(prob)
    c.set_state(b.get_state())
    c.step(6)
    assert np.array_equal(c.get_state(), a.get_state())


# (precision, nk, operator bar, shift bar, step bar)
SMALLEST = [("W2_F64", 8, 1e-12, 1e-13, 1e-10), ("W2_F64_SLICED", 16, 2e-12, 1e-13, 1e-10),
            ("W2_F32_TF32X3", 16, 2e-6, 1e-6, 1e-6), ("W2_F32_BF16X3", 16, 2e-6, 1e-6, 1e-6)]


@pytest.mark.parametrize("nx", [4, 5])
@pytest.mark.parametrize("prec,nk,bar_theta,bar_adv,bar_step", SMALLEST)
def test_smallest_spatial_grids(nx, prec, nk, bar_theta, bar_adv, bar_step):
    """The smallest grids the API takes (nx = 4 and 5: periodic lines of four
    or five points, shorter than the spline start sums and split into
    recursion pieces of two or three points): operator, shift and three steps
    against the oracle on every element, for every precision."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=nx, nk=nk)
    ctx = w2.Context.from_problem(prob, precision=getattr(w2, prec))
    f = np.ascontiguousarray(f0, dtype=ctx.np_dtype)
    f64 = f.astype(np.float64)
    o = oracle.Oracle(prob)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.theta(d, out)
    assert rel(out.cpu().numpy().astype(np.float64), o.theta(f64)) < bar_theta
    ctx.advect(d, out)
    assert rel(out.cpu().numpy().astype(np.float64), o.advect(f64)) < bar_adv
    ctx.set_state(d)
    ctx.step(3)
    assert rel(ctx.get_state().astype(np.float64), o.step(f64, 3)) < bar_step


@pytest.mark.parametrize("prec", ["W2_F64_SLICED", "W2_F32_TF32X3", "W2_F32_BF16X3"])
def test_staged_host_input_pipeline(prec):
    """w2_stage_state / w2_use_staged_state: three host states streamed with
    the copy of the next one queued while the current one steps give the same
    bits as w2_set_state before each step; nothing staged is W2_ERR_STATE."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=16, nk=16)
    p = getattr(w2, prec)
    ref = w2.Context.from_problem(prob, precision=p)
    hosts = [torch.from_numpy(np.ascontiguousarray(f0 * (1.0 + 0.1 * k), dtype=ref.np_dtype)).pin_memory()
             for k in range(3)]
    want = []
    for h in hosts:
        ref.set_state(h.numpy())
        ref.step(2)
        want.append((ref.get_state(), ref.observables().energy))
    ctx = w2.Context.from_problem(prob, precision=p)
    with pytest.raises(w2.W2Error) as e:
        ctx.use_staged_state()
    assert e.value.name == "W2_ERR_STATE"
    ctx.stage_state(hosts[0])
    for k in range(3):
        ctx.use_staged_state()
        if k + 1 < 3:
            ctx.stage_state(hosts[k + 1])
        ctx.step(2)
        ob = ctx.observables()
        assert ob.step == 2
        assert np.array_equal(ctx.get_state(), want[k][0]) and ob.energy == want[k][1], k


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED", "W2_F32_TF32X3"])
def test_observables_enqueue_collect(prec):
    """The two-slot asynchronous observables (w2_observables_enqueue /
    _collect) give the bits of w2_observables for the state at enqueue time,
    with that step count, while later steps are queued; a slot that was not
    enqueued, or a slot other than 0 and 1, is refused."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell(nx=32, nk=32)
    ctx = w2.Context.from_problem(prob, precision=getattr(w2, prec))
    ctx.set_state(np.ascontiguousarray(f0, dtype=ctx.np_dtype))
    ctx.step(2)
    want2 = ctx.observables()
    ctx.observables_enqueue(0)
    ctx.step(1)
    want3 = ctx.observables()
    ctx.observables_enqueue(1)
    ctx.step(1)
    got2 = ctx.observables_collect(0)
    got3 = ctx.observables_collect(1)
    for got, want, n in ((got2, want2, 2), (got3, want3, 3)):
        assert got.step == want.step == n
        assert (got.mass, got.energy, got.purity, got.l2norm) == (want.mass, want.energy, want.purity, want.l2norm)
        assert np.array_equal(got.n1, want.n1) and np.array_equal(got.n12, want.n12)
    with pytest.raises(w2.W2Error) as e:
        ctx.observables_collect(0)
    assert e.value.name == "W2_ERR_STATE"
    with pytest.raises(w2.W2Error) as e:
        ctx.observables_enqueue(2)
    assert e.value.name == "W2_ERR_ARG"
    ctx.close()


def test_sliced_nonfinite_and_unsupported():
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=8, nk=16)
    ctx = _ctx(prob)
    bad = f0.copy()
    bad[1, 2, 3, 4] = np.inf
    out = torch.empty(*bad.shape, dtype=torch.float64, device="cuda")
    ctx.theta(_dev(bad), out)
    assert bool(torch.isnan(out[1, 2]).all())
    ctx.set_state(bad)
    assert ctx.observables().status == "W2_ERR_NONFINITE"
    for nk in (8, 24, 128):  # slices need nk in {16, 32, 48, 64}
        with pytest.raises(w2.W2Error) as e:
            w2.Context(8, nk, 1.0, 0.01, precision=w2.W2_F64_SLICED)
        assert e.value.name == "W2_ERR_UNSUPPORTED"


def test_sliced_learned_pair_term_matches_fp64_pipe():
    """The learned form's hook (a supplied two-body term) on the sliced path."""
    from paper_2511_11354_gb300 import learned, w2
    prob, f0 = inputs.workload_dwell(nx=16, nk=32)
    zero = learned.zero_network(prob.nk, hidden=32, max_rows=prob.nx * prob.nx)
    outs = []
    for prec in (w2.W2_F64, w2.W2_F64_SLICED):
        c = w2.Context.from_problem(prob, precision=prec)
        c.set_state(f0)
        c.attach_learned(zero, 0, 1e30)
        c.step(5)
        outs.append(c.get_state())
    assert rel(outs[1], outs[0]) < 1e-11

