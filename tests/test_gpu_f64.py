"""GPU parity of the FP64 CUDA path against the FP64 oracle (through the C ABI).

Bars: the pseudo-difference operator and the spline shift alone agree to
1e-12 relative L2 (they differ from the oracle only by the order of FP64
rounding); whole time steps agree to <= 1e-10 relative L2, the FP64 bar for
the plain path.
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
    return w2.Context.from_problem(prob)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [(8, 8), (12, 24), (20, 16), (32, 32), (24, 48), (16, 64), (36, 40)]


@pytest.mark.parametrize("nx,nk", SHAPES)
def test_theta_parity(nx, nk):
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=11, noise=0.05)
    ctx = _ctx(prob)
    out = torch.empty(prob.nx, prob.nx, prob.nk, prob.nk, dtype=torch.float64, device="cuda")
    ctx.theta(_dev(f), out)
    ref = oracle.Oracle(prob).theta(f)
    assert rel(out.cpu().numpy(), ref) < 1e-12


def test_theta_parity_xc_and_hartree():
    prob, f = inputs.workload_small(nx=16, nk=24)
    prob.c_xc, prob.xc_kind = -0.7, 2
    ctx = _ctx(prob)
    out = torch.empty(*f.shape, dtype=torch.float64, device="cuda")
    ctx.theta(_dev(f), out)
    assert rel(out.cpu().numpy(), oracle.Oracle(prob).theta(f)) < 1e-12


@pytest.mark.parametrize("nx,nk", [(8, 8), (12, 24), (33, 16), (64, 32)])
def test_advect_parity(nx, nk):
    prob, _ = inputs.workload_small(nx=nx, nk=nk)
    prob.dt = 0.37  # shifts of several cells (no potential: the shift alone)
    prob.vext, prob.vee, prob.gamma, prob.c_hartree = inputs.zero_potential(), inputs.zero_potential(), 0.0, 0.0
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=5, noise=0.1)
    ctx = _ctx(prob)
    out = torch.empty(*f.shape, dtype=torch.float64, device="cuda")
    ctx.advect(_dev(f), out)
    assert rel(out.cpu().numpy(), oracle.Oracle(prob).advect(f)) < 1e-13


def test_step_parity_small_workload():
    """32^4, L=20, cosine well, soft-Coulomb pair, Hartree on: 20 steps."""
    prob, f0 = inputs.workload_small()
    ctx = _ctx(prob)
    ctx.set_state(f0)
    ctx.step(20)
    got = ctx.get_state()
    ref = oracle.Oracle(prob).step(f0, 20)
    assert rel(got, ref) < 1e-10


@pytest.mark.parametrize("nx,nk,steps", [(16, 16, 10), (20, 24, 5), (40, 8, 3)])
def test_step_parity_dwell_shapes(nx, nk, steps):
    prob, f0 = inputs.workload_dwell(nx=nx, nk=nk)
    ctx = _ctx(prob)
    ctx.set_state(_dev(f0))
    ctx.step(steps)
    assert rel(ctx.get_state(), oracle.Oracle(prob).step(f0, steps)) < 1e-10


def test_step_parity_full_size_workload():
    """64^4 double well (the benchmark workload), 2 steps, full comparison."""
    prob, f0 = inputs.workload_dwell()
    ctx = _ctx(prob)
    ctx.set_state(_dev(f0))
    ctx.step(2)
    got = ctx.get_state()
    ref = oracle.Oracle(prob).step(f0, 2)
    assert rel(got, ref) < 1e-10
    # exchange symmetry is kept to rounding
    assert np.abs(got - got.transpose(1, 0, 3, 2)).max() < 1e-13 * np.abs(got).max()


@pytest.mark.parametrize("nx,nk", [(32, 32), (24, 64)])
def test_observables_parity(nx, nk):
    prob, f0 = inputs.workload_small(nx=nx, nk=nk)
    ctx = _ctx(prob)
    ctx.set_state(f0)
    ctx.step(3)
    f = ctx.get_state()
    ob = ctx.observables()
    ref = oracle.Oracle(prob).observables(f)
    for k in ("mass", "energy", "purity", "entropy_lin", "l2norm"):
        assert abs(getattr(ob, k) - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    np.testing.assert_allclose(ob.n1, ref["n1"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(ob.n12, ref["n12"], rtol=0, atol=1e-13)
    assert ob.step == 3 and ob.status == "W2_OK"


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
def test_observables_wide_range_state_64(prec):
    """The 64-point reduction (warp butterfly for the row sums) on a state of
    both signs spanning ten decades per block, against the oracle; a NaN in
    one block gives W2_ERR_NONFINITE with the outputs still written."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=12, nk=64)
    rng = np.random.default_rng(8)
    f = f0 * np.exp(rng.uniform(-11.5, 11.5, f0.shape)) * np.sign(rng.standard_normal(f0.shape))
    ctx = w2.Context.from_problem(prob, precision=getattr(w2, prec))
    ctx.set_state(f)
    ob = ctx.observables()
    ref = oracle.Oracle(prob).observables(f)
    for k in ("mass", "energy", "purity", "l2norm"):
        assert abs(getattr(ob, k) - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    np.testing.assert_allclose(ob.n1, ref["n1"], rtol=1e-12, atol=1e-13 * np.abs(ref["n1"]).max())
    assert ctx.observables().mass == ob.mass  # deterministic
    g = f.copy()
    g[3, 7, 40, 2] = np.nan
    ctx.set_state(g)
    bad = ctx.observables()
    assert bad.status == "W2_ERR_NONFINITE" and np.isnan(bad.mass)
    with pytest.raises(w2.W2Error) as e:
        ctx.observables(raise_nonfinite=True)
    assert e.value.code == -6


def test_checkpoint_resume_bitwise_and_determinism():
    prob, f0 = inputs.workload_small(nx=16, nk=16)
    a = _ctx(prob)
    a.set_state(f0)
    a.step(20)
    fa = a.get_state()
    b = _ctx(prob)
    b.set_state(f0)
    b.step(10)
    mid = b.get_state()
    c = _ctx(prob)
    c.set_state(mid)
    c.step(10)
    assert np.array_equal(c.get_state(), fa)
    a2 = _ctx(prob)
    a2.set_state(f0)
    a2.step(20)
    assert np.array_equal(a2.get_state(), fa)
    assert a.observables().energy == a2.observables().energy


def test_error_paths():
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=8, nk=8)
    ctx = w2.Context(prob.nx, prob.nk, prob.L, prob.dt)
    with pytest.raises(w2.W2Error) as e:
        ctx.step(1)
    assert e.value.name == "W2_ERR_STATE"
    with pytest.raises(w2.W2Error) as e:
        ctx.set_state(f0)
    assert e.value.name == "W2_ERR_STATE"
    # literal (uncapped) double well: refused by the stability precheck
    pl, _ = inputs.workload_dwell(nx=16, nk=16, literal=True)
    c2 = w2.Context(pl.nx, pl.nk, pl.L, pl.dt)
    with pytest.raises(w2.W2Error) as e:
        c2.set_potentials(pl.vext, pl.vee, pl.gamma, pl.c_hartree)
    assert e.value.name == "W2_ERR_UNSTABLE"
    # NaN planted in the host state is reported by the observables
    ctx.set_potentials(prob.vext, prob.vee, prob.gamma, prob.c_hartree)
    bad = f0.copy()
    bad[1, 2, 3, 4] = np.nan
    ctx.set_state(bad)
    assert ctx.observables().status == "W2_ERR_NONFINITE"
    with pytest.raises(w2.W2Error):
        w2.Context(8, 7, 1.0, 0.01)
