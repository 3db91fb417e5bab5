"""GPU parity of the tcgen05 sliced sweep (k_theta_t: every 8-bit digit
product of the pseudo-difference operator on tcgen05.mma with the
accumulators in tensor memory, N_k = 64) against the FP64 oracle and against
the warp-level mma.sync sweep of the same slices.

Bars: the operator within 2e-12 relative L2 of the oracle (the bar of the
sliced path); the two tensor-core paths within 1e-13 of each other (they
differ only in the rounding of the lowest slice diagonal, below 2^-50 of each
block's scale); whole steps within 1e-10 of the oracle.  The smallest grid
runs first, so a wrong layout shows there before any large launch.
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


def _ctx(prob, tcgen05=True):
    """A sliced context on the tcgen05 path (tcgen05=False: the mma.sync path)."""
    from paper_2511_11354_gb300 import w2
    c = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    c.set_tensor_path(tcgen05)
    return c


def _both(prob, f):
    """The operator on f through the tcgen05 path and the mma.sync path."""
    ctx = _ctx(prob)
    d = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    outs = []
    for tc in (True, False):
        ctx.set_tensor_path(tc)
        o = torch.empty_like(d)
        ctx.theta(d, o)
        outs.append(o.cpu().numpy())
    ctx.close()
    return outs


def test_smallest_grid_first():
    prob, _ = inputs.workload_small(nx=4, nk=64)
    f = inputs.initial_state(prob, centres=(-2.5, 3.0), seed=11, noise=0.05)
    t, s = _both(prob, f)
    assert np.all(np.isfinite(t))
    assert rel(t, oracle.Oracle(prob).theta(f)) < 2e-12
    assert rel(t, s) < 1e-13


@pytest.mark.parametrize("nx", [5, 7, 16, 33])
def test_theta_wide_range_both_signs(nx):
    """H-L exchange-correlation and Hartree on, a state of both signs whose
    magnitudes span six decades inside each block."""
    prob, f = inputs.workload_small(nx=nx, nk=64)
    prob.c_xc, prob.xc_kind = -0.7, 2
    rng = np.random.default_rng(nx)
    f = f * np.exp(rng.uniform(-7, 7, f.shape)) * np.sign(rng.standard_normal(f.shape))
    t, s = _both(prob, f)
    assert rel(t, oracle.Oracle(prob).theta(f)) < 2e-12
    assert rel(t, s) < 1e-13


def test_nonfinite_block():
    """A NaN in one block makes that whole block NaN (the block exponent sees
    it); the two paths agree on which outputs are NaN and on the rest."""
    prob, f = inputs.workload_small(nx=8, nk=64)
    prob.c_hartree = 0.0
    f = f.copy()
    f[2, 5, 10, 20] = np.nan
    t, s = _both(prob, f)
    assert np.all(np.isnan(t[2, 5]))
    assert np.array_equal(np.isnan(t), np.isnan(s))
    ok = ~np.isnan(t)
    if ok.any():
        assert rel(t[ok], s[ok]) < 1e-13


def test_full_size_steps_tcgen05_against_mma_sync():
    """20 steps of the 64^4 double-well workload on each path."""
    prob, f0 = inputs.workload_dwell()
    runs = []
    for tc in (True, False):
        c = _ctx(prob, tc)
        c.set_state(f0)
        c.step(20)
        runs.append((c.get_state(), c.observables()))
        c.close()
    (a, oa), (b, ob) = runs
    assert rel(a, b) < 1e-12
    assert abs(oa.mass - ob.mass) < 1e-13 * abs(ob.mass)
    assert abs(oa.energy - ob.energy) < 1e-12 * abs(ob.energy)


def test_exchange_symmetric_tcgen05():
    prob, f0 = inputs.workload_dwell(nx=12, nk=64)
    outs = []
    for sym in (False, True):
        c = _ctx(prob)
        c.set_exchange_symmetry(sym)
        c.set_state(f0)
        c.step(3)
        outs.append(c.get_state())
        c.close()
    assert rel(outs[1], outs[0]) < 1e-13
    assert rel(outs[0], oracle.Oracle(prob).step(f0, 3)) < 1e-10


def test_timeout_is_reported_and_recovered():
    """Host-requested stall: the sweep leaves one batch of products and its
    completion signal out, its next bounded wait (2e5 clocks) runs out, the
    blocks turn NaN and w2_observables reports W2_ERR_TIMEOUT; after the
    stall is lifted the context steps as a fresh one."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=8, nk=64)
    ref = _ctx(prob)
    ref.set_state(f0)
    ref.step(2)
    want = ref.get_state()
    ref.close()
    c = _ctx(prob)
    c.set_state(f0)
    c.debug_sweep_stall(True, 200000)
    c.step(1)
    with pytest.raises(w2.W2Error) as e:
        c.observables()
    assert e.value.code == -7
    assert np.isnan(c.get_state()).any()
    c.debug_sweep_stall(False)
    c.set_state(f0)
    c.step(2)
    c.observables()
    np.testing.assert_array_equal(c.get_state(), want)
    c.close()


@pytest.mark.parametrize("sym", [False, True])
def test_full_size_steps_against_the_oracle(sym):
    """The 64^4 double-well workload, 2 steps on the tcgen05 path (persistent
    CTAs over runs of 27 blocks; with exchange symmetry over the 2080 blocks
    i1 <= i2), every element against the oracle."""
    prob, f0 = inputs.workload_dwell()
    c = _ctx(prob)
    c.set_exchange_symmetry(sym)
    c.set_state(f0)
    c.step(2)
    got = c.get_state()
    c.close()
    assert rel(got, oracle.Oracle(prob).step(f0, 2)) < 1e-10
    assert np.abs(got - got.transpose(1, 0, 3, 2)).max() < 1e-13 * np.abs(got).max()


@pytest.mark.parametrize("nx", [5, 13, 33])
def test_steps_on_ragged_grids(nx):
    """Whole steps where the blocks do not divide evenly over the CTAs (the
    last CTA's run is shorter) and the A1 matrices change inside a run."""
    prob, f0 = inputs.workload_small(nx=nx, nk=64)
    c = _ctx(prob)
    c.set_state(f0)
    c.step(3)
    got = c.get_state()
    c.close()
    assert rel(got, oracle.Oracle(prob).step(f0, 3)) < 1e-10


def test_setter_errors():
    """w2_set_tensor_path: W2_ERR_ARG for a value other than 0 or 1,
    W2_ERR_UNSUPPORTED for tcgen05 = 1 outside W2_F64_SLICED; tcgen05 = 1 at
    an nk the tcgen05 sweep does not take runs the mma.sync sweep (the same
    operator).  w2_debug_sweep_stall: W2_ERR_ARG for a bad flag or a negative
    wait."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=8, nk=32)
    c = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    lib = w2.load()
    assert lib.w2_set_tensor_path(c.h, 2) == -1
    assert lib.w2_debug_sweep_stall(c.h, 2, 0) == -1
    assert lib.w2_debug_sweep_stall(c.h, 1, -5) == -1
    c.set_tensor_path(True)
    c.set_state(f0)
    c.step(2)
    assert rel(c.get_state(), oracle.Oracle(prob).step(f0, 2)) < 1e-10
    c.close()
    p = w2.Context.from_problem(prob, precision=w2.W2_F64)
    assert lib.w2_set_tensor_path(p.h, 1) == -8
    assert lib.w2_set_tensor_path(p.h, 0) == 0
    p.close()
