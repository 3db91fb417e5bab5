"""Allocation failures, injected on the host (w2_debug_fail_alloc): every
allocation of each allocating call is made to fail in turn.  The call must
return W2_ERR_OOM, release what it had taken (the device's free memory comes
back), and leave the library usable: the same call succeeds afterwards and
its results equal those of an object that never saw a failure.  Nothing on
the device fails; the hook refuses the allocation before it is attempted."""
import gc

import numpy as np
import pytest

from paper_2511_11354_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

OOM = -3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11354_gb300 import build
    build.build()


@pytest.fixture(autouse=True)
def _disarm():
    from paper_2511_11354_gb300 import w2
    yield
    w2.debug_fail_alloc(-1)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _count(make):
    """Allocations one call of make() attempts (its object is released)."""
    from paper_2511_11354_gb300 import w2
    c0 = w2.debug_alloc_count()
    obj = make()
    n = w2.debug_alloc_count() - c0
    obj.close()
    return n


def _sweep(make, n):
    """Fail allocation k of make() for k = 0 .. n - 1: each raises W2_ERR_OOM."""
    from paper_2511_11354_gb300 import w2
    for k in range(n):
        w2.debug_fail_alloc(k)
        with pytest.raises(w2.W2Error) as e:
            obj = make()
            obj.close()
        assert e.value.code == OOM, (k, e.value)
        e = None  # the traceback holds the half-built object: let it go
        gc.collect()
    w2.debug_fail_alloc(-1)


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F32_TF32X3", "W2_F64_SLICED"])
def test_context_creation(prec):
    """w2_create and w2_set_potentials of the 64^2 x 32^2 double well (32 MB
    per FP64 state array): every allocation failed in turn; afterwards no
    memory is held and a new context steps exactly as one made before."""
    from paper_2511_11354_gb300 import w2
    p = getattr(w2, prec)
    prob, f0 = inputs.workload_dwell(nx=64, nk=32)

    def make():
        return w2.Context.from_problem(prob, precision=p)

    ref = make()
    ref.set_state(f0)
    ref.step(2)
    want = ref.get_state()
    ref.close()
    n = _count(make)
    assert n >= 10
    free0 = _free_bytes()
    _sweep(make, n)
    assert _free_bytes() >= free0 - (16 << 20)
    ctx = make()
    ctx.set_state(f0)
    ctx.step(2)
    np.testing.assert_array_equal(ctx.get_state(), want)
    ctx.close()


def test_context_buffers_taken_later():
    """Buffers a context takes on first use: the patch tables (w2_set_patches),
    the staging buffer (w2_stage_state) and the density-matrix scratch
    (w2_occupations).  A failed call leaves the context as it was; the retry
    gives the results of a context that never failed."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell(nx=64, nk=16)
    ref = w2.Context.from_problem(prob, precision=w2.W2_F64)
    ref.set_state(f0)
    occ_ref, s_ref = ref.occupations()
    ref.set_patches(2, 2)
    ref.step(2)
    want = ref.get_state()
    ref.close()

    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
    ctx.set_state(f0)
    c0 = w2.debug_alloc_count()
    ctx.occupations()
    n_occ = w2.debug_alloc_count() - c0
    ctx.close()
    for k in range(n_occ):
        ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
        ctx.set_state(f0)
        w2.debug_fail_alloc(k)
        with pytest.raises(w2.W2Error) as e:
            ctx.occupations()
        assert e.value.code == OOM
        occ, s = ctx.occupations()
        np.testing.assert_allclose(occ, occ_ref, rtol=0, atol=1e-13)
        assert abs(s - s_ref) < 1e-12
        ctx.close()

    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
    ctx.set_state(f0)
    c0 = w2.debug_alloc_count()
    ctx.set_patches(2, 2)
    n_pm = w2.debug_alloc_count() - c0
    ctx.close()
    assert n_pm >= 5
    for k in range(n_pm):
        ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
        ctx.set_state(f0)
        w2.debug_fail_alloc(k)
        with pytest.raises(w2.W2Error) as e:
            ctx.set_patches(2, 2)
        assert e.value.code == OOM
        ctx.set_patches(2, 2)
        ctx.step(2)
        np.testing.assert_array_equal(ctx.get_state(), want)
        ctx.close()

    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64)
    w2.debug_fail_alloc(0)
    with pytest.raises(w2.W2Error) as e:
        ctx.stage_state(f0)
    assert e.value.code == OOM
    ctx.stage_state(f0)
    ctx.use_staged_state()
    ctx.set_patches(2, 2)
    ctx.step(2)
    np.testing.assert_array_equal(ctx.get_state(), want)
    ctx.close()


def test_batch_creation():
    """w2_batch_create of two 32^2 x 16^2 instances (each instance's context,
    the plan and its pinned error word): every allocation failed in turn."""
    from paper_2511_11354_gb300 import w2
    probs = [inputs.workload_small(nx=32, nk=16)[0] for _ in range(2)]

    def make():
        return w2.Batch(probs)

    n = _count(make)
    assert n >= 20
    free0 = _free_bytes()
    _sweep(make, n)
    assert _free_bytes() >= free0 - (4 << 20)
    b = make()
    b.close()


def test_network_creation_and_first_training_step():
    """w2_mlp_create (both kinds) and the scratch of a kernel network's first
    training step: each allocation failed in turn; the retried step returns
    the loss of a network that never failed."""
    from paper_2511_11354_gb300 import w2
    for kind in ("pair", "kernel"):
        def make():
            return w2.MLP(16, hidden=64, max_rows=32, kind=kind)
        n = _count(make)
        assert n >= 10
        _sweep(make, n)

    prob, f0 = inputs.workload_dwell(nx=16, nk=16)
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    rng = np.random.default_rng(1)
    rows = 8
    F = torch.from_numpy(rng.standard_normal((rows, 256))).cuda()
    P = torch.from_numpy(rng.standard_normal((rows, 256))).cuda()
    D = torch.from_numpy(rng.integers(0, 16, rows).astype(np.int32)).cuda()
    ref = w2.MLP(16, hidden=64, max_rows=16, kind="kernel")
    params = ref.get_params()
    c0 = w2.debug_alloc_count()
    want = ref.kernel_train_step(ctx, F, P, D, 1e-3)
    n = w2.debug_alloc_count() - c0
    ref.close()
    assert n >= 6
    for k in range(n):
        m = w2.MLP(16, hidden=64, max_rows=16, kind="kernel")
        m.set_params(params)
        w2.debug_fail_alloc(k)
        with pytest.raises(w2.W2Error) as e:
            m.kernel_train_step(ctx, F, P, D, 1e-3)
        assert e.value.code == OOM
        assert m.kernel_train_step(ctx, F, P, D, 1e-3) == want
        m.close()
    ctx.close()


def test_sem_context_creation():
    """w2_sem_create and its potentials on a 17^2 x 12^2 correlated problem."""
    from paper_2511_11354_gb300 import w2
    prob, _ = inputs.workload_correlated("IV", nx=17, ncell=2, nq=6, L=12.0)

    def make():
        return w2.SemContext.from_problem(prob, precision=w2.W2_F64)

    n = _count(make)
    assert n >= 5
    _sweep(make, n)
    make().close()


def test_disarmed_hook_and_counter():
    """n < 0 disarms: nothing fails; the counter counts every attempt."""
    from paper_2511_11354_gb300 import w2
    w2.debug_fail_alloc(3)
    w2.debug_fail_alloc(-1)
    prob, _ = inputs.workload_small(nx=32, nk=16)
    c0 = w2.debug_alloc_count()
    ctx = w2.Context.from_problem(prob)
    assert w2.debug_alloc_count() > c0
    ctx.close()
