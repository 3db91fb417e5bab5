"""GPU checks of the batching form: a batch of uneven problems advanced by the
one persistent graph-captured launch per step gives, bit for bit, what each
problem gives in its own precision-form context, before and after autotuning
of its tile shapes; it stays within the precision form's tolerance of the FP64
oracle (an instance of every momentum size of the workload, nk = 64
included); and a wait that runs out (injected on the host) is reported as
W2_ERR_TIMEOUT without harming the CUDA context."""
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


def test_batch_matches_single_contexts_bitwise():
    from paper_2511_11354_gb300 import w2
    probs, states = inputs.workload_batch(n=7, seed=5)
    # make sure several momentum sizes and grid sizes are present
    assert len({p.nk for p in probs}) >= 2 and len({p.nx for p in probs}) >= 2
    b = w2.Batch(probs)
    for i, f in enumerate(states):
        b.set_state(i, f.astype(np.float32))
    b.step(6)
    got = [b.get_state(i) for i in range(len(probs))]
    for i, p in enumerate(probs):
        c = w2.Context.from_problem(p, precision=w2.W2_F32_TF32X3)
        c.set_state(states[i].astype(np.float32))
        c.step(6)
        assert np.array_equal(got[i], c.get_state()), i
        c.close()
    tuning = b.autotune()
    assert tuning["grid"] > 0 and tuning["shapes_tried"] >= 2 and tuning["shift_cols"] in (32, 64)
    assert tuning["theta_split"] in (1, 2)
    # the states were restored: stepping on continues from step 6
    after = [b.get_state(i) for i in range(len(probs))]
    for i in range(len(probs)):
        assert np.array_equal(after[i], got[i]), i
    b2 = w2.Batch(probs)
    for i, f in enumerate(states):
        b2.set_state(i, f.astype(np.float32))
    b2.autotune()
    b2.step(6)
    for i in range(len(probs)):
        assert np.array_equal(b2.get_state(i), got[i]), i
    ob = b2.observables(0)
    assert ob.step == 6 and ob.status == "W2_OK"


def test_batch_with_128_point_lines():
    """The batch's largest lines (nx = 128, eight recursion pieces per line)
    beside a small instance: the shift slabs of 64 columns would need 512
    threads, so the batch takes 32-column slabs (the autotuner only tries
    shapes that fit) and still matches single contexts bit for bit."""
    from paper_2511_11354_gb300 import w2
    probs = [inputs.Problem(nx=128, nk=64, L=20.0, dt=0.01, vext=inputs.cos_potential(0.5, 20.0),
                            vee=inputs.soft_coulomb(1.0), gamma=1.0),
             inputs.Problem(nx=24, nk=32, L=20.0, dt=0.01, vext=inputs.cos_potential(0.5, 20.0),
                            vee=inputs.soft_coulomb(1.0), gamma=0.5)]
    states = [inputs.initial_state(q, centres=(-2.0, 2.5), seed=i) for i, q in enumerate(probs)]
    b = w2.Batch(probs)
    for i, f in enumerate(states):
        b.set_state(i, f.astype(np.float32))
    b.step(2)
    tuning = b.autotune()
    assert tuning["shift_cols"] == 32
    b.step(1)
    for i, q in enumerate(probs):
        c = w2.Context.from_problem(q, precision=w2.W2_F32_TF32X3)
        c.set_state(states[i].astype(np.float32))
        c.step(3)
        assert np.array_equal(b.get_state(i), c.get_state()), i
        c.close()
    b.close()


def test_batch_instance_vs_oracle():
    """Instances of each momentum size of the workload (32, 48, 64) and of
    uneven spatial sizes, 10 steps, each against the FP64 oracle."""
    from paper_2511_11354_gb300 import w2
    probs, _ = inputs.workload_batch(n=3, seed=9)
    shapes = [(16, 32), (24, 48), (16, 64)]
    small = []
    for p, (nx, nk) in zip(probs, shapes):
        small.append(inputs.Problem(nx=nx, nk=nk, L=p.L, dt=p.dt, vext=p.vext, vee=p.vee, gamma=p.gamma,
                                    c_hartree=p.c_hartree))
    fs = [inputs.initial_state(q, centres=inputs.draw_centres(i), seed=i) for i, q in enumerate(small)]
    b = w2.Batch(small)
    for i, f in enumerate(fs):
        b.set_state(i, f.astype(np.float32))
    b.step(10)
    for i, q in enumerate(small):
        ref = oracle.Oracle(q).step(fs[i], 10)
        got = b.get_state(i).astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6, (i, q.nx, q.nk)


@pytest.mark.parametrize("phase", [0, 2, 4])
def test_batch_wait_timeout_is_reported(phase):
    """Failure detection without a GPU fault: the host stops the counting of
    one phase of one instance, the next phase's items wait until their limit
    (0.2 s), the launch ends and the batch reports W2_ERR_TIMEOUT; the CUDA
    context stays usable (a fresh batch steps and matches a single context)."""
    from paper_2511_11354_gb300 import w2
    probs, states = inputs.workload_batch(n=2, seed=5)
    probs = [inputs.Problem(nx=8, nk=16, L=p.L, dt=p.dt, vext=p.vext, vee=p.vee, gamma=p.gamma) for p in probs]
    fs = [inputs.initial_state(q, centres=(-2.0, 2.0), seed=i) for i, q in enumerate(probs)]
    b = w2.Batch(probs)
    for i, f in enumerate(fs):
        b.set_state(i, f.astype(np.float32))
    b.set_wait_limit(0.2)
    b.step(1)
    assert b.sync() == 0
    b.inject_stall(phase, 1)
    b.step(1)
    assert w2.STATUS[b.sync()] == "W2_ERR_TIMEOUT"
    with pytest.raises(w2.W2Error):
        b.get_state(0)
    b.close()
    torch.cuda.synchronize()
    c = w2.Batch(probs)
    for i, f in enumerate(fs):
        c.set_state(i, f.astype(np.float32))
    c.step(2)
    assert c.sync() == 0
    s = w2.Context.from_problem(probs[1], precision=w2.W2_F32_TF32X3)
    s.set_state(fs[1].astype(np.float32))
    s.step(2)
    assert np.array_equal(c.get_state(1), s.get_state())
    c.close()
    s.close()
