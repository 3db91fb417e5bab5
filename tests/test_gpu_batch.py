"""GPU checks of the batching form: a batch of uneven problems advanced by the
persistent graph-captured kernels gives, bit for bit, what each problem gives
in its own precision-form context, before and after autotuning; and it stays
within the precision form's tolerance of the FP64 oracle."""
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
    assert tuning["xsum"] > 0 and len(tuning["classes"]) == len({p.nk for p in probs})
    b2 = w2.Batch(probs)
    for i, f in enumerate(states):
        b2.set_state(i, f.astype(np.float32))
    b2.autotune()
    b2.step(6)
    for i in range(len(probs)):
        assert np.array_equal(b2.get_state(i), got[i]), i
    ob = b2.observables(0)
    assert ob.step == 6 and ob.status == "W2_OK"


def test_batch_instance_vs_oracle():
    from paper_2511_11354_gb300 import w2
    probs, states = inputs.workload_batch(n=3, seed=9)
    small = []
    for p in probs:  # shrink to oracle-friendly sizes, keeping uneven shapes
        q = inputs.Problem(nx=16 if p.nx < 48 else 24, nk=32 if p.nk < 64 else 48, L=p.L, dt=p.dt, vext=p.vext,
                           vee=p.vee, gamma=p.gamma, c_hartree=p.c_hartree)
        small.append(q)
    fs = [inputs.initial_state(q, centres=inputs.draw_centres(i), seed=i) for i, q in enumerate(small)]
    b = w2.Batch(small)
    for i, f in enumerate(fs):
        b.set_state(i, f.astype(np.float32))
    b.step(10)
    for i, q in enumerate(small):
        ref = oracle.Oracle(q).step(fs[i], 10)
        got = b.get_state(i).astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6, i
