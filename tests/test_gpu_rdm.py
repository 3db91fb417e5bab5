"""GPU checks of the occupation numbers and the correlation entropy: the
batched Jacobi eigensolver against numpy's Hermitian eigensolver, and the
device reconstruction rho1 -> occupations -> entropy against the numpy
reference (oracle/rdm_ref.py) on the same state."""
import math

import numpy as np
import pytest

from oracle import rdm_ref
from paper_2511_11354_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11354_gb300 import build
    build.build()


@pytest.mark.parametrize("n,batch", [(1, 2), (2, 3), (5, 3), (16, 4), (64, 2), (97, 1), (201, 2), (320, 1),
                                     (321, 1)])
def test_batched_hermitian_eigvals(n, batch):
    """Householder tridiagonal reduction + bisection up to n = 320 (the rows
    in the shared memory of a cluster of 8 CTAs), cyclic Jacobi beyond."""
    from paper_2511_11354_gb300 import w2
    rng = np.random.default_rng(n)
    b = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    h = b + np.conj(np.transpose(b, (0, 2, 1)))
    a = torch.from_numpy(h.copy()).cuda()
    eig = w2.hermitian_eigvals(a).cpu().numpy()
    for k in range(batch):
        want = np.sort(np.linalg.eigvalsh(h[k]))[::-1]
        assert np.abs(eig[k] - want).max() < 1e-12 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("kind", ["diagonal", "scaled_identity", "zero", "graded", "block"])
def test_hermitian_eigvals_structured(kind):
    """Matrices where reflections are skipped (a zero column below the
    diagonal), every eigenvalue is the same, or the spectrum spans 30
    decades like the occupations of a nearly pure state (absolute bar)."""
    from paper_2511_11354_gb300 import w2
    n = 57
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    if kind == "diagonal":
        want = rng.standard_normal(n)
        h = np.diag(want).astype(np.complex128)
    elif kind == "scaled_identity":
        want = np.full(n, 3.0)
        h = 3.0 * np.eye(n, dtype=np.complex128)
    elif kind == "zero":
        want = np.zeros(n)
        h = np.zeros((n, n), dtype=np.complex128)
    elif kind == "graded":
        want = 10.0 ** -np.linspace(0, 30, n)
        h = (q * want) @ q.conj().T
    else:  # two decoupled Hermitian blocks
        b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        b[:20, 20:] = 0
        b[20:, :20] = 0
        h = b + b.conj().T
        want = np.linalg.eigvalsh(h)
    h = 0.5 * (h + h.conj().T)
    eig = w2.hermitian_eigvals(torch.from_numpy(h[None].copy()).cuda()).cpu().numpy()[0]
    want = np.sort(want)[::-1]
    assert np.all(np.diff(eig) <= 1e-15 * max(1.0, np.abs(want).max()))
    assert np.abs(eig - want).max() <= 1e-13 * max(1.0, np.abs(want).max())


def _reference(prob, f):
    f1 = rdm_ref.f1_from_state(np.asarray(f, dtype=np.float64), prob.dx, prob.dp)
    occ = rdm_ref.occupations(rdm_ref.rho1_from_f1(f1, prob.nx, prob.nk, prob.dp), prob.dx)
    return occ, rdm_ref.correlation_entropy(occ)


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED", "W2_F32_TF32X3"])
def test_occupations_of_an_evolved_state(prec):
    """The small workload after 10 steps (a correlated state): occupations
    and entropy from the device against the reference on the same state."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_small(nx=32, nk=32)
    p = getattr(w2, prec)
    ctx = w2.Context.from_problem(prob, precision=p)
    ctx.set_state(f0.astype(ctx.np_dtype))
    ctx.step(10)
    occ, s = ctx.occupations()
    ref_occ, ref_s = _reference(prob, ctx.get_state())
    assert np.abs(occ - ref_occ).max() < 1e-11 * ref_occ[0]
    assert abs(s - ref_s) < 1e-10 * max(1.0, abs(ref_s))
    assert abs(occ.sum() - ctx.observables().mass) < 1e-10 * occ.sum()


def test_occupations_of_a_product_of_pure_states():
    """f = W_a(x1, p1) W_b(x2, p2) with pure Gaussian packets: particle 1 is
    in a pure state, one occupation equal to its mass, the rest ~0, entropy
    ~0 (box large enough that the periodic images are negligible)."""
    from paper_2511_11354_gb300 import w2
    prob = inputs.Problem(nx=64, nk=64, L=30.0, dt=0.01, vext=inputs.zero_potential(), vee=inputs.zero_potential(),
                          gamma=0.0, c_hartree=0.0)
    x, p = prob.x(), prob.p()

    def wig(x0, p0, s):
        return np.exp(-(x[:, None] - x0) ** 2 / (2 * s * s) - 2 * s * s * (p[None, :] - p0) ** 2) / math.pi

    wa, wb = wig(-2.0, 0.5, 1.3), wig(3.0, -0.4, 1.1)
    f = np.ascontiguousarray(wa[:, None, :, None] * wb[None, :, None, :])
    ctx = w2.Context.from_problem(prob)
    ctx.set_state(f)
    occ, s = ctx.occupations()
    mass_b = wb.sum() * prob.dx * prob.dp
    assert abs(occ[0] - mass_b) < 1e-8 * mass_b and np.abs(occ[1:]).max() < 1e-8
    # eigenvalues at the 1e-8 level of the discretisation each add
    # lam ln lam ~ -2e-7 to the entropy
    assert abs(s - math.log(mass_b)) < 2e-6
