"""GPU parity of the non-periodic path (Chebyshev spectral elements in
momentum, natural-boundary spline in position, Sec. 3.2 and 4.1) against the
numpy oracle, through the C ABI (include/w2_sem.h).

Sizes span several 64-wide product tiles and ragged tails (odd and even nx,
nq not a power of two, np not a multiple of the tile); the last case is the
strongly correlated example's mesh (201^2 x 128^2) checked on sampled
spatial points, where the two-body chain runs in many chunks of X with a
ragged last chunk.  Bars: operator 1e-12, shift 1e-13, steps 1e-10
(relative L2), observables 1e-12.
"""
import math

import numpy as np
import pytest

from oracle import SemOracle
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


def _perturbed(f, seed=2):
    rng = np.random.default_rng(seed)
    g = f * (1.0 + 0.1 * rng.standard_normal(f.shape))
    return np.ascontiguousarray(0.5 * (g + g.transpose(1, 0, 3, 2)))


# (nx, ncell, nq, L, hamiltonian)
CASES = [(17, 2, 6, 12.0, "IV"), (20, 3, 5, 10.0, "III"), (33, 4, 16, 14.0, "IV"), (25, 1, 32, 16.0, "II")]


def _case(nx, ncell, nq, L, ham, soft=1.0):
    prob, f = inputs.workload_correlated(ham, soft=soft, nx=nx, ncell=ncell, nq=nq, L=L)
    return prob, _perturbed(f)


def _ctx(prob, prec="W2_F64"):
    from paper_2511_11354_gb300 import w2
    return w2.SemContext.from_problem(prob, precision=getattr(w2, prec))


# operator bars: FP64 pipe, and the tensor-core products from 47-bit slices
# (each product of the chain rounds near 2^-47 of its line scales; measured
# at the level of the FP64 pipe, about 1e-13)
THETA_BAR = {"W2_F64": 1e-12, "W2_F64_SLICED": 1e-12}


def test_momenta_and_weights():
    prob, _ = _case(17, 3, 7, 12.0, "I")
    p, w = _ctx(prob).momenta()
    o = SemOracle(prob)
    np.testing.assert_allclose(p, o.p, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, o.w, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
@pytest.mark.parametrize("case", CASES)
def test_theta_parity(case, prec):
    prob, f = _case(*case)
    ctx = _ctx(prob, prec)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.theta(d, out)
    err = rel(out.cpu().numpy(), SemOracle(prob).theta(f))
    print(f"theta {case} {prec}: {err:.3e}")
    assert err < THETA_BAR[prec]


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
@pytest.mark.parametrize("which", ["one_body", "two_body"])
def test_theta_terms_separately(which, prec):
    prob, f = _case(21, 2, 8, 12.0, "IV", soft=0.01)
    if which == "one_body":
        prob.gamma = 0.0
    else:
        prob.c_hartree, prob.c_xc, prob.vext = 0.0, 0.0, inputs.zero_potential()
    ctx = _ctx(prob, prec)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.theta(d, out)
    err = rel(out.cpu().numpy(), SemOracle(prob).theta(f))
    print(f"theta {which} {prec}: {err:.3e}")
    assert err < THETA_BAR[prec]


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
@pytest.mark.parametrize("case", CASES[:3] + [(101, 2, 4, 30.0, "IV"), (151, 2, 4, 30.0, "IV"),
                                   (201, 2, 4, 30.0, "IV")])
def test_advect_parity(case, prec):
    """The FP64-pipe context shifts in FP64, the sliced one in double-float
    pairs (about 2^-47 per operation); at 101, 151 and 201 points per line
    the sliced shift solves each line in two, three and four pieces started
    from geometric sums."""
    prob, f = _case(*case)
    prob.dt = 0.37  # feet several cells away, some outside the box
    ctx = _ctx(prob, prec)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.advect(d, out)
    err = rel(out.cpu().numpy(), SemOracle(prob).advect(f))
    print(f"advect {case} {prec}: {err:.3e}")
    assert err < 1e-13


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], (41, 4, 8, 30.0, "IV")])
def test_steps_parity(case, prec):
    prob, f = _case(*case)
    ctx = _ctx(prob, prec)
    ctx.set_state(f)
    ctx.step(5)
    ref = SemOracle(prob).step(f, 5)
    err = rel(ctx.get_state(), ref)
    print(f"steps {case} {prec}: {err:.3e}")
    assert err < 1e-10


def test_observables_parity():
    prob, f = _case(17, 2, 6, 12.0, "IV")
    ctx = _ctx(prob)
    ctx.set_state(f)
    ob = ctx.observables()
    ref = SemOracle(prob).observables(f)
    for k in ("mass", "energy", "purity", "l2norm"):
        assert abs(getattr(ob, k) - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    np.testing.assert_allclose(ob.n1, ref["n1"], rtol=1e-12, atol=1e-15)
    assert ob.step == 0


def test_errors():
    from paper_2511_11354_gb300 import w2
    with pytest.raises(w2.W2Error):
        w2.SemContext(7, 2, 4, 10.0, 5.0, 0.01)         # nx too small
    with pytest.raises(w2.W2Error):
        w2.SemContext(17, 2, 33, 10.0, 5.0, 0.01)       # nq too large
    with pytest.raises(w2.W2Error):
        w2.SemContext(257, 2, 4, 10.0, 5.0, 0.01, precision=w2.W2_F64_SLICED)  # sliced lines too long
    ctx = w2.SemContext(17, 2, 4, 10.0, 5.0, 0.01)
    with pytest.raises(w2.W2Error) as e:
        ctx.step(1)                                     # no potentials, no state
    assert e.value.name == "W2_ERR_STATE"
    d = torch.zeros(ctx.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(w2.W2Error) as e:
        ctx.advect(d, d)                                # overlapping arrays
    assert e.value.name == "W2_ERR_ARG"


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
def test_paper_mesh_sampled(prec):
    """The strongly correlated example's mesh: 201^2 x (8 x 16)^2 on
    [-15, 15]^2 x [-10 pi/3, 10 pi/3]^2, Hamiltonian IV; the operator at 24
    sampled spatial points (its potentials from the whole state) and one
    step's exchange symmetry."""
    prob, f = inputs.workload_correlated("IV", soft=1.0)
    ctx = _ctx(prob, prec)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.theta(d, out)
    xs = np.random.default_rng(5).choice(prob.nx * prob.nx, 24, replace=False)
    got = out.view(prob.nx * prob.nx, prob.np_, prob.np_)[torch.from_numpy(xs).cuda()].cpu().numpy()
    err = rel(got, SemOracle(prob).theta_sample(f, xs))
    print(f"paper mesh {prec}: {err:.3e}")
    assert err < THETA_BAR[prec]
    del out
    ctx.set_state(d)
    ctx.step(1)
    g = ctx.get_state(torch.empty_like(d))
    asym = (g - g.permute(1, 0, 3, 2)).abs().max().item()
    assert math.isfinite(asym) and asym <= (1e-13 if prec == "W2_F64" else 1e-11) * g.abs().max().item()


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
def test_occupations_parity(prec):
    """Occupation numbers and correlation entropy of an evolved correlated
    state against the oracle (exact inverse Wigner transform over the cells,
    numpy's Hermitian eigensolver)."""
    from oracle.rdm_ref import correlation_entropy
    prob, f = _case(21, 2, 8, 12.0, "IV")
    ctx = _ctx(prob, prec)
    ctx.set_state(f)
    ctx.step(2)
    g = ctx.get_state()
    occ, s = ctx.occupations()
    ref = SemOracle(prob).occupations(g)
    assert np.abs(occ - ref).max() < 1e-11 * ref[0]
    assert abs(s - correlation_entropy(ref)) < 1e-10 * max(1.0, abs(s))
    assert abs(occ.sum() - ctx.observables().mass) < 1e-10 * occ.sum()


def test_occupations_of_a_two_packet_mixture():
    """f = f1 (x) f1 with f1 the 50/50 mixture of two unit-width Gaussians 4
    apart: occupations (1 +- e^-2)/2 (the overlap of the packets is e^-2)."""
    prob = inputs.sem_correlated_problem("I", nx=121, ncell=8, nq=12, L=30.0)
    o = SemOracle(prob)
    x, p = o.x, o.p
    f1 = sum(np.exp(-0.5 * (x[:, None] - c) ** 2 - 2 * p[None, :] ** 2) for c in (-2.0, 2.0)) / (2 * math.pi)
    m1 = o.dx * np.dot(f1.sum(axis=0), o.w)
    f = np.einsum("ac,bd->abcd", f1, f1 / m1)
    ctx = _ctx(prob)
    ctx.set_state(f)
    occ, s = ctx.occupations()
    e = math.exp(-2.0)
    assert abs(occ[0] - 0.5 * (1 + e)) < 1e-5 and abs(occ[1] - 0.5 * (1 - e)) < 1e-5, occ[:3]
    exact = sum(v * math.log(v) for v in (0.5 * (1 + e), 0.5 * (1 - e)))
    assert abs(s - exact) < 5e-3


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
def test_smallest_mesh(prec):
    """The smallest mesh the API takes: 8 points per axis (y grid of 7), one
    momentum cell of two Chebyshev points (np = 2, every product far below
    one tile): operator, shift and two steps against the oracle."""
    prob, f = _case(8, 1, 2, 10.0, "IV")
    f = f / np.abs(f).max()  # two momentum nodes far out in the packet's tails: rescale to O(1)
    prob.dt = 0.37
    ctx = _ctx(prob, prec)
    o = SemOracle(prob)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.theta(d, out)
    assert rel(out.cpu().numpy(), o.theta(f)) < THETA_BAR[prec]
    ctx.advect(d, out)
    assert rel(out.cpu().numpy(), o.advect(f)) < 1e-13
    prob.dt = 0.001  # |Theta f| is about 500 |f| on this mesh: a stable step
    ctx = _ctx(prob, prec)
    ctx.set_state(f)
    ctx.step(2)
    ref = SemOracle(prob).step(f, 2)
    assert np.linalg.norm(ref) < 2 * np.linalg.norm(f)
    assert rel(ctx.get_state(), ref) < 1e-10


@pytest.mark.parametrize("prec", ["W2_F64", "W2_F64_SLICED"])
def test_theta_parity_widest_momentum_axis(prec):
    """The largest momentum axis (8 cells x 32 points = 256: contractions over
    2 np = 512 split in two on the sliced path) on the smallest box (8 points,
    y grid of 7)."""
    prob, f = _case(8, 8, 32, 10.0, "IV")
    ctx = _ctx(prob, prec)
    d = torch.from_numpy(f).cuda()
    out = torch.empty_like(d)
    ctx.theta(d, out)
    err = rel(out.cpu().numpy(), SemOracle(prob).theta(f))
    print(f"theta widest {prec}: {err:.3e}")
    assert err < THETA_BAR[prec]
