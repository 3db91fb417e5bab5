"""GPU checks of the learned form: the training kernels' gradients against the
FP64 numpy reference network, the judge and fallback, and what a trained
network gains over the method without the two-body term."""
import numpy as np
import pytest

from oracle import mlp_ref
from paper_2511_11354_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11354_gb300 import build
    build.build()


def _bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def test_mlp_gradients_match_reference():
    """BF16 products with FP32 accumulation against FP64 on the same
    BF16-rounded weights and inputs: relative L2 error of the whole gradient."""
    from paper_2511_11354_gb300 import w2
    nk, hidden, rows = 8, 32, 48
    m = w2.MLP(nk, hidden, max_rows=rows)
    rng = np.random.default_rng(1)
    p = (rng.standard_normal(m.nparams) * 0.3).astype(np.float32)
    m.set_params(p)
    x = rng.standard_normal((rows, m.din)).astype(np.float32)
    t = rng.standard_normal((rows, nk * nk)).astype(np.float32)
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    tt = torch.from_numpy(t).cuda()
    g, loss = m.gradients(xb, tt)
    # the reference sees the parameters as the tensor cores do (weights in BF16, biases FP32)
    pr = p.astype(np.float64).copy()
    for name, off, shape in m.layout():
        if name.startswith("W"):
            n = int(np.prod(shape))
            pr[off:off + n] = _bf16_round(p[off:off + n])
    lref, gref = mlp_ref.loss_and_grad(pr, _bf16_round(x).astype(np.float64), t.astype(np.float64),
                                       m.din, hidden, nk * nk)
    assert abs(loss - lref) < 2e-2 * lref
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 5e-2
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert cos > 0.998
    # one training step lowers the loss on the same batch
    l0 = m.train_step(xb, tt, 1e-3)
    l1 = m.train_step(xb, tt, 1e-3)
    assert l1 < l0


def _small_dwell():
    prob, f0 = inputs.workload_dwell(nx=16, nk=32)
    return prob, f0


def test_judge_and_fallback():
    from paper_2511_11354_gb300 import learned, w2
    prob, f0 = _small_dwell()
    zero = learned.zero_network(prob.nk, hidden=32, max_rows=prob.nx * prob.nx)
    # a network that is plainly wrong (zero) falls back to the exact term at the first judgement
    out, rep = learned.run(prob, f0, 12, zero, judge_every=5, tol=0.1)
    assert rep["judged"] == 1 and not rep["active"] and rep["last_err"] == pytest.approx(1.0, abs=1e-6)
    # ... and from then on the step is the exact one: 5 steps without, 7 with the pair term
    ctx = w2.Context.from_problem(prob)
    ctx.set_state(f0)
    ctx.attach_learned(zero, 0, 1e30)
    ctx.step(5)
    ctx.attach_learned(None)
    ctx.step(7)
    assert np.array_equal(ctx.get_state(), out)


def test_trained_network_beats_dropping_the_two_body_term():
    """Trained on a short exact trajectory of the double-well physics, the
    network stands in for the two-body term over the next 40 steps: the state
    stays closer to the exact run than the run without the two-body term, and
    the judge reports an error well below 1."""
    from paper_2511_11354_gb300 import learned, w2
    prob, f0 = _small_dwell()
    torch.manual_seed(0)
    mlp = w2.MLP(prob.nk, hidden=256, max_rows=max(512, prob.nx * prob.nx))
    X, T = learned.make_dataset(prob, f0, mlp, snapshots=120, stride=1, points_per_snapshot=96, seed=0)
    losses = learned.train(mlp, X, T, steps=1500, batch=512, lr=2e-3, lr_final=1e-4, seed=0)
    assert losses[-1] < 0.2 * losses[0]
    exact, _ = learned.run(prob, f0, 40)
    net, rep = learned.run(prob, f0, 40, mlp, judge_every=20, tol=0.9)
    nopair, _ = learned.run(prob, f0, 40, learned.zero_network(prob.nk, 32, prob.nx * prob.nx))
    e_net = np.linalg.norm(net - exact) / np.linalg.norm(exact)
    e_nopair = np.linalg.norm(nopair - exact) / np.linalg.norm(exact)
    assert rep["judged"] == 2 and rep["active"], rep
    assert rep["last_err"] < 0.5, rep
    assert e_net < 0.5 * e_nopair, (e_net, e_nopair)


def test_feature_rows_match_their_definition():
    """Input rows of the network (w2_features): the scaled block, the scaled
    reduced one-body function at x1 and at x2, and eight harmonics of the pair
    distance, each within BF16 rounding of its definition."""
    from paper_2511_11354_gb300 import w2
    prob, f0 = inputs.workload_dwell(nx=8, nk=16)
    nx, nk, P = prob.nx, prob.nk, prob.nk * prob.nk
    ctx = w2.Context.from_problem(prob)
    mlp = w2.MLP(nk, 32, max_rows=64)
    mlp.set_scales(2.0, 3.0, 1.0)
    pts = [0, 5, 17, 63]
    xs = torch.tensor(pts, dtype=torch.int32, device="cuda")
    X = torch.empty(len(pts), mlp.din, dtype=torch.bfloat16, device="cuda")
    ctx.features(mlp, torch.from_numpy(f0).cuda(), xs, X)
    got = X.float().cpu().numpy()
    f1 = f0.sum(axis=(1, 3)) * prob.dx * prob.dp  # [x1][p1]
    for r, Xi in enumerate(pts):
        i1, i2 = divmod(Xi, nx)
        want = np.zeros(mlp.din)
        want[:P] = 2.0 * f0[i1, i2].ravel()
        want[P:P + nk] = 3.0 * f1[i1]
        want[P + nk:P + 2 * nk] = 3.0 * f1[i2]
        for m in range(1, 9):
            u = 2 * np.pi * m * (i1 - i2) / nx
            want[P + 2 * nk + 2 * (m - 1)] = np.sin(u)
            want[P + 2 * nk + 2 * (m - 1) + 1] = np.cos(u)
        assert np.all(np.abs(got[r] - want) <= 2.0 ** -8 * np.abs(want) + 1e-6), r


@pytest.mark.parametrize("nk,hidden,rows", [(8, 32, 200), (16, 64, 300), (64, 256, 4096)])
def test_inference_forward_matches_reference(nk, hidden, rows):
    """The inference forward (pipelined BF16 GEMMs with fused bias/SiLU
    epilogues) against the FP64 reference network with the same BF16
    roundings: BF16 weights and inputs, hidden activations rounded to BF16
    between layers.  The shapes cover ragged row and column tiles, a K tail
    below one 32-wide step and the timed size."""
    from paper_2511_11354_gb300 import w2
    m = w2.MLP(nk, hidden, max_rows=rows)
    rng = np.random.default_rng(nk)
    p = (rng.standard_normal(m.nparams) * 0.2).astype(np.float32)
    m.set_params(p)
    x = (rng.standard_normal((rows, m.din)) * 0.5).astype(np.float32)
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    y = torch.empty(rows, nk * nk, dtype=torch.float32, device="cuda")
    m.forward(xb, y)
    got = y.cpu().numpy().astype(np.float64)
    pr = p.astype(np.float64).copy()
    for name, off, shape in m.layout():
        if name.startswith("W"):
            n = int(np.prod(shape))
            pr[off:off + n] = _bf16_round(p[off:off + n])
    a = _bf16_round(x).astype(np.float64)
    for l, (W, b) in enumerate(mlp_ref.unpack(pr, m.din, hidden, nk * nk)):
        z = a @ W + b
        a = _bf16_round(mlp_ref.silu(z)).astype(np.float64) if l < 3 else z
    err = np.linalg.norm(got - a) / np.linalg.norm(a)
    assert err < 5e-3, err


def _tc_gradient_error(m, hidden, dout, rows, seed):
    """Relative L2 error of the kernels' gradient against the FP64 reference
    with the same BF16 roundings (weights, inputs, activations, dz)."""
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(m.nparams) * 0.05).astype(np.float32)
    m.set_params(p)
    x = rng.standard_normal((rows, m.din)).astype(np.float32)
    t = rng.standard_normal((rows, dout)).astype(np.float32)
    g, loss = m.gradients(torch.from_numpy(x).to(torch.bfloat16).cuda(), torch.from_numpy(t).cuda())
    lref, gref = mlp_ref.loss_and_grad_tc(p.astype(np.float64), x, t.astype(np.float64), m.din, hidden, dout)
    return abs(loss - lref) / lref, float(np.linalg.norm(g - gref) / np.linalg.norm(gref))


def test_mlp_gradients_at_the_trained_shapes():
    """The two trained shapes: the pair-term network of the 64^4 workload
    (input 4256, width 256, output 4096, batch 1024) and the kernel network
    (input 32, width 256, output 64, one row per pair distance), against the
    reference applying the kernels' BF16 roundings: within 2e-3."""
    from paper_2511_11354_gb300 import w2
    pair = w2.MLP(64, 256, max_rows=1024)
    el, eg = _tc_gradient_error(pair, 256, 64 * 64, 1024, 5)
    assert el < 1e-3 and eg < 2e-3, (el, eg)
    pair.close()
    kern = w2.MLP(64, 256, max_rows=64, kind="kernel")
    el, eg = _tc_gradient_error(kern, 256, 64, 64, 6)
    assert el < 1e-3 and eg < 2e-3, (el, eg)
    kern.close()


def test_kernel_network_loss_and_output_gradient_vs_reference():
    """The operator side of the kernel network's training chain (features,
    forward, the predicted term's residuals and the gradient of the relative
    loss with respect to the network outputs) against the FP64 reference of
    oracle/mlp_ref.py on the same outputs: trajectory rows of the 16^2 x 32^2
    double well, loss within 1e-12 and dL/dy within 1e-10 relative."""
    from paper_2511_11354_gb300 import learned, w2
    prob, f0 = _small_dwell()
    F, P, D = learned.make_kernel_dataset(prob, f0, snapshots=6, stride=2, points_per_snapshot=20, seed=3)
    mlp = w2.MLP(prob.nk, hidden=64, max_rows=prob.nx, kind="kernel")
    s_y = 3.0 * float(F.square().mean().sqrt()) / float(P.square().mean().sqrt())
    mlp.set_scales(1.0, 1.0, s_y)
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    loss, y, g = mlp.kernel_loss_grad(ctx, F, P, D)
    nk = prob.nk
    Fh = F.cpu().numpy().reshape(-1, nk, nk)
    Ph = P.cpu().numpy().reshape(-1, nk, nk)
    # the kernels scale the outputs by the FP32 reciprocal of s_y
    s_eff = 1.0 / float(np.float32(1.0) / np.float32(mlp.scales[2]))
    lref, gref = mlp_ref.pair_kernel_loss_grad(Fh, Ph, D.cpu().numpy(), y.astype(np.float64), s_eff)
    assert abs(loss - lref) < 1e-12 * lref, (loss, lref)
    assert np.linalg.norm(g - gref) < 1e-10 * np.linalg.norm(gref), np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert np.all(g[:, 0] == 0.0)
    # the training step reports the same loss before its update
    assert mlp.kernel_train_step(ctx, F, P, D, 1e-3) == loss
    ctx.close()
    mlp.close()


def test_kernel_network_learns_the_two_body_term():
    """A kernel network trained on snapshots of an exact trajectory (random
    spatial points of each) stands in for the two-body term: the judge's
    error is small, the state stays close to the exact run, and far closer
    than the run without the two-body term."""
    from paper_2511_11354_gb300 import learned, w2
    prob, f0 = _small_dwell()
    torch.manual_seed(0)
    F, P, D = learned.make_kernel_dataset(prob, f0, snapshots=150, stride=1, points_per_snapshot=24, seed=0)
    mlp = w2.MLP(prob.nk, hidden=256, max_rows=prob.nx, kind="kernel")
    s_y = 3.0 * float(F.square().mean().sqrt()) / float(P.square().mean().sqrt())
    mlp.set_scales(1.0, 1.0, s_y)
    losses = learned.train_kernel(mlp, prob, F, P, D, steps=4000, batch=1024, lr=1e-3, lr_final=1e-5, seed=0)
    assert np.mean(losses[-50:]) < 1e-4 * losses[0], (losses[0], np.mean(losses[-50:]))
    exact, _ = learned.run(prob, f0, 40, precision=w2.W2_F64_SLICED)
    net, rep = learned.run(prob, f0, 40, mlp, judge_every=20, tol=0.05, precision=w2.W2_F64_SLICED)
    nopair, _ = learned.run(prob, f0, 40, learned.zero_network(prob.nk, 32, prob.nx * prob.nx),
                            precision=w2.W2_F64_SLICED)
    e_net = np.linalg.norm(net - exact) / np.linalg.norm(exact)
    e_nopair = np.linalg.norm(nopair - exact) / np.linalg.norm(exact)
    assert rep["judged"] == 2 and rep["active"], rep
    assert rep["last_err"] < 2e-2, rep
    assert e_net < 0.05 * e_nopair, (e_net, e_nopair)
