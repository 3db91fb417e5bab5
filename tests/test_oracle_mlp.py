"""Pin of the numpy reference network (oracle/mlp_ref.py) that checks the
learned form's CUDA training kernels: its analytic gradient equals central
finite differences of its loss."""
import numpy as np

from oracle import mlp_ref


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    din, hidden, dout, rows = 7, 5, 4, 6
    n = din * hidden + hidden + 2 * (hidden * hidden + hidden) + hidden * dout + dout
    p = rng.standard_normal(n) * 0.5
    x = rng.standard_normal((rows, din))
    t = rng.standard_normal((rows, dout))
    loss, g = mlp_ref.loss_and_grad(p, x, t, din, hidden, dout)
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (mlp_ref.loss_and_grad(p + e, x, t, din, hidden, dout)[0]
                 - mlp_ref.loss_and_grad(p - e, x, t, din, hidden, dout)[0]) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())
    y = mlp_ref.forward(p, x, din, hidden, dout)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14


def test_bf16_rounding_and_tensor_core_reference():
    """The BF16 rounding of the tensor-core reference against torch's
    conversion (ties to even), and the reference itself: with inputs and
    weights already BF16-exact and roundings of the intermediates switched
    off it is the plain reference (same loss and gradient)."""
    import torch
    rng = np.random.default_rng(2)
    a = (rng.standard_normal(4096) * 10.0 ** rng.integers(-8, 8, 4096)).astype(np.float32)
    a[:4] = [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 2.0 ** -130]  # ties, a subnormal
    want = torch.from_numpy(a).to(torch.bfloat16).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(mlp_ref.bf16(a), want)
    din, hidden, dout, rows = 7, 5, 4, 6
    n = din * hidden + hidden + 2 * (hidden * hidden + hidden) + hidden * dout + dout
    p = mlp_ref.bf16(rng.standard_normal(n) * 0.5)
    x = mlp_ref.bf16(rng.standard_normal((rows, din)))
    t = rng.standard_normal((rows, dout))
    keep = mlp_ref.bf16
    try:
        mlp_ref.bf16 = lambda v: np.asarray(v, dtype=np.float64)
        l1, g1 = mlp_ref.loss_and_grad_tc(p, x, t, din, hidden, dout)
    finally:
        mlp_ref.bf16 = keep
    l0, g0 = mlp_ref.loss_and_grad(p, x, t, din, hidden, dout)
    assert abs(l1 - l0) < 1e-15 * max(1.0, l0)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-15 * np.abs(g0).max())
