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
