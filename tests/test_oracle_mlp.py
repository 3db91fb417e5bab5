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


def test_pair_kernel_gradient_matches_finite_differences():
    """The kernel network's loss gradient with respect to its outputs (the
    reference the CUDA training chain is checked against) equals central
    differences of its loss, at several outputs of several distances."""
    rng = np.random.default_rng(3)
    nx, nk, rows, s_y = 5, 8, 12, 2.5
    F = rng.standard_normal((rows, nk, nk))
    P = rng.standard_normal((rows, nk, nk))
    D = rng.integers(0, nx, rows)
    y = rng.standard_normal((nx, nk))
    loss, g = mlp_ref.pair_kernel_loss_grad(F, P, D, y, s_y)
    assert np.all(g[:, 0] == 0.0)
    h = 1e-6
    for d, j in [(0, 1), (1, 3), (D[0], nk - 1), (D[1], 2), (4, 5)]:
        e = np.zeros_like(y)
        e[d, j] = h
        fd = (mlp_ref.pair_kernel_loss_grad(F, P, D, y + e, s_y)[0]
              - mlp_ref.pair_kernel_loss_grad(F, P, D, y - e, s_y)[0]) / (2 * h)
        assert abs(g[d, j] - fd) < 1e-7 * max(1.0, abs(fd)), (d, j, g[d, j], fd)
    K = y / s_y
    K[:, 0] = 0
    R = mlp_ref.pair_apply(F, K[D]) - P
    assert abs(loss - np.sum(R * R) / np.sum(P * P)) < 1e-14


def _pair_term_residual(prob, f, apply):
    """Least-squares fit of one kernel row per pair distance to the oracle's
    exact two-body term through `apply`; the relative residual."""
    import oracle
    o = oracle.Oracle(prob)
    U0 = np.zeros((prob.nx, 2 * prob.nk))  # one-body potentials: not used by the two-body term
    P = o.theta_with(f, U0, U0, 4)
    nx, nk = prob.nx, prob.nk
    F = f.reshape(nx * nx, nk, nk)
    P = P.reshape(nx * nx, nk, nk)
    res2 = 0.0
    for d in range(nx):
        xs = [i1 * nx + i2 for i1 in range(nx) for i2 in range(nx) if (i1 - i2) % nx == d]
        cols = []
        for j in range(1, nk):
            K = np.zeros((len(xs), nk))
            K[:, j] = 1.0
            cols.append(apply(F[xs], K).ravel())
        A = np.stack(cols, axis=1)
        coef, *_ = np.linalg.lstsq(A, P[xs].ravel(), rcond=None)
        res2 += float(np.sum((A @ coef - P[xs].ravel()) ** 2))
    return np.sqrt(res2 / float(np.sum(P * P)))


def test_exact_two_body_term_has_the_kernel_form():
    """The oracle's two-body term (its own DFT-mode construction) is, at every
    pair distance, Theta_K F for one kernel row K: a least-squares fit through
    the reference's pair_apply leaves a residual at rounding level, and a
    planted mistake in the shift directions does not fit."""
    from paper_2511_11354_gb300 import inputs
    prob, f = inputs.workload_dwell(nx=8, nk=16)
    assert _pair_term_residual(prob, f, mlp_ref.pair_apply) < 1e-12

    def wrong(F, K):  # F(n1 + j, n2 + j) - F(n1 - j, n2 - j): the anti-diagonal taken as the diagonal
        nk = F.shape[1]
        out = np.zeros_like(F)
        for j in range(1, nk):
            a = np.zeros_like(F)
            b = np.zeros_like(F)
            a[:, :nk - j, :nk - j] = F[:, j:, j:]
            b[:, j:, j:] = F[:, :nk - j, :nk - j]
            out += K[:, j, None, None] * (a - b)
        return out
    assert _pair_term_residual(prob, f, wrong) > 1e-2
