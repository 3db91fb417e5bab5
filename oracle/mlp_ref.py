"""Plain FP64 numpy reference of the learned form's networks (test
infrastructure only): forward pass and the gradient of the mean squared error
with respect to every packed parameter, written out layer by layer, and the
kernel network's operator-side loss and gradient.  Used to check the CUDA
training kernels; pinned by central finite differences and against the FP64
oracle's two-body term in tests/test_oracle_mlp.py.

Network: x -> silu(x W0 + b0) -> silu(. W1 + b1) -> silu(. W2 + b2) -> . W3 + b3,
silu(z) = z / (1 + exp(-z)); loss = mean((y - t)^2).
"""
import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def unpack(p, din, hidden, dout):
    dims = [(din, hidden), (hidden, hidden), (hidden, hidden), (hidden, dout)]
    layers, off = [], 0
    for i, o in dims:
        W = p[off:off + i * o].reshape(i, o)
        off += i * o
        b = p[off:off + o]
        off += o
        layers.append((W, b))
    assert off == p.size
    return layers


def forward(p, x, din, hidden, dout):
    a = x
    for l, (W, b) in enumerate(unpack(p, din, hidden, dout)):
        z = a @ W + b
        a = silu(z) if l < 3 else z
    return a


def loss_and_grad(p, x, t, din, hidden, dout):
    p = np.asarray(p, dtype=np.float64)
    layers = unpack(p, din, hidden, dout)
    acts, zs = [np.asarray(x, dtype=np.float64)], []
    a = acts[0]
    for l, (W, b) in enumerate(layers):
        z = a @ W + b
        if l < 3:
            zs.append(z)
            a = silu(z)
            acts.append(a)
        else:
            y = z
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    grads = []
    dz = 2.0 * (y - t) / n
    for l in range(3, -1, -1):
        W, b = layers[l]
        grads.append((acts[l].T @ dz, dz.sum(axis=0)))
        if l > 0:
            dz = (dz @ W.T) * dsilu(zs[l - 1])
    grads = grads[::-1]
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, g


def bf16(a):
    """Round to the nearest BF16 (ties to even), through FP32, as numbers."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grad_tc(p, x, t, din, hidden, dout):
    """loss_and_grad with the roundings the tensor-core kernels apply, in
    FP64 otherwise: weights and inputs in BF16; each hidden activation
    silu(z) stored in BF16 for the next product and for its weight gradient;
    the output gradient 2 (y - t)/n and each back-propagated dz rounded to
    BF16 for the products (the bias gradients sum the unrounded dz)."""
    p = np.asarray(p, dtype=np.float64)
    layers = unpack(p, din, hidden, dout)
    Wb = [bf16(W) for W, _ in layers]
    acts, zs = [bf16(x)], []
    a = acts[0]
    for l, (W, b) in enumerate(layers):
        z = a @ Wb[l] + b
        if l < 3:
            zs.append(z)
            a = bf16(silu(z))
            acts.append(a)
        else:
            y = z
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    grads = []
    dz = 2.0 * (y - t) / n
    for l in range(3, -1, -1):
        dzb = bf16(dz)
        grads.append((acts[l].T @ dzb, dz.sum(axis=0)))
        if l > 0:
            dz = (dzb @ Wb[l].T) * dsilu(zs[l - 1])
    grads = grads[::-1]
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, g


# ---------------------------------------------------------------------------
# Kernel network (the two-body term's structure): reference of its loss and
# of the loss gradient with respect to the network's outputs.  The two-body
# term of Eq. two_body_FSM at one spatial point, with the shift kernel K of
# its pair distance: Theta_K F(n1, n2) = sum_{j >= 1} K(j) [F(n1 + j, n2 - j)
# - F(n1 - j, n2 + j)], F zero outside the momentum window.
# ---------------------------------------------------------------------------

def _pair_shifts(F, j):
    """(F(n1 + j, n2 - j), F(n1 - j, n2 + j)) for blocks F [rows][nk][nk]."""
    nk = F.shape[1]
    a = np.zeros_like(F)
    b = np.zeros_like(F)
    a[:, :nk - j, j:] = F[:, j:, :nk - j]
    b[:, j:, :nk - j] = F[:, :nk - j, j:]
    return a, b


def pair_apply(F, K):
    """Theta_K F for blocks F [rows][nk][nk] and one kernel row per block,
    K [rows][nk] (K[:, 0] is not used)."""
    F = np.asarray(F, dtype=np.float64)
    out = np.zeros_like(F)
    for j in range(1, F.shape[1]):
        a, b = _pair_shifts(F, j)
        out += np.asarray(K, dtype=np.float64)[:, j, None, None] * (a - b)
    return out


def pair_kernel_loss_grad(F, P, D, y, s_y):
    """Relative loss L = sum |Theta_{K[D_b]} F_b - P_b|^2 / sum |P_b|^2 with
    the kernel table K = y / s_y (column 0 unused) of the network outputs y
    [nx][nk], and dL/dy [nx][nk] (column 0 zero)."""
    F = np.asarray(F, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    D = np.asarray(D, dtype=np.int64)
    K = np.array(y, dtype=np.float64) / s_y
    K[:, 0] = 0.0
    R = pair_apply(F, K[D]) - P
    p2 = float(np.sum(P * P))
    loss = float(np.sum(R * R)) / p2
    G = np.zeros((D.size, F.shape[1]))
    for j in range(1, F.shape[1]):
        a, b = _pair_shifts(F, j)
        G[:, j] = np.sum(R * (a - b), axis=(1, 2))
    dK = np.zeros(K.shape)
    np.add.at(dK, D, G)
    return loss, 2.0 * dK / p2 / s_y
