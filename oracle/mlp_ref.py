"""Plain FP64 numpy reference of the learned form's network (test
infrastructure only): forward pass and the gradient of the mean squared error
with respect to every packed parameter, written out layer by layer.  Used to
check the CUDA training kernels; pinned by central finite differences in
tests/test_oracle_mlp.py.

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
