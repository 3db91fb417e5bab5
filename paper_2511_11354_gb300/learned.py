"""Learned form driver: data from trajectories of the exact method, training
through the library's own kernels, and runs with the network standing in for
the two-body term (judged against the exact term and falling back to it).

All arithmetic runs in the CUDA library (w2_features, w2_theta_pair,
w2_mlp_train_step, w2_step); PyTorch holds the device buffers and gathers
training batches.
"""
from __future__ import annotations

import numpy as np

from . import w2


def _torch():
    import torch
    return torch


def make_dataset(prob, f0, mlp, snapshots, stride, points_per_snapshot, seed=0, ctx=None, scale="max"):
    """Run the exact FP64 method from f0 and collect, every `stride` steps,
    input rows and scaled two-body targets for `points_per_snapshot` random
    spatial points.  Sets the network's input/output scales from the first
    snapshot: the reciprocal maximum (scale="max") or root mean square
    ("rms") of f, f1 and the two-body term.  Returns (X bf16 [rows][din],
    T f32 [rows][nk^2])."""
    torch = _torch()
    own = ctx is None
    if own:
        ctx = w2.Context.from_problem(prob)
    nx, nk = prob.nx, prob.nk
    ctx.set_state(torch.from_numpy(np.ascontiguousarray(f0, dtype=np.float64)).cuda())
    f = torch.empty(ctx.shape, dtype=torch.float64, device="cuda")
    pair = torch.empty_like(f)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    rows = snapshots * points_per_snapshot
    X = torch.empty(rows, mlp.din, dtype=torch.bfloat16, device="cuda")
    T = torch.empty(rows, nk * nk, dtype=torch.float32, device="cuda")
    for s in range(snapshots):
        if s:
            ctx.step(stride)
        ctx.get_state(f)
        ctx.theta_pair(f, pair)
        if s == 0:
            f1 = f.sum(dim=(1, 3)) * prob.dx * prob.dp
            if scale == "rms":
                mlp.set_scales(1.0 / float(f.square().mean().sqrt()), 1.0 / float(f1.square().mean().sqrt()),
                               1.0 / float(pair.square().mean().sqrt()))
            else:
                mlp.set_scales(1.0 / float(f.abs().max()), 1.0 / float(f1.abs().max()),
                               1.0 / float(pair.abs().max()))
        xs = torch.randperm(nx * nx, generator=gen)[:points_per_snapshot].to(torch.int32).cuda()
        r0 = s * points_per_snapshot
        ctx.features(mlp, f, xs, X[r0:r0 + points_per_snapshot])
        T[r0:r0 + points_per_snapshot] = (pair.view(nx * nx, nk * nk)[xs.long()] * mlp.scales[2]).float()
    if own:
        ctx.close()
    return X, T


def train(mlp, X, T, steps, batch, lr, seed=0, lr_final=None, log_every=0):
    """Adam on random batches; the learning rate decays geometrically from lr
    to lr_final.  Returns the list of losses."""
    torch = _torch()
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    losses = []
    lr_final = lr if lr_final is None else lr_final
    for it in range(steps):
        idx = torch.randint(0, n, (batch,), generator=gen).cuda()
        rate = lr * (lr_final / lr) ** (it / max(1, steps - 1))
        loss = mlp.train_step(X[idx].contiguous(), T[idx].contiguous(), rate)
        losses.append(loss)
        if log_every and it % log_every == 0:
            print(f"train step {it}: loss {loss:.4e} lr {rate:.2e}")
    return losses


def zero_network(nk, hidden=256, max_rows=4096):
    """A network whose output is identically zero: the method without the
    two-body term."""
    m = w2.MLP(nk, hidden, max_rows)
    m.set_params(np.zeros(m.nparams, dtype=np.float32))
    m.set_scales(1.0, 1.0, 1.0)
    return m


def run(prob, f0, steps, mlp=None, judge_every=0, tol=1e30, precision=w2.W2_F64):
    """Advance the FP64 method (W2_F64 or W2_F64_SLICED) `steps` steps, with
    `mlp` for the two-body term when given.  Returns (final state, learned
    report or None)."""
    torch = _torch()
    ctx = w2.Context.from_problem(prob, precision=precision)
    ctx.set_state(torch.from_numpy(np.ascontiguousarray(f0, dtype=np.float64)).cuda())
    if mlp is not None:
        ctx.attach_learned(mlp, judge_every, tol)
    ctx.step(steps)
    out = ctx.get_state()
    rep = ctx.learned_report() if mlp is not None else None
    ctx.close()
    return out, rep


# ---------------------------------------------------------------------------
# Kernel networks: the two-body term's structure (linear in f, a shift kernel
# that depends on the pair distance only); the network predicts the kernel.
# ---------------------------------------------------------------------------

def make_kernel_dataset(prob, f0, snapshots, stride, points_per_snapshot, seed=0, precision=None):
    """Run the exact FP64 method from f0 and collect, every `stride` steps,
    `points_per_snapshot` random spatial points: their state blocks, the
    exact two-body term there and their pair distance index d = (i1 - i2)
    mod nx.  Returns device tensors (F float64 [rows][nk^2], P float64
    [rows][nk^2], d int32 [rows])."""
    torch = _torch()
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED if precision is None else precision)
    nx, nk = prob.nx, prob.nk
    ctx.set_state(torch.from_numpy(np.ascontiguousarray(f0, dtype=np.float64)).cuda())
    f = torch.empty(ctx.shape, dtype=torch.float64, device="cuda")
    pair = torch.empty_like(f)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    rows = snapshots * points_per_snapshot
    F = torch.empty(rows, nk * nk, dtype=torch.float64, device="cuda")
    P = torch.empty_like(F)
    D = torch.empty(rows, dtype=torch.int32, device="cuda")
    for s in range(snapshots):
        if s:
            ctx.step(stride)
        ctx.get_state(f)
        ctx.theta_pair(f, pair)
        xs = torch.randperm(nx * nx, generator=gen)[:points_per_snapshot]
        r0 = s * points_per_snapshot
        F[r0:r0 + points_per_snapshot] = f.view(nx * nx, nk * nk)[xs.cuda()]
        P[r0:r0 + points_per_snapshot] = pair.view(nx * nx, nk * nk)[xs.cuda()]
        D[r0:r0 + points_per_snapshot] = ((xs // nx - xs % nx) % nx).to(torch.int32).cuda()
    ctx.close()
    return F, P, D


def train_kernel(mlp, prob, F, P, D, steps, batch, lr, lr_final=None, seed=0, log_every=0):
    """Adam on random batches of the kernel dataset, through the library's
    kernel-network training step; the learning rate decays geometrically from
    lr to lr_final.  Returns the list of relative losses."""
    torch = _torch()
    ctx = w2.Context.from_problem(prob, precision=w2.W2_F64_SLICED)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = F.shape[0]
    lr_final = lr if lr_final is None else lr_final
    losses = []
    for it in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=gen).cuda()
        rate = lr * (lr_final / lr) ** (it / max(1, steps - 1))
        loss = mlp.kernel_train_step(ctx, F[idx].contiguous(), P[idx].contiguous(), D[idx].contiguous(), rate)
        losses.append(loss)
        if log_every and it % log_every == 0:
            print(f"kernel train step {it}: relative loss {loss:.4e} lr {rate:.2e}")
    ctx.close()
    return losses
