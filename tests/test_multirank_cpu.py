"""Multi-rank paths on CPU with gloo: the replica timing of bench.py (the job
time is the maximum over ranks, the rate counts every replica), and the
sharded Lawson step of the distributed scheme (Sec. 4.2) on two ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    my_ms = 100.0 + 50.0 * rank          # rank 1 is the slow replica
    ms = bench.reduce_max(my_ms, dist, "cpu")
    rate = bench.whole_job_rate(1000, 10, world, ms)
    q.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    assert all(abs(o[2] - 1000 * 10 * 2 / 0.150) < 1e-6 for o in out)


# ---------------------------------------------------------------------------
# The sharded step (Sec. 4.2) on two gloo ranks: x1 cut into two patches, one
# per rank.  The pseudo-difference operator and the x2 shift are local; the
# densities are summed over the ranks (all_reduce) before each operator; the
# x1 shift solves one local spline per patch with perfectly matched boundary
# conditions, each rank sending its neighbour the part of the end-slope
# stencil over its own points and its G boundary samples (point-to-point).
# The ranks' arithmetic is the FP64 oracle's operator and line shift plus the
# local spline written out here; the assembled result must match the
# oracle's unsharded step.
# ---------------------------------------------------------------------------

NNB = 26


def _slope_stencil(nx, h):
    z = np.sqrt(3.0) - 2.0
    zn = z ** nx

    def beta(m):
        m %= nx
        return np.sqrt(3.0) * (z ** m + z ** (nx - m)) / (1.0 - zn)
    return np.array([(beta(j - 1) - beta(j + 1)) / (2 * h) for j in range(-NNB, NNB + 1)])


def _bspline_weights(th):
    return np.array([(1 - th) ** 3 / 6, (3 * th ** 3 - 6 * th ** 2 + 4) / 6,
                     (-3 * th ** 3 + 3 * th ** 2 + 3 * th + 1) / 6, th ** 3 / 6])


def _x1_shift_patch(own, prob, D, G, recv_left, recv_right):
    """own: [M, nx, nk, nk] rows of this patch; recv_*: (slope part, ghost
    rows) from the neighbours.  Returns the shifted own rows."""
    M, nx, nk = own.shape[0], prob.nx, prob.nk
    h, n = prob.dx, M + 2 * G
    lines = own.reshape(M, -1)
    pl = recv_left[0] + sum(D[NNB + (m + G)] * lines[m] for m in range(0, -G + NNB + 1))
    hi = M + G - 1
    pr = recv_right[0] + sum(D[NNB + (m - hi)] * lines[m] for m in range(hi - NNB, M))
    vals = np.concatenate([recv_left[1], lines, recv_right[1]])   # points -G .. M + G - 1
    T = np.zeros((n, n))
    for v in range(n):
        T[v, v] = 4.0
        if v > 0:
            T[v, v - 1] = 1.0
        if v < n - 1:
            T[v, v + 1] = 1.0
    T[0, 1] = 2.0
    T[n - 1, n - 2] = 2.0
    rhs = 6.0 * vals
    rhs[0] += 2 * h * pl
    rhs[n - 1] -= 2 * h * pr
    eta = np.linalg.solve(T, rhs)
    ext = np.concatenate([(eta[1] - 2 * h * pl)[None], eta, (eta[n - 2] + 2 * h * pr)[None]])
    out = np.empty_like(lines).reshape(M, nx, nk, nk)
    e4 = ext.reshape(n + 2, nx, nk, nk)
    for a in range(nk):
        s = prob.dt * (a - nk // 2) * prob.dp / (prob.mass * h)
        k0 = int(np.floor(-s))
        w = _bspline_weights(-s - k0)
        for v in range(M):
            r = G + v + k0
            out[v, :, a, :] = sum(w[q] * e4[r + q, :, a, :] for q in range(4))
    return out


def _send_parts(own, D, G):
    M = own.shape[0]
    lines = own.reshape(M, -1)
    cl, cr = G - 1, M - G
    to_left = sum(D[NNB + (m - cl)] * lines[m] for m in range(0, cl + NNB + 1))
    to_right = sum(D[NNB + (m - cr)] * lines[m] for m in range(cr - NNB, M))
    return (to_left, lines[:G].copy()), (to_right, lines[M - G:].copy())


def _exchange(rank, world, parts):
    """Send (slope part, ghost rows) to each neighbour and receive theirs."""
    left, right = (rank - 1) % world, (rank + 1) % world
    to_left, to_right = parts
    bufs = {}
    reqs = []
    for tag, (dst, (s, g)) in enumerate(((left, to_left), (right, to_right))):
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(s)), dst, tag=10 * tag))
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(g)), dst, tag=10 * tag + 1))
    # what the left neighbour sent to its right (tag 10) and the right one to its left (tag 0)
    for src, tag, key in ((left, 10, "L"), (right, 0, "R")):
        s = torch.empty(to_left[0].shape, dtype=torch.float64)
        g = torch.empty(to_left[1].shape, dtype=torch.float64)
        dist.recv(s, src, tag=tag)
        dist.recv(g, src, tag=tag + 1)
        bufs[key] = (s.numpy(), g.numpy())
    for r in reqs:
        r.wait()
    return bufs["L"], bufs["R"]


def _shard_rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_2511_11354_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, f0 = inputs.workload_small(nx=64, nk=8)
    nx, nk, M = prob.nx, prob.nk, prob.nx // world
    o = oracle.Oracle(prob)
    D = _slope_stencil(nx, prob.dx)
    k0s = [int(np.floor(-prob.dt * (a - nk // 2) * prob.dp / (prob.mass * prob.dx))) for a in range(nk)]
    G = max(1, max(max(-k, k + 1) for k in k0s))
    rows = slice(rank * M, (rank + 1) * M)

    def full(own):
        z = np.zeros((nx, nx, nk, nk))
        z[rows] = own
        return z

    def theta(own):
        # densities of the sharded state: each rank sums its rows, all ranks add
        n1p, n2p = o.marginals(full(own))
        n = torch.from_numpy(np.stack([n1p, n2p]))
        dist.all_reduce(n)
        U1, U2 = o.potential_fine(n[0].numpy()), o.potential_fine(n[1].numpy())
        return o.theta_with(full(own), U1, U2, 7)[rows]

    def shift(own):
        a = np.empty_like(own)
        for i in range(M):   # x2 lines are local
            for p1 in range(nk):
                for p2 in range(nk):
                    s2 = prob.dt * (p2 - nk // 2) * prob.dp / prob.mass
                    a[i, :, p1, p2] = o.shift_line(own[i, :, p1, p2], s2)
        recv_l, recv_r = _exchange(rank, world, _send_parts(a, D, G))
        return _x1_shift_patch(a, prob, D, G, recv_l, recv_r)

    own = f0[rows].copy()
    shifted = shift(own)
    tau = prob.dt
    g = theta(own)
    a, b = shifted, shift(g)
    ft = a + tau * b
    c = theta(ft)
    step = a + 0.5 * tau * (b + c)
    parts = [torch.zeros(M, nx, nk, nk, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(np.ascontiguousarray(step)))
    sh = [torch.zeros(M, nx, nk, nk, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(sh, torch.from_numpy(np.ascontiguousarray(shifted)))
    if rank == 0:
        got = np.concatenate([p.numpy() for p in parts])
        got_shift = np.concatenate([p.numpy() for p in sh])
        ref = o.step(f0, 1)
        ref_shift = o.advect(f0)
        q.put((float(np.linalg.norm(got_shift - ref_shift) / np.linalg.norm(ref_shift)),
               float(np.linalg.norm(got - ref) / np.linalg.norm(ref))))
    dist.destroy_process_group()


def test_two_gloo_ranks_sharded_step_matches_oracle():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    err_shift, err_step = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert err_shift < 1e-13, err_shift
    assert err_step < 1e-12, err_step
