"""The multi-replica path of bench.py on CPU: two gloo ranks, each timing its
own replica; the job time is the maximum over ranks and the rate counts the
points of every replica (weak scaling)."""
import os
import socket

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
