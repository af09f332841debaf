"""The multi-rank aggregation of bench.py on CPU: two gloo ranks, each with its own timings; every
rank gets the maximum of each timing over the ranks, and the whole-job value counts both replicas."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [1.0 + rank, 10.0 - rank, 3.0]
    out = bench.max_over_ranks(local, dist, "cpu")
    q.put((rank, out, bench.job_value(1000, world, out[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_timing():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out, value in res:
        assert out == [2.0, 10.0, 3.0]
        # 1000 DOF per replica, 2 replicas, 3 stages, 2 ms per step
        assert value == pytest.approx(1000 * 3 * 2 / 2e-3)
