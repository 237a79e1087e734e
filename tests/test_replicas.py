"""The multi-GPU path is replicas only: each rank solves its own maps and the
job's throughput is the total over the slowest rank.  Exercised here with two
gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) seconds for its 3 solves; the job took 2 s
    v = bench.job_throughput(float(rank + 1), 3, world)
    dist.destroy_process_group()
    q.put((rank, v))


def test_job_throughput_is_total_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == pytest.approx(6 / 2.0) and out[1] == pytest.approx(6 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_throughput(0.5, 5, 1) == pytest.approx(10.0)
