"""The multi-GPU path of bench.py runs independent replicas (no data-path
collective): the only cross-rank step is the max over ranks of the timed
region.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = [2.0, 3.5][rank]
    t = bench.slowest_rank(local_seconds, dist, "cpu")
    v = bench.replica_throughput(1000.0, world, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 3.5
        assert v == pytest.approx(2 * 1000.0 / 3.5)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank(1.25) == 1.25
    assert bench.replica_throughput(10.0, 1, 2.0) == 5.0
