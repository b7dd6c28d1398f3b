"""The N-replica path of bench.py on CPU: two gloo ranks agree on the slowest rank's timings and
the whole-job throughput sums the replicas (the path does not shard: replicas only)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = bench.slowest_rank([1.0 + rank, 10.0 - rank, 0.5 * (rank + 1)], world, device="cpu")
    thr = bench.replica_throughput(1000, times[0], world)
    dist.barrier()
    q.put((rank, times, thr))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, thr in out:
        assert times == [2.0, 10.0, 1.0]
        assert thr == pytest.approx(2 * 1000 / 2.0)


def test_single_replica_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.replica_throughput(10, 2.0, 1) == 5.0
