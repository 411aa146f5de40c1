"""The benchmark's N > 1 path (independent replicas, one per GPU) on CPU:
world_size 2 over gloo.  Each rank reports its own time; the job's time is
the slowest rank's and the job's throughput counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(1.0 + rank, dist, device="cpu")
    v = bench.replica_throughput(1000.0, world, t)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]  # both ranks see the slowest rank's time
    assert [o[2] for o in out] == [1000.0, 1000.0]  # 2 ranks x 1000 units / 2 s
