"""The multi-GPU path of bench.py is replicas only: each rank registers its own
pairs (disjoint seeds) and the job's throughput uses the maximum step time over
ranks.  Checked with two gloo processes on the CPU (no GPU, no data-path
collective besides that one max)."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms = bench.aggregate_ms(ms_local, world, dist, "cpu")
    seeds = bench.rank_seeds(rank)
    out.put((rank, ms, seeds, bench.throughput(ms, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate_with_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    import bench
    assert all(ms == 150.0 for _, ms, _, _ in res)
    s0, s1 = set(res[0][2]), set(res[1][2])
    assert len(s0) == bench.PAIRS and not (s0 & s1)
    assert abs(res[0][3] - world * bench.PAIRS * 1e3 / 150.0) < 1e-9
