"""The multi-rank logic of bench.py on CPU: two gloo ranks agree on the slowest
rank's time, split the independent systems of the batched workload without
overlap, and report whole-job throughput (replicas and shards need no data-path
collective; the only collective is this timing reduction)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = bench.shard(64, rank, world)
    ms = bench.max_over_ranks(100.0 + 25.0 * rank, dist, device="cpu")
    value = bench.throughput(4 * 1000 * 5, world, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, ms, value))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict()
    for _ in procs:
        r, mine, ms, value = q.get(timeout=120)
        res[r] = (mine, ms, value)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == 125.0              # the slowest rank's time, on every rank
    assert res[0][2] == pytest.approx(2 * 20000 / 0.125)  # units of both ranks over that time
    assert res[0][0] == list(range(0, 32)) and res[1][0] == list(range(32, 64))


def test_shard_covers_every_system_once():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for world in (1, 2, 3, 4, 7, 8):
        got = sorted(k for r in range(world) for k in bench.shard(64, r, world))
        assert got == list(range(64))
    assert bench.max_over_ranks(3.5, None) == 3.5
