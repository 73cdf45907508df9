"""The multi-GPU path of the benchmark on CPU: two gloo ranks.

Instances are independent, so ranks share no data; each rank solves its own
block of the workload and the job's time is the slowest rank's. Checked here
with world size 2 (no GPU): every instance of a step goes to exactly one rank,
the blocks are the same on every rank, and the maximum over ranks is what the
bench reports."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        mine = {s: b.shard_indices(rank, world, s, 4) for s in range(3)}
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        times = b.max_over_ranks([1.0 + rank, 10.0 - rank], dist, "cpu")
        q.put((rank, gathered, times))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_the_workload_and_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    b = _bench()
    for rank, gathered, times in out:
        assert times == [2.0, 10.0]                       # max over ranks, element-wise
        for s in range(3):
            blocks = [gathered[r][s] for r in range(2)]
            flat = [i for blk in blocks for i in blk]
            assert len(flat) == len(set(flat)) == 8          # disjoint, 4 per rank
            assert sorted(flat) == sorted((s * 8 + j) % b.WORKLOADS["ksg30"]["n_inst"] for j in range(8))
    assert out[0][1] == out[1][1]                          # every rank sees the same plan
