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


def _collect(q, procs, limit):
    """One result per rank; fails as soon as a rank exits without one."""
    import queue
    import time
    out, t0 = [], time.time()
    while len(out) < len(procs):
        try:
            out.append(q.get(timeout=2))
        except queue.Empty:
            dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
            if dead or time.time() - t0 > limit:
                for p in procs:
                    if p.is_alive():
                        p.kill()
                raise AssertionError(f"a rank failed (exit codes {[p.exitcode for p in procs]})")
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


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
    out = _collect(q, procs, 120)
    b = _bench()
    for rank, gathered, times in out:
        assert times == [2.0, 10.0]                       # max over ranks, element-wise
        for s in range(3):
            blocks = [gathered[r][s] for r in range(2)]
            flat = [i for blk in blocks for i in blk]
            assert len(flat) == len(set(flat)) == 8          # disjoint, 4 per rank
            assert sorted(flat) == sorted((s * 8 + j) % b.WORKLOADS["ksg30"]["n_inst"] for j in range(8))
    assert out[0][1] == out[1][1]                          # every rank sees the same plan


def _shard_rank(rank, world, port, q):
    """One rank of a branch-sharded solve with the oracle standing in for the
    device: the same host search on every rank, leaves i = rank (mod world), each
    leaf solved exactly (transfer matrix, fixed spins pinned by strong fields), the
    maximum exchanged by an all-reduce and the partial counting sums by an
    all-gather."""
    import json

    import torch.distributed as dist

    import oracle
    import paper_2602_05470_gb300 as P
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_answers.json")) as f:
            g = json.load(f)["spin_large_f6"][0]
        inst = synth.square_lattice(g["L"], seed=g["seed"])
        s = P.Solver(mode=P.MODE_BBTN, space_cap_log2=12, use_symmetry=False)
        fx, total = s.search_leaves(inst, max_leaves=4096)
        mine = list(range(rank, total, world))
        big = 8 * (sum(abs(j) for j in inst.J) + 1)
        vals = {}
        for i in mine:
            row = fx[i]
            h2 = [h + (big if f == 1 else -big if f == 0 else 0) for h, f in zip(inst.h2, row)]
            e2, d, _ = oracle.spin_square_tm(synth.Instance(**{**inst.__dict__, "h2": h2}))
            vals[i] = (-(e2 + big * int((row >= 0).sum())), d)        # max-plus value, count
        local = max((v for v, _ in vals.values()), default=-(1 << 62))
        t = torch.tensor([local], dtype=torch.int64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        gmax = int(t[0])
        part = (gmax, sum(d for v, d in vals.values() if v == gmax)) if any(
            v == gmax for v, _ in vals.values()) else (-(1 << 62), 0)
        parts, shares = [None] * world, [None] * world
        dist.all_gather_object(parts, part)
        dist.all_gather_object(shares, mine)
        best = max(p[0] for p in parts)
        count = sum(c for v, c in parts if v == best)
        q.put((rank, total, shares, -best, count, (g["e2"], int(g["count"]))))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_one_instance_by_branches():
    """Branch sharding protocol on two gloo ranks: the leaf shares are disjoint and
    cover the host search's leaves, and the counting sum of the ranks' partial
    results (largest value, counts of the ranks that attain it) equals the oracle's
    energy and degeneracy of the whole 16 x 16 lattice."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = _collect(q, procs, 600)
    for rank, total, shares, e2, count, want in out:
        flat = sorted(i for sh in shares for i in sh)
        assert flat == list(range(total)) and total > 1
        assert (e2, count) == want
