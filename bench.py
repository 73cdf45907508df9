"""Benchmark: exact ground-state counting with the branch-and-bound tensor network.

Workload (one "step" = one pass of the whole path over a batch of instances):
unweighted MIS on random King's subgraphs, 30 x 30 grid, site filling 0.8
(32 seeded instances; a step solves 8 of them, --streams at a time, each in its
own context on its own CUDA stream), branch-and-bound contraction with a space cap
of 2^24 elements per tensor, exact degeneracy in three count planes (two residues
mod 30-bit primes per word) plus the overflow-check plane, recombined by CRT.
Metric: time-to-exact-count per instance (seconds, lower is better), with tropical
GOP/s and the roofline fractions of the contraction kernels alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID, FILLING, CAP, N_INST = 30, 0.8, 24, 32
# integer-ALU peak for the tiled kernel (one add+max instruction per tropical
# multiply-add): 152 SMs x 64 ALU lanes per SM per clock x 2.07 GHz
ALU_PEAK_TOPS = 152 * 64 * 2.07e9 / 1e12
METRIC = "time-to-exact-count per instance (KSG 30x30 MIS, BBTN)"
WORKLOAD = "mis_kings_subgraph_30x30_filling0.8_cap2^24_bbtn_counting"


def shard_indices(rank: int, world: int, step: int, per_step: int):
    """Workload instances of one rank in one step: the ranks of a step take
    consecutive, disjoint blocks of per_step instances (weak scaling)."""
    return [(step * per_step * world + rank * per_step + j) % N_INST for j in range(per_step)]


def instances(rank: int, world: int, step: int, per_step: int):
    import synth
    return [(idx, synth.kings_subgraph(N_GRID, FILLING, seed=synth.config_seed(2, idx)))
            for idx in shard_indices(rank, world, step, per_step)]


def max_over_ranks(values, dist, device):
    """Element-wise maximum of a list of floats over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "launch_list_ksg30x30_bbtn.md")
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, instance 0 of this workload "
                  "(profiles/launch_list_ksg30x30_bbtn.md)")


def ncu_traffic():
    """DRAM bytes per launch of each kernel from the committed ncu summary of this
    workload (its table rows read '| `kernel` (...) | launches | read + write | N MB |')."""
    out = {}
    try:
        import re
        for line in open(TRAFFIC_FILE):
            m = re.match(r"\|\s*`([^`]+)`.*\|\s*([\d.]+)\s*MB\s*\|\s*$", line)
            if m:
                out[m.group(1)] = float(m.group(2)) * 1e6
    except OSError:
        pass
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler run during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                t = [x.strip() for x in line.split(",")]
                if len(t) < 9:
                    continue
                try:
                    sm.append(float(t[1]))
                    smax = float(t[2])
                except ValueError:
                    continue
                for nm, v in zip(names, t[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_time(per: int, start: int = 0):
    """Time the CPU oracle (King's-subgraph transfer matrix, one host core) on
    `per` instances of the workload; returns (seconds per instance, description)."""
    import oracle
    import synth
    oracle.build()
    t = 0.0
    idxs = []
    for j in range(per):
        idx = (start + j) % N_INST
        inst = synth.kings_subgraph(N_GRID, FILLING, seed=synth.config_seed(2, idx))
        t0 = time.perf_counter()
        oracle.mwis_ksg_tm(inst)
        t += time.perf_counter() - t0
        idxs.append(idx)
    return t / per, f"instances {idxs} of the 32 (full 30x30 instances, exact count)"


def run_reference(args, rank, world):
    """--impl reference: the oracle as it stands, on the host cores, rank 0 only."""
    if rank != 0:
        return
    for w in range(args.warmup):
        oracle_time(1, start=w)
    samples = []
    for s in range(args.steps):
        v, _ = oracle_time(1, start=args.warmup + s)
        samples.append(v)
    value = sum(samples) / len(samples)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s/instance",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * value,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded King's subgraphs)",
        "config": {"workload": WORKLOAD, "instances_per_step": 1, "l2": "inputs are host-side graphs"},
        "cpu_baseline": {"value": value, "unit": "s/instance", "cores": 1, "kind": "oracle",
                         "sample": "one full 30x30 instance per step, transfer-matrix oracle, single thread"},
        "e2e": {"value": value, "unit": "s/instance", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2602_05470_gb300 as P
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")     # 256 MiB > L2
    per = args.instances_per_step

    def make_solver(profile=False, st=None):
        return P.Solver(mode=P.MODE_BBTN, space_cap_log2=CAP, n_primes=3, batch=64, profile=profile,
                        leaf_trials=args.leaf_trials, stream=(st or stream).cuda_stream)

    # S solver contexts, each on its own CUDA stream and host thread, take the
    # step's instances round-robin: one instance's many small launches leave most of
    # the GPU idle, and another instance's launches fill it
    S = max(1, args.streams)
    streams = [stream] + [torch.cuda.Stream() for _ in range(S - 1)]
    solvers = [make_solver(st=streams[w]) for w in range(S)]
    # host-side helpers: find each worker's next instance's contraction order (into
    # the library's order cache) on another thread while the current one is solved
    preps = [make_solver(st=streams[w]) for w in range(S)]

    per_inst_ms = {}

    def one_step(step, timed):
        insts = instances(rank, world, step, per)
        # no order survives from an earlier step: every step finds its own
        P.clear_order_cache()
        t0 = time.perf_counter()
        sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sa.record(stream)
        for w in range(1, S):
            streams[w].wait_event(sa)
        parts, errors = [None] * S, []

        def worker(w):
            try:
                st_sum, h2d, d2h = {}, 0, 0
                mine = insts[w::S]
                for j, (idx, inst) in enumerate(mine):
                    th = None
                    if not args.no_pipeline and j + 1 < len(mine):
                        th = threading.Thread(target=preps[w].prepare, args=(mine[j + 1][1],))
                        th.start()
                    solvers[w].load(inst)
                    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ea.record(streams[w])
                    res = solvers[w].solve(count=True, config=False)
                    eb.record(streams[w])
                    eb.synchronize()
                    if th is not None:
                        th.join()
                    if timed:
                        per_inst_ms[idx] = ea.elapsed_time(eb)
                    for k in ("launches", "tropical_ops", "bytes_moved", "leaves", "nodes", "kernel_ms", "t_plan_s",
                              "t_device_s", "t_total_s"):
                        st_sum[k] = st_sum.get(k, 0) + res.stats[k]
                    h2d += 16 * len(inst.edges) + 8 * inst.n          # network tensor values uploaded
                    d2h += 4 * (res.stats["leaves"] + res.stats["nodes"]) + 4 + 8 * 4   # leaf maxima + result
                    if timed and step == 0 and args.check:
                        import json as _j
                        row = _j.load(open(os.path.join(ROOT, "tests", "golden", "oracle_answers.json")))["ksg_30x30_f2"][idx]
                        assert res.alpha == row["alpha"] and res.count == int(row["count"]), "mismatch with oracle"
                parts[w] = (st_sum, h2d, d2h)
            except BaseException as e:   # re-raised on the main thread
                errors.append(e)

        if S == 1:
            worker(0)
        else:
            ths = [threading.Thread(target=worker, args=(w,)) for w in range(S)]
            for th in ths:
                th.start()
            for th in ths:
                th.join()
        if errors:
            raise errors[0]
        for w in range(1, S):
            ew = torch.cuda.Event()
            ew.record(streams[w])
            stream.wait_event(ew)
        sb.record(stream)
        sb.synchronize()
        dev_ms = sa.elapsed_time(sb)          # the whole step on the device clock
        wall = time.perf_counter() - t0
        st_sum, h2d, d2h = {}, 0, 0
        for part in parts:
            for k, v in part[0].items():
                st_sum[k] = st_sum.get(k, 0) + v
            h2d += part[1]
            d2h += part[2]
        return dev_ms, wall, st_sum, h2d, d2h

    for w in range(args.warmup):
        one_step(w + 1000, False)
    clocks = Clocks(local_rank) if not args.no_clocks else None
    tot_dev, tot_wall, stats, H2D, D2H = 0.0, 0.0, {}, 0, 0
    if clocks:
        clocks.start()
    for s in range(args.steps):
        flush.fill_(s)                                    # evict L2 between timed steps
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        dev_ms, wall, st, h2d, d2h = one_step(s, True)
        torch.cuda.synchronize()
        tot_dev += dev_ms / 1000.0
        tot_wall += wall
        H2D += h2d
        D2H += d2h
        for k, v in st.items():
            stats[k] = stats.get(k, 0) + v
    ck = clocks.stop() if clocks else {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
    tot_dev, tot_wall = max_over_ranks([tot_dev, tot_wall], dist, "cuda")
    n_inst = per * args.steps * world
    # roofline: one more pass over the timed instances with every contraction launch
    # bracketed by CUDA events on this stream (not part of the timed region)
    keys = ("prof_ms", "prof_bytes", "prof_ops", "prof_launches", "prof_stream_ms", "prof_stream_bytes",
            "prof_stream_launches", "prof_scount_ms", "prof_scount_bytes", "prof_scount_launches",
            "prof_tiled_ms", "prof_tiled_ops", "prof_tiled_launches", "prof_tiled16_launches", "prof_tcount_ms",
            "prof_tcount_ops", "prof_tcount_launches")
    pb = {k: 0.0 for k in keys}
    if not args.no_profile_pass:
        prof = make_solver(profile=True)
        for s in range(args.steps):
            P.clear_order_cache()
            for _, inst in instances(rank, world, s, per):
                r = prof.solve(inst, count=True, config=False)
                for k in pb:
                    pb[k] += r.stats[k]
    peak, peak_kind = measured_peaks()
    traffic = ncu_traffic()

    def entry(kernel, ncu_name, bound, ms, work, launches, pk, unit, source, scale):
        ach = work / (ms * scale) if ms else 0.0
        return {"bound": bound, "achieved": ach, "peak": pk, "unit": unit, "frac": ach / pk if pk else None,
                "traffic": traffic.get(ncu_name), "traffic_source": TRAFFIC_SOURCE if ncu_name in traffic else None,
                "algorithmic_bytes_per_launch": (pb_bytes.get(ncu_name, 0.0) / max(launches, 1)) or None,
                "kernel": kernel, "launches": int(launches), "avg_launch_us": 1000 * ms / max(launches, 1),
                "device_ms": ms, "peak_source": source}

    pb_bytes = {"k_contract4<0, 1, 16, 0>": pb["prof_stream_bytes"], "k_contract4<4, 1, 1, 1>": pb["prof_scount_bytes"]}
    all16 = pb["prof_tiled_launches"] > 0 and pb["prof_tiled16_launches"] == pb["prof_tiled_launches"]
    alu_src = "derived: 152 SMs x 64 ALU lanes x 2.07 GHz, one add+max instruction per op"
    kernels = [
        entry("k_contract4 value-only (streaming gather, K1v)", "k_contract4<0, 1, 16, 0>", "hbm",
              pb["prof_stream_ms"], pb["prof_stream_bytes"], pb["prof_stream_launches"], peak, "GB/s",
              peak_kind + " HBM copy", 1e6),
        entry("k_contract4 counting (streaming gather, K1v, 4 count planes of residue pairs)", "k_contract4<4, 1, 1, 1>", "hbm",
              pb["prof_scount_ms"], pb["prof_scount_bytes"], pb["prof_scount_launches"], peak, "GB/s",
              peak_kind + " HBM copy", 1e6),
        entry("k_tiled value-only (register-tiled, K1t" + (", two 16-bit lanes per instruction)" if all16 else ")"),
              "k_tiled<0, 16, 1, 64, 0>" if all16 else "k_tiled<0, 16, 0, 64, 0>", "alu", pb["prof_tiled_ms"], pb["prof_tiled_ops"],
              pb["prof_tiled_launches"], ALU_PEAK_TOPS * (2 if all16 else 1), "T tropical ops/s",
              alu_src + (" x 2 lanes" if all16 else ""), 1e9),
        entry("k_tiled counting (register-tiled, K1t, 4 count planes of residue pairs)", "k_tiled<4, 1, 0, 64, 1>", "alu",
              pb["prof_tcount_ms"], pb["prof_tcount_ops"], pb["prof_tcount_launches"], ALU_PEAK_TOPS,
              "T tropical ops/s", alu_src + " (ties add modular products on top)", 1e9),
    ]
    order = sorted(range(len(kernels)), key=lambda i: -kernels[i]["device_ms"])
    dominant = dict(kernels[order[0]])
    dominant["share_of_contraction_time"] = dominant["device_ms"] / max(pb["prof_ms"], 1e-9)
    dominant["other_kernels"] = [dict(kernels[i], share_of_contraction_time=kernels[i]["device_ms"] /
                                      max(pb["prof_ms"], 1e-9)) for i in order[1:]]
    # plain tensor-network contraction (dynamic slicing until the cap holds, every
    # slice contracted, no pruning) on a bounded sample of the timed instances
    ttn = None
    if rank == 0 and args.ttn_instances > 0:
        sl = P.Solver(mode=P.MODE_SLICED, space_cap_log2=CAP, n_primes=3, batch=64, stream=stream.cuda_stream)
        t_ttn, t_bb, idxs, slices = 0.0, 0.0, [], []
        for idx, inst in instances(rank, world, 0, per)[:args.ttn_instances]:
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sl.load(inst)
            ea.record(stream)
            r = sl.solve(count=True, config=False)
            eb.record(stream)
            eb.synchronize()
            t_ttn += ea.elapsed_time(eb) / 1000.0
            t_bb += per_inst_ms.get(idx, float("nan")) / 1000.0
            idxs.append(idx)
            slices.append(r.stats["slices_log2"])
        k = len(idxs)
        ttn = {"value": t_ttn / k, "unit": "s/instance", "instances": idxs, "slices_log2": slices,
               "bbtn_same_instances": t_bb / k, "bbtn_speedup": t_ttn / t_bb if t_bb else None,
               "what": "same kernels, dynamic slicing to the same cap, all slices contracted with counts, one "
                       "instance at a time; bbtn_same_instances is each instance's own span in the timed "
                       "steps, where --streams instances share the GPU"}
        sl.close()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, sample = oracle_time(args.cpu_instances)
        cpu = {"value": v, "unit": "s/instance", "cores": 1, "kind": "oracle", "sample": sample}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": tot_dev / n_inst, "unit": "s/instance",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot_dev / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32+u64(two residues mod 2^30-d)", "data": "synthetic (seeded King's subgraphs)",
        "config": {"workload": WORKLOAD, "instances_per_step": per, "instances_total": n_inst,
                   "pipeline": "off" if args.no_pipeline else
                   "the next instance's contraction order is found on a host thread during the current solve",
                   "streams": S,
                   "timing": "CUDA events around each whole step on the main stream, which the other solver "
                             "streams join at both ends",
                   "space_cap_log2": CAP, "n_primes": 3, "l2": "256 MiB flush between steps; tensors up to 470 MB"},
        "e2e": {"value": tot_wall / n_inst, "unit": "s/instance",
                "h2d_bytes_per_step": H2D // args.steps, "d2h_bytes_per_step": D2H // args.steps},
        "gpu_launches": int(stats.get("launches", 0)),
        "tropical_gops": stats.get("tropical_ops", 0) / tot_dev / 1e9 if tot_dev else 0.0,
        "leaves_per_instance": stats.get("leaves", 0) / (per * args.steps),
        # where an instance's time goes (library counters, per instance): host planning
        # (branching, leaf plans and orders), host wall time waiting on leaf windows, and
        # the device time of those windows
        "time_split_ms": {k: 1000 * stats.get(s, 0) / (per * args.steps) for k, s in
                          (("solve_wall", "t_total_s"), ("host_plan", "t_plan_s"), ("device_wait", "t_device_s"))}
        | {"device_windows": stats.get("kernel_ms", 0) / (per * args.steps),
           "kernels": pb["prof_ms"] / (per * args.steps) if not args.no_profile_pass else None},
        "leaf_trials": args.leaf_trials,
        "plain_ttn": ttn,
        "roofline": dominant,
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


KERNEL_CASES = {
    # name: (A labels, B labels, C labels, count planes); tiled: m 0-19, k 20-39, n 40-59, batch 60+
    # streaming step: a rank-26 tensor absorbs an edge matrix, one label summed
    "stream": ([200] + list(range(100, 125)), [200, 300], list(range(100, 125)) + [300], 0),
    "stream_count": ([200] + list(range(100, 123)), [200, 300], list(range(100, 123)) + [300], 4),
    # big x big step of the 30x30 workload: batch 2, m 11, n 11, k 10
    "tiled": (list(range(0, 11)) + list(range(20, 30)) + [60, 61], list(range(20, 30)) + list(range(40, 51)) + [60, 61],
              list(range(0, 11)) + list(range(40, 51)) + [60, 61], 0),
    "tiled_count": (list(range(0, 10)) + list(range(20, 30)) + [60, 61], list(range(20, 30)) + list(range(40, 50)) + [60, 61],
                    list(range(0, 10)) + list(range(40, 50)) + [60, 61], 4),
    # a big x big step with only 4 B-only labels (64 x 16 tiles): batch 4, m 8, n 4, k 12
    "tiled_narrow": (list(range(0, 8)) + list(range(20, 32)) + [60, 61, 62, 63],
                     list(range(20, 32)) + list(range(40, 44)) + [60, 61, 62, 63],
                     list(range(0, 8)) + list(range(40, 44)) + [60, 61, 62, 63], 0),
    # the same big x big step with 16-bit lanes (value-only leaves of small-range instances)
    "tiled16": (list(range(0, 11)) + list(range(20, 30)) + [60, 61], list(range(20, 30)) + list(range(40, 51)) + [60, 61],
                list(range(0, 11)) + list(range(40, 51)) + [60, 61], -1),
}


def run_kernel_case(args):
    """One representative contraction step through the C ABI, timed with CUDA events."""
    import torch
    import paper_2602_05470_gb300 as P
    la, lb, lc, np_ = KERNEL_CASES[args.kernel_case]
    v16 = np_ < 0
    np_ = max(np_, 0)
    gen = torch.Generator(device="cuda").manual_seed(0)
    va = torch.randint(-4, 4, (1 << len(la),), dtype=torch.int32, device="cuda", generator=gen)
    vb = torch.randint(-4, 4, (1 << len(lb),), dtype=torch.int32, device="cuda", generator=gen)
    # counts in the solver's form: two residues per word (each below its 30-bit prime)
    def pair_counts(r):
        lo = torch.randint(0, 1 << 29, (np_, 1 << r), dtype=torch.int64, device="cuda", generator=gen)
        hi = torch.randint(0, 1 << 29, (np_, 1 << r), dtype=torch.int64, device="cuda", generator=gen)
        return lo | (hi << 32)

    ca = pair_counts(len(la)) if np_ else None
    cb = pair_counts(len(lb)) if np_ else None
    primes = P.prime_pairs(np_)
    out = (torch.empty(1 << len(lc), dtype=torch.int32, device="cuda"),
           torch.empty((np_, 1 << len(lc)), dtype=torch.int64, device="cuda") if np_ else None)
    def step():
        if v16:
            P.contract_values16(la, va, lb, vb, lc, out=out[0])
        else:
            P.contract(la, va, ca, lb, vb, cb, lc, primes, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.steps):
        step()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    elem = 4 + 8 * np_
    union = set(la) | set(lb)
    byts = elem * (2 ** len(la) + 2 ** len(lb) + 2 ** len(lc))
    ops = 2.0 ** len(union)
    peak, kind = measured_peaks()
    print(json.dumps({"kernel_case": args.kernel_case, "ms": ms, "algorithmic_bytes": byts, "tropical_ops": ops,
                      "gbs": byts / ms / 1e6, "hbm_frac": byts / ms / 1e6 / peak, "tops": ops / ms / 1e9,
                      "peak_gbs": peak, "peak_source": kind}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel-case", choices=sorted(KERNEL_CASES), default=None,
                    help="time one representative contraction step instead of the workload")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances-per-step", type=int, default=8)
    ap.add_argument("--cpu-instances", type=int, default=2)
    ap.add_argument("--ttn-instances", type=int, default=2,
                    help="timed instances also solved by plain sliced contraction (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="skip the nvidia-smi clock sampler")
    ap.add_argument("--no-profile-pass", action="store_true", help="skip the per-launch roofline pass")
    ap.add_argument("--check", action="store_true", help="compare step 0 with the stored oracle answers")
    ap.add_argument("--streams", type=int, default=3,
                    help="solver contexts solving a step's instances concurrently, one CUDA stream and host thread each")
    ap.add_argument("--leaf-trials", type=int, default=0,
                    help="annealing trials for the contraction order of each counting leaf (0: the root order)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="do not find the next instance's contraction order while the current one is solved")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.kernel_case:
        run_kernel_case(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
