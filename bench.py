"""Benchmark: exact ground-state counting with the branch-and-bound tensor network.

Default workload (one "step" = one pass of the whole path over a batch of
instances): unweighted MIS on random King's subgraphs, 30 x 30 grid, site filling
0.8 (32 seeded instances; a step solves 8 of them, --streams at a time, each in its
own context on its own CUDA stream), branch-and-bound contraction with a space cap
of 2^24 elements per tensor, exact degeneracy in three count planes (two residues
mod 30-bit primes per word) plus the overflow-check plane, recombined by CRT.
Every solved instance is compared with the stored oracle answer after its step,
outside the timed region.

--workload spin32: the +-J spin glass on the open 32 x 32 square lattice (no
field, 16 seeded instances), branch-and-bound at a space cap of 2^26, counts as
residues mod three 61-bit primes recombined by CRT, and one ground state from the
tropical backward pass. No oracle reaches 32 x 32, so each instance is checked by
invariants (the configuration attains the energy, the count is even, every tensor
fits the cap).

Metric: time-to-exact-count per instance (seconds, lower is better), with tropical
GOP/s, the roofline fractions of the contraction kernels and plain sliced
tensor-network contraction on the same GPU alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ksg30|spin32] [--kernel-case NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_answers.json")


def _ksg30(idx):
    import synth
    return synth.kings_subgraph(30, 0.8, seed=synth.config_seed(2, idx))


def _spin32(idx):
    import synth
    return synth.square_lattice(32, seed=synth.config_seed(3, idx))


WORKLOADS = {
    "ksg30": {
        "metric": "time-to-exact-count per instance (KSG 30x30 MIS, BBTN)",
        "name": "mis_kings_subgraph_30x30_filling0.8_cap2^24_bbtn_counting",
        "gen": _ksg30, "n_inst": 32, "cap": 24, "n_primes": 3, "wide": False, "config": False,
        "per_step": 8, "streams": 4, "golden": "ksg_30x30_f2", "order_restarts": 16,
        "dtype": "int32+u64(two residues mod 2^30-d)", "data": "synthetic (seeded King's subgraphs)",
        "l2": "256 MiB flush between steps; tensors up to 470 MB",
    },
    "spin32": {
        "metric": "time-to-exact-count per instance (+-J 32x32 spin glass, BBTN, with one ground state)",
        "name": "spin_glass_pmJ_32x32_open_nofield_cap2^26_bbtn_counting_3x61bit_primes_ground_state",
        "gen": _spin32, "n_inst": 16, "cap": 26, "n_primes": 3, "wide": True, "config": True,
        "per_step": 2, "streams": 2, "golden": None, "order_restarts": 0,
        "dtype": "int32+u64(one residue mod 2^61-c)", "data": "synthetic (seeded +-J lattices)",
        "l2": "256 MiB flush between steps; tensors up to 2.4 GB",
    },
}


def shard_indices(rank: int, world: int, step: int, per_step: int, n_inst: int = 32):
    """Workload instances of one rank in one step: the ranks of a step take
    consecutive, disjoint blocks of per_step instances (weak scaling)."""
    return [(step * per_step * world + rank * per_step + j) % n_inst for j in range(per_step)]


def max_over_ranks(values, dist, device):
    """Element-wise maximum of a list of floats over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


RATIO_FILE = os.path.join(ROOT, "profiles", "dram_traffic_kernel_cases.md")


def ncu_ratios():
    """DRAM bytes over algorithmic bytes per kernel on the bench's kernel cases (rows
    '| `kernel` | case | algorithmic MB | read MB | write MB | ratio |')."""
    out = {}
    try:
        import re
        for line in open(RATIO_FILE):
            m = re.match(r"\|\s*`([^`]+)`\s*\|.*\|\s*([\d.]+)\s*\|\s*$", line)
            if m:
                out[m.group(1)] = float(m.group(2))
    except OSError:
        pass
    return out


def measured_peaks():
    """(measured HBM copy GB/s, "measured"), else the recipe's fallback figure."""
    hbm, src = 6800.0, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        hbm, src = float(m["hbm_gbs"]), "measured"
    except Exception:
        pass
    return hbm, src


ALU_PEAK_FILE = os.path.join(ROOT, "profiles", "alu_peak_gb300.md")


def alu_peak():
    """Integer-ALU peak (T tropical ops/s at one add+max instruction per op, at the
    maximum SM clock) from the committed microbenchmark record, else the figure
    derived from 152 SMs x 64 lanes x 2.07 GHz."""
    try:
        import re
        for line in open(ALU_PEAK_FILE):
            m = re.match(r"\|\s*viaddmax_s32 at max clock\s*\|\s*([\d.]+)\s*\|", line)
            if m:
                return float(m.group(1)), "measured (profiles/alu_peak_gb300.md: independent __viaddmax_s32 chains)"
    except OSError:
        pass
    return 152 * 64 * 2.07e9 / 1e12, "derived: 152 SMs x 64 ALU lanes x 2.07 GHz"


class Clocks:
    """nvidia-smi sampler run during the timed region (samples go to a temp file)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.fh = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = tempfile.TemporaryFile(mode="w+")
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        self.fh.seek(0)
        for line in self.fh:
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
        self.fh.close()
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_time(wl, per: int, start: int = 0):
    """The CPU oracle on the host cores (one core) on a bounded sample of the
    workload: (seconds per instance, description, estimate flag). The 30x30 King's
    subgraphs are solved whole by the sparse transfer matrix. The 32 x 32 lattice
    is beyond the oracle (2^32 frontier states with big-integer counts), so the
    lattice transfer matrix is timed on 20 x 20 lattices and scaled by its cost
    L^2 2^L to L = 32: an estimate, labelled as such."""
    import oracle
    import synth
    oracle.build()
    t, idxs = 0.0, []
    for j in range(per):
        idx = (start + j) % wl["n_inst"]
        if wl is WORKLOADS["spin32"]:
            inst = synth.square_lattice(20, seed=synth.config_seed(3, idx))
            t0 = time.perf_counter()
            oracle.spin_square_tm(inst)
        else:
            inst = wl["gen"](idx)
            t0 = time.perf_counter()
            oracle.solve(inst)
        t += time.perf_counter() - t0
        idxs.append(idx)
    if wl is WORKLOADS["spin32"]:
        scale = (32 * 32 * 2.0 ** 32) / (20 * 20 * 2.0 ** 20)
        return (t / per) * scale, (f"20x20 +-J lattices (seeds of instances {idxs}), lattice transfer-matrix oracle, "
                                   f"one core, {t / per:.2f} s each, scaled by L^2 2^L to 32x32 (x{scale:.0f})"), True
    return t / per, f"instances {idxs} of the {wl['n_inst']} (whole instances, exact count)", False


def run_reference(args, rank, world, wl):
    """--impl reference: the oracle as it stands, on the host cores, rank 0 only."""
    if rank != 0:
        return
    for w in range(args.warmup):
        oracle_time(wl, 1, start=w)
    samples, desc, est = [], "", False
    for s in range(args.steps):
        v, desc, est = oracle_time(wl, 1, start=args.warmup + s)
        samples.append(v)
    value = sum(samples) / len(samples)
    line = {
        "impl": "reference", "metric": wl["metric"], "value": value, "unit": "s/instance",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * value,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": wl["data"],
        "config": {"workload": wl["name"], "instances_per_step": 1, "l2": "inputs are host-side graphs"},
        "cpu_baseline": {"value": value, "unit": "s/instance", "cores": 1, "kind": "oracle",
                         "sample": "one instance per step: " + desc, "estimate": est},
        "e2e": {"value": value, "unit": "s/instance", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def check_answers(wl, answers):
    """Compare solved instances (idx -> (optimum, count, config, sc_log2)) with the
    stored oracle answers, or, where no oracle reaches, with invariants. Raises on
    any mismatch; returns the number of instances checked."""
    if wl["golden"]:
        with open(GOLDEN) as f:
            rows = json.load(f)[wl["golden"]]
        for idx, (opt, cnt, _, sc) in answers.items():
            row = rows[idx]
            if (opt, cnt) != (row["alpha"], int(row["count"])):
                raise AssertionError(f"instance {idx}: ({opt}, {cnt}) differs from the oracle's "
                                     f"({row['alpha']}, {row['count']})")
            if sc > wl["cap"]:
                raise AssertionError(f"instance {idx}: a tensor of 2^{sc} elements exceeds the cap")
        return len(answers)
    for idx, (e2, cnt, cfg, sc) in answers.items():
        inst = wl["gen"](idx)
        e = sum(-2 * J * cfg[i] * cfg[j] for (i, j), J in zip(inst.edges, inst.J))
        if e != e2:
            raise AssertionError(f"instance {idx}: the returned configuration has 2H = {e}, not {e2}")
        if not (-2 * inst.m <= e2 < 0) or cnt <= 0 or cnt % 2:
            raise AssertionError(f"instance {idx}: E2 = {e2}, D = {cnt} violate the invariants")
        if sc > wl["cap"]:
            raise AssertionError(f"instance {idx}: a tensor of 2^{sc} elements exceeds the cap")
    return len(answers)


def run_ours(args, rank, world, local_rank, wl):
    import torch
    import paper_2602_05470_gb300 as P
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")     # 256 MiB > L2
    per = args.instances_per_step or wl["per_step"]
    cap, spin = wl["cap"], wl["golden"] is None

    # root contraction-order search: 16 restarts, every odd one from a min-fill order,
    # on the 30x30 King's subgraphs (measured: the same answers at 0.066 against 0.111
    # s/instance with the default four restarts)
    order_restarts = wl["order_restarts"] if args.order_restarts < 0 else args.order_restarts

    def make_solver(profile=False, st=None, mode=None, **kw):
        return P.Solver(mode=P.MODE_BBTN if mode is None else mode, space_cap_log2=cap, n_primes=wl["n_primes"],
                        wide_counts=wl["wide"], batch=64, profile=profile, leaf_trials=args.leaf_trials,
                        chain_fusion=not args.no_chain_fusion, order_restarts=order_restarts,
                        stream=(st or stream).cuda_stream, **kw)

    def step_instances(step):
        return [(idx, wl["gen"](idx)) for idx in shard_indices(rank, world, step, per, wl["n_inst"])]

    # S solver contexts, each on its own CUDA stream and host thread, take the
    # step's instances round-robin: one instance's many small launches leave most of
    # the GPU idle, and another instance's launches fill it
    S = max(1, args.streams or wl["streams"])
    streams = [stream] + [torch.cuda.Stream() for _ in range(S - 1)]
    solvers = [make_solver(st=streams[w]) for w in range(S)]
    # host-side helpers: find each worker's next instance's contraction order (into
    # the library's order cache) on another thread while the current one is solved
    preps = [make_solver(st=streams[w]) for w in range(S)]
    per_inst_ms = {}

    def one_step(step, timed):
        insts = step_instances(step)
        # no order survives from an earlier step: every step finds its own
        P.clear_order_cache()
        t0 = time.perf_counter()
        sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sa.record(stream)
        for w in range(1, S):
            streams[w].wait_event(sa)
        parts, errors, answers = [None] * S, [], {}

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
                    res = solvers[w].solve(count=True, config=wl["config"])
                    eb.record(streams[w])
                    eb.synchronize()
                    if th is not None:
                        th.join()
                    if timed:
                        per_inst_ms[idx] = ea.elapsed_time(eb)
                    answers[idx] = (res.energy2 if spin else res.alpha, res.count, res.config, res.stats["sc_log2"])
                    for k in ("launches", "tropical_ops", "bytes_moved", "leaves", "nodes", "kernel_ms", "t_plan_s",
                              "t_device_s", "t_total_s", "chains", "chained_steps"):
                        st_sum[k] = st_sum.get(k, 0) + res.stats[k]
                    h2d += 16 * len(inst.edges) + 8 * inst.n          # network tensor values uploaded
                    d2h += 4 * (res.stats["leaves"] + res.stats["nodes"]) + 4 + 8 * 4   # leaf maxima + result
                    if wl["config"]:
                        d2h += inst.n
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
        return dev_ms, wall, st_sum, h2d, d2h, answers

    for w in range(args.warmup):
        one_step(w + 1000, False)
    clocks = Clocks(local_rank) if not args.no_clocks else None
    tot_dev, tot_wall, stats, H2D, D2H, checked, timed_idx = 0.0, 0.0, {}, 0, 0, 0, []
    if clocks:
        clocks.start()
    for s in range(args.steps):
        flush.fill_(s)                                    # evict L2 between timed steps
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        dev_ms, wall, st, h2d, d2h, answers = one_step(s, True)
        torch.cuda.synchronize()
        tot_dev += dev_ms / 1000.0
        tot_wall += wall
        H2D += h2d
        D2H += d2h
        for k, v in st.items():
            stats[k] = stats.get(k, 0) + v
        timed_idx += sorted(answers)
        if not args.no_check:                             # outside the timed bracket
            checked += check_answers(wl, answers)
    ck = clocks.stop() if clocks else {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
    tot_dev, tot_wall = max_over_ranks([tot_dev, tot_wall], dist, "cuda")
    n_inst = per * args.steps * world
    distinct = sorted(set(timed_idx))
    # roofline: one more pass over the distinct timed instances with every contraction
    # launch bracketed by CUDA events on the solver's stream (not part of the timed region)
    keys = ("prof_ms", "prof_bytes", "prof_ops", "prof_launches", "prof_stream_ms", "prof_stream_bytes",
            "prof_stream_launches", "prof_scount_ms", "prof_scount_bytes", "prof_scount_launches",
            "prof_tiled_ms", "prof_tiled_ops", "prof_tiled_launches", "prof_tiled16_launches", "prof_tcount_ms",
            "prof_tcount_ops", "prof_tcount_launches", "prof_chain_ms", "prof_chain_bytes", "prof_chain_launches",
            "prof_tiled_bytes", "prof_tcount_bytes")
    pb = {k: 0.0 for k in keys}
    prof_idx = distinct[:args.profile_instances if args.profile_instances >= 0 else (2 if spin else 32)]
    if not args.no_profile_pass:
        prof = make_solver(profile=True)
        for idx in prof_idx:
            P.clear_order_cache()
            r = prof.solve(wl["gen"](idx), count=True, config=False)
            for k in pb:
                pb[k] += r.stats[k]
        prof.close()
    peak, peak_kind = measured_peaks()
    alu, alu_src = alu_peak()
    ratios = ncu_ratios()

    def entry(kernel, ncu_name, bound, ms, work, launches, pk, unit, source, scale, bytes_=None):
        ach = work / (ms * scale) if ms else 0.0
        per_launch = (bytes_ / max(launches, 1)) if bytes_ else None
        # traffic per launch: the kernel's measured DRAM bytes over algorithmic bytes
        # on its bench case, times this workload's algorithmic bytes per launch (the
        # same launches the achieved figure averages)
        tr, tsrc = None, None
        if per_launch and ncu_name in ratios:
            tr = ratios[ncu_name] * per_launch
            tsrc = (f"ncu DRAM bytes / algorithmic bytes = {ratios[ncu_name]:.3f} on this kernel's bench case "
                    "(profiles/dram_traffic_kernel_cases.md), times this workload's algorithmic bytes per launch")
        return {"bound": bound, "achieved": ach, "peak": pk, "unit": unit, "frac": ach / pk if pk else None,
                "traffic": tr, "traffic_source": tsrc,
                "algorithmic_bytes_per_launch": per_launch,
                "kernel": kernel, "launches": int(launches), "avg_launch_us": 1000 * ms / max(launches, 1),
                "device_ms": ms, "peak_source": source}

    def tiled_entry(kernel, ncu_name, ms, ops, byts, launches, alu_pk, alu_src):
        # Roofline of a register-tiled kernel: its arithmetic intensity (tropical ops
        # per algorithmic byte, summed over its launches) against the ridge point
        # alu_pk / HBM peak decides which resource bounds it. A counting step's output
        # carries 36 bytes per entry, so steps with short sums sit left of the ridge.
        ai = ops / byts if byts else float("inf")
        ridge = alu_pk * 1e12 / (peak * 1e9)
        if ai < ridge:
            e = entry(kernel, ncu_name, "hbm", ms, byts, launches, peak, "GB/s", peak_kind + " HBM copy", 1e6, byts)
        else:
            e = entry(kernel, ncu_name, "alu", ms, ops, launches, alu_pk, "T tropical ops/s", alu_src, 1e9)
        e.update({"intensity_ops_per_byte": ai, "ridge_ops_per_byte": ridge,
                  "alu_frac": ops / (ms * 1e9) / alu_pk if ms and alu_pk else None,
                  "hbm_frac": byts / (ms * 1e6) / peak if ms and peak else None})
        return e

    all16 = pb["prof_tiled_launches"] > 0 and pb["prof_tiled16_launches"] == pb["prof_tiled_launches"]
    planes = wl["n_primes"] + 1
    cform = "residue pairs" if not wl["wide"] else "61-bit residues"
    kernels = [
        entry("k_contract4 value-only (streaming gather, K1v)", "k_contract4<0, 1, 16, 0>", "hbm",
              pb["prof_stream_ms"], pb["prof_stream_bytes"], pb["prof_stream_launches"], peak, "GB/s",
              peak_kind + " HBM copy", 1e6, pb["prof_stream_bytes"]),
        entry(f"k_contract4 + k_outer4 counting (streaming gather K1v and its one-term form, {planes} count planes of {cform})",
              "k_contract4<4, 1, 1, 1>", "hbm", pb["prof_scount_ms"], pb["prof_scount_bytes"],
              pb["prof_scount_launches"], peak, "GB/s", peak_kind + " HBM copy", 1e6, pb["prof_scount_bytes"]),
        tiled_entry("k_tiled value-only (register-tiled, K1t" + (", two 16-bit lanes per instruction)" if all16 else ")"),
                    "k_tiled<0, 16, 1, 64, 0>" if all16 else "k_tiled<0, 16, 0, 64, 0>", pb["prof_tiled_ms"],
                    pb["prof_tiled_ops"], pb["prof_tiled_bytes"], pb["prof_tiled_launches"],
                    alu * (2 if all16 else 1), alu_src + (" x 2 lanes" if all16 else "")),
        entry("k_chain value-only (fused chains of streaming steps, K1m)", "k_chain", "hbm", pb["prof_chain_ms"],
              pb["prof_chain_bytes"], pb["prof_chain_launches"], peak, "GB/s", peak_kind + " HBM copy", 1e6,
              pb["prof_chain_bytes"]),
        tiled_entry(f"k_tiled counting (register-tiled, K1t, {planes} count planes of {cform})",
                    "k_tiled<4, 1, 0, 64, 1>", pb["prof_tcount_ms"], pb["prof_tcount_ops"], pb["prof_tcount_bytes"],
                    pb["prof_tcount_launches"], alu, alu_src + " (ties add modular products on top)"),
    ]
    order = sorted(range(len(kernels)), key=lambda i: -kernels[i]["device_ms"])
    dominant = dict(kernels[order[0]])
    dominant["share_of_contraction_time"] = dominant["device_ms"] / max(pb["prof_ms"], 1e-9)
    dominant["profiled_instances"] = prof_idx
    dominant["other_kernels"] = [dict(kernels[i], share_of_contraction_time=kernels[i]["device_ms"] /
                                      max(pb["prof_ms"], 1e-9)) for i in order[1:]]
    # plain tensor-network contraction (dynamic slicing until the cap holds, every
    # slice contracted, no pruning) against BBTN, each instance alone on the GPU,
    # on a sample spread over the timed instances
    ttn = None
    if rank == 0 and args.ttn_instances != 0:
        k = args.ttn_instances if args.ttn_instances > 0 else (2 if spin else 8)
        pick = distinct[::max(1, len(distinct) // k)][:k]
        sample = 0 if not spin else 16
        sl = make_solver(mode=P.MODE_SLICED, slice_sample=sample)
        alone = make_solver()
        prof_alone = make_solver(profile=True)
        rows = []
        for idx in pick:
            inst = wl["gen"](idx)
            times = []
            for sv in (sl, alone):
                P.clear_order_cache()
                sv.load(inst)
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ea.record(stream)
                r = sv.solve(count=True, config=wl["config"] and sv is alone)
                eb.record(stream)
                eb.synchronize()
                times.append((ea.elapsed_time(eb) / 1000.0, r))
            (t_sl, r_sl), (t_bb, r_bb) = times
            full = 2 ** r_sl.stats["slices_log2"]
            ran = r_sl.stats["slices_run"]
            if ran == full and (r_sl.energy2 if spin else r_sl.alpha, r_sl.count) != (
                    r_bb.energy2 if spin else r_bb.alpha, r_bb.count):
                raise AssertionError(f"instance {idx}: sliced and BBTN answers differ")
            # the same solve once more with every launch timed: the summed kernel time
            # against the solve's span bounds what fewer or persistent launches could save
            P.clear_order_cache()
            rk = prof_alone.solve(inst, count=True, config=wl["config"])
            kern = rk.stats["prof_ms"] / 1000.0
            rows.append({"instance": idx, "slices_log2": r_sl.stats["slices_log2"], "slices_run": ran,
                         "ttn_s": t_sl * full / ran, "bbtn_alone_s": t_bb,
                         "speedup": t_sl * full / ran / t_bb, "bbtn_kernels_s": kern,
                         "device_idle_share": max(0.0, 1.0 - kern / t_bb) if t_bb else None,
                         "launches": rk.stats["launches"]})
        sl.close()
        alone.close()
        prof_alone.close()
        import math
        ttn = {"unit": "s/instance", "instances": rows,
               "ttn_mean_s": sum(r["ttn_s"] for r in rows) / len(rows),
               "bbtn_alone_mean_s": sum(r["bbtn_alone_s"] for r in rows) / len(rows),
               "speedup_geomean": math.exp(sum(math.log(r["speedup"]) for r in rows) / len(rows)),
               "device_idle_share_mean": sum(r["device_idle_share"] or 0.0 for r in rows) / len(rows),
               "estimate": bool(sample),
               "what": "each instance alone on the GPU, its contraction order found inside the timed call: plain "
                       "TTN = the same kernels with dynamic slicing to the same cap, every slice contracted with "
                       "counts, no pruning" + (f" (estimate: the first {sample} slices timed and scaled by "
                                               "2^slices_log2 / slices_run, the paper's own estimate)" if sample else "")
                       + "; BBTN alone = the same solve as in the timed steps without other instances sharing the GPU"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, sample_desc, est = oracle_time(wl, args.cpu_instances)
        cpu = {"value": v, "unit": "s/instance", "cores": 1, "kind": "oracle", "sample": sample_desc, "estimate": est}
    if rank != 0:
        return
    line = {
        "metric": wl["metric"], "value": tot_dev / n_inst, "unit": "s/instance",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot_dev / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": wl["dtype"], "data": wl["data"],
        "config": {"workload": wl["name"], "instances_per_step": per, "instances_total": n_inst,
                   "pipeline": "off" if args.no_pipeline else
                   "the next instance's contraction order is found on a host thread during the current solve",
                   "streams": S,
                   "timing": "CUDA events around each whole step on the main stream, which the other solver "
                             "streams join at both ends",
                   "space_cap_log2": cap, "n_primes": wl["n_primes"], "l2": wl["l2"]},
        "checked": (not args.no_check) and checked == len(timed_idx),
        "checked_instances": checked,
        "check": ("every timed instance against the stored oracle answer (optimum and exact count), after its "
                  "step" if wl["golden"] else "every timed instance by invariants (configuration energy, even "
                  "count, cap), after its step") if not args.no_check else "off",
        "e2e": {"value": tot_wall / n_inst, "unit": "s/instance",
                "h2d_bytes_per_step": H2D // args.steps, "d2h_bytes_per_step": D2H // args.steps},
        "gpu_launches": int(stats.get("launches", 0)),
        "tropical_gops": stats.get("tropical_ops", 0) / tot_dev / 1e9 if tot_dev else 0.0,
        "leaves_per_instance": stats.get("leaves", 0) / (per * args.steps),
        "nodes_per_instance": stats.get("nodes", 0) / (per * args.steps),
        "chain_fusion": {"on": not args.no_chain_fusion,
                         "chains_per_instance": stats.get("chains", 0) / (per * args.steps),
                         "steps_replaced_per_instance": stats.get("chained_steps", 0) / (per * args.steps)},
        # where an instance's time goes (library counters, per instance): host planning
        # (branching, leaf plans and orders), host wall time waiting on leaf windows, and
        # the device time of those windows
        "time_split_ms": {k: 1000 * stats.get(s, 0) / (per * args.steps) for k, s in
                          (("solve_wall", "t_total_s"), ("host_plan", "t_plan_s"), ("device_wait", "t_device_s"))}
        | {"device_windows": stats.get("kernel_ms", 0) / (per * args.steps),
           "kernels": pb["prof_ms"] / max(len(prof_idx), 1) if not args.no_profile_pass else None},
        "single_instance_s": ttn["bbtn_alone_mean_s"] if ttn else None,
        "leaf_trials": args.leaf_trials,
        "order_restarts": order_restarts,
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


def run_alu_peak(args):
    """Integer-ALU peak: independent dependency chains of the add+max instruction
    the tiled kernel issues per tropical multiply-add (__viaddmax_s32), and of its
    two-lane 16-bit form, on 152 x 8 blocks of 256 threads, timed with CUDA events;
    the SM clock is sampled meanwhile and the rate is also given at the maximum clock."""
    import torch
    import paper_2602_05470_gb300 as P
    torch.cuda.set_device(0)
    out = {"kernel_case": "alu_peak"}
    clocks = Clocks(0)
    for which, name in ((0, "viaddmax_s32"), (1, "viaddmax_s16x2")):
        P.bench_alu(which, 152 * 8, 256, 4096)                      # warm-up
        clocks.start()
        best = None
        for _ in range(max(args.steps, 3)):
            ops, ms = P.bench_alu(which, 152 * 8, 256, 1 << 16)
            rate = ops / ms / 1e9
            best = rate if best is None else max(best, rate)
        ck = clocks.stop()
        at_max = best * ck["sm_max_mhz"] / ck["sm_mhz"] if ck.get("sm_mhz") else None
        out[name] = {"tops": best, "unit": "T tropical ops/s", "sm_mhz": ck.get("sm_mhz"),
                     "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons"), "tops_at_max_clock": at_max,
                     "per_sm_per_clock": (at_max or best) * 1e12 / 152 / ((ck.get("sm_max_mhz") or 2070) * 1e6)}
    print(json.dumps(out), flush=True)


PERMUTE_CASES = {
    # name: (rank, permutation (output bit q <- input bit perm[q]), count planes)
    "permute_tma": (26, list(range(13, 26)) + list(range(13)), 0),          # 8192 x 8192 transpose
    "permute_tma_count": (24, list(range(12, 24)) + list(range(12)), 4),    # with four count planes
    "permute_gather": (26, [1, 0] + list(range(2, 26)), 0),                 # a single-bit run at bit 0: K2
}


CHAIN_CASES = {
    # name: (rank of A, steps [(B labels, output labels)]) -- a frontier tensor absorbing
    # four edge matrices (two of them adding and summing a label), as on the workload
    "chain": (24, [([3, 17], list(range(24))), ([17, 30], list(range(24)) + [30]),
                   ([5, 30], [x for x in range(24) if x != 5] + [30]), ([9, 21], [x for x in range(24) if x != 5] + [30])]),
}


def run_chain_case(args):
    """bbtn_contract_chain on a rank-24 tensor, timed with CUDA events: algorithmic
    bytes = A read once and the result written once."""
    import torch
    import paper_2602_05470_gb300 as P
    ra, steps = CHAIN_CASES[args.kernel_case]
    va = torch.randint(-4, 4, (1 << ra,), dtype=torch.int32, device="cuda")
    dsteps = [(lb, torch.randint(-2, 3, (1 << len(lb),), dtype=torch.int32, device="cuda"), lc) for lb, lc in steps]
    rc = len(steps[-1][1])
    out = torch.empty(1 << rc, dtype=torch.int32, device="cuda")
    for _ in range(max(args.warmup, 1)):
        P.contract_chain(list(range(ra)), va, dsteps, out=out)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.steps):
        P.contract_chain(list(range(ra)), va, dsteps, out=out)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    byts = 4 * ((1 << ra) + (1 << rc))
    peak, kind = measured_peaks()
    print(json.dumps({"kernel_case": args.kernel_case, "ms": ms, "algorithmic_bytes": byts, "gbs": byts / ms / 1e6,
                      "hbm_frac": byts / ms / 1e6 / peak, "peak_gbs": peak, "peak_source": kind,
                      "unfused_steps": len(steps)}), flush=True)


def run_permute_case(args):
    """bbtn_permute on a large tensor, timed with CUDA events: algorithmic bytes =
    every plane read once and written once."""
    import torch
    import paper_2602_05470_gb300 as P
    r, perm, np_ = PERMUTE_CASES[args.kernel_case]
    vin = torch.randint(-4, 4, (1 << r,), dtype=torch.int32, device="cuda")
    cin = torch.randint(0, 1 << 29, (np_, 1 << r), dtype=torch.int64, device="cuda") if np_ else None
    tma = P._lib.load().bbtn_permute_uses_tma(r, P.i32_array(perm), vin.data_ptr(),
                                              cin.data_ptr() if np_ else None, vin.data_ptr(),
                                              cin.data_ptr() if np_ else None, np_)
    for _ in range(max(args.warmup, 1)):
        P.permute(perm, vin, cin)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ms = []
    for _ in range(args.steps):
        ev[0].record()
        P.permute(perm, vin, cin)
        ev[1].record()
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
    t = sorted(ms)[len(ms) // 2]
    byts = 2 * (4 + 8 * np_) * (1 << r)
    peak, kind = measured_peaks()
    print(json.dumps({"kernel_case": args.kernel_case, "tma": bool(tma), "ms_median": t, "algorithmic_bytes": byts,
                      "gbs": byts / t / 1e6, "hbm_frac": byts / t / 1e6 / peak, "peak_gbs": peak,
                      "peak_source": kind}), flush=True)


def run_kernel_case(args):
    """One representative contraction step through the C ABI, timed with CUDA events."""
    import torch
    import paper_2602_05470_gb300 as P
    if args.kernel_case == "alu_peak":
        return run_alu_peak(args)
    if args.kernel_case in PERMUTE_CASES:
        return run_permute_case(args)
    if args.kernel_case in CHAIN_CASES:
        return run_chain_case(args)
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


def run_scorer(args):
    """The learned branch scorer against the plain heuristic (its fallback and judge):
    lookahead training rows from args.scorer_graphs seeded King's subgraphs of 20x20 to
    24x24 (caps 2^12 to 2^14, host searches in parallel processes, spawned before the
    first GPU call), training on the GPU by the library's forward / backward / Adam
    kernels, then held-out 30x30 King's subgraphs at cap 2^16 solved with and without
    the scorer: leaves of the search, time-to-exact-count (CUDA events around each
    solve), identical answers."""
    import numpy as np
    from paper_2602_05470_gb300 import gnn
    import synth
    specs = [("mis", 20 + i % 5, synth.config_seed(4, 2000 + i), 12 + i % 3, 200, 8, 8)
             for i in range(args.scorer_graphs)]
    t0 = time.perf_counter()
    data = [(inst, rows) for inst, rows in gnn.branch_dataset(specs) if rows]
    t_rows = time.perf_counter() - t0
    import torch
    import paper_2602_05470_gb300 as P
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    model = gnn.GNN(seed=3)
    held = data[-8:]
    before = gnn.top1_agreement(model, held)
    t0 = time.perf_counter()
    losses = gnn.train(model, data[:-8], epochs=args.scorer_epochs, lr=2e-3, rng=np.random.default_rng(0))
    t_train = time.perf_counter() - t0
    after = gnn.top1_agreement(model, held)
    rows = []
    for idx in range(args.scorer_instances):
        inst = synth.kings_subgraph(30, 0.8, seed=synth.config_seed(4, 3000 + idx))
        row = {"instance": idx}
        for use in (False, True):
            s = P.Solver(mode=P.MODE_BBTN, space_cap_log2=16, use_gnn=use, stream=stream.cuda_stream)
            if use:
                s.set_gnn(branch=model)
            leaves = s.analyze(inst)["bb_leaves"]
            P.clear_order_cache()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            r = s.solve(inst, count=True, config=False)
            eb.record(stream)
            eb.synchronize()
            key = "scorer" if use else "heuristic"
            row[key] = {"leaves_host_search": leaves, "nodes": r.stats["nodes"], "s": ea.elapsed_time(eb) / 1000,
                        "answer": [r.alpha, str(r.count)]}
            s.close()
        if row["scorer"]["answer"] != row["heuristic"]["answer"]:
            raise AssertionError(f"instance {idx}: the scorer changed the answer")
        rows.append(row)
    import math
    gm = lambda k: math.exp(sum(math.log(r["scorer"][k] / r["heuristic"][k]) for r in rows) / len(rows))
    print(json.dumps({
        "kind": "learned branch scorer vs heuristic",
        "train": {"graphs": len(data) - 8, "graphs_requested": args.scorer_graphs, "sizes": "20x20..24x24 King's subgraphs",
                  "caps_log2": [12, 13, 14], "rows": sum(len(r) for _, r in data[:-8]), "epochs": args.scorer_epochs,
                  "rows_host_s": t_rows, "train_gpu_s": t_train, "loss_first_last": [losses[0], losses[-1]],
                  "top1_agreement_held_out": [before, after]},
        "eval": {"instances": rows, "workload": "30x30 King's subgraphs (filling 0.8), cap 2^16, exact count",
                 "leaves_ratio_geomean": gm("leaves_host_search"), "time_ratio_geomean": gm("s")},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["scorer30"], default="ksg30",
                    help="scorer30: train the learned branch scorer and compare it with the heuristic")
    ap.add_argument("--scorer-graphs", type=int, default=200)
    ap.add_argument("--scorer-epochs", type=int, default=20)
    ap.add_argument("--scorer-instances", type=int, default=6)
    ap.add_argument("--kernel-case", choices=sorted(KERNEL_CASES) + sorted(PERMUTE_CASES) + sorted(CHAIN_CASES) +
                    ["alu_peak"], default=None,
                    help="time one representative contraction step (or the integer-ALU peak) instead of the workload")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances-per-step", type=int, default=0, help="0: the workload's default")
    ap.add_argument("--cpu-instances", type=int, default=2)
    ap.add_argument("--ttn-instances", type=int, default=-1,
                    help="timed instances also solved alone by plain sliced contraction and by BBTN "
                         "(-1: 8 for ksg30, 2 for spin32; 0: skip)")
    ap.add_argument("--profile-instances", type=int, default=-1,
                    help="distinct timed instances in the per-launch roofline pass (-1: 32 for ksg30, 2 for spin32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="skip the nvidia-smi clock sampler")
    ap.add_argument("--no-profile-pass", action="store_true", help="skip the per-launch roofline pass")
    ap.add_argument("--no-check", action="store_true", help="skip the check of every timed instance's answer")
    ap.add_argument("--streams", type=int, default=0,
                    help="solver contexts solving a step's instances concurrently, one CUDA stream and host thread "
                         "each (0: the workload's default, 4 for ksg30, 2 for spin32)")
    ap.add_argument("--leaf-trials", type=int, default=0,
                    help="annealing trials for the contraction order of each counting leaf (0: the root order)")
    ap.add_argument("--order-restarts", type=int, default=-1,
                    help="restarts of the root contraction-order search, every odd one from a min-fill "
                         "elimination order (0: the library default, four restarts; -1: the workload's "
                         "setting, 16 for ksg30 and 0 for spin32)")
    ap.add_argument("--no-chain-fusion", action="store_true",
                    help="run every value-only step as its own launch (no fused chains; same results)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="do not find the next instance's contraction order while the current one is solved")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.workload == "scorer30":
        return run_scorer(args)
    wl = WORKLOADS[args.workload]
    if args.kernel_case:
        run_kernel_case(args)
    elif args.impl == "reference":
        run_reference(args, rank, world, wl)
    else:
        run_ours(args, rank, world, local_rank, wl)


if __name__ == "__main__":
    main()
