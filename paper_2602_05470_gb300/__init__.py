"""GB300 (sm_103a) Branch-and-Bound Tensor Networks -- Python binding.

Wang, Gao, Zhang, Pan, Liu, "Branch-and-Bound Tensor Networks for Exact
Ground-State Characterization" (arXiv:2602.05470).

Thin layer over the C ABI of ``libbbtn.so`` (include/bbtn.h): it marshals
arguments and uses PyTorch only for device memory and streams. Every step of the
contraction path runs in the library's CUDA kernels; if the library is missing
the import of a compute function fails (there is no CPU fallback).

Device-level calls (one contraction step, permute, aggregate, backward):
    contract, permute, aggregate, contract_backward
Solver (host-driven plain / sliced / branch-and-bound contraction):
    Solver(opts...).solve(instance) -> Result
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

from . import _lib
from ._lib import (BBTNError, FINITE_MIN, MAX_PRIMES, MODE_BBTN, MODE_PLAIN, MODE_SLICED, NEG,  # noqa: F401
                   Opts, Stats, check, i32_array, u64_array)

__all__ = ["clear_order_cache", "primes", "crt", "contract", "contract_values16", "permute", "aggregate", "contract_backward", "Solver", "Result",
           "BBTNError", "NEG", "FINITE_MIN", "MODE_PLAIN", "MODE_SLICED", "MODE_BBTN", "lib_path"]


def clear_order_cache():
    """Empty the library's process-wide cache of root contraction orders."""
    check(_lib.load().bbtn_clear_order_cache())


def lib_path() -> str:
    return _lib.LIB_PATH


def primes(n: int = 3):
    """The first n count primes p_t = 2^61 - c_t of the library."""
    lib = _lib.load()
    buf = (C.c_uint64 * max(n, 1))()
    check(lib.bbtn_primes(n, buf))
    return [int(buf[i]) for i in range(n)]


def prime_pairs(n: int = 3):
    """The first n pair moduli q1 << 32 | q0 (primes q = 2^30 - d): a count plane with
    such a modulus holds two residues per word, mod q0 (low half) and q1 (high half)."""
    lib = _lib.load()
    buf = (C.c_uint64 * max(n, 1))()
    check(lib.bbtn_prime_pairs(n, buf))
    return [int(buf[i]) for i in range(n)]


def crt(residues, moduli) -> int:
    """The integer in [0, prod moduli) with the given residues (host Garner recombination)."""
    lib = _lib.load()
    k = len(residues)
    r, p, need = u64_array(residues), u64_array(moduli), C.c_size_t()
    check(lib.bbtn_crt_decimal(k, r, p, None, 0, C.byref(need)))
    buf = C.create_string_buffer(need.value)
    check(lib.bbtn_crt_decimal(k, r, p, buf, need.value, C.byref(need)))
    return int(buf.value.decode())


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


def contract(la, va, ca, lb, vb, cb, lc, primes_, out=None, stream=None):
    """One counting-tropical pairwise contraction on the device.

    va/vb: int32 CUDA tensors of 2^r values; ca/cb: uint64-as-int64 CUDA tensors of
    shape [np, 2^r] or None (unit counts). lb=None: single-operand reduction.
    Returns (vc, cc) CUDA tensors (cc None when np == 0).
    """
    import torch
    lib = _lib.load()
    np_ = len(primes_)
    rc = len(lc)
    dev = va.device
    if out is None:
        vc = torch.empty(1 << rc, dtype=torch.int32, device=dev)
        cc = torch.empty((np_, 1 << rc), dtype=torch.int64, device=dev) if np_ else None
    else:
        vc, cc = out
    rb = 0 if lb is None else len(lb)
    check(lib.bbtn_contract(len(la), i32_array(la), _ptr(va), _ptr(ca),
                            rb, i32_array(lb or []), _ptr(vb), _ptr(cb),
                            rc, i32_array(lc), _ptr(vc), _ptr(cc), np_, u64_array(primes_),
                            _stream(stream)))
    return vc, cc


def contract_values16(la, va, lb, vb, lc, out=None, stream=None):
    """Value-only contraction with 16-bit lanes for operands whose finite values lie
    in (-2^12, 2^12); feasible outputs equal contract()'s, infeasible ones are below
    FINITE_MIN. lb=None: single-operand reduction."""
    import torch
    lib = _lib.load()
    vc = torch.empty(1 << len(lc), dtype=torch.int32, device=va.device) if out is None else out
    rb = 0 if lb is None else len(lb)
    check(lib.bbtn_contract_values16(len(la), i32_array(la), _ptr(va), rb, i32_array(lb or []), _ptr(vb),
                                     len(lc), i32_array(lc), _ptr(vc), _stream(stream)))
    return vc


def contract_chain(la, va, steps, out=None, stream=None):
    """Value-only chain of steps in one pass: steps = [(lb, vb, lc), ...] (vb a
    device int32 tensor of 2^len(lb) values, lc the step's output labels); returns
    the last step's values (device int32[2^len(lc_last)])."""
    import torch
    lib = _lib.load()
    L = len(steps)
    rb = [len(lb) for lb, _, _ in steps]
    rc = [len(lc) for _, _, lc in steps]
    lbs = [x for lb, _, _ in steps for x in lb]
    lcs = [x for _, _, lc in steps for x in lc]
    vbs = (C.c_void_p * max(L, 1))(*[vb.data_ptr() for _, vb, _ in steps])
    vc = torch.empty(1 << rc[-1], dtype=torch.int32, device=va.device) if out is None else out
    check(lib.bbtn_contract_chain(len(la), i32_array(la), _ptr(va), L, i32_array(rb), i32_array(lbs), vbs,
                                  i32_array(rc), i32_array(lcs), _ptr(vc), _stream(stream)))
    return vc


def permute(perm, vin, cin, stream=None):
    """out bit q <- in bit perm[q] for the value plane and the count planes."""
    import torch
    lib = _lib.load()
    r = len(perm)
    vout = torch.empty_like(vin)
    cout = torch.empty_like(cin) if cin is not None else None
    np_ = 0 if cin is None else cin.shape[0]
    check(lib.bbtn_permute(r, i32_array(perm), _ptr(vin), _ptr(cin), _ptr(vout), _ptr(cout), np_,
                           _stream(stream)))
    return vout, cout


def aggregate(vals, cnts, primes_, stream=None):
    """Counting-sum over n scalars: (max value, sum of counts at the max)."""
    import torch
    lib = _lib.load()
    np_ = len(primes_)
    ov = torch.empty(1, dtype=torch.int32, device=vals.device)
    oc = torch.empty(max(np_, 1), dtype=torch.int64, device=vals.device)
    check(lib.bbtn_aggregate(vals.numel(), _ptr(vals), _ptr(cnts), np_, u64_array(primes_), _ptr(ov),
                             _ptr(oc), _stream(stream)))
    return ov, oc[:np_]


def contract_backward(la, va, lb, vb, lc, vc, sel_o, stream=None):
    """Tropical arg-max of one step: linear indices of A and B attaining C[sel_o]."""
    import torch
    lib = _lib.load()
    q = sel_o.numel()
    sa = torch.empty(q, dtype=torch.int64, device=va.device)
    sb = torch.empty(q, dtype=torch.int64, device=va.device)
    rb = 0 if lb is None else len(lb)
    check(lib.bbtn_contract_backward(len(la), i32_array(la), _ptr(va), rb, i32_array(lb or []), _ptr(vb),
                                     len(lc), i32_array(lc), _ptr(vc), q, _ptr(sel_o), _ptr(sa), _ptr(sb),
                                     _stream(stream)))
    return sa, sb


def bench_alu(which: int, blocks: int, threads: int, iters: int, stream=None):
    """Integer-ALU microbenchmark (0: __viaddmax_s32, 1: __viaddmax_s16x2):
    (tropical multiply-adds executed, kernel milliseconds)."""
    lib = _lib.load()
    ops, ms = C.c_double(), C.c_float()
    check(lib.bbtn_bench_alu(which, blocks, threads, iters, C.byref(ops), C.byref(ms), _stream(stream)))
    return ops.value, ms.value


@dataclasses.dataclass
class Result:
    kind: str
    energy2: Optional[int]        # 2 H* (spin glass)
    alpha: Optional[int]          # MWIS optimum
    count: Optional[int]          # exact degeneracy (CRT)
    residues: list
    primes: list
    config: Optional[list]
    stats: dict


class Solver:
    """Owns one library context (a CUDA stream + device arena). Keyword options
    mirror `bbtn_opts` in include/bbtn.h; among them `n_primes` count planes (two
    residues mod 30-bit primes per word, or one mod a 61-bit prime with
    `wide_counts=True`), `leaf_trials` (own contraction orders for counting
    leaves, off by default) and `order_restarts` (restarts of the root order search,
    every odd one from a min-fill order; 0: the default four). Contexts on different streams may solve concurrently
    from different host threads."""

    def __init__(self, mode: int = MODE_BBTN, space_cap_log2: int = 24, n_primes: int = 3, seed: int = 1,
                 sa_iters: int = 20, region_size: int = 8, batch: int = 64, use_gnn: bool = False,
                 count_check: int = -1, use_symmetry: bool = True, max_slices_log2: int = 30,
                 profile: bool = False, branch_lookahead: int = 1, leaf_trials: int = 0, autotune: bool = False,
                 wide_counts: bool = False, slice_sample: int = 0, arena_budget_mb: int = 0,
                 chain_fusion: bool = True, order_restarts: int = 0, stream=None, workspace=None):
        lib = _lib.load()
        o = Opts()
        lib.bbtn_default_opts(C.byref(o))
        o.mode, o.space_cap_log2, o.n_primes, o.seed = mode, space_cap_log2, n_primes, seed
        o.sa_iters, o.region_size, o.batch, o.use_gnn = sa_iters, region_size, batch, int(use_gnn)
        o.count_check, o.use_symmetry = count_check, int(use_symmetry)
        o.max_slices_log2, o.profile, o.branch_lookahead = max_slices_log2, int(profile), branch_lookahead
        o.leaf_trials, o.autotune, o.wide_counts = leaf_trials, int(autotune), int(wide_counts)
        o.slice_sample, o.arena_budget_mb = int(slice_sample), int(arena_budget_mb)
        o.no_chain_fusion = int(not chain_fusion)
        o.order_restarts = int(order_restarts)
        self._ctx = C.c_void_p()
        check(lib.bbtn_create(C.byref(o), C.byref(self._ctx)))
        if stream is not None:
            check(lib.bbtn_set_stream(self._ctx, int(stream)))
        self._ws = workspace
        if workspace is not None:
            check(lib.bbtn_set_workspace(self._ctx, workspace.data_ptr(), workspace.numel() * workspace.element_size()))

    def close(self):
        if self._ctx:
            _lib.load().bbtn_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gnn(self, branch=None, value=None):
        """Attach learned scorers (paper_2602_05470_gb300.gnn.GNN), used when use_gnn is set:
        `branch` picks the seed of each branching region, `value` predicts an optimum."""
        check(_lib.load().bbtn_set_gnn(self._ctx, branch._h if branch is not None else None,
                                       value._h if value is not None else None))
        self._gnn = (branch, value)

    def branch_samples(self, inst, max_rows: int, lookahead: int):
        """Host-side search rows for the branch scorer: (fx, score, gamma), each max_rows' x n."""
        import numpy as np
        self.load(inst)
        n = inst.n
        fx = np.zeros((max_rows, n), dtype=np.int8)
        sc = np.zeros((max_rows, n), dtype=np.float32)
        ga = np.zeros((max_rows, n), dtype=np.float32)
        rows = C.c_int()
        f32 = C.POINTER(C.c_float)
        check(_lib.load().bbtn_branch_samples(self._ctx, max_rows, lookahead, fx.ctypes.data_as(_lib._i8p),
                                              sc.ctypes.data_as(f32), ga.ctypes.data_as(f32), C.byref(rows)))
        r = rows.value
        return fx[:r], sc[:r], ga[:r]

    def prepare(self, inst):
        """Host-only: find the instance's root contraction order into the library's
        order cache (a later solve of the same structure reuses it). Releases the GIL
        while it runs, so it can overlap another context's solve."""
        self.load(inst)
        check(_lib.load().bbtn_prepare(self._ctx))

    def search_leaves(self, inst, max_leaves: int = 4096):
        """Host-side search: (fixings of the first max_leaves leaves as an int8 array
        leaves' x n, -1 free / 0 / 1; number of leaves of the whole search)."""
        import numpy as np
        self.load(inst)
        fx = np.zeros((max_leaves, inst.n), dtype=np.int8)
        total = C.c_int64()
        check(_lib.load().bbtn_search_leaves(self._ctx, max_leaves, fx.ctypes.data_as(_lib._i8p), C.byref(total)))
        return fx[:min(max_leaves, total.value)], total.value

    def load(self, inst):
        """inst: object with kind ('spin'|'mwis'), n, edges, J, h2, w (e.g. synth.Instance)."""
        lib = _lib.load()
        flat = [v for e in inst.edges for v in e]
        if inst.kind == "spin":
            h2 = getattr(inst, "h2", None)
            check(lib.bbtn_load_spin_glass(self._ctx, inst.n, len(inst.edges), i32_array(flat),
                                           i32_array(inst.J), i32_array(h2) if h2 is not None else None))
        else:
            w = getattr(inst, "w", None)
            check(lib.bbtn_load_mwis(self._ctx, inst.n, len(inst.edges), i32_array(flat),
                                     i32_array(w) if w is not None else None))
        self._kind, self._n = inst.kind, inst.n

    def load_file(self, path: str, kind: str, n: int):
        check(_lib.load().bbtn_load_file(self._ctx, path.encode()))
        self._kind, self._n = kind, n

    def analyze(self, inst=None, dump_path: Optional[str] = None) -> dict:
        """Host-only planning summary (order, slicing, step list); needs no GPU."""
        if inst is not None:
            self.load(inst)
        info = _lib.PlanInfo()
        check(_lib.load().bbtn_analyze(self._ctx, C.byref(info), dump_path.encode() if dump_path else None))
        return info.as_dict()

    def solve(self, inst=None, count: bool = True, config: bool = False) -> Result:
        lib = _lib.load()
        if inst is not None:
            self.load(inst)
        check(lib.bbtn_solve(self._ctx, int(count), int(config)))
        e = C.c_int64()
        check(lib.bbtn_get_energy(self._ctx, C.byref(e)))
        res, prs, k = (C.c_uint64 * (2 * MAX_PRIMES))(), (C.c_uint64 * (2 * MAX_PRIMES))(), C.c_int()
        check(lib.bbtn_get_count_residues(self._ctx, res, prs, C.byref(k)))
        cnt = None
        if count:
            need = C.c_size_t()
            check(lib.bbtn_get_count_dec(self._ctx, None, 0, C.byref(need)))
            buf = C.create_string_buffer(need.value)
            check(lib.bbtn_get_count_dec(self._ctx, buf, need.value, C.byref(need)))
            cnt = int(buf.value.decode())
        cfg = None
        if config:
            arr = (C.c_int8 * self._n)()
            check(lib.bbtn_get_config(self._ctx, arr))
            cfg = [int(arr[i]) for i in range(self._n)]
        st = Stats()
        check(lib.bbtn_get_stats(self._ctx, C.byref(st)))
        spin = self._kind == "spin"
        return Result(self._kind, e.value if spin else None, None if spin else e.value, cnt,
                      [int(res[i]) for i in range(k.value)], [int(prs[i]) for i in range(k.value)], cfg,
                      st.as_dict())

    # ------------------------------------------------------------ branch sharding

    def shard_values(self, rank: int, world: int, count: bool = True, inst=None) -> int:
        """Step 1 of branch sharding (bbtn_shard_values): value-only contraction of
        this rank's leaves; returns the largest leaf maximum (max-plus convention)."""
        if inst is not None:
            self.load(inst)
        m = C.c_int64()
        check(_lib.load().bbtn_shard_values(self._ctx, rank, world, int(count), C.byref(m)))
        return m.value

    def shard_counts(self, global_max: int, config: bool = False):
        """Step 3 (bbtn_shard_counts): this rank's part of the counting sum as
        (value, planes, moduli, n_crt_planes, config or None)."""
        lib = _lib.load()
        v, np_, ncrt, have = C.c_int32(), C.c_int(), C.c_int(), C.c_int()
        planes, moduli = (C.c_uint64 * (MAX_PRIMES + 1))(), (C.c_uint64 * (MAX_PRIMES + 1))()
        cfg = (C.c_int8 * self._n)()
        check(lib.bbtn_shard_counts(self._ctx, int(global_max), int(config), C.byref(v), planes, moduli,
                                    C.byref(np_), C.byref(ncrt), cfg, C.byref(have)))
        k = np_.value
        x = [int(cfg[i]) for i in range(self._n)] if (config and have.value) else None
        return v.value, [int(planes[t]) for t in range(k)], [int(moduli[t]) for t in range(k)], ncrt.value, x


def count_decimal(planes, moduli, n_crt_planes: int) -> int:
    """Exact count from count-plane words (bbtn_count_decimal: CRT and overflow check)."""
    lib = _lib.load()
    need = C.c_size_t()
    check(lib.bbtn_count_decimal(len(planes), n_crt_planes, u64_array(planes), u64_array(moduli), None, 0,
                                 C.byref(need)))
    buf = C.create_string_buffer(need.value)
    check(lib.bbtn_count_decimal(len(planes), n_crt_planes, u64_array(planes), u64_array(moduli), buf, need.value,
                                 C.byref(need)))
    return int(buf.value.decode())


def combine_shards(parts, stream=None):
    """Counting sum of the ranks' partial results [(value, planes, moduli, n_crt), ...]
    on the device (bbtn_aggregate), then the exact count: (value, count)."""
    import numpy as np
    import torch
    moduli, ncrt = parts[0][2], parts[0][3]
    vals = torch.tensor([p[0] for p in parts], dtype=torch.int32, device="cuda")
    if not moduli:
        ov, _ = aggregate(vals, None, [], stream=stream)
        return int(ov.cpu()[0]), None
    words = np.array([p[1] for p in parts], dtype=np.uint64).T.copy()        # [np][world]
    cnts = torch.from_numpy(words.view(np.int64)).cuda()
    ov, oc = aggregate(vals, cnts, moduli, stream=stream)
    torch.cuda.current_stream().synchronize()
    v = int(ov.cpu()[0])
    planes = [int(x) for x in oc.cpu().numpy().view(np.uint64)]
    return v, count_decimal(planes, moduli, ncrt)


def solve_sharded(solver, inst, rank: int, world: int, dist=None, count: bool = True, config: bool = False):
    """One rank's part of a branch-sharded solve: every rank calls this with the same
    instance and options. The ranks exchange the largest leaf maximum (all-reduce)
    and their partial counting sums (all-gather) through torch.distributed `dist`
    (not needed when world == 1), combine them on the device, and return the
    instance's (optimum, count, configuration or None); the configuration comes from
    the rank holding an optimal leaf and is shared with the others."""
    import torch
    local = solver.shard_values(rank, world, count, inst=inst)
    g = torch.tensor([local], dtype=torch.int64, device="cuda")
    if dist is not None and world > 1:
        dist.all_reduce(g, op=dist.ReduceOp.MAX)
    gmax = int(g.cpu()[0])
    if gmax < FINITE_MIN:
        raise BBTNError(-7, "no feasible configuration")
    v, planes, moduli, ncrt, x = solver.shard_counts(gmax, config)
    part = (v, planes, moduli, ncrt, x)
    parts = [part]
    if dist is not None and world > 1:
        parts = [None] * world
        dist.all_gather_object(parts, part)
    value, cnt = combine_shards([p[:4] for p in parts])
    cfg = next((p[4] for p in parts if p[4] is not None), None)
    opt = -value if inst.kind == "spin" else value
    return opt, cnt, cfg
