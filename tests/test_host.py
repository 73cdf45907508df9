"""Host-side checks of the C-ABI library that need no GPU.

The library is built in-tree if it is missing or stale. Everything here runs
host code only: symbol exports, the prime table, the CRT recombination, the
planner (bbtn_analyze), argument validation, and the GNN feature rows.
"""
import ctypes as C
import os
import random
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2602_05470_gb300 import build
    build.build()
    import paper_2602_05470_gb300 as P
    return P


def _declared():
    txt = open(os.path.join(ROOT, "include", "bbtn.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bbtn_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(P):
    lib = C.CDLL(P.lib_path())
    names = _declared()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_structs_match_the_header(P):
    """The ctypes copies of bbtn_opts, bbtn_stats and bbtn_plan_info have the
    library's sizes (a field added on one side only would shift every later one)."""
    lib = P._lib.load()
    lib.bbtn_struct_size.restype = C.c_size_t
    lib.bbtn_struct_size.argtypes = [C.c_int]
    assert lib.bbtn_struct_size(0) == C.sizeof(P._lib.Opts)
    assert lib.bbtn_struct_size(1) == C.sizeof(P._lib.Stats)
    assert lib.bbtn_struct_size(2) == C.sizeof(P._lib.PlanInfo)
    assert lib.bbtn_struct_size(3) == 0


def test_version_and_error_strings(P):
    lib = P._lib.load()
    assert b"sm_103a" in lib.bbtn_version()
    assert lib.bbtn_primes(-1, None) == P._lib.EINVAL
    assert lib.bbtn_last_error()


def _is_prime(n):
    import sympy
    return sympy.isprime(n)


def test_prime_table(P):
    """2^61 - c_t with c_t ascending, all prime, and no prime 2^61 - c between them."""
    ps = P.primes(9)
    cs = [2**61 - p for p in ps]
    assert cs == sorted(cs) and cs[0] == 1
    assert all(_is_prime(p) for p in ps)
    for c in range(1, cs[-1]):
        if c not in cs:
            assert not _is_prime(2**61 - c), c


def test_prime_pair_table(P):
    """Pair moduli q1 << 32 | q0: the primes 2^30 - d in ascending d, taken two per
    modulus, none skipped; above 2^61, so they never read as a 2^61 - c prime."""
    ms = P.prime_pairs(9)
    qs = [q for m in ms for q in (m & 0xFFFFFFFF, m >> 32)]
    ds = [2**30 - q for q in qs]
    assert ds == sorted(ds) and len(set(ds)) == 18 and ds[-1] < 1024
    assert all(_is_prime(q) for q in qs)
    for d in range(1, ds[-1]):
        if d not in ds:
            assert not _is_prime(2**30 - d), d
    assert all(m >= 2**61 for m in ms)
    assert P._lib.load().bbtn_prime_pairs(10, None) == P._lib.EINVAL


@pytest.mark.parametrize("k", [2, 6, 16])
def test_crt_roundtrip_pair_primes(P, k):
    """Garner recombination over the unpacked 30-bit primes (what a solve with pair
    moduli reports)."""
    qs = [q for m in P.prime_pairs(8) for q in (m & 0xFFFFFFFF, m >> 32)][:k]
    M = 1
    for q in qs:
        M *= q
    rng = random.Random(k)
    for x in [0, 1, M - 1] + [rng.randrange(M) for _ in range(20)]:
        assert P.crt([x % q for q in qs], qs) == x


@pytest.mark.parametrize("k", [1, 2, 3, 8])
def test_crt_roundtrip(P, k):
    ps = P.primes(k)
    M = 1
    for p in ps:
        M *= p
    rng = random.Random(k)
    for x in [0, 1, M - 1, M // 2] + [rng.randrange(M) for _ in range(20)]:
        assert P.crt([x % p for p in ps], ps) == x


def test_crt_small_moduli(P):
    """Textbook case: x = 2 mod 3, 3 mod 5, 2 mod 7 -> 23."""
    assert P.crt([2, 3, 2], [3, 5, 7]) == 23


def test_crt_rejects_bad_input(P):
    with pytest.raises(P.BBTNError):
        P.crt([1, 2], [15, 7])       # 15 is not prime
    with pytest.raises(P.BBTNError):
        P.crt([7], [7])              # residue not below modulus
    with pytest.raises(P.BBTNError):
        P.crt([1, 1], [7, 7])        # repeated modulus


def test_context_without_device_plans_on_host(P):
    inst = synth.kings_subgraph(12, 0.8, seed=3)
    s = P.Solver(mode=P.MODE_PLAIN, space_cap_log2=30)
    info = s.analyze(inst)
    assert info["steps"] > 0 and info["sc_log2"] >= 1 and info["ops"] > 0
    assert info["tc_log2"] >= info["sc_log2"]


def test_sliced_plan_respects_cap(P, tmp_path):
    """After dynamic slicing every tensor of a slice's plan has at most 2^cap entries."""
    inst = synth.kings_subgraph(14, 0.8, seed=4)
    plain = P.Solver(mode=P.MODE_PLAIN, space_cap_log2=30).analyze(inst)
    cap = max(4, plain["sc_log2"] // 2)       # far below the width of any order: slicing is needed
    s = P.Solver(mode=P.MODE_SLICED, space_cap_log2=cap)
    path = str(tmp_path / "steps.csv")
    info = s.analyze(inst, dump_path=path)
    assert info["slices_log2"] > 0
    rows = [list(map(float, l.split(","))) for l in open(path).read().splitlines() if l and l[0].isdigit()]
    assert rows and max(max(r[0], r[1], r[2]) for r in rows) <= cap


def test_analyze_dump_lists_every_step(P, tmp_path):
    inst = synth.square_lattice(6, seed=1)
    s = P.Solver(mode=P.MODE_PLAIN, space_cap_log2=30)
    path = str(tmp_path / "steps.csv")
    info = s.analyze(inst, dump_path=path)
    rows = [l for l in open(path).read().splitlines() if l and l[0].isdigit()]
    assert len(rows) == info["steps"]


def test_invalid_instances_are_rejected(P):
    s = P.Solver()
    bad = synth.Instance(kind="mwis", n=3, edges=[(0, 3)], J=None, h2=None, w=[1, 1, 1], geometry=None)
    with pytest.raises(P.BBTNError) as e:
        s.load(bad)
    assert e.value.code == P._lib.EINVAL
    bad = synth.Instance(kind="mwis", n=2, edges=[(0, 1)], J=None, h2=None, w=[1, 0], geometry=None)
    with pytest.raises(P.BBTNError):
        s.load(bad)


def test_solve_without_device_fails_loudly(P):
    """No CPU fallback: on a machine without a GPU the solve reports a CUDA error."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    s = P.Solver()
    s.load(synth.path_graph(5))
    with pytest.raises(P.BBTNError) as e:
        s.solve()
    assert e.value.code == P._lib.ECUDA


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gnn_features_match_oracle(P, seed):
    from oracle import gnn as G
    from paper_2602_05470_gb300 import gnn
    inst = synth.kings_subgraph(9, 0.8, seed=seed, weights="uniform10" if seed else "unit")
    rng = np.random.default_rng(seed)
    fixed = rng.integers(-1, 2, inst.n)
    score = rng.random(inst.n).astype(np.float32) if seed else None
    got = gnn.features(inst, fixed, score)
    want = G.features(inst.n, inst.edges, inst.w, fixed, score)
    np.testing.assert_allclose(got, want, rtol=1e-7, atol=0)
    assert gnn.GNN.param_count() == G.param_count()


def _leaf_sum(P, inst, cap, use_symmetry):
    """(E2, D) of an instance from the host search's leaves, each solved by the
    transfer-matrix oracle with its fixed spins pinned by strong fields."""
    import oracle
    s = P.Solver(mode=P.MODE_BBTN, space_cap_log2=cap, use_symmetry=use_symmetry)
    fx, total = s.search_leaves(inst, max_leaves=4096)
    assert len(fx) == total > 0
    big = 8 * (sum(abs(j) for j in inst.J) + 1)
    best, count = None, 0
    for row in fx:
        h2 = [h + (big if f == 1 else -big if f == 0 else 0) for h, f in zip(inst.h2, row)]
        leaf = synth.Instance(**{**inst.__dict__, "h2": h2})
        e2, d, _ = oracle.spin_square_tm(leaf)
        e2 += big * int((row >= 0).sum())
        if best is None or e2 < best:
            best, count = e2, 0
        if e2 == best:
            count += d
    return best, count * (2 if use_symmetry else 1)


@pytest.mark.parametrize("row,cap", [(0, 14), (1, 12)])
@pytest.mark.parametrize("use_symmetry", [True, False])
def test_search_leaves_cover_every_ground_state(P, row, cap, use_symmetry):
    """The branch-and-bound leaves partition the optimal configurations: summing
    the leaves' exact optima and degeneracies (oracle) gives the lattice's.
    16 x 16 +-J lattices with stored oracle answers; regions of 8 spins, whose
    local values (fields from fixed neighbours, couplings inside the region)
    decide which configurations each branching keeps."""
    import json
    with open(os.path.join(ROOT, "tests", "golden", "oracle_answers.json")) as f:
        g = json.load(f)["spin_large_f6"][row]
    inst = synth.square_lattice(g["L"], seed=g["seed"])
    assert _leaf_sum(P, inst, cap, use_symmetry) == (g["e2"], int(g["count"]))


def test_prepared_order_is_reused_and_identical(P):
    """bbtn_prepare leaves the root order in the process-wide cache: a later plan of
    the same network reuses it (same tree cost, much faster) and clearing the cache
    makes the planner search again for the same tree."""
    import time
    inst = synth.kings_subgraph(20, 0.8, seed=11)
    P.clear_order_cache()
    s = P.Solver(mode=P.MODE_BBTN, space_cap_log2=16)
    t0 = time.perf_counter()
    s.prepare(inst)
    t_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    s.prepare(inst)
    t_cached = time.perf_counter() - t0
    a = s.analyze(inst)
    P.clear_order_cache()
    b = P.Solver(mode=P.MODE_BBTN, space_cap_log2=16).analyze(inst)
    assert a == b
    assert t_cached < t_first


@pytest.mark.parametrize("which", ["mixed", "pair_not_prime", "pair_equal", "pair_far", "wide_not_prime"])
def test_plane_moduli_rejected_before_any_device_work(P, which):
    """The contraction and both aggregation entry points check every plane modulus
    (all primes 2^61 - c, or all pairs q1 << 32 | q0 of distinct primes 2^30 - d)
    before they touch a buffer: bad moduli return BBTN_EINVAL, here without a GPU
    (the buffer arguments are never dereferenced)."""
    lib = P._lib.load()
    wide, pair = P.primes(2), P.prime_pairs(2)
    q0, q1 = pair[0] & 0xFFFFFFFF, pair[0] >> 32
    bad = {"mixed": [wide[0], pair[1]],
           "pair_not_prime": [pair[0], ((q1 - 1) << 32) | q0],      # q1 - 1 is even
           "pair_equal": [pair[0], (q0 << 32) | q0],
           "pair_far": [pair[0], (((1 << 30) - 1100) << 32) | q0],   # d >= 1024 is not a pair prime
           "wide_not_prime": [wide[0], wide[1] - 1]}[which]
    primes = (C.c_uint64 * 2)(*bad)
    la = (C.c_int32 * 2)(0, 1)
    lb = (C.c_int32 * 2)(1, 2)
    lc = (C.c_int32 * 2)(0, 2)
    fake = C.c_void_p(1 << 20)    # never dereferenced: validation fails first
    rc = lib.bbtn_contract(2, la, fake, fake, 2, lb, fake, fake, 2, lc, fake, fake, 2, primes, None)
    err = lib.bbtn_last_error()
    assert rc == P._lib.EINVAL and (b"modul" in err or b"prime" in err), err
    for fn in (lib.bbtn_aggregate, lib.bbtn_aggregate_noalloc):
        assert fn(4, fake, fake, 2, primes, fake, fake, None) == P._lib.EINVAL


def test_contract_chain_rejects_what_the_kernel_cannot_run(P):
    """The fused-chain entry point refuses chains outside the kernel's limits with
    BBTN_EINVAL before touching any buffer (the pointers here are never used)."""
    lib = P._lib.load()
    fake = C.c_void_p(0x1000)

    def call(la, steps, L=None):
        L = len(steps) if L is None else L
        rb = P.i32_array([len(s[0]) for s in steps])
        rc = P.i32_array([len(s[1]) for s in steps])
        lb = P.i32_array([x for s in steps for x in s[0]])
        lc = P.i32_array([x for s in steps for x in s[1]])
        vbs = (C.c_void_p * max(len(steps), 1))(*([0x2000] * len(steps)))
        return lib.bbtn_contract_chain(len(la), P.i32_array(la), fake, L, rb, lb, vbs, rc, lc, fake, None)

    la = list(range(8))
    ok_step = ([0, 1], la)
    assert call(la, [ok_step] * 9) == P._lib.EINVAL                          # more than 8 steps
    assert call(la, [([0, 1, 2, 3, 4], la)]) == P._lib.EINVAL                # B of rank 5
    four_sums = [([0], la[1:]), ([1], la[2:]), ([2], la[3:]), ([3], la[4:])]
    assert call(la, four_sums) == P._lib.EINVAL                              # 4 summed labels
    assert call(la, [([0], la + [50])]) == P._lib.EINVAL                     # output label from nowhere
    assert call(la, [([0], [0])]) == P._lib.EINVAL                           # result of rank 1
    assert "chain" in lib.bbtn_last_error().decode()


def test_shard_counts_needs_shard_values(P):
    """bbtn_shard_counts on a context whose leaf list was never built (or was
    discarded by loading an instance) is an out-of-order call, refused on the host."""
    lib = P._lib.load()
    import ctypes as C
    s = P.Solver(mode=P.MODE_BBTN, space_cap_log2=6)
    s.load(synth.kings_subgraph(6, 0.8, seed=1))
    v, npl, ncrt, have = C.c_int32(), C.c_int(), C.c_int(), C.c_int()
    planes, moduli = (C.c_uint64 * 9)(), (C.c_uint64 * 9)()
    rc = lib.bbtn_shard_counts(s._ctx, 0, 0, C.byref(v), planes, moduli, C.byref(npl), C.byref(ncrt), None,
                               C.byref(have))
    assert rc == P._lib.ESTATE
    assert b"shard_values" in lib.bbtn_last_error()
    s.close()


def test_order_restarts_option(P):
    """opts.order_restarts: 0..64 accepted, anything else rejected; with several
    min-fill restarts the root orders of eight 30x30 workload instances take less
    work in total than the default search's (host planning only)."""
    for bad in (-1, 65):
        with pytest.raises(P.BBTNError) as e:
            P.Solver(order_restarts=bad)
        assert e.value.code == P._lib.EINVAL
    total = {}
    for r in (0, 16):
        ops = []
        for idx in range(8):
            inst = synth.kings_subgraph(30, 0.8, seed=synth.config_seed(2, idx))
            s = P.Solver(mode=P.MODE_BBTN, space_cap_log2=24, order_restarts=r)
            P.clear_order_cache()
            ops.append(s.analyze(inst)["ops"])
            s.close()
        total[r] = ops
    assert sum(total[16]) < sum(total[0])
