"""Kernel-level parity: every device call through the C ABI against the CPU oracle,
element by element, on seeded inputs (bit-exact: all arithmetic is integer)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05470_gb300 as P
    return P


def _rand(rng, r, np_, lo=-3, hi=3, neg_frac=0.0, unit=False):
    v = rng.integers(lo, hi + 1, size=1 << r).astype(np.int32)
    if neg_frac:
        v[rng.random(1 << r) < neg_frac] = oracle.NEG
    if unit:
        c = np.where(v >= -(1 << 28), 1, 0).astype(np.uint64)[None, :].repeat(np_, 0)
    else:
        c = rng.integers(0, 2**61 - 1024, size=(np_, 1 << r), dtype=np.uint64)
        c[:, v < -(1 << 28)] = 0
    return v, c


def _dev(v, c):
    dv = torch.from_numpy(v).cuda()
    dc = torch.from_numpy(c.view(np.int64)).cuda() if c is not None and c.size else None
    return dv, dc


def _run(P, la, A, lb, B, lc, primes, unitA=False, unitB=False):
    va, ca = _dev(*A)
    if unitA:
        ca = None
    if lb is None:
        vb = cb = None
    else:
        vb, cb = _dev(*B)
        if unitB:
            cb = None
    vc, cc = P.contract(la, va, ca, lb, vb, cb, lc, primes)
    torch.cuda.synchronize()
    out_c = cc.cpu().numpy().view(np.uint64) if cc is not None else np.zeros((0, 1 << len(lc)), np.uint64)
    return vc.cpu().numpy(), out_c


CASES = [
    # (la, lb, lc) -- covers batch/m/n/k roles, private labels, outer products,
    # permuted outputs, scalars, and several thread blocks
    ([0, 1, 2, 3], [2, 3, 4, 5], [0, 1, 4, 5]),                      # plain matmul-like
    ([0, 1, 2, 3, 4, 5], [4, 5, 6, 7], [0, 1, 2, 3, 6, 7]),
    ([0, 1, 2], [1, 2, 3], [3, 0]),                                  # permuted output
    ([5, 1, 7, 3], [3, 7, 9], [9, 5, 1]),                            # scattered labels
    ([0, 1, 2, 3], [2, 3, 4], [0, 1, 2, 3, 4]),                      # batch labels, no sum
    ([0, 1, 2, 3], [4, 5], [0, 1, 2, 3, 4, 5]),                      # outer product
    ([0, 1, 2, 3], [3, 4], [0, 4]),                                  # private labels 1, 2
    ([0, 1], [0, 1], []),                                            # full contraction to a scalar
    (list(range(12)), [10, 11, 12, 13], list(range(10)) + [12, 13]), # 4096 outputs x 4
    (list(range(3, 16)), [0, 1, 2, 3], list(range(0, 3)) + list(range(4, 16))),  # 2^15 outputs, low bits from B
    (list(range(14)), [12, 13, 14], [14] + list(range(12))),         # big output, permuted top bit
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("np_", [0, 1, 3])
def test_contract_parity(P, case, np_):
    la, lb, lc = CASES[case]
    rng = np.random.default_rng(100 + case)
    primes = P.primes(np_)
    A = _rand(rng, len(la), max(np_, 1), neg_frac=0.1)
    B = _rand(rng, len(lb), max(np_, 1), neg_frac=0.1)
    A = (A[0], A[1][:np_])
    B = (B[0], B[1][:np_])
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov)
    assert np.array_equal(cc, oc)


def _labels(prefix_ids):
    return list(prefix_ids)


# shapes that take the register-tiled kernel: >= 6 A-only and B-only labels and
# 4..13 summed labels; label ids: m 0-9, n 10-19, k 20-33, batch 40-43
TILED = [
    # (m, n, k, batch, A's first group, B's first group, C order)
    (6, 6, 4, 1, "m", "k", "mnb"),
    (6, 6, 4, 1, "k", "n", "nmb"),
    (7, 6, 6, 2, "k", "k", "bnm"),
    (6, 7, 5, 0, "m", "n", "mn"),
    (6, 6, 8, 2, "k", "k", "nbm"),       # 2^14 outputs, 8 summed: below the split-K range
    (6, 4, 6, 2, "m", "k", "mnb"),       # 4 B-only labels: 64 x 16 tiles
    (7, 5, 8, 1, "k", "n", "bnm"),       # 5 B-only labels
]


def _tiled_case(m, n, k, b, afirst, bfirst, corder, private=False):
    M = list(range(0, m))
    N = list(range(10, 10 + n))
    K = list(range(20, 20 + k))
    Bt = list(range(40, 40 + b))
    la = (K + M + Bt) if afirst == "k" else (M + K + Bt)
    lb = (K + N + Bt) if bfirst == "k" else (N + K + Bt)
    if private:
        lb = lb + [50]               # summed label private to B
    groups = {"m": M, "n": N, "b": Bt}
    lc = [x for g in corder for x in groups[g]]
    return la, lb, lc


@pytest.mark.parametrize("case", range(len(TILED)))
@pytest.mark.parametrize("np_", [0, 1, 3])
def test_contract_tiled_parity(P, case, np_):
    la, lb, lc = _tiled_case(*TILED[case])
    rng = np.random.default_rng(500 + case)
    primes = P.primes(np_)
    A = _rand(rng, len(la), max(np_, 1), -4, 4, neg_frac=0.05)
    B = _rand(rng, len(lb), max(np_, 1), -4, 4, neg_frac=0.05)
    A = (A[0], A[1][:np_])
    B = (B[0], B[1][:np_])
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov)
    assert np.array_equal(cc, oc)


def test_contract_tiled_private_label(P):
    la, lb, lc = _tiled_case(6, 6, 4, 0, "m", "k", "mn", private=True)
    rng = np.random.default_rng(77)
    primes = P.primes(3)
    A = _rand(rng, len(la), 3, -2, 2)
    B = _rand(rng, len(lb), 3, -2, 2)
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)


@pytest.mark.parametrize("np_", [2, 8, 9])
def test_contract_many_planes(P, np_):
    la, lb, lc = [0, 1, 2, 3, 4], [3, 4, 5, 6], [0, 1, 2, 5, 6]
    rng = np.random.default_rng(7)
    primes = P.primes(np_)
    A = _rand(rng, 5, np_, -1, 1)
    B = _rand(rng, 4, np_, -1, 1)
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)


def test_contract_unit_counts(P):
    """Counts omitted (NULL): implied 1 for finite entries, 0 for -infinity."""
    la, lb, lc = [0, 1, 2, 3], [2, 3, 4], [0, 1, 4]
    rng = np.random.default_rng(8)
    primes = P.primes(3)
    A = _rand(rng, 4, 3, -2, 2, neg_frac=0.2, unit=True)
    B = _rand(rng, 3, 3, -2, 2, neg_frac=0.2, unit=True)
    vc, cc = _run(P, la, A, lb, B, lc, primes, unitA=True, unitB=True)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)


@pytest.mark.parametrize("rs", [12, 13, 14])
def test_contract_large_summed_extent(P, rs):
    """More summed labels than the shared-memory table covers (2^12)."""
    la = list(range(rs + 2))
    lb = list(range(2, rs + 3))
    lc = [0, 1, rs + 2]
    rng = np.random.default_rng(rs)
    primes = P.primes(2)
    A = _rand(rng, len(la), 2, -2, 2)
    B = _rand(rng, len(lb), 2, -2, 2)
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)


@pytest.mark.parametrize("la,lc", [([0, 1, 2, 3, 4], [1, 3]), ([0, 1, 2], []), (list(range(16)), list(range(4, 16)))])
def test_reduce_parity(P, la, lc):
    rng = np.random.default_rng(len(la))
    primes = P.primes(3)
    A = _rand(rng, len(la), 3, -2, 2, neg_frac=0.05)
    vc, cc = _run(P, la, A, None, None, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], None, None, None, lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)


@pytest.mark.parametrize("r,seed", [(1, 0), (4, 1), (7, 2), (11, 3), (16, 4), (20, 5)])
def test_permute_parity(P, r, seed):
    rng = np.random.default_rng(seed)
    perm = [int(x) for x in rng.permutation(r)]
    primes = P.primes(3)
    v, c = _rand(rng, r, 3, -5, 5)
    dv, dc = _dev(v, c)
    ov_, oc_ = P.permute(perm, dv, dc)
    torch.cuda.synchronize()
    # the permutation is the single-operand contraction with relabelled output bits
    la = list(range(r))
    lc = [perm[q] for q in range(r)]
    ev, ec = oracle.contract(la, v, c, None, None, None, lc, primes)
    assert np.array_equal(ov_.cpu().numpy(), ev)
    assert np.array_equal(oc_.cpu().numpy().view(np.uint64), ec)


@pytest.mark.parametrize("n", [0, 1, 7, 256, 257, 1000, 70000])
def test_aggregate_parity(P, n):
    rng = np.random.default_rng(n)
    primes = P.primes(3)
    v = rng.integers(-3, 1, size=n).astype(np.int32)
    c = rng.integers(0, 2**61 - 1024, size=(3, n), dtype=np.uint64)
    dv = torch.from_numpy(v).cuda()
    dc = torch.from_numpy(c.view(np.int64).copy()).cuda()
    ov_, oc_ = P.aggregate(dv, dc, primes)
    torch.cuda.synchronize()
    # oracle: pad to a power of two with (-inf, 0) and reduce every label
    r = max(0, int(np.ceil(np.log2(max(n, 1)))))
    pv = np.full(1 << r, oracle.NEG, np.int32)
    pc = np.zeros((3, 1 << r), np.uint64)
    pv[:n] = v
    pc[:, :n] = c
    ev, ec = oracle.contract(list(range(r)), pv, pc, None, None, None, [], primes)
    assert int(ov_.cpu()[0]) == int(ev[0])
    assert np.array_equal(oc_.cpu().numpy().view(np.uint64), ec[:, 0])


def test_backward_selects_a_maximiser(P):
    la, lb, lc = [0, 1, 2, 3, 4], [3, 4, 5, 6], [0, 1, 5, 6]
    rng = np.random.default_rng(11)
    va = rng.integers(-3, 3, size=32).astype(np.int32)
    vb = rng.integers(-3, 3, size=16).astype(np.int32)
    primes = P.primes(1)
    ov, _ = oracle.contract(la, va, np.ones((1, 32), np.uint64), lb, vb, np.ones((1, 16), np.uint64), lc, primes)
    dva, dvb, dvc = torch.from_numpy(va).cuda(), torch.from_numpy(vb).cuda(), torch.from_numpy(ov).cuda()
    sel = torch.arange(16, dtype=torch.int64, device="cuda")
    sa, sb = P.contract_backward(la, dva, lb, dvb, lc, dvc, sel)
    sa, sb = sa.cpu().numpy(), sb.cpu().numpy()
    for o in range(16):
        ia, ib = int(sa[o]), int(sb[o])
        assert va[ia] + vb[ib] == ov[o]
        # the output labels agree with o
        bits = {lc[i]: (o >> i) & 1 for i in range(len(lc))}
        for i, l in enumerate(la):
            if l in bits:
                assert (ia >> i) & 1 == bits[l]
        for i, l in enumerate(lb):
            if l in bits:
                assert (ib >> i) & 1 == bits[l]
        # shared summed labels agree between A and B
        for i, l in enumerate(la):
            if l in lb and l not in bits:
                assert (ia >> i) & 1 == (ib >> lb.index(l)) & 1


# few outputs, long sums: the split-K kernel (<= 2^12 outputs, >= 2^12 summed
# assignments); labels: outputs 0-9, summed 100+
SPLITK = [
    ([0, 1] + list(range(100, 114)), list(range(100, 114)) + [16, 17, 18, 19], [0, 1, 16, 17, 18, 19]),
    ([0, 1, 2] + list(range(100, 112)), list(range(100, 112)) + [20, 21], [0, 20, 1, 21, 2]),   # 32 outputs x 2^12
    (list(range(7)) + list(range(100, 109)), list(range(100, 109)) + list(range(10, 17)), list(range(7)) + list(range(10, 17))),  # 2^14 x 2^9
    ([0, 1, 2, 3] + list(range(100, 108)), list(range(100, 108)) + [4, 5, 6, 7, 8], list(range(9))),   # 2^9 outputs x 2^8
    (list(range(100, 118)), list(range(117, 99, -1)), []),
    ([0, 1, 2] + list(range(100, 116)), None, [2, 0, 1]),
]


@pytest.mark.parametrize("case", range(len(SPLITK)))
@pytest.mark.parametrize("np_", [0, 3, 4])
def test_contract_splitk_parity(P, case, np_):
    la, lb, lc = SPLITK[case]
    rng = np.random.default_rng(900 + case)
    primes = P.primes(np_)
    A = _rand(rng, len(la), max(np_, 1), -3, 3, neg_frac=0.05)
    A = (A[0], A[1][:np_])
    B = None
    if lb is not None:
        B = _rand(rng, len(lb), max(np_, 1), -3, 3, neg_frac=0.05)
        B = (B[0], B[1][:np_])
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, None if B is None else B[0], None if B is None else B[1], lc, primes)
    assert np.array_equal(vc, ov)
    assert np.array_equal(cc, oc)


def test_contract_tiled_long_sum(P):
    """13 summed labels over 2^16 outputs (above the split-K range): tiled."""
    la, lb, lc = _tiled_case(8, 8, 13, 0, "k", "k", "mn")
    rng = np.random.default_rng(1414)
    primes = P.primes(1)
    A = _rand(rng, len(la), 1, -3, 3, neg_frac=0.02)
    B = _rand(rng, len(lb), 1, -3, 3, neg_frac=0.02)
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)


# Paths of the four-outputs-per-thread streaming kernel: 128-bit loads of A when
# the two lowest output bits are A's two lowest bits and A is 16-byte aligned,
# scalar loads otherwise; 128-bit stores when C is 16-byte aligned; B constant or
# varying over the four outputs; summed labels at A's low bits; reductions.
VEC = [
    # (la, lb, lc, shift_a, shift_c)
    (list(range(16)), [15, 16], list(range(15)) + [16], 0, 0),        # growth step, summed top bit
    (list(range(16)), [15, 16], list(range(15)) + [16], 1, 0),        # A not 16-byte aligned
    (list(range(16)), [15, 16], list(range(15)) + [16], 0, 3),        # C not 16-byte aligned
    (list(range(14)), [3, 20], list(range(14)) + [20], 1, 1),         # no summed label, both shifted
    (list(range(14)), [0, 20], [20] + list(range(1, 14)), 0, 0),      # low output bit from B, A's bit 0 summed
    ([30] + list(range(14)), [30, 31], list(range(14)) + [31], 0, 0),  # summed label at A's bit 0
    (list(range(15)), [0, 1, 40], list(range(15)) + [40], 0, 0),      # B varies over the low bits
    (list(range(12)) + [50, 51], None, list(range(12)), 1, 2),         # single-operand reduction, shifted
    (list(range(12)) + [50, 51], None, list(range(12)), 0, 0),         # single-operand reduction, aligned
    (list(range(2, 17)) + [0, 1], [0, 1, 60], list(range(2, 17)) + [60], 0, 0),  # summed at A's top bits
    (list(range(14)), [13, 20, 21], list(range(13)) + [20, 21], 0, 0),  # two B-only output bits on top
    (list(range(14)), [13, 20, 21], [21] + list(range(13)) + [20], 1, 1),  # B-only bits at 0 and top, shifted
    ([5, 0, 3, 1, 2, 4, 6, 7, 8, 9, 10, 11], [4, 30], [30, 0, 1, 2, 3] + list(range(5, 12)), 0, 0),  # scattered A
    (list(range(14)), [12, 13], list(range(12)) + [13], 0, 0),        # B inside A: 128-bit residue loads/stores
    (list(range(14)), [12, 13], list(range(12)) + [13], 1, 0),        # the same with A not 16-byte aligned
]


@pytest.mark.parametrize("case", range(len(VEC)))
@pytest.mark.parametrize("np_", [0, 4])
def test_contract_vector_paths(P, case, np_):
    la, lb, lc, sa, sc = VEC[case]
    rng = np.random.default_rng(700 + case)
    primes = P.primes(np_)
    A = _rand(rng, len(la), max(np_, 1), neg_frac=0.1)
    A = (A[0], A[1][:np_])
    va_full = torch.zeros((1 << len(la)) + sa, dtype=torch.int32, device="cuda")
    va_full[sa:] = torch.from_numpy(A[0]).cuda()
    va = va_full[sa:]
    ca = torch.from_numpy(A[1].view(np.int64)).cuda() if np_ else None
    if lb is None:
        B = (None, np.zeros((np_, 0), np.uint64))
        vb = cb = None
    else:
        B = _rand(rng, len(lb), max(np_, 1), neg_frac=0.1)
        B = (B[0], B[1][:np_])
        vb, cb = _dev(*B)
        if not np_:
            cb = None
    vc_full = torch.zeros((1 << len(lc)) + sc, dtype=torch.int32, device="cuda")
    cc = torch.zeros((np_, 1 << len(lc)), dtype=torch.int64, device="cuda") if np_ else None
    P.contract(la, va, ca, lb, vb, cb, lc, primes, out=(vc_full[sc:], cc))
    torch.cuda.synchronize()
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc_full[sc:].cpu().numpy(), ov)
    if np_:
        assert np.array_equal(cc.cpu().numpy().view(np.uint64), oc)


@pytest.mark.parametrize("case", range(len(TILED) + 2))
def test_contract_values16(P, case):
    """16-bit-lane value-only contraction: feasible outputs equal the oracle's,
    infeasible ones stay below FINITE_MIN. Values span (-2^12, 2^12)."""
    if case < len(TILED):
        la, lb, lc = _tiled_case(*TILED[case])
    else:
        la, lb, lc = CASES[8 + case - len(TILED)][:3]
    rng = np.random.default_rng(900 + case)
    va = rng.integers(-2000, 2000, size=1 << len(la)).astype(np.int32)
    vb = rng.integers(-2000, 2000, size=1 << len(lb)).astype(np.int32)
    # enough infeasible entries that both feasible and infeasible outputs occur
    frac = 0.9 if case < len(TILED) else 0.3
    va[rng.random(va.size) < frac] = oracle.NEG
    vb[rng.random(vb.size) < frac] = oracle.NEG
    vc = P.contract_values16(la, torch.from_numpy(va).cuda(), lb, torch.from_numpy(vb).cuda(), lc)
    torch.cuda.synchronize()
    got = vc.cpu().numpy()
    ov, _ = oracle.contract(la, va, np.zeros((0, va.size), np.uint64), lb, vb, np.zeros((0, vb.size), np.uint64),
                            lc, [])
    feas = ov >= -(1 << 28)
    assert feas.any() and (~feas).any()
    assert np.array_equal(got[feas], ov[feas])
    assert (got[~feas] < -(1 << 28)).all()


# ---- count planes with pair moduli: two residues per word, mod primes 2^30 - d.
# The oracle contracts the low halves mod q0 and the high halves mod q1 separately.
M32 = np.uint64(0xFFFFFFFF)


def _pair_planes(rng, v, moduli):
    planes = []
    for m in moduli:
        q0, q1 = m & 0xFFFFFFFF, m >> 32
        lo = rng.integers(0, q0, size=v.size, dtype=np.uint64)
        hi = rng.integers(0, q1, size=v.size, dtype=np.uint64)
        w = lo | (hi << np.uint64(32))
        w[v < -(1 << 28)] = 0
        planes.append(w)
    return np.stack(planes) if planes else np.zeros((0, v.size), np.uint64)


def _oracle_pair(la, va, ca, lb, vb, cb, lc, moduli):
    q0 = [m & 0xFFFFFFFF for m in moduli]
    q1 = [m >> 32 for m in moduli]
    half = lambda c, s: None if c is None else (c >> np.uint64(s)) & M32
    ov, lo = oracle.contract(la, va, half(ca, 0), lb, vb, half(cb, 0), lc, q0)
    _, hi = oracle.contract(la, va, half(ca, 32), lb, vb, half(cb, 32), lc, q1)
    return ov, lo | (hi << np.uint64(32))


def _pair_case(P, la, lb, lc, np_, seed, lo=-3, hi=3, neg=0.05, unitA=False, unitB=False):
    rng = np.random.default_rng(seed)
    moduli = P.prime_pairs(np_)
    va = rng.integers(lo, hi + 1, size=1 << len(la)).astype(np.int32)
    va[rng.random(va.size) < neg] = oracle.NEG
    ca = _pair_planes(rng, va, moduli)
    vb = cb = None
    if lb is not None:
        vb = rng.integers(lo, hi + 1, size=1 << len(lb)).astype(np.int32)
        vb[rng.random(vb.size) < neg] = oracle.NEG
        cb = _pair_planes(rng, vb, moduli)
    one = np.uint64(0x100000001)
    if unitA:
        ca = np.where(va >= -(1 << 28), one, np.uint64(0))[None, :].repeat(np_, 0)
    if unitB and lb is not None:
        cb = np.where(vb >= -(1 << 28), one, np.uint64(0))[None, :].repeat(np_, 0)
    vc, cc = _run(P, la, (va, ca), lb, None if lb is None else (vb, cb), lc, moduli, unitA=unitA, unitB=unitB)
    ov, oc = _oracle_pair(la, va, ca, lb, vb, cb, lc, moduli)
    assert np.array_equal(vc, ov)
    assert np.array_equal(cc, oc)


PAIR_CASES = ([CASES[i] for i in (0, 3, 6, 7, 8, 9)] + [_tiled_case(*t) for t in TILED] +
              [(la, lb, lc) for la, lb, lc in SPLITK] + [(la, lb, lc) for la, lb, lc, _, _ in VEC[:7]])


@pytest.mark.parametrize("case", range(len(PAIR_CASES)))
@pytest.mark.parametrize("np_", [1, 4])
def test_contract_pair_moduli(P, case, np_):
    """Every kernel family (streaming, four-outputs streaming, register-tiled 64- and
    16-wide, split-K, reductions) with pair-modulus count planes."""
    la, lb, lc = PAIR_CASES[case]
    _pair_case(P, la, lb, lc, np_, 1300 + case, lo=-4, hi=4)


@pytest.mark.parametrize("case", [0, 8, 12, 13])
def test_contract_pair_unit_counts(P, case):
    """Unit counts (implied by the values) enter as 1 in both halves of the word."""
    la, lb, lc = PAIR_CASES[case]
    _pair_case(P, la, lb, lc, 3, 1400 + case, unitA=True, unitB=case % 2 == 0)


def test_contract_pair_dense_ties(P):
    """All values equal: every summed assignment ties, so a tiled chunk adds 16
    products per output half (the most its 64-bit sums take before reduction)."""
    la, lb, lc = _tiled_case(6, 6, 8, 1, "k", "n", "mnb")
    _pair_case(P, la, lb, lc, 4, 1500, lo=0, hi=0, neg=0.0)


def test_contract_pair_rejects_mixed_moduli(P):
    la, lb, lc = CASES[0]
    rng = np.random.default_rng(1)
    v = rng.integers(-2, 3, size=16).astype(np.int32)
    c = np.zeros((2, 16), np.uint64)
    with pytest.raises(P.BBTNError):
        _run(P, la, (v, c), lb, (v, c), lc, [P.primes(1)[0], P.prime_pairs(1)[0]])


@pytest.mark.parametrize("n", [1, 257, 70000])
def test_aggregate_pair_moduli(P, n):
    rng = np.random.default_rng(77 + n)
    moduli = P.prime_pairs(3)
    v = rng.integers(-2, 1, size=n).astype(np.int32)
    c = _pair_planes(rng, v, moduli)
    ov_, oc_ = P.aggregate(torch.from_numpy(v).cuda(), torch.from_numpy(c.view(np.int64).copy()).cuda(), moduli)
    torch.cuda.synchronize()
    r = max(0, int(np.ceil(np.log2(max(n, 1)))))
    pv = np.full(1 << r, oracle.NEG, np.int32)
    pc = np.zeros((3, 1 << r), np.uint64)
    pv[:n], pc[:, :n] = v, c
    ev, ec = _oracle_pair(list(range(r)), pv, pc, None, None, None, [], moduli)
    assert int(ov_.cpu()[0]) == int(ev[0])
    assert np.array_equal(oc_.cpu().numpy().view(np.uint64), ec[:, 0])


@pytest.mark.parametrize("np_", [0, 3])
def test_contract_tiled_swapped_operands(P, np_):
    """4 A-only and 12 B-only labels: too few rows for the tile as given, so the
    operands are exchanged (max-plus addition commutes) and the step is tiled."""
    M, N, K = [0, 1, 2, 3], list(range(10, 22)), list(range(30, 36))
    la, lb, lc = K + M, N + K, M + N
    rng = np.random.default_rng(2200 + np_)
    primes = P.primes(np_)
    A = _rand(rng, len(la), max(np_, 1), -4, 4, neg_frac=0.05)
    B = _rand(rng, len(lb), max(np_, 1), -4, 4, neg_frac=0.05)
    A, B = (A[0], A[1][:np_]), (B[0], B[1][:np_])
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)
    _pair_case(P, la, lb, lc, 2, 2300 + np_, lo=-4, hi=4)


# ---------------------------------------------------------------- fused chains (K1m)

def _oracle_chain(la, va, steps):
    """The chain step by step through the oracle's single contraction (values only)."""
    lab, v = list(la), va
    for lb, vb, lc in steps:
        v, _ = oracle.contract(lab, v, np.zeros((0, 1 << len(lab)), np.uint64), lb, vb,
                               np.zeros((0, 1 << len(lb)), np.uint64), lc, [])
        lab = list(lc)
    return v


def _random_chain(rng, ra, L, max_sum=3, new_low=False):
    """A random chain: each step's B holds one or two labels of the current tensor
    and possibly a new one; some labels are summed (at most max_sum over the chain).
    Output labels keep the current order with new labels inserted at random places
    (or at the bottom, new_low) and summed ones dropped."""
    cur = list(range(ra))
    nxt = 100
    steps, summed = [], 0
    for _ in range(L):
        k = int(rng.integers(1, 3))
        lb = [int(x) for x in rng.choice(cur, size=min(k, len(cur)), replace=False)]
        out = list(cur)
        if rng.random() < 0.5:
            lb.append(nxt)
            pos = 0 if new_low else int(rng.integers(0, len(out) + 1))
            out.insert(pos, nxt)
            nxt += 1
        rng.shuffle(lb)
        if summed < max_sum and rng.random() < 0.4 and len(out) > 3:
            drop = lb[int(rng.integers(0, len(lb)))]
            out.remove(drop)
            summed += 1
        vb = rng.integers(-4, 5, size=1 << len(lb)).astype(np.int32)
        if rng.random() < 0.3:
            vb[int(rng.integers(0, len(vb)))] = oracle.NEG          # a hard constraint
        steps.append((lb, vb, out))
        cur = out
    return steps


@pytest.mark.parametrize("seed", range(12))
def test_contract_chain_parity(P, seed):
    """Random chains of 1..8 steps (ranks 6..20, up to three summed labels, new
    labels, hard constraints): the one-pass kernel equals the step-by-step oracle
    element by element, infeasible entries included."""
    rng = np.random.default_rng(1000 + seed)
    for trial in range(6):
        ra = int(rng.integers(6, 21))
        L = int(rng.integers(1, 9))
        steps = _random_chain(rng, ra, L, max_sum=3 if L <= 2 else 2 if L <= 4 else 1, new_low=trial % 2 == 1)
        va = rng.integers(-6, 7, size=1 << ra).astype(np.int32)
        va[rng.random(1 << ra) < 0.1] = oracle.NEG
        want = _oracle_chain(list(range(ra)), va, steps)
        dsteps = [(lb, torch.from_numpy(vb).cuda(), lc) for lb, vb, lc in steps]
        got = P.contract_chain(list(range(ra)), torch.from_numpy(va).cuda(), dsteps)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), want), (seed, trial, L)


@pytest.mark.parametrize("offset", [0, 1])
def test_contract_chain_vector_and_misaligned(P, offset):
    """Edge matrices added to a rank-18 tensor whose two lowest bits pass through
    (the 128-bit load and store path), and the same from a misaligned start."""
    rng = np.random.default_rng(7)
    ra = 18
    la = list(range(ra))
    steps = [([5, 9], rng.integers(-3, 4, 4).astype(np.int32), la),
             ([9, 12], rng.integers(-3, 4, 4).astype(np.int32), la),
             ([12, 17], rng.integers(-3, 4, 4).astype(np.int32), [x for x in la if x != 17])]
    buf = rng.integers(-5, 6, size=(1 << ra) + 4).astype(np.int32)
    va = buf[offset:offset + (1 << ra)]
    want = _oracle_chain(la, va, steps)
    dbuf = torch.from_numpy(buf).cuda()
    out = torch.empty((1 << (ra - 1)) + 4, dtype=torch.int32, device="cuda")
    dsteps = [(lb, torch.from_numpy(vb).cuda(), lc) for lb, vb, lc in steps]
    got = P.contract_chain(la, dbuf[offset:offset + (1 << ra)], dsteps, out=out[offset:offset + (1 << (ra - 1))])
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)


def test_contract_chain_smallest_and_positive_after_neg(P):
    """Rank-2 results; a positive B entry after a hard constraint (the floor at
    NEG is applied after every step, so NEG + 4 stays NEG + 4, not NEG)."""
    la = [0, 1, 2]
    va = np.array([oracle.NEG, 3, -2, oracle.NEG, 0, 1, 5, -7], np.int32)
    steps = [([0], np.array([-1, 2], np.int32), [1, 2, 0]),
             ([1, 7], np.array([4, oracle.NEG, 3, 1], np.int32), [2, 7, 1]),
             ([2], np.array([4, 4], np.int32), [7, 1])]
    want = _oracle_chain(la, va, steps)
    dsteps = [(lb, torch.from_numpy(vb).cuda(), lc) for lb, vb, lc in steps]
    got = P.contract_chain(la, torch.from_numpy(va).cuda(), dsteps)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)


def _blocks(r, cuts, order):
    """A permutation made of the input bit ranges split at `cuts`, put in `order`."""
    edges = [0] + list(cuts) + [r]
    blocks = [list(range(edges[i], edges[i + 1])) for i in range(len(edges) - 1)]
    return [b for k in order for b in blocks[k]]


TMA_PERMS = [
    (12, _blocks(12, [6], [1, 0]), 3),                 # transpose of two 6-bit runs
    (16, _blocks(16, [2, 9, 13], [2, 0, 3, 1]), 3),    # four runs, short ones at both ends
    (20, _blocks(20, [10], [1, 0]), 0),                # a 1024 x 1024 transpose, values only
    (18, _blocks(18, [3, 7, 12, 15], [4, 1, 0, 3, 2]), 2),   # five runs
    (14, _blocks(14, [5], [0, 1]), 3),                 # identity (one run: plain tiled copy)
    (17, _blocks(17, [4, 11], [0, 2, 1]), 1),          # low run kept in place, upper runs swapped
    (22, _blocks(22, [2, 20], [2, 1, 0]), 1),          # runs of 2, 18 and 2 bits
]


@pytest.mark.parametrize("case", range(len(TMA_PERMS)))
def test_permute_tma_parity(P, case):
    """Permutations the TMA-staged kernel takes (at most five runs of consecutive
    bits): element-wise equal to the oracle's single-operand contraction with
    relabelled outputs, value plane and count planes."""
    r, perm, np_ = TMA_PERMS[case]
    rng = np.random.default_rng(50 + case)
    primes = P.primes(max(np_, 1))[:np_]
    v, c = _rand(rng, r, np_, -5, 5)
    dv, dc = _dev(v, c)
    lib = P._lib.load()
    assert lib.bbtn_permute_uses_tma(r, P.i32_array(perm), dv.data_ptr(), dc.data_ptr() if dc is not None else None,
                                     dv.data_ptr(), dc.data_ptr() if dc is not None else None, np_) == 1
    ov_, oc_ = P.permute(perm, dv, dc)
    torch.cuda.synchronize()
    la = list(range(r))
    lc = [perm[q] for q in range(r)]
    ev, ec = oracle.contract(la, v, c, None, None, None, lc, primes)
    assert np.array_equal(ov_.cpu().numpy(), ev)
    if np_:
        assert np.array_equal(oc_.cpu().numpy().view(np.uint64), ec)


def test_permute_tma_declines_what_it_cannot_tile(P):
    """Six runs, a single-bit run at bit 0, or a misaligned buffer: the
    shared-memory kernel runs instead (and still matches)."""
    lib = P._lib.load()
    buf = torch.zeros(1 << 13, dtype=torch.int32, device="cuda")
    ptr = buf.data_ptr()
    six = _blocks(12, [2, 4, 6, 8, 10], [5, 4, 3, 2, 1, 0])
    assert lib.bbtn_permute_uses_tma(12, P.i32_array(six), ptr, None, ptr, None, 0) == 0
    lowbit = [0] + [x + 1 for x in _blocks(11, [5], [1, 0])]      # input bit 0 a run of one bit
    assert lib.bbtn_permute_uses_tma(12, P.i32_array(lowbit), ptr, None, ptr, None, 0) == 0
    ok = _blocks(12, [6], [1, 0])
    assert lib.bbtn_permute_uses_tma(12, P.i32_array(ok), ptr + 4, None, ptr, None, 0) == 0
    v, _ = _rand(np.random.default_rng(3), 12, 0)
    ov_, _ = P.permute(six, torch.from_numpy(v).cuda(), None)
    torch.cuda.synchronize()
    ev, _ = oracle.contract(list(range(12)), v, np.zeros((0, 1 << 12), np.uint64), None, None, None, six, [])
    assert np.array_equal(ov_.cpu().numpy(), ev)


# ---- counting steps with no summed label (one product per output) take their own
# kernel: 128-bit count-word loads and stores where A's and C's count planes start
# on 16 bytes and the four outputs of a thread are A's and C's two lowest bits,
# scalar words otherwise (count tensors offset by one word); unit counts on either
# side (the product is then the other operand's count).
OUTER = [
    # (la, lb, lc)
    (list(range(14)), [12, 13], list(range(14))),                  # B inside A: vector loads and stores
    (list(range(14)), [13, 20], list(range(14)) + [20]),           # a B-only label on top
    (list(range(14)), [0, 20], [20] + list(range(14))),            # a B-only label at C's bit 0
    ([3, 0, 1, 2] + list(range(4, 14)), [0, 1], list(range(14))),  # A's bits permuted against C's
    (list(range(15)), [40], list(range(15)) + [40]),               # a vertex-like B on top
]


def _outer_run(P, la, lb, lc, pair, seed, sa=0, sc=0, unitA=False, unitB=False, neg=0.05):
    rng = np.random.default_rng(seed)
    moduli = P.prime_pairs(4) if pair else P.primes(3)
    np_ = len(moduli)
    va = rng.integers(-4, 5, size=1 << len(la)).astype(np.int32)
    va[rng.random(va.size) < neg] = oracle.NEG
    vb = rng.integers(-4, 5, size=1 << len(lb)).astype(np.int32)
    vb[rng.random(vb.size) < neg] = oracle.NEG

    def planes(v, unit):
        if unit:
            one = np.uint64(0x100000001) if pair else np.uint64(1)
            return np.where(v >= -(1 << 28), one, np.uint64(0))[None, :].repeat(np_, 0)
        if pair:
            return _pair_planes(rng, v, moduli)
        c = np.stack([rng.integers(0, int(m), size=v.size, dtype=np.uint64) for m in moduli])
        c[:, v < -(1 << 28)] = 0
        return c

    ca, cb = planes(va, unitA), planes(vb, unitB)
    # count tensors placed sa / sc words past a 16-byte boundary
    ca_full = torch.zeros(np_ * va.size + sa, dtype=torch.int64, device="cuda")
    ca_full[sa:] = torch.from_numpy(ca.reshape(-1).view(np.int64)).cuda()
    cc_full = torch.zeros(np_ * (1 << len(lc)) + sc, dtype=torch.int64, device="cuda")
    vc = torch.empty(1 << len(lc), dtype=torch.int32, device="cuda")
    cc = cc_full[sc:].view(np_, 1 << len(lc))
    dva, dvb = torch.from_numpy(va).cuda(), torch.from_numpy(vb).cuda()
    dca = None if unitA else ca_full[sa:].view(np_, va.size)
    dcb = None if unitB else torch.from_numpy(cb.view(np.int64)).cuda()
    P.contract(la, dva, dca, lb, dvb, dcb, lc, moduli, out=(vc, cc))
    torch.cuda.synchronize()
    if pair:
        ov, oc = _oracle_pair(la, va, ca, lb, vb, cb, lc, moduli)
    else:
        ov, oc = oracle.contract(la, va, ca, lb, vb, cb, lc, moduli)
    assert np.array_equal(vc.cpu().numpy(), ov)
    assert np.array_equal(cc.cpu().numpy().view(np.uint64), oc)


@pytest.mark.parametrize("case", range(len(OUTER)))
@pytest.mark.parametrize("form", ["pair", "wide"])
@pytest.mark.parametrize("shift", [(0, 0), (1, 0), (0, 1)])
def test_contract_outer_counting(P, case, form, shift):
    la, lb, lc = OUTER[case]
    _outer_run(P, la, lb, lc, form == "pair", 2000 + case, sa=shift[0], sc=shift[1])


@pytest.mark.parametrize("case", range(len(OUTER)))
@pytest.mark.parametrize("unit", [(True, False), (False, True), (True, True)])
def test_contract_outer_unit_counts(P, case, unit):
    la, lb, lc = OUTER[case]
    _outer_run(P, la, lb, lc, True, 2100 + case, unitA=unit[0], unitB=unit[1])


# The general streaming counting path with the same count-word layouts: summed
# labels on A's top bits, so a thread's four outputs are A's and C's two lowest bits
# (128-bit value and count-word loads of A, 128-bit count stores) when the count
# tensors start on 16 bytes, and one word at a time when they are offset by a word.
VEC_COUNT = [
    (list(range(15)), [14], list(range(14))),                 # one summed label, B a vertex-like tensor
    (list(range(16)), [14, 15], list(range(14))),             # two summed labels from B
    (list(range(15)), [14, 30], list(range(14)) + [30]),      # summed label plus a B-only label on top
]


@pytest.mark.parametrize("case", range(len(VEC_COUNT)))
@pytest.mark.parametrize("form", ["pair", "wide"])
@pytest.mark.parametrize("shift", [(0, 0), (1, 0), (0, 1)])
def test_contract_count_word_layouts(P, case, form, shift):
    la, lb, lc = VEC_COUNT[case]
    _outer_run(P, la, lb, lc, form == "pair", 2200 + case, sa=shift[0], sc=shift[1])


@pytest.mark.parametrize("case", range(len(VEC_COUNT)))
@pytest.mark.parametrize("unit", [(True, False), (False, True)])
def test_contract_count_word_layouts_unit(P, case, unit):
    la, lb, lc = VEC_COUNT[case]
    _outer_run(P, la, lb, lc, True, 2300 + case, unitA=unit[0], unitB=unit[1])


# Counting steps with long sums (64 to 256 summed assignments per output) whose
# shapes neither the register-tiled nor the split-K kernel takes (2^16 outputs, no
# or one B-only label): the streaming kernel's two passes, with many ties.
ONLINE = [
    (list(range(22)), list(range(16, 22)), list(range(16))),                       # 6 summed labels on A's top bits
    (list(range(100, 106)) + list(range(16)), list(range(100, 106)), list(range(16))),  # summed at A's low bits
    (list(range(21)), list(range(15, 21)) + [40], list(range(15)) + [40]),         # plus a B-only output label
    (list(range(24)), list(range(16, 24)), list(range(16))),                       # 8 summed labels
]


@pytest.mark.parametrize("case", range(len(ONLINE)))
@pytest.mark.parametrize("form", ["pair", "wide"])
def test_contract_one_pass_long_sums(P, case, form):
    la, lb, lc = ONLINE[case]
    _outer_run(P, la, lb, lc, form == "pair", 2400 + case, sc=case % 2)


@pytest.mark.parametrize("case", [0, 2])
@pytest.mark.parametrize("unit", [(True, False), (False, True)])
def test_contract_one_pass_unit_counts(P, case, unit):
    la, lb, lc = ONLINE[case]
    _outer_run(P, la, lb, lc, True, 2500 + case, unitA=unit[0], unitB=unit[1])


def test_contract_one_pass_infeasible_outputs(P):
    """Mostly infeasible operands: many outputs have no feasible assignment and keep
    their largest infeasible sum with count 0, as the oracle's definition stores them."""
    la, lb, lc = ONLINE[0]
    _outer_run(P, la, lb, lc, True, 2600, neg=0.95)


# Big-by-big steps whose sum is shorter than the tiled kernel's 16-deep chunk (4 or 8
# summed assignments): the streaming kernel gathers both operands.
TILED_SHORT = [
    # (m, n, k, batch, A's first group, B's first group, C order)
    (6, 6, 2, 1, "m", "k", "mnb"),   # 4 summed: three quarters of the chunk padded
    (6, 6, 3, 2, "k", "n", "nmb"),   # 8 summed
    (7, 4, 3, 1, "k", "k", "bnm"),   # 8 summed, 64 x 16 tiles
    (6, 5, 2, 0, "m", "n", "mn"),    # 4 summed, 5 B-only labels
]


@pytest.mark.parametrize("case", range(len(TILED_SHORT)))
@pytest.mark.parametrize("np_", [0, 1, 3])
def test_contract_tiled_short_sums(P, case, np_):
    la, lb, lc = _tiled_case(*TILED_SHORT[case])
    rng = np.random.default_rng(2700 + case)
    primes = P.primes(np_)
    A = _rand(rng, len(la), max(np_, 1), -4, 4, neg_frac=0.05)
    B = _rand(rng, len(lb), max(np_, 1), -4, 4, neg_frac=0.05)
    A = (A[0], A[1][:np_])
    B = (B[0], B[1][:np_])
    vc, cc = _run(P, la, A, lb, B, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, primes)
    assert np.array_equal(vc, ov)
    assert np.array_equal(cc, oc)


@pytest.mark.parametrize("case", range(len(TILED_SHORT)))
def test_contract_tiled_short_sums_pair(P, case):
    la, lb, lc = _tiled_case(*TILED_SHORT[case])
    _pair_case(P, la, lb, lc, 4, 2800 + case, lo=-4, hi=4)


@pytest.mark.parametrize("case", range(len(TILED_SHORT)))
def test_contract_tiled_short_sums_values16(P, case):
    la, lb, lc = _tiled_case(*TILED_SHORT[case])
    rng = np.random.default_rng(2900 + case)
    va = rng.integers(-2000, 2000, size=1 << len(la)).astype(np.int32)
    vb = rng.integers(-2000, 2000, size=1 << len(lb)).astype(np.int32)
    va[rng.random(va.size) < 0.8] = oracle.NEG
    vb[rng.random(vb.size) < 0.8] = oracle.NEG
    vc = P.contract_values16(la, torch.from_numpy(va).cuda(), lb, torch.from_numpy(vb).cuda(), lc)
    torch.cuda.synchronize()
    got = vc.cpu().numpy()
    ov, _ = oracle.contract(la, va, np.zeros((0, va.size), np.uint64), lb, vb, np.zeros((0, vb.size), np.uint64),
                            lc, [])
    feas = ov >= -(1 << 28)
    assert feas.any() and (~feas).any()
    assert np.array_equal(got[feas], ov[feas])
    assert (got[~feas] < -(1 << 28)).all()


# Steps with 2^16..2^18 outputs and long sums that the register-tiled kernel does not
# take (the streaming kernel then runs only 2^14..2^16 threads through the sums).
FEW_GROUPS = [
    (list(range(16)) + list(range(100, 106)), list(range(100, 106)) + [30], list(range(16)) + [30]),  # rc 17, rs 6
    (list(range(100, 108)) + list(range(16)), list(range(100, 108)), list(range(16))),  # summed at A's low bits
    (list(range(18)) + list(range(100, 106)), list(range(100, 106)) + [17], list(range(18))),  # rc 18, a batch label
]


@pytest.mark.parametrize("case", range(len(FEW_GROUPS)))
@pytest.mark.parametrize("form", ["pair", "wide"])
def test_contract_few_groups_long_sums(P, case, form):
    la, lb, lc = FEW_GROUPS[case]
    _outer_run(P, la, lb, lc, form == "pair", 3000 + case, sc=case % 2)


@pytest.mark.parametrize("case", range(len(FEW_GROUPS)))
def test_contract_few_groups_long_sums_values(P, case):
    la, lb, lc = FEW_GROUPS[case]
    rng = np.random.default_rng(3100 + case)
    A = _rand(rng, len(la), 1, -4, 4, neg_frac=0.05)
    B = _rand(rng, len(lb), 1, -4, 4, neg_frac=0.05)
    A, B = (A[0], A[1][:0]), (B[0], B[1][:0])
    vc, _ = _run(P, la, A, lb, B, lc, [])
    ov, _ = oracle.contract(la, A[0], A[1], lb, B[0], B[1], lc, [])
    assert np.array_equal(vc, ov)


def test_contract_few_groups_long_sums_reduction(P):
    """A single-operand reduction with 2^16 outputs of 64 terms each."""
    la, lc = list(range(22)), list(range(16))
    rng = np.random.default_rng(3200)
    primes = P.primes(3)
    A = _rand(rng, len(la), 3, -4, 4, neg_frac=0.05)
    vc, cc = _run(P, la, A, None, None, lc, primes)
    ov, oc = oracle.contract(la, A[0], A[1], None, None, None, lc, primes)
    assert np.array_equal(vc, ov) and np.array_equal(cc, oc)
