"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here touches the CUDA library. Each group pins one oracle routine to
something other than itself: closed forms, invariants, special cases that reduce
to a library routine, or brute force on tiny inputs.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

PRIMES = [2**61 - 1, 2**61 - 31, 2**61 - 45]


# ---------------------------------------------------------------- brute force, spin glass

@pytest.mark.parametrize("seed", range(6))
def test_tree_closed_form(seed):
    """A tree is unfrustrated: E0 = -sum |J|, and with h = 0 exactly the two
    spin-flip-related configurations attain it (Eq. (1))."""
    inst = synth.random_tree(14, seed=seed, dist="uniform")
    e2, d, cfg = oracle.spin_bruteforce(inst)
    assert e2 == -2 * sum(abs(j) for j in inst.J)
    assert d == 2


@pytest.mark.parametrize("n", [3, 4, 5, 8, 11])
@pytest.mark.parametrize("frustrated", [False, True])
def test_cycle_closed_form(n, frustrated):
    """+-1 cycle: unfrustrated -> E0 = -n, D = 2; frustrated (odd number of
    antiferro bonds) -> exactly one broken bond: E0 = -n + 2, D = 2n."""
    J = [1] * n
    if frustrated:
        J[0] = -1
    inst = synth.cycle_graph(n, kind="spin", J=J)
    e2, d, _ = oracle.spin_bruteforce(inst)
    if frustrated:
        assert (e2, d) == (2 * (-n + 2), 2 * n)
    else:
        assert (e2, d) == (-2 * n, 2)


def test_free_spins_closed_form():
    inst = synth.empty_graph(9, kind="spin")
    assert oracle.spin_bruteforce(inst)[:2] == (0, 2**9)
    h2 = [3, -1, 2, -5, 1, 1, -2, 4, 7]
    inst = synth.empty_graph(9, kind="spin", h2=h2)
    assert oracle.spin_bruteforce(inst)[:2] == (-sum(abs(h) for h in h2), 1)


@pytest.mark.parametrize("seed", range(8))
def test_spin_flip_parity(seed):
    """With h = 0, H(s) = H(-s): the degeneracy is even."""
    inst = synth.square_lattice(4, seed=seed)
    _, d, _ = oracle.spin_bruteforce(inst)
    assert d % 2 == 0


def test_bruteforce_config_attains_energy():
    for seed in range(4):
        inst = synth.square_lattice(4, seed=seed, h2=1)
        e2, _, cfg = oracle.spin_bruteforce(inst)
        cfg = [int(x) for x in cfg]
        e = sum(-2 * J * cfg[i] * cfg[j] for (i, j), J in zip(inst.edges, inst.J))
        e += sum(-h * s for h, s in zip(inst.h2, cfg))
        assert e == e2


# ---------------------------------------------------------------- brute force, MWIS

@pytest.mark.parametrize("n", range(1, 13))
def test_path_closed_form(n):
    """Path P_n: alpha = ceil(n/2); one MIS for odd n, n/2 + 1 for even n."""
    a, d, _ = oracle.mwis_bruteforce(synth.path_graph(n))
    assert a == (n + 1) // 2
    assert d == (1 if n % 2 else n // 2 + 1)


@pytest.mark.parametrize("n", range(3, 13))
def test_cycle_mis_closed_form(n):
    """Cycle C_n: alpha = floor(n/2); 2 maximum sets for even n, n for odd n."""
    a, d, _ = oracle.mwis_bruteforce(synth.cycle_graph(n))
    assert a == n // 2
    assert d == (2 if n % 2 == 0 else n)


def test_complete_empty_star_closed_forms():
    assert oracle.mwis_bruteforce(synth.complete_graph(7))[:2] == (1, 7)
    assert oracle.mwis_bruteforce(synth.empty_graph(7))[:2] == (7, 1)
    w = [5, 2, 9, 9, 1, 3]
    assert oracle.mwis_bruteforce(synth.complete_graph(6, w=w))[:2] == (9, 2)
    # star: either the centre alone or all leaves
    assert oracle.mwis_bruteforce(synth.star_graph(6))[:2] == (5, 1)
    assert oracle.mwis_bruteforce(synth.star_graph(6, w=[5, 1, 1, 1, 1, 1]))[:2] == (5, 2)


def test_mwis_config_is_independent():
    inst = synth.kings_subgraph(4, 0.8, seed=11, weights="uniform10")
    a, _, x = oracle.mwis_bruteforce(inst)
    assert all(not (x[i] and x[j]) for i, j in inst.edges)
    assert sum(w for w, xi in zip(inst.w, x) if xi) == a


# ---------------------------------------------------------------- square-lattice transfer matrix

@pytest.mark.parametrize("shape", [(1, 6), (2, 3), (3, 3), (3, 4), (4, 4), (4, 5), (5, 4)])
@pytest.mark.parametrize("h2", [0, 1])
@pytest.mark.parametrize("dist", ["pm1", "uniform"])
def test_square_tm_vs_bruteforce(shape, h2, dist):
    L, Lc = shape
    for seed in range(3):
        inst = synth.square_lattice(L, seed=seed, Lc=Lc, h2=h2, dist=dist, jmax=5)
        bf = oracle.spin_bruteforce(inst)[:2]
        tm = oracle.spin_square_tm(inst)[:2]
        assert tm == bf


@pytest.mark.parametrize("L", [2, 5, 8, 12])
@pytest.mark.parametrize("dist", ["ferro", "antiferro"])
def test_square_tm_unfrustrated(L, dist):
    """Ferromagnet (and antiferromagnet: the lattice is bipartite) with h = 0:
    every bond satisfied, E0 = -#bonds, D = 2."""
    inst = synth.square_lattice(L, dist=dist)
    e2, d, cfg = oracle.spin_square_tm(inst, want_config=True)
    assert (e2, d) == (-2 * inst.m, 2)


def test_square_tm_dominant_field():
    """A field stronger than all couplings pins every spin: unique ground state."""
    inst = synth.square_lattice(6, seed=3, h2=20)
    e2, d, cfg = oracle.spin_square_tm(inst, want_config=True)
    assert d == 1 and (cfg == 1).all()
    assert e2 == sum(-2 * J for J in inst.J) - 20 * inst.n


@pytest.mark.parametrize("seed", range(4))
def test_square_tm_config_and_parity(seed):
    inst = synth.square_lattice(7, seed=seed)
    e2, d, cfg = oracle.spin_square_tm(inst, want_config=True)
    cfg = [int(x) for x in cfg]
    assert d % 2 == 0
    e = sum(-2 * J * cfg[i] * cfg[j] for (i, j), J in zip(inst.edges, inst.J))
    assert e == e2


# ---------------------------------------------------------------- King's-subgraph transfer matrix

@pytest.mark.parametrize("shape", [(3, 3), (4, 4), (4, 5), (5, 4), (3, 7), (2, 9)])
@pytest.mark.parametrize("weights", ["unit", "uniform10"])
def test_ksg_tm_vs_bruteforce(shape, weights):
    N, Nc = shape
    for seed in range(4):
        inst = synth.kings_subgraph(N, 0.8, seed=seed, weights=weights, Nc=Nc)
        if inst.n > 22:
            continue
        assert oracle.mwis_ksg_tm(inst) == oracle.mwis_bruteforce(inst)[:2]


@pytest.mark.parametrize("L", [3, 5, 7, 9, 11])
def test_ksg_tm_full_odd_king(L):
    """Full (2k+1)^2 king graph: the (k+1)^2 sites with both coordinates even
    form the unique maximum independent set (each 2x2 block holds at most one)."""
    inst = synth.kings_subgraph(L, 1.0)
    assert oracle.mwis_ksg_tm(inst) == (((L + 1) // 2) ** 2, 1)


def test_ksg_tm_single_row_is_path():
    for n in range(1, 12):
        inst = synth.kings_subgraph(1, 1.0, Nc=n)
        a = (n + 1) // 2
        assert oracle.mwis_ksg_tm(inst) == (a, 1 if n % 2 else n // 2 + 1)


def test_ksg_tm_isolated_sites():
    # sites two apart in both directions: no king adjacency -> alpha = n, D = 1
    mask = [1 if (r % 2 == 0 and c % 2 == 0) else 0 for r in range(7) for c in range(7)]
    inst = synth.kings_subgraph(7, 1.0)
    inst.geometry["mask"] = mask
    inst.n = sum(mask)
    inst.w = [1] * inst.n
    assert oracle.mwis_ksg_tm(inst) == (16, 1)


# ---------------------------------------------------------------- counting-tropical contraction

def _rand_tensor(rng, r, lo=-4, hi=4, np_=3):
    v = rng.integers(lo, hi + 1, size=1 << r).astype(np.int32)
    c = rng.integers(0, 2**61 - 100, size=(np_, 1 << r), dtype=np.uint64)
    return v, c


def test_contract_outer_product_closed_form():
    """No summed label: value = a + b, count = cA * cB mod p."""
    rng = np.random.default_rng(0)
    va, ca = _rand_tensor(rng, 2)
    vb, cb = _rand_tensor(rng, 3)
    vc, cc = oracle.contract([0, 1], va, ca, [2, 3, 4], vb, cb, [0, 1, 2, 3, 4], PRIMES)
    for o in range(1 << 5):
        ia, ib = o & 3, o >> 2
        assert vc[o] == va[ia] + vb[ib]
        for t, p in enumerate(PRIMES):
            assert int(cc[t, o]) == int(ca[t, ia]) * int(cb[t, ib]) % p


def test_contract_reduce_matches_numpy_max():
    """Single operand: the value is numpy's max over the summed axes; counts are
    the sums over the arg-max positions."""
    rng = np.random.default_rng(1)
    va, ca = _rand_tensor(rng, 5, -2, 2)
    vc, cc = oracle.contract([0, 1, 2, 3, 4], va, ca, None, None, None, [1, 3], PRIMES)
    T = va.reshape(2, 2, 2, 2, 2)  # axes: (4,3,2,1,0) in C order
    ref = T.max(axis=(0, 2, 4))     # keep labels 3 (axis 1) and 1 (axis 3) -> [l3][l1]
    for l1 in range(2):
        for l3 in range(2):
            assert vc[l1 + 2 * l3] == ref[l3, l1]
            for t, p in enumerate(PRIMES):
                s = 0
                for rest in range(8):
                    l0, l2, l4 = rest & 1, (rest >> 1) & 1, rest >> 2
                    idx = l0 | (l1 << 1) | (l2 << 2) | (l3 << 3) | (l4 << 4)
                    if va[idx] == vc[l1 + 2 * l3]:
                        s += int(ca[t, idx])
                assert int(cc[t, l1 + 2 * l3]) == s % p


def test_contract_output_permutation_is_transpose():
    rng = np.random.default_rng(2)
    va, ca = _rand_tensor(rng, 4)
    vb, cb = _rand_tensor(rng, 3)
    v1, c1 = oracle.contract([0, 1, 2, 3], va, ca, [3, 4, 5], vb, cb, [0, 1, 4, 5], PRIMES)
    v2, c2 = oracle.contract([0, 1, 2, 3], va, ca, [3, 4, 5], vb, cb, [5, 0, 4, 1], PRIMES)
    # bit order [0,1,4,5] -> [5,0,4,1]: numpy transpose of the reversed-axis view
    t1 = v1.reshape(2, 2, 2, 2)       # axes (5,4,1,0)
    t2 = v2.reshape(2, 2, 2, 2)       # axes (1,4,0,5)
    assert (np.transpose(t1, (2, 1, 3, 0)) == t2).all()


def test_contract_associativity():
    """(A B) C == A (B C): the algebra of the paper is a commutative semiring."""
    rng = np.random.default_rng(3)
    va, ca = _rand_tensor(rng, 3, -1, 1)
    vb, cb = _rand_tensor(rng, 3, -1, 1)
    vc_, cc_ = _rand_tensor(rng, 3, -1, 1)
    la, lb, lc = [0, 1, 2], [2, 3, 4], [4, 5, 0]
    ab_v, ab_c = oracle.contract(la, va, ca, lb, vb, cb, [0, 1, 3, 4], PRIMES)
    r1v, r1c = oracle.contract([0, 1, 3, 4], ab_v, ab_c, lc, vc_, cc_, [1, 3, 5], PRIMES)
    bc_v, bc_c = oracle.contract(lb, vb, cb, lc, vc_, cc_, [2, 3, 5, 0], PRIMES)
    r2v, r2c = oracle.contract(la, va, ca, [2, 3, 5, 0], bc_v, bc_c, [1, 3, 5], PRIMES)
    assert (r1v == r2v).all() and (r1c == r2c).all()


def test_contract_neg_floor():
    """Entries whose every candidate lies below the -infinity sentinel are the
    sentinel with count 0 (hard constraint (inf, 0) of the MWIS paragraph)."""
    neg = oracle.NEG
    va = np.array([neg, neg], np.int32)
    ca = np.zeros((3, 2), np.uint64)
    vb = np.array([neg, -5], np.int32)
    cb = np.ones((3, 2), np.uint64)
    vc, cc = oracle.contract([0], va, ca, [0], vb, cb, [], PRIMES)
    assert vc[0] == neg and (cc == 0).all()


def _spin_tn(inst):
    """Max-plus tensors of E2 = 2H: per edge -2 B^{ij}, per vertex -2 w^i with
    s = 0 <-> sigma = -1 (the tensors printed after Eq. (1))."""
    ts = []
    for (i, j), J in zip(inst.edges, inst.J):
        v = np.zeros(4, np.int32)
        for si in range(2):
            for sj in range(2):
                v[si | (sj << 1)] = 2 * J * (2 * si - 1) * (2 * sj - 1)
        ts.append(([i, j], v))
    for i in range(inst.n):
        ts.append(([i], np.array([-inst.h2[i], inst.h2[i]], np.int32)))
    return ts


def _mwis_tn(inst):
    """Max-plus MWIS tensors: B = [[0,0],[0,-inf]] (count 0 at -inf), w = (0, w_i)."""
    ts = []
    for (i, j) in inst.edges:
        ts.append(([i, j], np.array([0, 0, 0, oracle.NEG], np.int32)))
    for i in range(inst.n):
        ts.append(([i], np.array([0, inst.w[i]], np.int32)))
    return ts


def _contract_all(ts, order_seed):
    rng = np.random.default_rng(order_seed)
    order = rng.permutation(len(ts))
    ts = [ts[k] for k in order]
    npr = len(PRIMES)
    lab, val = ts[0]
    cnt = np.where(val > oracle.NEG, 1, 0).astype(np.uint64)[None, :].repeat(npr, 0)
    for k in range(1, len(ts)):
        lb, vb = ts[k]
        cb = np.where(vb > oracle.NEG, 1, 0).astype(np.uint64)[None, :].repeat(npr, 0)
        rest = set()
        for l2, _ in ts[k + 1:]:
            rest |= set(l2)
        out = [x for x in list(dict.fromkeys(list(lab) + list(lb))) if x in rest]
        val, cnt = oracle.contract(lab, val, cnt, lb, vb, cb, out, PRIMES)
        lab = out
    assert lab == []
    return int(val[0]), [int(c) for c in cnt[:, 0]]


@pytest.mark.parametrize("seed", range(4))
def test_contract_network_equals_bruteforce_spin(seed):
    """Contracting the whole spin-glass network (Eq. (2)) pairwise gives the
    brute-force ground energy and degeneracy, for any contraction order."""
    inst = synth.square_lattice(3, seed=seed, Lc=4, h2=seed % 2)
    e2, d, _ = oracle.spin_bruteforce(inst)
    for order_seed in range(2):
        v, c = _contract_all(_spin_tn(inst), order_seed)
        assert v == -e2
        assert c == [d % p for p in PRIMES]


@pytest.mark.parametrize("seed", range(4))
def test_contract_network_equals_bruteforce_mwis(seed):
    inst = synth.kings_subgraph(4, 0.8, seed=seed, weights="uniform10" if seed % 2 else "unit")
    a, d, _ = oracle.mwis_bruteforce(inst)
    v, c = _contract_all(_mwis_tn(inst), seed)
    assert v == a
    assert c == [d % p for p in PRIMES]


# ---------------------------------------------------------------- multi-limb counts (closed forms)
#
# The transfer-matrix oracles add counts as little-endian 64-bit limbs and print
# them in decimal; every pin above has D < 2^64. These instances are disjoint
# unions of small components whose optimum and degeneracy are known, so the
# totals are closed forms that cross 2^64 (one carry into the second limb) and
# 2^128 (the routine runs out of its two default limbs and is retried with four).
# A dropped carry, a limb-order slip in the decimal conversion or a lost retry
# changes the result.

def _ksg_components(rows, pattern):
    """Mask of `rows` occupied rows (an empty row between consecutive ones, so no
    king move joins them), each holding the same row pattern."""
    Nc = len(pattern)
    N = 2 * rows - 1
    mask = []
    for r in range(N):
        mask += [int(ch) for ch in pattern] if r % 2 == 0 else [0] * Nc
    return synth.kings_mask_graph(N, Nc, mask)


def test_ksg_tm_seventy_dominoes():
    """70 isolated dominoes (two adjacent sites): each has alpha 1 and 2 maximum
    sets, so alpha = 70 and D = 2^70 (one carry out of the low limb)."""
    inst = _ksg_components(35, "11011")
    assert inst.n == 140 and inst.m == 70
    assert oracle.mwis_ksg_tm(inst) == (70, 2 ** 70)


def test_ksg_tm_paths_dominoes_singles():
    """Per row: a 4-site path (alpha 2, 3 maximum sets: {1,3}, {1,4}, {2,4}), a
    domino (1, 2) and a single site (1, 1), separated by empty columns. Over 50
    rows alpha = 50 * 4 and D = 3^50 * 2^50 = 6^50 > 2^129."""
    inst = _ksg_components(50, "1111011010")
    assert inst.n == 50 * 7
    a, d = oracle.mwis_ksg_tm(inst)
    assert (a, d) == (200, 6 ** 50)
    assert d > 2 ** 128


def test_ksg_tm_multilimb_with_a_coupled_block():
    """The same rows plus one full 3x3 king block (alpha 4 with the four corners as
    the unique maximum set) in an extra row band: alpha and D change by exactly
    that component's (4, 1)."""
    base = _ksg_components(40, "1111011010")
    N, Nc = base.geometry["N"], base.geometry["Nc"]
    mask = list(base.geometry["mask"]) + [0] * Nc
    for r in range(3):
        mask += [1, 1, 1] + [0] * (Nc - 3)
    inst = synth.kings_mask_graph(N + 4, Nc, mask)
    assert oracle.mwis_ksg_tm(inst) == (40 * 4 + 4, 6 ** 40)


def _square_with(L, Lc, bonds, h2):
    """L x Lc open lattice with every coupling 0 except `bonds` {(i, j): J}."""
    inst = synth.square_lattice(L, Lc=Lc, dist="ferro")
    inst.J = [bonds.get((i, j), 0) for (i, j) in inst.edges]
    inst.h2 = list(h2)
    return inst


def test_square_tm_free_spins_two_limbs():
    """9 x 9 lattice with every coupling and field 0: every configuration has
    energy 0, so D = 2^81."""
    inst = _square_with(9, 9, {}, [0] * 81)
    e2, d, _ = oracle.spin_square_tm(inst)
    assert (e2, d) == (0, 2 ** 81)


def test_square_tm_three_state_pairs_four_limbs():
    """14 x 12 lattice, couplings 0 except the horizontal bonds (c, c+1) for c in
    {0, 3, 6, 9} of each row, J = +1, with 2h = +2 on the left spin and -2 on the
    right one. Such a pair has H = -s_a s_b - s_a + s_b: -1 at (+,+), (+,-) and
    (-,-), +3 at (-,+) -- three ground states. The other spins are free (D = 2
    each). So E2 = 2 * (-1) * 56 and D = 3^56 * 2^56 = 6^56 > 2^144."""
    L, Lc = 14, 12
    bonds, h2 = {}, [0] * (L * Lc)
    for r in range(L):
        for c in (0, 3, 6, 9):
            a, b = r * Lc + c, r * Lc + c + 1
            bonds[(a, b)] = 1
            h2[a], h2[b] = 2, -2
    inst = _square_with(L, Lc, bonds, h2)
    e2, d, cfg = oracle.spin_square_tm(inst, want_config=True)
    assert (e2, d) == (-112, 6 ** 56)
    e = sum(-2 * J * cfg[i] * cfg[j] for (i, j), J in zip(inst.edges, inst.J)) - sum(
        h * s for h, s in zip(h2, cfg))
    assert e == e2
