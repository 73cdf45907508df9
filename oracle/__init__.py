"""CPU oracle for the counting-tropical contraction path (TEST INFRASTRUCTURE).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package. It shares no code with the CUDA library
(``paper_2602_05470_gb300``) and never imports it: both sides only share the
seeded graph generators in ``synth``.

The arithmetic lives in ``oracle.c`` (plain C, exact integers, big-integer
counts). This module compiles it with gcc and marshals arguments through
ctypes. Which paper passage each routine follows is stated in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# -infinity sentinel used by the max-plus form of the algebra (values are floored here)
NEG = -(1 << 29)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no GPU code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.POINTER
        i32p, u64p, i64p, i8p, u8p = P(C.c_int32), P(C.c_uint64), P(C.c_int64), P(C.c_int8), P(C.c_uint8)
        lib.oracle_spin_bruteforce.argtypes = [C.c_int, C.c_int, i32p, i32p, i32p, i64p, u64p, i8p]
        lib.oracle_mwis_bruteforce.argtypes = [C.c_int, C.c_int, i32p, i32p, i64p, u64p, i8p]
        lib.oracle_spin_square_tm.argtypes = [C.c_int, C.c_int, i32p, i32p, i32p, C.c_int, i64p,
                                              C.c_char_p, C.c_size_t, i8p]
        lib.oracle_mwis_ksg_tm.argtypes = [C.c_int, C.c_int, u8p, i32p, C.c_int, i64p, C.c_char_p,
                                           C.c_size_t, u64p]
        lib.oracle_contract.argtypes = [C.c_int, i32p, i32p, u64p, C.c_int, i32p, i32p, u64p,
                                        C.c_int, i32p, i32p, u64p, C.c_int, u64p, C.c_int32]
        for f in (lib.oracle_spin_bruteforce, lib.oracle_mwis_bruteforce, lib.oracle_spin_square_tm,
                  lib.oracle_mwis_ksg_tm, lib.oracle_contract):
            f.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def _i32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


# ---------------------------------------------------------------- problems

def spin_bruteforce(inst):
    """(E2 = 2*min H, degeneracy, one minimiser as +-1) by enumeration."""
    lib = _load()
    e = inst.edge_array()
    J, h2 = _i32(inst.J), _i32(inst.h2 if inst.h2 is not None else [0] * inst.n)
    e2, cnt = C.c_int64(), C.c_uint64()
    cfg = np.zeros(inst.n, np.int8)
    rc = lib.oracle_spin_bruteforce(inst.n, inst.m, _ptr(_i32(e.ravel()), C.c_int32),
                                    _ptr(J, C.c_int32), _ptr(h2, C.c_int32), C.byref(e2),
                                    C.byref(cnt), _ptr(cfg, C.c_int8))
    if rc:
        raise RuntimeError(f"oracle_spin_bruteforce rc={rc}")
    return e2.value, cnt.value, cfg


def mwis_bruteforce(inst):
    """(alpha, number of maximum-weight independent sets, one of them as 0/1)."""
    lib = _load()
    e = inst.edge_array()
    w = _i32(inst.w if inst.w is not None else [1] * inst.n)
    best, cnt = C.c_int64(), C.c_uint64()
    cfg = np.zeros(inst.n, np.int8)
    rc = lib.oracle_mwis_bruteforce(inst.n, inst.m, _ptr(_i32(e.ravel()), C.c_int32),
                                    _ptr(w, C.c_int32), C.byref(best), C.byref(cnt), _ptr(cfg, C.c_int8))
    if rc:
        raise RuntimeError(f"oracle_mwis_bruteforce rc={rc}")
    return best.value, cnt.value, cfg


def _square_couplings(inst):
    g = inst.geometry
    L, Lc = g["L"], g["Lc"]
    Jh = np.zeros((L, max(Lc - 1, 1)), np.int32)
    Jv = np.zeros((max(L - 1, 1), Lc), np.int32)
    for (i, j), J in zip(inst.edges, inst.J):
        ri, ci = divmod(i, Lc)
        rj, cj = divmod(j, Lc)
        if ri == rj and cj == ci + 1:
            Jh[ri, ci] = J
        elif ci == cj and rj == ri + 1:
            Jv[ri, ci] = J
        else:
            raise ValueError("edge is not a lattice bond")
    return L, Lc, Jh, Jv


def spin_square_tm(inst, want_config: bool = False, w64: int = 2):
    """(E2, exact degeneracy as int, minimiser or None) by the site-by-site sweep."""
    lib = _load()
    L, Lc, Jh, Jv = _square_couplings(inst)
    h2 = _i32(inst.h2 if inst.h2 is not None else [0] * inst.n)
    while True:
        e2 = C.c_int64()
        buf = C.create_string_buffer(8192)
        cfg = np.zeros(inst.n, np.int8) if want_config else None
        rc = lib.oracle_spin_square_tm(L, Lc, _ptr(_i32(Jh.ravel()), C.c_int32),
                                       _ptr(_i32(Jv.ravel()), C.c_int32), _ptr(h2, C.c_int32),
                                       w64, C.byref(e2), buf, 8192, _ptr(cfg, C.c_int8))
        if rc == -3:
            w64 *= 2
            continue
        if rc:
            raise RuntimeError(f"oracle_spin_square_tm rc={rc}")
        return e2.value, int(buf.value.decode()), cfg


def mwis_ksg_tm(inst, w64: int = 2):
    """(alpha, exact number of maximum-weight independent sets) on a King's subgraph."""
    lib = _load()
    g = inst.geometry
    N, Nc, mask = g["N"], g["Nc"], np.asarray(g["mask"], np.uint8)
    wsite = np.zeros(N * Nc, np.int32)
    sites = np.nonzero(mask)[0]
    wv = inst.w if inst.w is not None else [1] * inst.n
    for v, s in enumerate(sites):
        wsite[s] = wv[v]
    while True:
        best = C.c_int64()
        buf = C.create_string_buffer(8192)
        mx = C.c_uint64()
        rc = lib.oracle_mwis_ksg_tm(N, Nc, _ptr(mask, C.c_uint8), _ptr(wsite, C.c_int32), w64,
                                    C.byref(best), buf, 8192, C.byref(mx))
        if rc == -3:
            w64 *= 2
            continue
        if rc:
            raise RuntimeError(f"oracle_mwis_ksg_tm rc={rc}")
        return best.value, int(buf.value.decode())


def solve(inst, brute_limit: int = 22):
    """Exact optimum and degeneracy by whichever oracle route fits the instance.

    Spin glass: returns (E2 = 2 H*, D). MWIS: returns (alpha, D).
    """
    g = inst.geometry or {}
    if inst.kind == "spin":
        if g.get("kind") == "square" and min(g["L"], g["Lc"]) <= 24 and inst.n > brute_limit:
            if g["Lc"] <= g["L"]:
                e2, d, _ = spin_square_tm(inst)
                return e2, d
        if inst.n <= brute_limit:
            e2, d, _ = spin_bruteforce(inst)
            return e2, d
        if g.get("kind") == "square":
            e2, d, _ = spin_square_tm(inst)
            return e2, d
    else:
        if g.get("kind") == "ksg" and inst.n > brute_limit:
            return mwis_ksg_tm(inst)
        if inst.n <= brute_limit:
            a, d, _ = mwis_bruteforce(inst)
            return a, d
        if g.get("kind") == "ksg":
            return mwis_ksg_tm(inst)
    raise ValueError("no oracle route for this instance")


# ---------------------------------------------------------------- one contraction

def contract(la, va, ca, lb, vb, cb, lc, primes, neg: int = NEG):
    """Counting-tropical pairwise contraction by its definition.

    la/lb/lc: label lists (bit i of the linear index is variable label[i]).
    va: int32[2^ra]; ca: uint64[np, 2^ra] residues. lb=None -> single operand.
    Returns (vc int32[2^rc], cc uint64[np, 2^rc]).
    """
    lib = _load()
    primes = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
    npr = len(primes)
    la, lc = _i32(la), _i32(lc)
    ra, rc = len(la), len(lc)
    va = _i32(va)
    ca = np.ascontiguousarray(np.asarray(ca, dtype=np.uint64).reshape(npr, 1 << ra)) if npr else np.zeros(1, np.uint64)
    if lb is None:
        rb, lbp, vbp, cbp = -1, None, None, None
        lb_a = vb_a = cb_a = None
    else:
        lb_a = _i32(lb)
        rb = len(lb_a)
        vb_a = _i32(vb)
        cb_a = np.ascontiguousarray(np.asarray(cb, dtype=np.uint64).reshape(npr, 1 << rb)) if npr else np.zeros(1, np.uint64)
        lbp, vbp, cbp = _ptr(lb_a, C.c_int32), _ptr(vb_a, C.c_int32), _ptr(cb_a, C.c_uint64)
    vc = np.zeros(1 << rc, np.int32)
    cc = np.zeros((max(npr, 1), 1 << rc), np.uint64)
    r = lib.oracle_contract(ra, _ptr(la, C.c_int32), _ptr(va, C.c_int32), _ptr(ca, C.c_uint64),
                            rb, lbp, vbp, cbp, rc, _ptr(lc, C.c_int32), _ptr(vc, C.c_int32),
                            _ptr(cc, C.c_uint64), npr, _ptr(primes, C.c_uint64), int(neg))
    if r:
        raise RuntimeError(f"oracle_contract rc={r}")
    return vc, cc[:npr]
