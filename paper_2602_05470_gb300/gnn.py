"""Learned branch scorer: a thin binding of the ``bbtn_gnn_*`` entry points.

The model (3 message-passing layers, hidden width 64, fp32) and its forward,
backward and Adam kernels live in the library; this module only marshals host
arrays and builds training samples. The paper's discussion proposes learned
policies in place of its myopic branching heuristics; the solver uses this model
for a first incumbent and for the order of children (MWIS instances only), never
for pruning, so solver results do not depend on it.
"""
from __future__ import annotations

import ctypes as C
from typing import Iterable, Optional

import numpy as np

from . import _lib
from ._lib import check

N_FEATURES = 8


def _f32(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _flat_edges(inst):
    return np.ascontiguousarray(np.asarray(inst.edges, dtype=np.int32).reshape(-1))


def features(inst, fixed: Optional[Iterable[int]] = None, score=None) -> np.ndarray:
    """Feature rows (n x 8, float32); fixed[v] in {-1, 0, 1}; score: overflow shares."""
    lib = _lib.load()
    n = inst.n
    e = _flat_edges(inst)
    w = getattr(inst, "w", None)
    if inst.kind == "spin":
        h2 = getattr(inst, "h2", None)
        w = [abs(int(x)) for x in h2] if h2 is not None else [0] * n
    wv = np.ascontiguousarray(np.asarray(w, dtype=np.int32)) if w is not None else None
    sv = np.ascontiguousarray(np.asarray(score, dtype=np.float32)) if score is not None else None
    fx = np.ascontiguousarray(np.asarray(fixed, dtype=np.int8)) if fixed is not None else None
    out = np.zeros((n, N_FEATURES), dtype=np.float32)
    check(lib.bbtn_gnn_features(n, len(inst.edges), e.ctypes.data_as(_lib._i32p),
                                wv.ctypes.data_as(_lib._i32p) if wv is not None else None,
                                fx.ctypes.data_as(_lib._i8p) if fx is not None else None,
                                _f32(sv) if sv is not None else None, _f32(out)))
    return out


class GNN:
    """One model with its parameters, gradients and Adam moments on the device."""

    def __init__(self, seed: int = 0, stream=None):
        lib = _lib.load()
        self._h = C.c_void_p()
        check(lib.bbtn_gnn_create(seed, C.byref(self._h)))
        if stream is not None:
            check(lib.bbtn_gnn_set_stream(self._h, int(stream)))
        self.n = 0

    @staticmethod
    def param_count() -> int:
        return _lib.load().bbtn_gnn_param_count()

    def close(self):
        if self._h:
            _lib.load().bbtn_gnn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graph(self, inst):
        e = _flat_edges(inst)
        check(_lib.load().bbtn_gnn_set_graph(self._h, inst.n, len(inst.edges), e.ctypes.data_as(_lib._i32p)))
        self.n = inst.n

    def forward(self, feats: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(feats, dtype=np.float32)
        assert f.shape == (self.n, N_FEATURES)
        out = np.zeros(self.n, dtype=np.float32)
        check(_lib.load().bbtn_gnn_forward(self._h, _f32(f), _f32(out)))
        return out

    def train_step(self, feats, labels, mask, lr: float) -> float:
        f = np.ascontiguousarray(feats, dtype=np.float32)
        y = np.ascontiguousarray(labels, dtype=np.float32)
        m = np.ascontiguousarray(mask, dtype=np.float32)
        assert f.shape == (self.n, N_FEATURES) and y.shape == (self.n,) and m.shape == (self.n,)
        loss = C.c_float()
        check(_lib.load().bbtn_gnn_train_step(self._h, _f32(f), _f32(y), _f32(m), float(lr), C.byref(loss)))
        return loss.value

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.param_count(), dtype=np.float32)
        check(_lib.load().bbtn_gnn_get_params(self._h, _f32(p)))
        return p

    def set_params(self, p: np.ndarray):
        q = np.ascontiguousarray(p, dtype=np.float32)
        assert q.shape == (self.param_count(),)
        check(_lib.load().bbtn_gnn_set_params(self._h, _f32(q)))

    def get_grads(self) -> np.ndarray:
        g = np.zeros(self.param_count(), dtype=np.float32)
        check(_lib.load().bbtn_gnn_get_grads(self._h, _f32(g)))
        return g

    def save(self, path: str):
        np.save(path, self.get_params())

    def load(self, path: str):
        self.set_params(np.load(path))


def samples(inst, x_opt, rng: np.random.Generator, k: int, max_fixed: float = 0.5):
    """k training samples from one optimal configuration x_opt of an MWIS instance.

    Each sample fixes a random subset (a fraction in [0, max_fixed]) of the vertices
    to their values in x_opt -- a sub-problem of which x_opt is still optimal -- and
    asks for x_opt on the free vertices. Returns (feats, labels, mask) triples.
    """
    x = np.asarray(x_opt, dtype=np.float32)
    out = []
    for i in range(k):
        frac = 0.0 if i == 0 else rng.uniform(0.0, max_fixed)
        fix = rng.random(inst.n) < frac
        fixed = np.where(fix, x.astype(np.int8), -1).astype(np.int8)
        out.append((features(inst, fixed), x.copy(), (~fix).astype(np.float32)))
    return out


def train(model: GNN, data, epochs: int, lr: float = 3e-3, rng: Optional[np.random.Generator] = None):
    """Plain Adam training over a list of (inst, [(feats, labels, mask), ...]); returns epoch mean losses."""
    rng = rng or np.random.default_rng(0)
    hist = []
    for _ in range(epochs):
        tot, cnt = 0.0, 0
        for j in rng.permutation(len(data)):
            inst, smp = data[j]
            model.set_graph(inst)
            for f, y, m in smp:
                tot += model.train_step(f, y, m, lr)
                cnt += 1
        hist.append(tot / max(cnt, 1))
    return hist


def mean_loss(model: GNN, data) -> float:
    """Masked loss averaged over samples, without changing the parameters."""
    tot, cnt = 0.0, 0
    for inst, smp in data:
        model.set_graph(inst)
        for f, y, m in smp:
            tot += model.train_step(f, y, m, 0.0)
            cnt += 1
    return tot / max(cnt, 1)


# ---------------------------------------------------------------- branch scorer data

def branch_rows(inst, cap: int, max_rows: int, lookahead: int = 16, seed: int = 1, region_size: int = 8):
    """Training rows of the branch scorer from one instance (host-side search).

    Every expanded node of the lookahead search gives one row: features with the
    overflow shares, label 1 on the candidate seeds whose branching attains the
    smallest gamma, mask on the candidates. Rows where all candidates tie carry no
    signal and are dropped.
    """
    from . import Solver
    s = Solver(space_cap_log2=cap, seed=seed, region_size=region_size)
    fx, sc, ga = s.branch_samples(inst, max_rows, lookahead)
    s.close()
    out = []
    for r in range(len(fx)):
        g = ga[r]
        cand = g > 0
        if cand.sum() < 2:
            continue
        gmin = g[cand].min()
        y = (cand & (g <= gmin * (1 + 1e-6))).astype(np.float32)
        if y.sum() == cand.sum():
            continue
        out.append((features(inst, fx[r], sc[r]), y, cand.astype(np.float32)))
    return out


def _rows_job(args):
    kind, N, seed, cap, max_rows, lookahead = args[:6]
    region_size = args[6] if len(args) > 6 else 8
    import synth
    inst = synth.kings_subgraph(N, 0.8, seed=seed)
    return inst, branch_rows(inst, cap, max_rows, lookahead, region_size=region_size)


def branch_dataset(specs, workers: int = 0):
    """[(kind, N, seed, cap, max_rows, lookahead[, region_size])] -> [(inst, rows)], host
    processes in parallel."""
    import multiprocessing as mp
    import os
    workers = workers or max(1, (os.cpu_count() or 2) - 1)
    if workers == 1:
        return [_rows_job(a) for a in specs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_rows_job, specs, chunksize=1)


def top1_agreement(model: GNN, data) -> float:
    """Fraction of rows whose top-scored candidate is one of the best seeds."""
    hit = tot = 0
    for inst, rows in data:
        if not rows:
            continue
        model.set_graph(inst)
        for f, y, m in rows:
            s = model.forward(f)
            s = np.where(m > 0, s, -np.inf)
            hit += y[int(np.argmax(s))] > 0
            tot += 1
    return hit / max(tot, 1)
