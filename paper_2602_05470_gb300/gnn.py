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


def features(inst, fixed: Optional[Iterable[int]] = None) -> np.ndarray:
    """Feature rows (n x 8, float32) of an MWIS instance; fixed[v] in {-1, 0, 1}."""
    lib = _lib.load()
    n = inst.n
    e = _flat_edges(inst)
    w = getattr(inst, "w", None)
    wv = np.ascontiguousarray(np.asarray(w, dtype=np.int32)) if w is not None else None
    fx = np.ascontiguousarray(np.asarray(fixed, dtype=np.int8)) if fixed is not None else None
    out = np.zeros((n, N_FEATURES), dtype=np.float32)
    check(lib.bbtn_gnn_features(n, len(inst.edges), e.ctypes.data_as(_lib._i32p),
                                wv.ctypes.data_as(_lib._i32p) if wv is not None else None,
                                fx.ctypes.data_as(_lib._i8p) if fx is not None else None, _f32(out)))
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
