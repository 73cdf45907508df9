"""Seeded graph / coupling generators and the plain-text instance format.

Every random draw comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a 64-bit counter advanced by the
golden-ratio increment and finalised by two xor-shift-multiply rounds.

Workloads (paper, Applications section):
  * +-J spin glasses: couplings J_ij drawn from {+1, -1} with equal probability on
    open-boundary L x L square lattices (and 3D lattices / random regular graphs);
    the field h is an input (the paper's own counting runs use h = 0.5; fields are
    carried as the integer h2 = 2h so that energies stay integral).
  * Random King's subgraphs: each site of an N x N grid kept independently with
    probability equal to the filling rate (0.8 in the paper); kept sites are joined
    to their king-move neighbours (horizontal, vertical and diagonal distance 1).
    Vertices are numbered in row-major order of the kept sites.
  * Weighted MIS: integer vertex weights drawn uniformly from 1..10.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based 64-bit generator (published SplitMix64 finaliser)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Integer in [0, n) by rejection (unbiased)."""
        if n <= 0:
            raise ValueError("n must be positive")
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next_u64()
            if x < lim:
                return x % n

    def sign(self) -> int:
        return 1 if (self.next_u64() >> 63) else -1


def config_seed(config_id: int, idx: int) -> int:
    """Seed of instance `idx` of workload family `config_id`."""
    return 0xBB7A0000 + 1000 * config_id + idx


@dataclasses.dataclass
class Instance:
    kind: str                      # "spin" or "mwis"
    n: int
    edges: list                    # list of (i, j), i < j
    J: Optional[list] = None       # spin: coupling per edge
    h2: Optional[list] = None      # spin: 2*h per vertex
    w: Optional[list] = None       # mwis: weight per vertex
    geometry: Optional[dict] = None

    @property
    def m(self) -> int:
        return len(self.edges)

    def edge_array(self):
        import numpy as np
        return np.asarray(self.edges, dtype=np.int32).reshape(-1, 2)


# --------------------------------------------------------------------------
# spin-glass graphs
# --------------------------------------------------------------------------

def _couplings(rng: SplitMix64, m: int, dist: str, jmax: int):
    if dist == "pm1":
        return [rng.sign() for _ in range(m)]
    if dist == "ferro":
        return [1] * m
    if dist == "antiferro":
        return [-1] * m
    if dist == "uniform":              # nonzero integers in [-jmax, jmax]
        out = []
        for _ in range(m):
            v = rng.below(2 * jmax)          # [0, 2 jmax) -> [-jmax,-1] U [1,jmax]
            out.append(v - jmax if v < jmax else v - jmax + 1)
        return out
    raise ValueError(dist)


def square_lattice(L: int, seed: int = 0, dist: str = "pm1", h2=0, jmax: int = 1000,
                   Lc: Optional[int] = None) -> Instance:
    """Open-boundary L x Lc square lattice; vertex (r, c) -> r*Lc + c.

    Edges are listed site by site in row-major order: right neighbour first,
    then the one below. `h2` is an int (uniform 2h) or a list per vertex.
    """
    Lc = L if Lc is None else Lc
    rng = SplitMix64(seed)
    edges = []
    for r in range(L):
        for c in range(Lc):
            v = r * Lc + c
            if c + 1 < Lc:
                edges.append((v, v + 1))
            if r + 1 < L:
                edges.append((v, v + Lc))
    J = _couplings(rng, len(edges), dist, jmax)
    n = L * Lc
    h2l = list(h2) if isinstance(h2, (list, tuple)) else [int(h2)] * n
    return Instance("spin", n, edges, J=J, h2=h2l,
                    geometry={"kind": "square", "L": L, "Lc": Lc})


def cubic_lattice(L: int, seed: int = 0, dist: str = "pm1", h2=0, Ly: Optional[int] = None,
                  Lz: Optional[int] = None) -> Instance:
    """Open-boundary L x Ly x Lz cubic lattice (Ly = Lz = L by default); vertex
    (x, y, z) -> (x * Ly + y) * Lz + z. Edges site by site: +z, +y, +x."""
    Ly = L if Ly is None else Ly
    Lz = L if Lz is None else Lz
    rng = SplitMix64(seed)
    edges = []
    for x in range(L):
        for y in range(Ly):
            for z in range(Lz):
                v = (x * Ly + y) * Lz + z
                if z + 1 < Lz:
                    edges.append((v, v + 1))
                if y + 1 < Ly:
                    edges.append((v, v + Lz))
                if x + 1 < L:
                    edges.append((v, v + Ly * Lz))
    J = _couplings(rng, len(edges), dist, 1)
    n = L * Ly * Lz
    h2l = list(h2) if isinstance(h2, (list, tuple)) else [int(h2)] * n
    return Instance("spin", n, edges, J=J, h2=h2l, geometry={"kind": "cubic", "L": L, "Ly": Ly, "Lz": Lz})


def random_regular_graph(n: int, d: int, seed: int = 0, kind: str = "spin",
                         dist: str = "pm1", h2=0) -> Instance:
    """Random d-regular simple graph by the pairing model with restarts."""
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    rng = SplitMix64(seed)
    while True:
        stubs = [v for v in range(n) for _ in range(d)]
        for i in range(len(stubs) - 1, 0, -1):          # Fisher-Yates
            j = rng.below(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        es = set()
        ok = True
        for k in range(0, len(stubs), 2):
            a, b = stubs[k], stubs[k + 1]
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in es:
                ok = False
                break
            es.add(e)
        if ok:
            break
    edges = sorted(es)
    if kind == "spin":
        J = _couplings(rng, len(edges), dist, 1)
        h2l = list(h2) if isinstance(h2, (list, tuple)) else [int(h2)] * n
        return Instance("spin", n, edges, J=J, h2=h2l, geometry={"kind": "rrg", "d": d})
    return Instance("mwis", n, edges, w=[1] * n, geometry={"kind": "rrg", "d": d})


# --------------------------------------------------------------------------
# MIS graphs
# --------------------------------------------------------------------------

def kings_subgraph(N: int, filling: float = 0.8, seed: int = 0, weights: str = "unit",
                   Nc: Optional[int] = None) -> Instance:
    """Random King's subgraph on an N x Nc grid.

    Each site is kept when a uniform draw is below `filling`. `weights` is
    "unit" or "uniform10" (integers 1..10, drawn after the sites).
    geometry["mask"] is the row-major 0/1 occupancy of the N*Nc grid.
    """
    Nc = N if Nc is None else Nc
    rng = SplitMix64(seed)
    mask = [1 if rng.uniform() < filling else 0 for _ in range(N * Nc)]
    inst = kings_mask_graph(N, Nc, mask)
    if weights == "uniform10":
        inst.w = [1 + rng.below(10) for _ in range(inst.n)]
    elif weights != "unit":
        raise ValueError(weights)
    return inst


def kings_mask_graph(N: int, Nc: int, mask) -> Instance:
    """Unit-weight King's subgraph of a given row-major 0/1 site mask on an N x Nc
    grid: kept sites are numbered in row-major order and joined to the kept sites
    one king move away."""
    mask = [1 if m else 0 for m in mask]
    if len(mask) != N * Nc:
        raise ValueError("mask size")
    vid = [-1] * (N * Nc)
    n = 0
    for s in range(N * Nc):
        if mask[s]:
            vid[s] = n
            n += 1
    edges = []
    for r in range(N):
        for c in range(Nc):
            s = r * Nc + c
            if not mask[s]:
                continue
            for dr, dc in ((0, 1), (1, -1), (1, 0), (1, 1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < N and 0 <= cc < Nc and mask[rr * Nc + cc]:
                    edges.append((vid[s], vid[rr * Nc + cc]))
    edges.sort()
    return Instance("mwis", n, edges, w=[1] * n,
                    geometry={"kind": "ksg", "N": N, "Nc": Nc, "mask": mask})


def erdos_renyi(n: int, p: float, seed: int = 0, kind: str = "mwis", dist: str = "pm1",
                h2=0, weights: str = "unit") -> Instance:
    rng = SplitMix64(seed)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.uniform() < p]
    if kind == "spin":
        J = _couplings(rng, len(edges), dist, 1000)
        h2l = list(h2) if isinstance(h2, (list, tuple)) else [int(h2)] * n
        return Instance("spin", n, edges, J=J, h2=h2l, geometry={"kind": "er"})
    w = [1] * n if weights == "unit" else [1 + rng.below(10) for _ in range(n)]
    return Instance("mwis", n, edges, w=w, geometry={"kind": "er"})


def random_tree(n: int, seed: int = 0, kind: str = "spin", dist: str = "pm1", h2=0) -> Instance:
    """Random recursive tree: vertex v > 0 attaches to a uniform earlier vertex."""
    rng = SplitMix64(seed)
    edges = [(rng.below(v), v) for v in range(1, n)]
    edges.sort()
    if kind == "spin":
        J = _couplings(rng, len(edges), dist, 1000)
        h2l = list(h2) if isinstance(h2, (list, tuple)) else [int(h2)] * n
        return Instance("spin", n, edges, J=J, h2=h2l, geometry={"kind": "tree"})
    return Instance("mwis", n, edges, w=[1] * n, geometry={"kind": "tree"})


def _simple(kind, n, edges, J=None, h2=0, w=None, geom=None):
    if kind == "spin":
        J = [1] * len(edges) if J is None else list(J)
        h2l = list(h2) if isinstance(h2, (list, tuple)) else [int(h2)] * n
        return Instance("spin", n, edges, J=J, h2=h2l, geometry=geom)
    return Instance("mwis", n, edges, w=[1] * n if w is None else list(w), geometry=geom)


def path_graph(n: int, kind: str = "mwis", **kw) -> Instance:
    return _simple(kind, n, [(i, i + 1) for i in range(n - 1)], geom={"kind": "path"}, **kw)


def cycle_graph(n: int, kind: str = "mwis", **kw) -> Instance:
    edges = [(i, i + 1) for i in range(n - 1)] + ([(0, n - 1)] if n > 2 else [])
    return _simple(kind, n, edges, geom={"kind": "cycle"}, **kw)


def complete_graph(n: int, kind: str = "mwis", **kw) -> Instance:
    return _simple(kind, n, [(i, j) for i in range(n) for j in range(i + 1, n)],
                   geom={"kind": "complete"}, **kw)


def empty_graph(n: int, kind: str = "mwis", **kw) -> Instance:
    return _simple(kind, n, [], geom={"kind": "empty"}, **kw)


def star_graph(n: int, kind: str = "mwis", **kw) -> Instance:
    return _simple(kind, n, [(0, i) for i in range(1, n)], geom={"kind": "star"}, **kw)


# --------------------------------------------------------------------------
# plain-text instance files
# --------------------------------------------------------------------------
#   c <free text>                 comment (geometry is stored in comments)
#   p spin <n> <m> | p mwis <n> <m>
#   e <i> <j> <J>   (spin)  |  e <i> <j>   (mwis)      -- 0-based vertices
#   f <i> <h2>      (spin, omitted = 0)  |  w <i> <weight>  (mwis, omitted = 1)

def write_instance(inst: Instance, path: str) -> None:
    with open(path, "w") as f:
        g = inst.geometry or {}
        if g.get("kind") == "square":
            f.write(f"c geometry square {g['L']} {g['Lc']}\n")
        elif g.get("kind") == "ksg":
            f.write(f"c geometry ksg {g['N']} {g['Nc']} " + "".join(map(str, g["mask"])) + "\n")
        f.write(f"p {inst.kind} {inst.n} {inst.m}\n")
        for k, (i, j) in enumerate(inst.edges):
            if inst.kind == "spin":
                f.write(f"e {i} {j} {inst.J[k]}\n")
            else:
                f.write(f"e {i} {j}\n")
        if inst.kind == "spin":
            for i, h in enumerate(inst.h2 or []):
                if h:
                    f.write(f"f {i} {h}\n")
        else:
            for i, wv in enumerate(inst.w or []):
                if wv != 1:
                    f.write(f"w {i} {wv}\n")


def read_instance(path: str) -> Instance:
    kind = None
    n = 0
    edges, J = [], []
    geom = None
    fields = {}
    weights = {}
    with open(path) as f:
        for line in f:
            t = line.split()
            if not t:
                continue
            if t[0] == "c":
                if len(t) >= 3 and t[1] == "geometry":
                    if t[2] == "square":
                        geom = {"kind": "square", "L": int(t[3]), "Lc": int(t[4])}
                    elif t[2] == "ksg":
                        geom = {"kind": "ksg", "N": int(t[3]), "Nc": int(t[4]),
                                "mask": [int(ch) for ch in t[5]]}
            elif t[0] == "p":
                kind, n = t[1], int(t[2])
            elif t[0] == "e":
                edges.append((int(t[1]), int(t[2])))
                if kind == "spin":
                    J.append(int(t[3]))
            elif t[0] == "f":
                fields[int(t[1])] = int(t[2])
            elif t[0] == "w":
                weights[int(t[1])] = int(t[2])
    if kind == "spin":
        return Instance("spin", n, edges, J=J, h2=[fields.get(i, 0) for i in range(n)], geometry=geom)
    return Instance("mwis", n, edges, w=[weights.get(i, 1) for i in range(n)], geometry=geom)
