"""Writes tests/golden/*.json: exact oracle answers for the benchmark workloads.

Calls only the CPU oracle and the seeded generators. Run from the repo root:
    python tests/golden/make_golden.py
Workloads (seeds from synth.config_seed(family, index)):
  family 1: +-J spin glass, 8x8 open square lattice, no field, 1 instance
  family 2: unweighted MIS, random King's subgraph 30x30, filling 0.8, 32 instances
  family 6: +-J spin glass, 16x16 and 20x20 lattices, no field (cross-size checks)
  family 8: +-J spin glass, 20x20 lattices, field h = 0.5 (2h = 1), the paper's counting setting, 4 instances
  family 9: weighted MIS (weights 1..10), random King's subgraph 30x30, filling 0.8, 8 instances
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def main():
    out = {}
    t0 = time.time()
    inst = synth.square_lattice(8, seed=synth.config_seed(1, 0))
    e2, d = oracle.solve(inst)
    out["spin_8x8_f1"] = [{"seed": synth.config_seed(1, 0), "L": 8, "e2": e2, "count": str(d)}]
    rows = []
    for L, idx in ((16, 0), (16, 1), (20, 0)):
        seed = synth.config_seed(6, 100 * L + idx)
        e2, d = oracle.solve(synth.square_lattice(L, seed=seed))
        rows.append({"seed": seed, "L": L, "e2": e2, "count": str(d)})
    out["spin_large_f6"] = rows
    rows = []
    for idx in range(32):
        seed = synth.config_seed(2, idx)
        inst = synth.kings_subgraph(30, 0.8, seed=seed)
        a, d = oracle.mwis_ksg_tm(inst)
        rows.append({"seed": seed, "N": 30, "filling": 0.8, "n": inst.n, "alpha": a, "count": str(d)})
        print(idx, inst.n, a, d, f"{time.time() - t0:.1f}s", flush=True)
    out["ksg_30x30_f2"] = rows
    rows = []
    for idx in range(4):
        seed = synth.config_seed(8, idx)
        e2, d = oracle.solve(synth.square_lattice(20, seed=seed, h2=1))
        rows.append({"seed": seed, "L": 20, "h2": 1, "e2": e2, "count": str(d)})
        print("field", idx, e2, d, f"{time.time() - t0:.1f}s", flush=True)
    out["spin_20x20_field_f8"] = rows
    rows = []
    for idx in range(8):
        seed = synth.config_seed(9, idx)
        inst = synth.kings_subgraph(30, 0.8, seed=seed, weights="uniform10")
        a, d = oracle.mwis_ksg_tm(inst)
        rows.append({"seed": seed, "N": 30, "filling": 0.8, "weights": "uniform10", "n": inst.n, "alpha": a,
                     "count": str(d)})
        print("weighted", idx, inst.n, a, d, f"{time.time() - t0:.1f}s", flush=True)
    out["mwis_ksg_30x30_w10_f9"] = rows
    with open(os.path.join(HERE, "oracle_answers.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
