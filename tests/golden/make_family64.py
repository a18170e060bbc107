"""Writes tests/golden/family64.json: the FP64 oracle's converged C^H (elasticity) and
kappa^H (heat conduction) for one seeded 64^3 cell of each generator family, plus one
degenerate cell (a Schwarz-P network below its percolation threshold: isolated periodic
blobs, whose effective tensors are zero).

Cell i of family FAMILIES[i] uses the first seed seed0 + i + 16 k (k = 0, 1, ...) whose
oracle conductivity kappa^H has every diagonal entry above 1e-3 phi (a structure connected
across the cell in all three directions), so that every family cell has a nonzero tensor.

Only the oracle (assembled K, Jacobi-PCG to r <= 1e-10, energy-average C^H of App. F.1 /
F.2) and the seeded input generators are called; nothing here touches the CUDA library.
The GPU parity test regenerates the same cells from the same seeds and compares.

Run from the repository root:  python tests/golden/make_family64.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import solve  # noqa: E402
from paper_2604_26518_b300 import lattices as L  # noqa: E402

RES = 64
SEED0 = 5000
TOL = 1e-10


def connected(vox) -> bool:
    r = solve.solve_cell(vox, "heat", tol=1e-8)
    return bool(np.diag(r["CH"]).min() > 1e-3 * vox.mean())


def pick_seed(i: int, fam: str) -> int:
    for k in range(32):
        seed = SEED0 + i + 16 * k
        vox, _ = L.mixed_cell(seed, RES, families=(fam,))
        if connected(vox):
            return seed
    raise RuntimeError(f"no connected {fam} cell found")


def main():
    out = {"res": RES, "seed0": SEED0, "tol": TOL, "E": 1.0, "nu": 0.3, "k": 1.0,
           "note": "cell = lattices.mixed_cell(seed, res, families=(family,)); CH = oracle "
                   "C^H at r <= tol (elastic 6x6, heat 3x3); degenerate: the oracle's tensors "
                   "vanish (disconnected solid)",
           "cells": []}
    todo = [(fam, pick_seed(i, fam), False) for i, fam in enumerate(L.FAMILIES)]
    todo.append(("schwarz_p", SEED0 + 1, True))      # below the percolation threshold
    for fam, seed, degenerate in todo:
        vox, desc = L.mixed_cell(seed, RES, families=(fam,))
        rec = {"family": fam, "seed": seed, "phi": float(vox.mean()),
               "n_solid": int(vox.sum()), "degenerate": degenerate}
        for kind in ("elastic", "heat"):
            t = time.time()
            r = solve.solve_cell(vox, kind, tol=TOL)
            rec[kind] = {"CH": r["CH"].tolist(), "res": float(r["res"].max()),
                         "iters": int(r["iters"].max())}
            print(f"{fam:16s} {seed} {kind:8s} phi={rec['phi']:.4f} "
                  f"iters={rec[kind]['iters']} res={rec[kind]['res']:.2e} "
                  f"maxC={np.abs(r['CH']).max():.3e} {time.time() - t:.1f}s", flush=True)
        if degenerate:
            assert np.abs(np.array(rec["heat"]["CH"])).max() < 1e-10
        out["cells"].append(rec)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "family64.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
