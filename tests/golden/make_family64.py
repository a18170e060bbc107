"""Writes tests/golden/family64.json: the FP64 oracle's converged C^H (elasticity) and
kappa^H (heat conduction) for one seeded 64^3 cell of each generator family.

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


def cell(i: int, fam: str):
    """The 64^3 cell of family `fam` (index i in lattices.FAMILIES)."""
    return L.mixed_cell(SEED0 + i, RES, families=(fam,))


def main():
    out = {"res": RES, "seed0": SEED0, "tol": TOL, "E": 1.0, "nu": 0.3, "k": 1.0,
           "note": "cell i = lattices.mixed_cell(seed0 + i, res, families=(FAMILIES[i],)); "
                   "CH = oracle C^H at r <= tol (elastic 6x6, heat 3x3)",
           "cells": []}
    for i, fam in enumerate(L.FAMILIES):
        vox, desc = cell(i, fam)
        rec = {"family": fam, "seed": SEED0 + i, "phi": float(vox.mean()),
               "n_solid": int(vox.sum())}
        for kind in ("elastic", "heat"):
            t = time.time()
            r = solve.solve_cell(vox, kind, tol=TOL)
            rec[kind] = {"CH": r["CH"].tolist(), "res": float(r["res"].max()),
                         "iters": int(r["iters"].max())}
            print(f"{fam:16s} {kind:8s} phi={rec['phi']:.4f} iters={rec[kind]['iters']} "
                  f"res={rec[kind]['res']:.2e} {time.time() - t:.1f}s", flush=True)
        out["cells"].append(rec)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "family64.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
