"""Small, fixed launch sequences for profiling the library under ncu.

    python -m paper_2604_26518_b300.profile_case smoother   # k_stencil on one 128^3 cell
    python -m paper_2604_26518_b300.profile_case smoother16 # the same, FP16 coarse stencils
    python -m paper_2604_26518_b300.profile_case setup      # hierarchy + operators, twice
    python -m paper_2604_26518_b300.profile_case solve      # one solve + C^H of one cell

The `smoother` case builds the first cell of the benchmark batch (seed 2000, 128^3), then
runs two Jacobi sweeps on level 0 followed by two on level 1 (four k_stencil launches,
each preceded by layout-conversion kernels), so that `ncu -k regex:k_stencil -c 4`
captures the level-0 and a coarse-level smoother without profiling a full run.
"""
from __future__ import annotations

import sys

import numpy as np

from . import gmt, lattices

FAMILIES = ("gyroid", "schwarz_p", "diamond", "plate_gyroid", "plate_schwarz_p",
            "plate_diamond", "bcc", "octet")


def cell(seed: int = 2000, n: int = 128):
    return lattices.mixed_cell(seed, n, families=FAMILIES)[0]


def main(argv):
    import torch
    case = argv[1] if len(argv) > 1 else "smoother"
    vox = cell()
    if case in ("smoother", "smoother16"):
        h = gmt.Hierarchy(vox, gmt.default_options(coarse_fp16=int(case == "smoother16")))
        h.prepare(gmt.ELASTIC)
        rng = np.random.default_rng(0)
        for level in (0, 1):
            n = h.num_nodes(level)
            f = rng.standard_normal((n * 3, 6))
            u = rng.standard_normal((n * 3, 6))
            h.smooth(level, f, u, 2, gmt.FP32)
    elif case == "setup":
        v = torch.from_numpy(vox).cuda()
        for _ in range(2):
            h = gmt.Hierarchy(v)
            h.prepare(gmt.ELASTIC)
            h.free()
    elif case == "solve":
        h = gmt.Hierarchy(torch.from_numpy(vox).cuda())
        st, _, info = h.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
        h.homogenize(gmt.ELASTIC)
        print(info.as_dict())
    else:
        raise SystemExit(f"unknown case {case}")
    torch.cuda.synchronize()
    print("done", case)


if __name__ == "__main__":
    main(sys.argv)
