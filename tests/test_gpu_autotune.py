"""Solver-schedule autotuner (gmt_autotune): every candidate schedule solves the cell to the
tolerance (the twelve sweep schedules, then the fastest of them with the finer
true-residual replacement threshold), the chosen one is the fastest measured and is set on
the hierarchy, and a solve with it reaches the same C^H as the default schedule (within the
solve tolerance's reach, 1e-4 of the converged oracle)."""
import math

import numpy as np
import pytest

from oracle import solve
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("physics", ["elastic", "heat"])
def test_autotune_picks_the_fastest_converging_schedule(gmt_lib, physics):
    gmt = gmt_lib
    ph = gmt.ELASTIC if physics == "elastic" else gmt.HEAT
    vox = L.tpms_network("diamond", 48, 0.3)
    h = gmt.Hierarchy(vox)
    best, times = h.autotune(ph, tol=1e-5)
    assert times.shape == (gmt.AUTOTUNE_CANDIDATES,)
    assert np.all(np.isfinite(times)) and np.all(times > 0)    # every candidate converged
    i = int(np.argmin(times))
    j = int(np.argmin(times[:12])) if i == 12 else i     # candidate 12: 0..11's fastest
    assert (best.nu_pre, best.nu_post, best.nu_coarse, best.coarse_fp16) == \
        (1 + j // 6, 1 + j // 6, 1 + (j // 2) % 3, j % 2)
    assert best.inner_tol == (0.003 if i == 12 else gmt.default_options().inner_tol)
    st, _, info = h.solve(ph, tol=1e-5, want_field=False)
    assert st == gmt.OK and max(info.as_dict()["rel_residual"]) <= 1e-5
    CH = h.homogenize(ph)
    ref = solve.solve_cell(vox, physics, tol=1e-10)["CH"]
    assert np.abs(CH - ref).max() <= 1e-4 * np.abs(ref).max()
    h.free()


def test_autotune_fp64_skips_fp16_candidates(gmt_lib):
    gmt = gmt_lib
    h = gmt.Hierarchy(L.tpms_network("gyroid", 32, 0.3), gmt.default_options(precision=gmt.FP64))
    best, times = h.autotune(gmt.ELASTIC, tol=1e-5)
    assert all(math.isinf(t) for t in times[1:12:2])
    assert all(math.isfinite(t) for t in times[0:12:2])
    assert math.isinf(times[12])               # the inner-tolerance candidate is mixed only
    assert best.coarse_fp16 == 0 and best.precision == gmt.FP64
    h.free()
