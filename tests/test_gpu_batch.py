"""Uneven-resolution batches solved concurrently: cells on separate CUDA streams driven by
separate host threads give bitwise the same C^H as the same cells solved one after another
(every reduction has a fixed order and the hierarchies share no mutable state), and a
48^3 cell (dense 6^3 coarsest level) matches the oracle."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import solve
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu


def _solve(gmt, vox, stream):
    h = gmt.Hierarchy(vox, gmt.default_options(), stream)
    st, _, info = h.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
    CH = h.homogenize(gmt.ELASTIC)
    h.free()
    return CH, info.inner_total


def test_concurrent_streams_bitwise_equal_to_serial(gmt_lib):
    import torch
    gmt = gmt_lib
    cells = [L.batch_cell(3000 + i, resolutions=(32, 48, 64))[0] for i in range(6)]
    vox = [torch.from_numpy(v).cuda() for v in cells]
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    serial = [_solve(gmt, v, main) for v in vox]
    streams = [torch.cuda.Stream() for _ in range(3)]
    with ThreadPoolExecutor(max_workers=3) as ex:
        futs = [ex.submit(_solve, gmt, v, streams[i % 3]) for i, v in enumerate(vox)]
        conc = [f.result() for f in futs]
    torch.cuda.synchronize()
    for (a, ca), (b, cb) in zip(serial, conc):
        assert ca == cb
        assert np.array_equal(a, b)


def test_48_cell_matches_oracle(gmt_lib):
    gmt = gmt_lib
    vox = L.tpms_network("diamond", 48, 0.3)
    ref = solve.solve_cell(vox, "elastic", tol=1e-8)
    h = gmt.Hierarchy(vox)
    assert h.levels == 4 and h.level_res(3) == 6
    st, _, info = h.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
    CH = h.homogenize(gmt.ELASTIC)
    assert np.abs(CH - ref["CH"]).max() <= 1e-4 * np.abs(ref["CH"]).max()


def test_fp64_fallback_on_diverging_mixed_solve(gmt_lib):
    """A thin Schwarz-P cell (64^3, phi = 0.12) whose FP32 V-cycle is far from symmetric:
    the mixed-precision CG diverges, gmt_solve falls back to plain FP64 and converges to
    the FP64 solve's C^H."""
    gmt = gmt_lib
    vox, d = L.batch_cell(3026)
    assert d["family"] == "schwarz_p" and d["n"] == 64
    h = gmt.Hierarchy(vox)
    st, _, info = h.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
    assert st == gmt.OK and info.fp64_fallback == 1
    assert max(info.as_dict()["rel_residual"]) <= 1e-5
    CH = h.homogenize(gmt.ELASTIC)
    h64 = gmt.Hierarchy(vox, gmt.default_options(precision=gmt.FP64))
    st64, _, info64 = h64.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
    assert st64 == gmt.OK and info64.fp64_fallback == 0
    CH64 = h64.homogenize(gmt.ELASTIC)
    assert np.abs(CH - CH64).max() <= 1e-6 * np.abs(CH64).max()
    # without the fallback the mixed solve reports the divergence
    h2 = gmt.Hierarchy(vox, gmt.default_options(fp64_fallback=0))
    st2, _, info2 = h2.solve(gmt.ELASTIC, tol=1e-5, want_field=False, allow_not_converged=True)
    assert st2 == gmt.DIVERGED and info2.fp64_fallback == 0
