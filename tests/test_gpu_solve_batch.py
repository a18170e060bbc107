"""Batched solves (gmt_solve_batch): cells of different sizes and level counts solved
together, their mixed-precision V-cycles run as shared batched launches, give every cell
bitwise the field, V-cycle count and C^H of its own gmt_solve, a non-percolating cell's
FP64 fallback included; the C^H of one cell also matches the converged oracle."""
import numpy as np
import pytest

from oracle import solve
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu


def _cells():
    cells = [L.batch_cell(3000 + i, resolutions=(32, 48, 64))[0] for i in range(6)]
    vox, d = L.batch_cell(3026)          # 64^3 Schwarz-P below percolation: FP64 fallback
    assert d["family"] == "schwarz_p" and d["n"] == 64
    return cells + [vox, L.tpms_network("gyroid", 32, 0.3)]


def _single(gmt, vox, physics, tol):
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(physics, tol=tol, allow_not_converged=True)
    CH = h.homogenize(physics)
    h.free()
    return st, u, info, CH


@pytest.mark.parametrize("physics", ["elastic", "heat"])
def test_batch_solve_bitwise_equal_to_single(gmt_lib, physics):
    import torch
    gmt = gmt_lib
    ph = gmt.ELASTIC if physics == "elastic" else gmt.HEAT
    cells = _cells()
    ref = [_single(gmt, v, ph, 1e-5) for v in cells]
    hs = [gmt.Hierarchy(v) for v in cells]
    assert len({h.levels for h in hs}) > 1
    res = gmt.solve_batch(hs, ph, tol=1e-5, allow_not_converged=True)
    for (st, u, info, CH), (bst, bu, binfo), h in zip(ref, res, hs):
        assert bst == st
        assert torch.equal(bu, u)
        assert binfo.inner_total == info.inner_total and binfo.outer == info.outer
        assert binfo.fp64_fallback == info.fp64_fallback
        assert list(binfo.rel_residual) == list(info.rel_residual)
        assert np.array_equal(h.homogenize(ph), CH)
    if ph == gmt.ELASTIC:
        assert ref[6][2].fp64_fallback == 1          # the fallback ran inside the batch
        assert all(r[0] == gmt.OK for r in ref)
    for h in hs:
        h.free()


def test_batch_solve_warm_start_and_matches_oracle(gmt_lib):
    import torch
    gmt = gmt_lib
    cells = _cells()[:3] + [_cells()[7]]
    hs = [gmt.Hierarchy(v) for v in cells]
    res = gmt.solve_batch(hs, gmt.ELASTIC, tol=1e-3)
    # continue two of them from their tol-1e-3 fields, the others from zero
    u0 = [res[0][1], None, res[2][1], None]
    ref = []
    for v, x in zip(cells, u0):
        h = gmt.Hierarchy(v)
        st, u, info = h.solve(gmt.ELASTIC, tol=1e-6, u0=x)
        ref.append((u, info.inner_total, h.homogenize(gmt.ELASTIC)))
        h.free()
    hs2 = [gmt.Hierarchy(v) for v in cells]
    res2 = gmt.solve_batch(hs2, gmt.ELASTIC, tol=1e-6, u0s=u0)
    for (u, cyc, CH), (st, bu, binfo), h in zip(ref, res2, hs2):
        assert st == gmt.OK and torch.equal(bu, u) and binfo.inner_total == cyc
        assert np.array_equal(h.homogenize(gmt.ELASTIC), CH)
    oracle = solve.solve_cell(cells[3], "elastic", tol=1e-10)["CH"]
    CH = hs2[3].homogenize(gmt.ELASTIC)
    assert np.abs(CH - oracle).max() <= 1e-4 * np.abs(oracle).max()
    for h in hs + hs2:
        h.free()


def test_batch_solve_rejects_unsupported_options(gmt_lib):
    gmt = gmt_lib
    v = L.tpms_network("gyroid", 16, 0.3)
    a = gmt.Hierarchy(v)
    for opts in (dict(smoother=gmt.CHEBYSHEV), dict(precision=gmt.FP64), dict(cycle=gmt.CYCLE_W),
                 dict(omega=0.5)):
        b = gmt.Hierarchy(v, gmt.default_options(**opts))
        with pytest.raises(gmt.GmtError) as e:
            gmt.solve_batch([a, b], gmt.ELASTIC)
        assert e.value.status == gmt.ERR_ARG
        b.free()
    with pytest.raises(gmt.GmtError) as e:
        gmt.solve_batch([a, a], gmt.ELASTIC)
    assert e.value.status == gmt.ERR_ARG
    a.free()


def test_batch_of_one_without_fields(gmt_lib):
    """A batch of one cell, with no field copied out: the stored solution's C^H and the
    V-cycle count are gmt_solve's."""
    gmt = gmt_lib
    vox = L.tpms_plate("diamond", 48, 0.3)
    h1 = gmt.Hierarchy(vox)
    st, _, info = h1.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
    CH = h1.homogenize(gmt.ELASTIC)
    h2 = gmt.Hierarchy(vox)
    (bst, bu, binfo), = gmt.solve_batch([h2], gmt.ELASTIC, tol=1e-5, want_fields=False)
    assert bst == st == gmt.OK and bu is None and binfo.inner_total == info.inner_total
    assert np.array_equal(h2.homogenize(gmt.ELASTIC), CH)
    h1.free()
    h2.free()
