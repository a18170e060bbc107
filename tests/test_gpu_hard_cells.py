"""The hard cells of the uneven-resolution batch (seeds 3000 + i of lattices.batch_cell).

  * Non-percolating cells: the largest face-connected component does not reach across the
    periodic cell (a Schwarz-P network below its percolation threshold, seed 3026; a
    spinodal whose largest component is a small blob, seed 3025). Such a component is free
    to rotate as well as to translate, so K has rotational null modes that the zero-mean
    projection does not remove; the mixed-precision recurrence picks them up from FP32
    rounding and diverges, and gmt_solve's FP64 fallback solves the cell. The oracle's
    conductivity of these cells vanishes (the test that they do not percolate); their C^H
    vanishes too, so it is held to 1e-4 of the Voigt scale phi |C0|.
  * Slow spinodal cells (seeds 3010, 3041, 128^3, wavenumbers 9-10): the V-cycle contracts
    slowly (560-1100 cycles, the same in FP64), and they converge within the default cap.
    Checked through the oracle's matrix-free residual of the library's field, and C^H
    symmetric and below the Voigt bound phi C0.
"""
import numpy as np
import pytest

from oracle import fe, solve
from oracle.grid import Level
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [3026, 3025])
def test_non_percolating_cells_fall_back_and_converge(gmt_lib, seed):
    gmt = gmt_lib
    vox, desc = L.batch_cell(seed)
    kap = solve.solve_cell(vox, "heat", tol=1e-8)["CH"]
    assert np.abs(kap).max() < 1e-10, "cell percolates"
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(gmt.ELASTIC, tol=1e-5)
    assert st == gmt.OK, info.as_dict()
    Ke, x0, D, M, C0 = fe.physics("elastic")
    CH = h.homogenize(gmt.ELASTIC)
    assert np.abs(CH).max() <= 1e-4 * vox.mean() * np.abs(C0).max(), CH
    lev = Level(vox.astype(bool))
    U = u.detach().cpu().numpy().reshape(-1, M)
    F = solve.cancel_rounding(solve.load(lev, Ke, x0, D), solve.gross_load_norm(lev, Ke, x0, D))
    R = F - solve.apply_ebe(lev, Ke, U, D)
    fn = np.linalg.norm(F, axis=0)
    res = np.where(fn > 0, np.linalg.norm(R, axis=0) / np.where(fn > 0, fn, 1), 0)
    assert res.max() <= 1e-5 * 1.02, res


@pytest.mark.parametrize("seed", [3010, 3041])
def test_slow_spinodal_cells_converge(gmt_lib, seed):
    gmt = gmt_lib
    vox, desc = L.batch_cell(seed)
    assert desc["family"] == "spinodal" and desc["n"] == 128
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(gmt.ELASTIC, tol=1e-5)
    assert st == gmt.OK and info.inner_total > 320, info.as_dict()
    Ke, x0, D, M, C0 = fe.physics("elastic")
    lev = Level(vox.astype(bool))
    U = u.detach().cpu().numpy().reshape(-1, M)
    F = solve.cancel_rounding(solve.load(lev, Ke, x0, D), solve.gross_load_norm(lev, Ke, x0, D))
    R = F - solve.apply_ebe(lev, Ke, U, D)
    fn = np.linalg.norm(F, axis=0)
    res = np.linalg.norm(R, axis=0) / fn
    assert res.max() <= 1e-5 * 1.02, res
    CH = h.homogenize(gmt.ELASTIC)
    np.testing.assert_allclose(CH, CH.T, atol=1e-12)
    # Voigt bound (exact for FE): phi C0 - C^H is positive semidefinite
    assert np.linalg.eigvalsh(vox.mean() * C0 - CH).min() > -1e-6
    assert np.linalg.eigvalsh(CH).min() > 0
    # the library's C^H equals the oracle's energy average of the library's field
    C_of_gpu = solve.homogenize_chunked(lev, U, Ke, x0, D)
    assert np.abs(CH - C_of_gpu).max() <= 2e-7 * vox.mean() * np.abs(C0).max()


@pytest.mark.parametrize("seed,percolates", [(3026, False), (3025, False), (3000, True),
                                             (3001, True), (3010, True)])
def test_vcycle_symmetry_separates_the_non_percolating_cells(gmt_lib, seed, percolates):
    """The symmetry defect |<B f1, f2> - <f1, B f2>| / sqrt(<B f1, f1><B f2, f2>) of one
    V-cycle B on random zero-mean f1, f2. In FP64 it is rounding-level on every cell. In FP32
    it is 1e-8 or less on cells that percolate (the slow spinodal included) and 1e-4 or more
    on the two that do not, whose rotational null modes the FP32 cycle cannot keep apart:
    the located cause of their FP64 fallback (measured 2.6e-2 and 5.9e-4 there, 1e-10 to 1e-8
    elsewhere)."""
    gmt = gmt_lib
    vox, _ = L.batch_cell(seed)
    h = gmt.Hierarchy(vox)
    h.prepare(gmt.ELASTIC)
    n = h.num_nodes(0)
    rng = np.random.default_rng(1)
    f1 = rng.standard_normal((n, 3, 6))
    f2 = rng.standard_normal((n, 3, 6))
    f1 -= f1.mean(axis=0)
    f2 -= f2.mean(axis=0)

    def defect(prec):
        b1 = h.vcycle(f1, precision=prec).cpu().numpy()
        b2 = h.vcycle(f2, precision=prec).cpu().numpy()
        a, b = float((b1 * f2).sum()), float((f1 * b2).sum())
        return abs(a - b) / np.sqrt(abs(float((b1 * f1).sum()) * float((b2 * f2).sum())))

    assert defect(gmt.FP64) < 1e-8
    d32 = defect(gmt.FP32)
    if percolates:
        assert d32 < 1e-6, d32
    else:
        assert d32 > 1e-4, d32
