"""Converged-oracle parity of a full solve for every generator family at 64^3.

For one seeded 64^3 cell of each family (TPMS networks and plates, BCC / octet trusses,
spinodal; each connected across the cell), the library solves the cell problems to
r <= 1e-5 and returns C^H; the FP64 oracle's C^H at r <= 1e-10 is stored in
tests/golden/family64.json (written by tests/golden/make_family64.py, which calls only the
oracle and the seeded generators). One more cell is degenerate: a Schwarz-P network below
its percolation threshold (isolated periodic blobs), whose tensors vanish; there the
relative metric is undefined and C^H is held to 1e-4 of the Voigt bound's scale phi |C0|.

Checks per cell and physics:
  * C^H within 1e-4 of the oracle's, normalised by the largest entry (Sec. 5 error metric
    delta, read as max-entry relative);
  * the oracle's relative residual of the library's field (its own matrix-free product)
    at most the tolerance;
  * the library's C^H equals the oracle's energy average of the library's field;
  * the field's error in the energy norm. For the exact solution u* of K u* = f and any u,
    the energy average of App. F.1 satisfies
        N^3 (C_II(u) - C_II(u*)) = (u - u*)^T K (u - u*)      (K u* = f, f = sum A^T K_e x0),
    so the relative energy-norm error of case I is sqrt((C_II(u) - C*_II) / C*_II), computed
    from the oracle's energy average of the library's field and the stored converged C*.
    A residual of 1e-5 does not bound this error by 1e-4 on ill-conditioned cells: on the
    spinodal cell the library's field at r <= 1e-5 is 2.1e-4 away, and the oracle's own
    Jacobi-PCG field at r <= 1e-5 is 5.2e-4 away. The field check therefore continues the
    solve (warm start) to r <= 1e-6 and holds that field to 1e-4.
"""
import json
import os

import numpy as np
import pytest

from oracle import fe, solve
from oracle.grid import Level
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu
TOL = 1e-5
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "family64.json")


def _golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def _cells():
    g = _golden()
    return [(i, c["family"] + ("-degenerate" if c["degenerate"] else ""))
            for i, c in enumerate(g["cells"])]


@pytest.mark.parametrize("kind", ["elastic", "heat"])
@pytest.mark.parametrize("idx,family", _cells())
def test_family64_matches_converged_oracle(gmt_lib, idx, family, kind):
    gmt = gmt_lib
    g = _golden()
    rec = g["cells"][idx]
    vox, desc = L.mixed_cell(rec["seed"], g["res"], families=(rec["family"],))
    assert int(vox.sum()) == rec["n_solid"]
    C_star = np.array(rec[kind]["CH"])
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(ph, tol=TOL)
    assert st == gmt.OK, info.as_dict()
    CH = h.homogenize(ph)
    Ke, x0, D, M, C0 = fe.physics(kind)
    if rec["degenerate"]:
        scale = vox.mean() * np.abs(C0).max()
        assert np.abs(C_star).max() <= 1e-10 * scale
        assert np.abs(CH).max() <= 1e-4 * scale, (family, kind, CH)
        return
    err = np.abs(CH - C_star).max() / np.abs(C_star).max()
    assert err <= 1e-4, (family, kind, err, CH, C_star)

    lev = Level(vox.astype(bool))
    U = u.detach().cpu().numpy().reshape(-1, M)
    F = solve.cancel_rounding(solve.load(lev, Ke, x0, D), solve.gross_load_norm(lev, Ke, x0, D))
    R = F - solve.apply_ebe(lev, Ke, U, D)
    fn = np.linalg.norm(F, axis=0)
    res = np.where(fn > 0, np.linalg.norm(R, axis=0) / np.where(fn > 0, fn, 1), 0)
    assert res.max() <= TOL * 1.02, (family, kind, res)
    C_of_gpu = solve.homogenize_chunked(lev, U, Ke, x0, D)
    # the float-float energy path rounds each element's terms (of size ~|C0|) once in FP32;
    # summed over the phi N^3 elements that is an absolute error ~1e-7 phi |C0|, which on
    # soft cells (spinodal: C^H ~ phi |C0| / 20) exceeds 1e-7 of |C^H| itself
    assert np.abs(CH - C_of_gpu).max() <= 2e-7 * vox.mean() * np.abs(C0).max()
    diag = np.diag(C_star)
    st, u6, info6 = h.solve(ph, tol=1e-6, u0=u)
    assert st == gmt.OK, info6.as_dict()
    U6 = u6.detach().cpu().numpy().reshape(-1, M)
    excess = np.diag(solve.homogenize_chunked(lev, U6, Ke, x0, D)) - diag
    # the energy of any field is at least the minimum's (up to the oracle's 1e-10 residual)
    assert excess.min() >= -1e-9 * diag.max(), excess
    en = np.sqrt(np.maximum(excess, 0.0) / np.maximum(diag, 1e-300))
    assert en.max() <= 1e-4, (family, kind, en)
