"""BF16 V-cycle (gmt_options.precision = GMT_PREC_BF16): the V-cycle's vectors stored in
BF16 on every level with FP32 arithmetic, inside the FP32 Krylov loop and the float-float
solution. Solves reach the tolerance with C^H within 1e-4 of the converged oracle, for
elasticity and heat, network, plate and truss cells; C^H agrees with the FP32 solve's; the
warm-start sweeps (which run in FP32 scratch on a BF16 workspace) and a full-size 128^3 cell
of the benchmark's mix converge."""
import numpy as np
import pytest

from oracle import solve
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu
TOL = 1e-5

CELLS = {
    "gyroid32": lambda: L.tpms_network("gyroid", 32, 0.3),
    "plate24": lambda: L.tpms_plate("schwarz_p", 24, 0.35),
    "octet32": lambda: L.largest_component(L.truss("octet", 32, 0.09)),
}


@pytest.mark.parametrize("kind", ["elastic", "heat"])
@pytest.mark.parametrize("name", list(CELLS))
def test_bf16_solve_matches_oracle(gmt_lib, name, kind):
    gmt = gmt_lib
    vox = CELLS[name]()
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    ref = solve.solve_cell(vox, kind, tol=1e-10)["CH"]
    out = {}
    for prec in (gmt.FP32, gmt.BF16):
        h = gmt.Hierarchy(vox, gmt.default_options(precision=prec))
        st, _, info = h.solve(ph, tol=TOL, want_field=False)
        assert st == gmt.OK and not info.fp64_fallback
        assert max(info.as_dict()["rel_residual"]) <= TOL
        CH = h.homogenize(ph)
        assert np.abs(CH - ref).max() <= 1e-4 * np.abs(ref).max()
        out[prec] = (CH, info.inner_total)
        h.free()
    (c32, n32), (c16, n16) = out[gmt.FP32], out[gmt.BF16]
    assert np.abs(c16 - c32).max() <= 1e-4 * np.abs(c32).max()
    print(f"{name} {kind}: V-cycles FP32 {n32}, BF16 {n16}")


def test_bf16_warm_sweeps_and_full_size_128(gmt_lib):
    import torch
    gmt = gmt_lib
    vox = CELLS["gyroid32"]()
    h = gmt.Hierarchy(vox)
    st, u, _ = h.solve(gmt.ELASTIC, tol=TOL)
    CH = h.homogenize(gmt.ELASTIC)
    h.free()
    rough = u + 1e-3 * torch.randn(u.shape, dtype=u.dtype, device=u.device,
                                   generator=torch.Generator(device="cuda").manual_seed(2))
    # an odd sweep count ends in the FP32 scratch buffer, which is copied back
    hb = gmt.Hierarchy(vox, gmt.default_options(precision=gmt.BF16, warm_sweeps=3))
    st, _, info = hb.solve(gmt.ELASTIC, tol=TOL, u0=rough, want_field=False)
    assert st == gmt.OK and max(info.as_dict()["rel_residual"]) <= TOL
    assert np.abs(hb.homogenize(gmt.ELASTIC) - CH).max() <= 1e-4 * np.abs(CH).max()
    hb.free()
    vox, _ = L.mixed_cell(2002, 128)
    hb = gmt.Hierarchy(vox, gmt.default_options(precision=gmt.BF16))
    st, _, info = hb.solve(gmt.ELASTIC, tol=TOL, want_field=False)
    assert st == gmt.OK and max(info.as_dict()["rel_residual"]) <= TOL
    CH16 = hb.homogenize(gmt.ELASTIC)
    hb.free()
    h = gmt.Hierarchy(vox)
    h.solve(gmt.ELASTIC, tol=TOL, want_field=False)
    CH32 = h.homogenize(gmt.ELASTIC)
    h.free()
    assert np.abs(CH16 - CH32).max() <= 1e-4 * np.abs(CH32).max()


@pytest.mark.parametrize("smoother", ["chebyshev", "gs8"])
def test_bf16_solve_other_smoothers(gmt_lib, smoother):
    """The BF16 instances of the Chebyshev and 8-colour Gauss-Seidel sweeps: solves reach the
    tolerance with C^H within 1e-4 of the converged oracle."""
    gmt = gmt_lib
    vox = CELLS["gyroid32"]()
    ref = solve.solve_cell(vox, "elastic", tol=1e-10)["CH"]
    sm = gmt.CHEBYSHEV if smoother == "chebyshev" else gmt.GS8
    h = gmt.Hierarchy(vox, gmt.default_options(precision=gmt.BF16, smoother=sm))
    st, _, info = h.solve(gmt.ELASTIC, tol=TOL, want_field=False)
    assert st == gmt.OK and max(info.as_dict()["rel_residual"]) <= TOL
    assert np.abs(h.homogenize(gmt.ELASTIC) - ref).max() <= 1e-4 * np.abs(ref).max()
    h.free()
