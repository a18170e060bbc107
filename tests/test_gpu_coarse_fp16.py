"""FP16 copies of the coarse levels' stored stencils (gmt_options.coarse_fp16): the FP32
apply of every level >= 1 stays within FP16 rounding of the oracle's Galerkin operator
P^T K P, solves reach the same residual with C^H within 1e-4 of the converged oracle, and
the batched V-cycle with FP16 stencils is bitwise each lattice's own."""
import numpy as np
import pytest

from oracle import solve
from paper_2604_26518_b300 import lattices as L
from helpers import oracle_setup, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_coarse_apply_within_fp16_rounding(gmt_lib, kind):
    gmt = gmt_lib
    vox = L.tpms_network("gyroid", 32, 0.3)
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    h = gmt.Hierarchy(vox, gmt.default_options(coarse_fp16=1))
    h32 = gmt.Hierarchy(vox)
    O = oracle_setup(vox, kind, h.levels)
    h.prepare(ph)
    h32.prepare(ph)
    D, M = O["D"], O["M"]
    rng = np.random.default_rng(3)
    for l in range(h.levels - 1):
        n = h.num_nodes(l)
        u = rng.standard_normal((n * D, M))
        Ku = O["Ks"][l] @ u
        y = to_np(h.apply(l, u, gmt.FP32), D, M)
        y32 = to_np(h32.apply(l, u, gmt.FP32), D, M)
        if l == 0:    # level 0 forms its stencil from the masks in either mode
            assert np.array_equal(y, y32)
        else:         # FP16 coefficients: unit roundoff 2^-11 per coefficient
            assert rel_err(y, Ku) < 1e-3, (l, rel_err(y, Ku))
            if ph == gmt.ELASTIC:   # (the scaled heat stencils are dyadic: exact in FP16)
                assert rel_err(y, Ku) > 1e-6, (l, rel_err(y, Ku))
        # the FP64 apply never uses the FP16 copy
        assert rel_err(to_np(h.apply(l, u, gmt.FP64), D, M), Ku) < 1e-12
    h.free()
    h32.free()


@pytest.mark.parametrize("name", ["gyroid32", "plate24", "octet32"])
def test_solve_with_fp16_coarse_stencils(gmt_lib, name):
    gmt = gmt_lib
    vox = {"gyroid32": lambda: L.tpms_network("gyroid", 32, 0.3),
           "plate24": lambda: L.tpms_plate("schwarz_p", 24, 0.35),
           "octet32": lambda: L.largest_component(L.truss("octet", 32, 0.09))}[name]()
    ref = solve.solve_cell(vox, "elastic", tol=1e-10)["CH"]
    out = {}
    for fp16 in (0, 1):
        h = gmt.Hierarchy(vox, gmt.default_options(coarse_fp16=fp16))
        st, _, info = h.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
        assert st == gmt.OK and max(info.as_dict()["rel_residual"]) <= 1e-5
        CH = h.homogenize(gmt.ELASTIC)
        assert np.abs(CH - ref).max() <= 1e-4 * np.abs(ref).max()
        out[fp16] = info.inner_total
        h.free()
    assert out[1] <= out[0] + 2, out


def test_batched_vcycle_with_fp16_stencils(gmt_lib):
    import torch
    gmt = gmt_lib
    cells = [L.tpms_network("gyroid", 32, 0.3), L.tpms_plate("schwarz_p", 24, 0.35),
             L.tpms_network("diamond", 48, 0.3)]
    hs = [gmt.Hierarchy(v, gmt.default_options(coarse_fp16=1)) for v in cells]
    for h in hs:
        h.prepare(gmt.ELASTIC)
    g = torch.Generator(device="cpu").manual_seed(4)
    F = [torch.randn((h.num_nodes(0), 3, 6), generator=g, dtype=torch.float64).cuda() for h in hs]
    batch = gmt.vcycle_batch(hs, F)
    for h, f, b in zip(hs, F, batch):
        assert torch.equal(h.vcycle(f, None, gmt.FP32), b)
    mixed = gmt.Hierarchy(cells[0])
    mixed.prepare(gmt.ELASTIC)
    with pytest.raises(gmt.GmtError):
        gmt.vcycle_batch([hs[0], mixed], F[:1] + F[:1])
    for h in hs + [mixed]:
        h.free()
