"""V-cycle with injected coarse corrections (gmt_vcycle_inject, Alg. 2): every level l >= 1
of the first descent starts from a given field instead of zero. Against the oracle's cycle
with the same corrections (FP64 to 1e-10, FP32 to 1e-4), for elasticity and heat, bricked
and dense coarsest levels, from zero and from a given fine field; the coarsest level's
entry changes nothing; without corrections the call is bitwise gmt_vcycle; W-cycle
schedules and a wrong entry count are rejected."""
import numpy as np
import pytest

from oracle import vcycle
from paper_2604_26518_b300 import lattices as L
from helpers import oracle_setup, rel_err, to_np

pytestmark = pytest.mark.gpu

CELLS = {
    "gyroid32": lambda: L.tpms_network("gyroid", 32, 0.3),
    "plate24": lambda: L.tpms_plate("schwarz_p", 24, 0.35),       # coarsest 6^3: dense layout
    "diamond48": lambda: L.tpms_network("diamond", 48, 0.3),      # four levels
}


@pytest.mark.parametrize("kind", ["elastic", "heat"])
@pytest.mark.parametrize("name", list(CELLS))
def test_injected_vcycle_matches_oracle(gmt_lib, name, kind):
    import torch
    gmt = gmt_lib
    vox = CELLS[name]()
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    h = gmt.Hierarchy(vox)
    h.prepare(ph)
    O = oracle_setup(vox, kind, h.levels)
    D, M = O["D"], O["M"]
    o = gmt.default_options()
    vc = vcycle.VCycle(O["Ks"], O["Ps"], D, smoother="jacobi", nu_pre=o.nu_pre,
                       nu_post=o.nu_post, nu_coarse=o.nu_coarse)
    rng = np.random.default_rng(5)
    F = O["F"]
    scale = np.abs(vc.cycle(F)).max()
    e = [None] + [0.3 * scale * rng.standard_normal((h.num_nodes(l) * D, M))
                  for l in range(1, h.levels)]
    ref = vc.cycle(F, e=e)
    assert rel_err(vc.cycle(F), ref) > 1e-3               # the corrections matter
    got = to_np(h.vcycle(F, None, gmt.FP64, corrections=e), D, M)
    assert rel_err(got, ref) < 1e-10, rel_err(got, ref)
    got32 = to_np(h.vcycle(F, None, gmt.FP32, corrections=e), D, M)
    assert rel_err(got32, ref) < 1e-4, rel_err(got32, ref)
    # from a given fine field
    u0 = ref
    ref2 = vc.cycle(F, u0, e=e)
    got2 = to_np(h.vcycle(F, u0, gmt.FP64, corrections=e), D, M)
    assert rel_err(got2, ref2) < 1e-10
    # the coarsest level is solved exactly: its entry is not read
    e2 = list(e)
    e2[-1] = None
    assert torch.equal(h.vcycle(F, None, gmt.FP64, corrections=e2),
                       h.vcycle(F, None, gmt.FP64, corrections=e))
    # no corrections: the plain V-cycle, bit for bit
    for prec in (gmt.FP32, gmt.FP64):
        assert torch.equal(h.vcycle(F, None, prec, corrections=[None] * h.levels),
                           h.vcycle(F, None, prec))
    h.free()


@pytest.mark.parametrize("smoother", ["chebyshev", "gs8"])
def test_injected_vcycle_other_smoothers(gmt_lib, smoother):
    """The injected start goes through the Chebyshev and 8-colour Gauss-Seidel smoothers'
    nonzero-start paths: against the oracle's cycle with the same corrections."""
    gmt = gmt_lib
    vox = CELLS["gyroid32"]()
    sm = gmt.CHEBYSHEV if smoother == "chebyshev" else gmt.GS8
    h = gmt.Hierarchy(vox, gmt.default_options(smoother=sm))
    h.prepare(gmt.ELASTIC)
    O = oracle_setup(vox, "elastic", h.levels)
    o = gmt.default_options()
    kw = {}
    if smoother == "chebyshev":
        kw = {"cheb_lmax": [h.lambda_max(l) for l in range(h.levels - 1)]}
    else:
        kw = {"levels": O["levels"]}
    vc = vcycle.VCycle(O["Ks"], O["Ps"], 3, smoother=smoother, nu_pre=o.nu_pre,
                       nu_post=o.nu_post, nu_coarse=o.nu_coarse, **kw)
    rng = np.random.default_rng(9)
    F = O["F"]
    scale = np.abs(vc.cycle(F)).max()
    e = [None] + [0.3 * scale * rng.standard_normal((h.num_nodes(l) * 3, 6))
                  for l in range(1, h.levels)]
    ref = vc.cycle(F, e=e)
    got = to_np(h.vcycle(F, None, gmt.FP64, corrections=e), 3, 6)
    assert rel_err(got, ref) < 1e-10, rel_err(got, ref)
    h.free()


def test_injection_rejects_bad_calls(gmt_lib):
    gmt = gmt_lib
    vox = CELLS["gyroid32"]()
    h = gmt.Hierarchy(vox, gmt.default_options(cycle=gmt.CYCLE_W))
    h.prepare(gmt.ELASTIC)
    F = np.zeros((h.num_nodes(0) * 3, 6))
    with pytest.raises(gmt.GmtError) as err:
        h.vcycle(F, None, gmt.FP64, corrections=[None] * h.levels)
    assert err.value.status == gmt.ERR_ARG
    with pytest.raises(ValueError):
        h.vcycle(F, None, gmt.FP64, corrections=[None] * (h.levels + 1))
    h.free()
