"""Batched V-cycle (gmt_vcycle_batch): one launch per phase over the bricks of many
lattices gives every lattice bitwise the FP32 V-cycle that gmt_vcycle runs for it alone,
with bricked and dense coarsest levels and different level counts mixed in one batch, from
zero and from a given field, for elasticity and heat conduction, up to the largest batch;
the first lattice's result also matches the oracle's V-cycle (Alg. 1) to FP32 accuracy."""
import numpy as np
import pytest

from oracle import vcycle
from paper_2604_26518_b300 import lattices as L
from helpers import oracle_setup, rel_err, to_np

pytestmark = pytest.mark.gpu


def _cells():
    rng = np.random.default_rng(21)
    return [
        L.tpms_network("gyroid", 32, 0.3),                       # levels 32, 16, 8
        L.largest_component(L.truss("octet", 32, 0.09)),
        L.tpms_plate("schwarz_p", 24, 0.35),                      # levels 24, 12, 6 (dense)
        L.spinodal(32, 0.35, 3, np.random.default_rng(4)),
        L.random_binary(24, 0.5, rng),                            # dense coarsest too
    ]


def _loads(gmt, hs, seed):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    out = []
    for h in hs:
        D, M = h._dm()
        out.append(torch.randn((h.num_nodes(0), D, M), generator=g, dtype=torch.float64).cuda())
    return out


@pytest.mark.parametrize("physics", ["elastic", "heat"])
def test_batch_bitwise_equal_to_single(gmt_lib, physics):
    import torch
    gmt = gmt_lib
    ph = gmt.ELASTIC if physics == "elastic" else gmt.HEAT
    hs = [gmt.Hierarchy(v) for v in _cells()]
    for h in hs:
        h.prepare(ph)
    F = _loads(gmt, hs, 5)
    single = [h.vcycle(f, None, gmt.FP32) for h, f in zip(hs, F)]
    batch = gmt.vcycle_batch(hs, F)
    for a, b in zip(single, batch):
        assert torch.equal(a, b)
    # from a given field (no diagonal start)
    single2 = [h.vcycle(f, u, gmt.FP32) for h, f, u in zip(hs, F, single)]
    batch2 = gmt.vcycle_batch(hs, F, batch)
    for a, b in zip(single2, batch2):
        assert torch.equal(a, b)
    # a batch of one, and the batch in another order
    assert torch.equal(gmt.vcycle_batch(hs[2:3], F[2:3])[0], single[2])
    rev = gmt.vcycle_batch(hs[::-1], F[::-1])[::-1]
    for a, b in zip(single, rev):
        assert torch.equal(a, b)
    for h in hs:
        h.free()


def test_batch_first_lattice_matches_oracle(gmt_lib):
    gmt = gmt_lib
    cells = _cells()
    hs = [gmt.Hierarchy(v) for v in cells[:3]]
    for h in hs:
        h.prepare(gmt.ELASTIC)
    O = oracle_setup(cells[0], "elastic", hs[0].levels)
    o = gmt.default_options()
    vc = vcycle.VCycle(O["Ks"], O["Ps"], 3, smoother="jacobi", nu_pre=o.nu_pre,
                       nu_post=o.nu_post, nu_coarse=o.nu_coarse)
    F = [O["F"]] + _loads(gmt, hs[1:], 6)
    u = gmt.vcycle_batch(hs, F)
    assert rel_err(to_np(u[0], 3, 6), vc.cycle(O["F"])) < 1e-4
    for h in hs:
        h.free()


def test_largest_batch(gmt_lib):
    import torch
    gmt = gmt_lib
    rng = np.random.default_rng(77)
    hs = []
    for i in range(gmt.BATCH_MAX):
        kind = i % 3
        if kind == 0:
            v = L.random_binary(16, 0.55, rng)
        elif kind == 1:
            v = L.spinodal(16, 0.4, 2, np.random.default_rng(100 + i))
        else:
            v = L.tpms_network("gyroid", 16, 0.25 + 0.002 * i)
        if not v.any():
            v[0, 0, 0] = 1
        hs.append(gmt.Hierarchy(v))
    for h in hs:
        h.prepare(gmt.ELASTIC)
    F = _loads(gmt, hs, 9)
    batch = gmt.vcycle_batch(hs, F)
    for h, f, b in zip(hs, F, batch):
        assert torch.equal(h.vcycle(f, None, gmt.FP32), b)
    with pytest.raises(ValueError):
        gmt.vcycle_batch(hs + hs[:1], F + F[:1])
    for h in hs:
        h.free()


def test_batch_rejects_mismatched_hierarchies(gmt_lib):
    gmt = gmt_lib
    cells = _cells()
    a = gmt.Hierarchy(cells[0])
    b = gmt.Hierarchy(cells[1])
    a.prepare(gmt.ELASTIC)
    b.prepare(gmt.ELASTIC, E=2.0)
    F = _loads(gmt, [a, b], 1)
    with pytest.raises(gmt.GmtError) as e:
        gmt.vcycle_batch([a, b], F)
    assert e.value.status == gmt.ERR_ARG
    b.prepare(gmt.ELASTIC)
    with pytest.raises(gmt.GmtError) as e:
        gmt.vcycle_batch([a, a], [F[0], F[0]])
    assert e.value.status == gmt.ERR_ARG
    c = gmt.Hierarchy(cells[0], gmt.default_options(smoother=gmt.CHEBYSHEV))
    c.prepare(gmt.ELASTIC)
    with pytest.raises(gmt.GmtError) as e:
        gmt.vcycle_batch([a, c], [F[0], F[0]])
    assert e.value.status == gmt.ERR_ARG
    d = gmt.Hierarchy(cells[0])
    d.prepare(gmt.HEAT)
    with pytest.raises(gmt.GmtError) as e:
        gmt.vcycle_batch([a, d], [F[0], _loads(gmt, [d], 2)[0]])
    assert e.value.status == gmt.ERR_ARG
    for h in (a, b, c, d):
        h.free()


def test_batch_with_different_level_counts(gmt_lib):
    """Lattices of 2, 3 and 4 levels in one batch: each takes its coarsest solve at its own
    coarsest level, bitwise as alone."""
    import torch
    gmt = gmt_lib
    cells = [L.tpms_network("gyroid", 16, 0.3), _cells()[0], L.tpms_plate("schwarz_p", 24, 0.35),
             L.tpms_network("diamond", 48, 0.3), L.spinodal(64, 0.35, 4, np.random.default_rng(8))]
    hs = [gmt.Hierarchy(v) for v in cells]
    assert sorted({h.levels for h in hs}) == [2, 3, 4]
    for h in hs:
        h.prepare(gmt.ELASTIC)
    F = _loads(gmt, hs, 12)
    batch = gmt.vcycle_batch(hs, F)
    for h, f, b in zip(hs, F, batch):
        assert torch.equal(h.vcycle(f, None, gmt.FP32), b)
    for h in hs:
        h.free()
