"""Parity of every hot-path step of the CUDA library (through the C ABI) against the CPU
oracle: hierarchy (bit-exact), operator apply per level, transfers, smoothers, coarsest
solve and one full V-cycle."""
import numpy as np
import pytest

from oracle import grid, solve, vcycle
from paper_2604_26518_b300 import lattices as L
from helpers import oracle_setup, rel_err, to_np

pytestmark = pytest.mark.gpu


def _cells():
    rng = np.random.default_rng(11)
    return {
        "gyroid32": L.tpms_network("gyroid", 32, 0.3),
        "random8": L.random_binary(8, 0.45, rng),
        "octet16": L.largest_component(L.truss("octet", 16, 0.11)),
        "plate24": L.tpms_plate("schwarz_p", 24, 0.35),      # coarsest 6^3: dense layout
        "spinodal20": L.spinodal(20, 0.3, 3, np.random.default_rng(3)),
    }


CELLS = _cells()


@pytest.mark.parametrize("name", list(CELLS))
def test_hierarchy_bit_exact(gmt_lib, name):
    gmt = gmt_lib
    vox = CELLS[name]
    h = gmt.Hierarchy(vox)
    lv = grid.hierarchy(vox, h.levels)
    assert h.levels == grid.choose_levels(vox.shape[0])
    for l, o in enumerate(lv):
        assert h.level_res(l) == o.n
        assert h.num_nodes(l) == o.num_nodes and h.num_elements(l) == o.num_elements
        xyz, m = h.node_coords(l)
        np.testing.assert_array_equal(xyz.cpu().numpy(), o.node_xyz())
        np.testing.assert_array_equal(m.cpu().numpy(), o.node_mask_list())
        exyz, cm = h.element_coords(l)
        np.testing.assert_array_equal(exyz.cpu().numpy(), o.elem_xyz())
        if l > 0:
            fine = lv[l - 1].active
            e = o.elem_xyz()
            expect = np.zeros(len(e), dtype=np.uint8)
            for c in range(8):
                cx, cy, cz = c & 1, (c >> 1) & 1, c >> 2
                expect |= (fine[2 * e[:, 2] + cz, 2 * e[:, 1] + cy, 2 * e[:, 0] + cx].astype(np.uint8) << c)
            np.testing.assert_array_equal(cm.cpu().numpy(), expect)
        if l + 1 < len(lv):
            idx, w = h.transfer_stencil(l)
            oi, ow = grid.transfer_stencil(o, lv[l + 1])
            np.testing.assert_array_equal(idx.cpu().numpy(), oi)
            np.testing.assert_array_equal(w.cpu().numpy(), ow)


@pytest.mark.parametrize("name", ["gyroid32", "octet16", "plate24", "random8"])
@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_operator_transfer_and_smoother_parity(gmt_lib, name, kind):
    gmt = gmt_lib
    vox = CELLS[name]
    h = gmt.Hierarchy(vox)
    O = oracle_setup(vox, kind, h.levels)
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    h.prepare(ph)
    D, M = O["D"], O["M"]
    rng = np.random.default_rng(7)
    for l in range(h.levels):
        n = h.num_nodes(l)
        u = rng.standard_normal((n * D, M))
        Ku = O["Ks"][l] @ u
        if h.num_bricks(l) > 0:
            y64 = to_np(h.apply(l, u, gmt.FP64), D, M)
            assert rel_err(y64, Ku) < 1e-12, (l, rel_err(y64, Ku))
            y32 = to_np(h.apply(l, u, gmt.FP32), D, M)
            assert rel_err(y32, Ku) < 2e-5, (l, rel_err(y32, Ku))
            if l + 1 < h.levels:   # damped block-Jacobi, from zero and from u
                Di = vcycle.block_diag_inverse(O["Ks"][l], D)
                f = rng.standard_normal((n * D, M))
                s1 = to_np(h.smooth(l, f, None, 1), D, M)
                assert rel_err(s1, 0.6 * (Di @ f)) < 1e-13
                s2 = to_np(h.smooth(l, f, u, 2), D, M)
                ref = u
                for _ in range(2):
                    ref = ref + 0.6 * (Di @ (f - O["Ks"][l] @ ref))
                assert rel_err(s2, ref) < 1e-12, (l, rel_err(s2, ref))
        if l + 1 < h.levels:
            P = O["Ps"][l]
            fc = to_np(h.restrict(l, u), D, M)
            assert rel_err(fc, P.T @ u) < 1e-14
            uc = rng.standard_normal((h.num_nodes(l + 1) * D, M))
            uf = to_np(h.prolong(l, uc, u), D, M)
            assert rel_err(uf, u + P @ uc) < 1e-14


@pytest.mark.parametrize("name", ["gyroid32", "plate24"])
def test_coarsest_solve_parity(gmt_lib, name):
    gmt = gmt_lib
    vox = CELLS[name]
    h = gmt.Hierarchy(vox)
    O = oracle_setup(vox, "elastic", h.levels)
    h.prepare(gmt.ELASTIC)
    KL = O["Ks"][-1]
    f = solve.gauge(np.random.default_rng(2).standard_normal((KL.shape[0], 6)), 3)
    u = to_np(h.coarse_solve(f), 3, 6)
    ref = np.linalg.solve(vcycle.coarsest_matrix(KL, 3), f)
    assert rel_err(u, ref) < 1e-9
    assert rel_err(KL @ u, f) < 1e-9


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("name", ["gyroid32", "octet16", "plate24"])
def test_vcycle_parity(gmt_lib, name, smoother):
    gmt = gmt_lib
    vox = CELLS[name]
    sm = gmt.JACOBI if smoother == "jacobi" else gmt.CHEBYSHEV
    h = gmt.Hierarchy(vox, gmt.default_options(smoother=sm))
    O = oracle_setup(vox, "elastic", h.levels)
    h.prepare(gmt.ELASTIC)
    kw = {}
    if smoother == "chebyshev":
        kw = {"cheb_lmax": [h.lambda_max(l) for l in range(h.levels - 1)]}
    o = gmt.default_options()
    vc = vcycle.VCycle(O["Ks"], O["Ps"], 3, smoother=smoother, nu_pre=o.nu_pre,
                       nu_post=o.nu_post, nu_coarse=o.nu_coarse, **kw)
    F = O["F"]
    u1 = to_np(h.vcycle(F, None, gmt.FP64), 3, 6)
    r1 = vc.cycle(F)
    assert rel_err(u1, r1) < 1e-10, rel_err(u1, r1)
    u2 = to_np(h.vcycle(F, u1, gmt.FP64), 3, 6)
    r2 = vc.cycle(F, r1)
    assert rel_err(u2, r2) < 1e-10
    u32 = to_np(h.vcycle(F, None, gmt.FP32), 3, 6)
    assert rel_err(u32, r1) < 1e-4


def test_lambda_max_estimate(gmt_lib):
    import scipy.sparse.linalg as spla
    gmt = gmt_lib
    vox = CELLS["gyroid32"]
    h = gmt.Hierarchy(vox, gmt.default_options(smoother=gmt.CHEBYSHEV))
    O = oracle_setup(vox, "elastic", h.levels)
    h.prepare(gmt.ELASTIC)
    for l in range(h.levels - 1):
        A = vcycle.block_diag_inverse(O["Ks"][l], 3) @ O["Ks"][l]
        lam = float(np.abs(spla.eigs(A, k=1, which="LM", return_eigenvectors=False))[0])
        est = h.lambda_max(l)
        assert 0.9 * lam <= est <= lam * (1 + 1e-6), (l, est, lam)


@pytest.mark.parametrize("smoother,kind", [("gs8", "V"), ("jacobi", "W"), ("jacobi", "F"),
                                           ("gs8", "W")])
@pytest.mark.parametrize("name", ["gyroid32", "octet16"])
def test_cycle_schedules_and_gs8_parity(gmt_lib, name, smoother, kind):
    """8-colour Gauss-Seidel smoothing and W-/F-cycles against the oracle's cycle."""
    gmt = gmt_lib
    vox = CELLS[name]
    sm = gmt.GS8 if smoother == "gs8" else gmt.JACOBI
    cyc = {"V": gmt.CYCLE_V, "W": gmt.CYCLE_W, "F": gmt.CYCLE_F}[kind]
    h = gmt.Hierarchy(vox, gmt.default_options(smoother=sm, cycle=cyc))
    O = oracle_setup(vox, "elastic", h.levels)
    h.prepare(gmt.ELASTIC)
    o = gmt.default_options()
    vc = vcycle.VCycle(O["Ks"], O["Ps"], 3, smoother=smoother, kind=kind, levels=O["levels"],
                       nu_pre=o.nu_pre, nu_post=o.nu_post, nu_coarse=o.nu_coarse)
    F = O["F"]
    u1 = to_np(h.vcycle(F, None, gmt.FP64), 3, 6)
    r1 = vc.cycle(F)
    assert rel_err(u1, r1) < 1e-10, rel_err(u1, r1)
    u2 = to_np(h.vcycle(F, u1, gmt.FP64), 3, 6)
    assert rel_err(u2, vc.cycle(F, r1)) < 1e-10
    assert rel_err(to_np(h.vcycle(F, None, gmt.FP32), 3, 6), r1) < 1e-4


@pytest.mark.parametrize("smoother,kind", [("gs8", "V"), ("jacobi", "W"), ("jacobi", "F")])
def test_solve_with_other_schedules(gmt_lib, smoother, kind):
    gmt = gmt_lib
    vox = CELLS["gyroid32"]
    sm = gmt.GS8 if smoother == "gs8" else gmt.JACOBI
    cyc = {"V": gmt.CYCLE_V, "W": gmt.CYCLE_W, "F": gmt.CYCLE_F}[kind]
    ref = solve.solve_cell(vox, "elastic", tol=1e-8)
    h = gmt.Hierarchy(vox, gmt.default_options(smoother=sm, cycle=cyc))
    st, u, info = h.solve(gmt.ELASTIC, tol=1e-5)
    assert st == gmt.OK
    CH = h.homogenize(gmt.ELASTIC)
    assert np.abs(CH - ref["CH"]).max() <= 1e-4 * np.abs(ref["CH"]).max()
