"""End-to-end parity of gmt_solve + gmt_homogenize against the FP64 oracle: C^H within
1e-4 (normalised by the largest entry) at relative residual 1e-5, fields in the energy norm,
closed forms, edge cases, determinism, and a full-size 128^3 cell checked through
properties the oracle evaluates on the library's field."""
import numpy as np
import pytest

from oracle import fe, grid, solve
from paper_2604_26518_b300 import lattices as L
from helpers import rel_err, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def gyroid32():
    vox = L.tpms_network("gyroid", 32, 0.30)
    return vox, solve.solve_cell(vox, "elastic"), solve.solve_cell(vox, "heat")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("krylov", [1, 0])
@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_config1_gyroid32(gmt_lib, gyroid32, precision, krylov, kind):
    gmt = gmt_lib
    vox, el, th = gyroid32
    ref = el if kind == "elastic" else th
    prec = gmt.FP64 if precision == "fp64" else gmt.FP32
    opts = gmt.default_options(precision=prec, krylov=krylov, max_inner=200, levels=3)
    h = gmt.Hierarchy(vox, opts)
    assert h.levels == 3
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    st, u, info = h.solve(ph, tol=TOL)
    D, M = ref["D"], ref["NC"]
    U = to_np(u, D, M)
    res = solve.relative_residual(ref["K"], ref["F"], U)      # oracle's own SpMV
    assert res.max() <= TOL * 1.02, (res, info.as_dict())
    # the library's outer residual: float-float difference form, accurate to ~1e-7 of ||f||
    np.testing.assert_allclose(np.array(info.as_dict()["rel_residual"]), res, rtol=0.05, atol=3e-7)
    CH = h.homogenize(ph)
    err = np.abs(CH - ref["CH"]).max() / np.abs(ref["CH"]).max()
    assert err <= 1e-4, err
    # the library's C^H of its own field equals the oracle's energy average of that field
    C_orc_of_gpu = solve.homogenize(ref["level"], U, ref["Ke"], ref["x0"], D)
    assert np.abs(CH - C_orc_of_gpu).max() <= (1e-12 if precision == "fp64" else 2e-7) * np.abs(ref["CH"]).max()
    en = solve.energy_norm_error(ref["K"], U, ref["U"], ref["Ke"], ref["x0"], ref["level"], D)
    assert en.max() <= 1e-4, en
    # gauge: zero mean per component and case
    assert np.abs(U.reshape(-1, D, M).mean(axis=0)).max() < 1e-9 * max(np.abs(U).max(), 1)


def test_solid_cell_and_laminates_closed_forms(gmt_lib):
    gmt = gmt_lib
    E, nu = 1.0, 0.3
    h = gmt.Hierarchy(np.ones((16, 16, 16), dtype=np.uint8))
    st, u, info = h.solve(gmt.ELASTIC, E=E, nu=nu, tol=TOL)
    assert float(u.abs().max()) == 0.0
    np.testing.assert_allclose(h.homogenize(gmt.ELASTIC, E=E, nu=nu), fe.elastic_C0(E, nu), atol=1e-12)
    vox = L.laminate_z(16, [0, 1, 2, 3, 8, 9])
    phi = 6 / 16
    h = gmt.Hierarchy(vox)
    h.solve(gmt.ELASTIC, tol=1e-8)
    C = h.homogenize(gmt.ELASTIC)
    expect = np.zeros((6, 6))
    expect[0, 0] = expect[1, 1] = phi * E / (1 - nu ** 2)
    expect[0, 1] = expect[1, 0] = phi * E * nu / (1 - nu ** 2)
    expect[5, 5] = phi * E / (2 * (1 + nu))
    assert np.abs(C - expect).max() < 1e-6
    h.solve(gmt.HEAT, tol=1e-8)
    np.testing.assert_allclose(h.homogenize(gmt.HEAT), np.diag([phi, phi, 0.0]), atol=1e-6)
    vox = L.rods_x(16, 4, 2, 2)
    h = gmt.Hierarchy(vox)
    h.solve(gmt.ELASTIC, tol=1e-8)
    C = h.homogenize(gmt.ELASTIC)
    expect = np.zeros((6, 6))
    expect[0, 0] = vox.mean() * E
    assert np.abs(C - expect).max() < 1e-6


@pytest.mark.parametrize("n", [4, 8])
def test_single_level_direct_solve_brute_force(gmt_lib, n):
    gmt = gmt_lib
    vox = L.largest_component(L.random_binary(n, 0.6, np.random.default_rng(n)))
    h = gmt.Hierarchy(vox)
    assert h.levels == 1
    st, u, info = h.solve(gmt.ELASTIC, tol=1e-9)
    Ub, Cb = solve.brute_force(vox, "elastic")
    assert np.abs(h.homogenize(gmt.ELASTIC) - Cb).max() <= 2e-7 * np.abs(Cb).max()


def test_edge_cases_report_status(gmt_lib):
    gmt = gmt_lib
    with pytest.raises(gmt.GmtError) as e:
        gmt.Hierarchy(np.zeros((16, 16, 16), dtype=np.uint8))
    assert e.value.status == gmt.ERR_EMPTY
    with pytest.raises(gmt.GmtError) as e:
        gmt.Hierarchy(np.ones((18, 18, 18), dtype=np.uint8))
    assert e.value.status == gmt.ERR_RES
    with pytest.raises(gmt.GmtError) as e:
        gmt.Hierarchy(np.ones((16, 16, 16), dtype=np.uint8), gmt.default_options(levels=4))
    assert e.value.status == gmt.ERR_RES
    h = gmt.Hierarchy(L.tpms_network("gyroid", 16, 0.3))
    with pytest.raises(gmt.GmtError) as e:
        h.solve(gmt.ELASTIC, nu=0.5)
    assert e.value.status == gmt.ERR_ARG
    with pytest.raises(gmt.GmtError) as e:
        h.homogenize(gmt.ELASTIC)                   # nothing solved yet
    assert e.value.status == gmt.ERR_STATE
    # an iteration cap the solve cannot meet returns NOT_CONVERGED with the best field
    h.set_options(gmt.default_options(max_outer=1, max_inner=1))
    st, u, info = h.solve(gmt.ELASTIC, tol=1e-12, allow_not_converged=True)
    assert st == gmt.NOT_CONVERGED and max(info.as_dict()["rel_residual"]) > 1e-12


def test_repeat_runs_bitwise_identical(gmt_lib):
    gmt = gmt_lib
    vox = L.tpms_plate("diamond", 32, 0.25)
    out = []
    for _ in range(2):
        h = gmt.Hierarchy(vox)
        st, u, info = h.solve(gmt.ELASTIC, tol=TOL)
        out.append((u.cpu().numpy().copy(), h.homogenize(gmt.ELASTIC)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_binding_rejects_mis_sized_inputs(gmt_lib):
    """A field, density vector or voxel array of the wrong size never reaches the library:
    the binding raises ValueError (the library reads exactly the sizes it expects)."""
    import torch
    gmt = gmt_lib
    h = gmt.Hierarchy(L.tpms_network("gyroid", 16, 0.3))
    h.prepare(gmt.ELASTIC)
    n = h.num_nodes(0)
    for bad in (np.zeros((n - 1) * 18), torch.zeros(n * 18 + 6, dtype=torch.float64)):
        with pytest.raises(ValueError):
            h.apply(0, bad, gmt.FP64)
    with pytest.raises(ValueError):
        h.vcycle(np.zeros(n * 18), None, gmt.FP64,
                 corrections=[None, np.zeros(5)] + [None] * (h.levels - 2))
    with pytest.raises(ValueError):
        h.set_densities(np.ones(h.num_elements(0) + 1))
    with pytest.raises(ValueError):
        gmt.Hierarchy(np.zeros((8, 8, 4), dtype=np.uint8))
    with pytest.raises(ValueError):
        gmt.Hierarchy(torch.zeros((8, 8, 4), dtype=torch.uint8))
    h.free()


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_stored_solution_survives_other_calls(gmt_lib, kind):
    """Calls between gmt_solve and C^H of the stored solution leave that solution as it was:
    per-step applies that switch the workspace to the other precision and back, an FP64
    residual, and C^H or sensitivities of another field."""
    gmt = gmt_lib
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    vox = L.tpms_network("gyroid", 32, 0.30)
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(ph, tol=TOL)
    assert st == gmt.OK
    CH = h.homogenize(ph)
    other = u * 0.5
    h.apply(0, u, gmt.FP64)              # the FP64 workspace takes the solution over
    CH64 = h.homogenize(ph)
    assert np.abs(CH64 - CH).max() <= 1e-6 * np.abs(CH).max()
    h.residual(u, gmt.FP64)
    h.homogenize(ph, u=other)
    h.sensitivities(ph, u=other)
    assert np.array_equal(h.homogenize(ph), CH64)
    h.apply(0, u, gmt.FP32)              # and back: the float-float pair round-trips exactly
    assert np.array_equal(h.homogenize(ph), CH)
    h.homogenize(ph, u=other)
    h.sensitivities(ph, u=other)
    h.residual(other, gmt.FP64)
    h.residual(other, gmt.FP32)
    assert np.array_equal(h.homogenize(ph), CH)
    assert not np.allclose(h.homogenize(ph, u=other), CH)
    h.free()


def test_warm_start_resumes(gmt_lib):
    gmt = gmt_lib
    vox = L.largest_component(L.truss("bcc", 32, 0.09))
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(gmt.ELASTIC, tol=TOL)
    st2, u2, info2 = h.solve(gmt.ELASTIC, tol=TOL, u0=u)
    assert info2.outer == 0 and info2.inner_total == 0


@pytest.mark.slow
def test_full_size_128_properties(gmt_lib):
    """A 128^3 cell of the mixed workload at the launch configuration the benchmark times:
    the oracle evaluates the residual and the energy average on the library's field (matrix-
    free, chunked) instead of solving the 2M-dof system itself."""
    gmt = gmt_lib
    vox, desc = L.mixed_cell(2002, 128)
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(gmt.ELASTIC, tol=TOL)
    lev = grid.Level(vox)
    Ke, x0, D, M, C0 = fe.physics("elastic")
    U = to_np(u, D, M)
    F = solve.load(lev, Ke, x0, D)
    R = F - solve.apply_ebe(lev, Ke, U, D)
    res = np.linalg.norm(R, axis=0) / np.linalg.norm(F, axis=0)
    assert res.max() <= TOL * 1.02, res
    CH = h.homogenize(gmt.ELASTIC)
    Co = solve.homogenize_chunked(lev, U, Ke, x0, D)
    assert np.abs(CH - Co).max() <= 2e-7 * np.abs(Co).max()
    phi = vox.mean()
    assert np.linalg.eigvalsh(phi * C0 - CH).min() > -1e-9       # Voigt bound
    assert np.linalg.eigvalsh(CH).min() > -1e-9 and np.abs(CH - CH.T).max() < 1e-12


def test_trace_totals_cover_the_solve(gmt_lib):
    gmt = gmt_lib
    h = gmt.Hierarchy(L.tpms_network("gyroid", 32, 0.30))
    h.trace(True)
    h.solve(gmt.ELASTIC, tol=1e-5, want_field=False)
    h.homogenize(gmt.ELASTIC)
    tot = h.trace_totals()
    for k in ("smooth_l0", "resid_l0", "apply_l0", "outer_resid", "restrict", "prolong",
              "coarse_solve", "energy", "vector", "setup_operators", "setup_coarse_inverse"):
        n, ms, b = tot[k]
        assert n > 0 and ms > 0.0, (k, tot[k])
    assert tot["smooth_l0"][2] > 0


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_graph_replayed_vcycles_match_direct_launches(gmt_lib, kind):
    """On a stream of its own, gmt_solve replays its V-cycles from captured CUDA graphs; the
    result is bitwise the one of the same solve with every kernel launched directly."""
    import torch
    gmt = gmt_lib
    vox, _ = L.batch_cell(3003)          # a 64^3 spinodal cell: 40 V-cycles at 1e-5
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    out = {}
    for graphs in (0, 1):   # (a form is captured after 16 direct V-cycles)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            h = gmt.Hierarchy(vox, gmt.default_options(graphs=graphs), s)
            n0 = gmt.launch_count()
            st, u, info = h.solve(ph, tol=1e-6 if kind == "elastic" else 1e-9)
            launches = gmt.launch_count() - n0
            CH = h.homogenize(ph)
            s.synchronize()
        assert st == gmt.OK and info.inner_total > 18, info.as_dict()
        out[graphs] = (u.cpu().numpy(), CH, info.inner_total, launches)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    assert out[0][3] == out[1][3]     # replays count the kernels of their graph


def test_warm_sweeps_smooth_a_rough_initial_field(gmt_lib):
    """gmt_options.warm_sweeps: damped-Jacobi sweeps applied to a given initial field before
    the iteration. A converged field plus high-frequency noise is mostly rough error, which
    the sweeps remove: the solve from the smoothed start needs no more V-cycles, and both
    reach the same C^H (FP32 and FP64 solves)."""
    import torch
    gmt = gmt_lib
    vox = L.tpms_network("gyroid", 32, 0.3)
    h = gmt.Hierarchy(vox)
    _, u, _ = h.solve(gmt.ELASTIC, tol=1e-8)
    g = torch.Generator(device="cpu").manual_seed(3)
    noisy = u + 0.3 * u.abs().max() * torch.randn(u.shape, generator=g, dtype=torch.float64).cuda()
    h.free()
    for prec in (gmt.FP32, gmt.FP64):
        res = {}
        for sweeps in (0, 4):
            h = gmt.Hierarchy(vox, gmt.default_options(precision=prec, warm_sweeps=sweeps))
            st, _, info = h.solve(gmt.ELASTIC, tol=1e-5, u0=noisy, want_field=False)
            assert st == gmt.OK and max(info.as_dict()["rel_residual"]) <= 1e-5
            res[sweeps] = (info.inner_total, h.homogenize(gmt.ELASTIC))
            h.free()
        assert res[4][0] <= res[0][0], res
        CH0, CH4 = res[0][1], res[4][1]
        assert np.abs(CH4 - CH0).max() <= 1e-4 * np.abs(CH0).max()
