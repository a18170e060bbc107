"""Element densities of the SIMP interpolation (App. F.3) on the GPU, against the oracle's
coefficient path: C_e = (rho_min + rho_e^p) C0 per element.

  * every level's operator (level 0 from the stored per-node stencils with coefficients,
    levels >= 1 the element-local Galerkin products of the weighted element matrices) against
    the oracle's global P^T K P of the assembled weighted matrix;
  * full solves: C^H within 1e-4 of the oracle's converged C^H, the oracle's residual of the
    library's field, and the library's C^H equal to the oracle's energy average of that
    field;
  * sensitivities p rho_e^(p-1) / N^3 (x0 - u_e)^T K0 (x0 - u_e) against the oracle's on the
    library's field;
  * unit densities with rho_min = 0 reproduce the binary design, and clearing the densities
    returns to it; bad densities are rejected.
"""
import numpy as np
import pytest

from oracle import fe, galerkin, grid, solve
from paper_2604_26518_b300 import lattices as L
from helpers import rel_err, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5
RHO_MIN, P = 1e-3, 3.0


def _cell(name):
    if name == "gyroid24":
        return L.tpms_network("gyroid", 24, 0.4)
    if name == "octet16":
        return L.largest_component(L.truss("octet", 16, 0.11))
    if name == "random8":
        return L.largest_component(L.random_binary(8, 0.6, np.random.default_rng(4)))
    raise ValueError(name)


def _rho(n_elems, seed):
    return np.random.default_rng(seed).uniform(0.2, 1.0, n_elems)


def _oracle(vox, kind, levels, rho):
    lv = grid.hierarchy(vox, levels)
    Ke, x0, D, M, C0 = fe.physics(kind)
    coef = solve.simp_coef(lv[0], rho, RHO_MIN, P)
    K1 = solve.assemble(lv[0], Ke, D, coef)
    Ks, Ps = galerkin.galerkin_hierarchy(lv, K1, D)
    return lv, coef, Ks, Ps, D, M


@pytest.mark.parametrize("name", ["gyroid24", "octet16"])
@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_operators_with_densities(gmt_lib, name, kind):
    gmt = gmt_lib
    vox = _cell(name)
    h = gmt.Hierarchy(vox)
    rho = _rho(h.num_elements(0), 1)
    h.set_densities(rho, RHO_MIN, P)
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    h.prepare(ph)
    lv, coef, Ks, Ps, D, M = _oracle(vox, kind, h.levels, rho)
    rng = np.random.default_rng(9)
    for l in range(h.levels):
        if h.num_bricks(l) == 0:
            continue
        u = rng.standard_normal((h.num_nodes(l) * D, M))
        Ku = Ks[l] @ u
        y64 = to_np(h.apply(l, u, gmt.FP64), D, M)
        assert rel_err(y64, Ku) < 1e-12, (l, rel_err(y64, Ku))
        y32 = to_np(h.apply(l, u, gmt.FP32), D, M)
        assert rel_err(y32, Ku) < 2e-5, (l, rel_err(y32, Ku))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_solve_with_densities_matches_oracle(gmt_lib, kind, precision):
    gmt = gmt_lib
    vox = _cell("gyroid24")
    prec = gmt.FP64 if precision == "fp64" else gmt.FP32
    h = gmt.Hierarchy(vox, gmt.default_options(precision=prec))
    rho = _rho(h.num_elements(0), 2)
    h.set_densities(rho, RHO_MIN, P)
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    st, u, info = h.solve(ph, tol=TOL)
    assert st == gmt.OK, info.as_dict()
    lev = grid.Level(vox.astype(bool))
    coef = solve.simp_coef(lev, rho, RHO_MIN, P)
    ref = solve.solve_cell(vox, kind, coef=coef, tol=1e-10)
    D, M = ref["D"], ref["NC"]
    U = to_np(u, D, M)
    res = solve.relative_residual(ref["K"], ref["F"], U)
    assert res.max() <= TOL * 1.02, (res, info.as_dict())
    CH = h.homogenize(ph)
    assert np.abs(CH - ref["CH"]).max() <= 1e-4 * np.abs(ref["CH"]).max()
    C_of_gpu = solve.homogenize(ref["level"], U, ref["Ke"], ref["x0"], D, coef)
    tol = 1e-12 if precision == "fp64" else 2e-7
    assert np.abs(CH - C_of_gpu).max() <= tol * np.abs(ref["CH"]).max()
    # sensitivities of the library's field
    sens = h.sensitivities(ph, p=P).cpu().numpy()
    expect = solve.sensitivities(ref["level"], U, ref["Ke"], ref["x0"], D, P, rho=rho)
    stol = 1e-12 if precision == "fp64" else 2e-6
    assert np.abs(sens - expect).max() <= stol * np.abs(expect).max()
    with pytest.raises(gmt.GmtError):
        h.sensitivities(ph, p=2.0)        # p must be the densities' p


@pytest.mark.parametrize("name", ["random8", "octet16"])
def test_small_hierarchies_with_densities(gmt_lib, name):
    """A single-level (8^3: level 0 is the coarsest, solved directly) and a multi-level cell,
    against the brute-force dense solve with the same coefficients."""
    gmt = gmt_lib
    vox = _cell(name)
    h = gmt.Hierarchy(vox, gmt.default_options(precision=gmt.FP64))
    rho = _rho(h.num_elements(0), 3)
    h.set_densities(rho, RHO_MIN, P)
    st, u, info = h.solve(gmt.ELASTIC, tol=1e-9)
    assert st == gmt.OK, info.as_dict()
    lev = grid.Level(vox.astype(bool))
    _, C = solve.brute_force(vox, "elastic", coef=solve.simp_coef(lev, rho, RHO_MIN, P))
    assert np.abs(h.homogenize(gmt.ELASTIC) - C).max() <= 1e-7 * np.abs(C).max()


def test_unit_densities_reproduce_the_binary_design(gmt_lib):
    gmt = gmt_lib
    vox = _cell("gyroid24")
    h = gmt.Hierarchy(vox, gmt.default_options(precision=gmt.FP64))
    h.solve(gmt.ELASTIC, tol=1e-8)
    C_bin = h.homogenize(gmt.ELASTIC)
    h.set_densities(np.ones(h.num_elements(0)), 0.0, P)
    st, _, _ = h.solve(gmt.ELASTIC, tol=1e-8)
    assert st == gmt.OK
    C_unit = h.homogenize(gmt.ELASTIC)
    assert np.abs(C_unit - C_bin).max() <= 1e-7 * np.abs(C_bin).max()
    # uniform density 0.5: the tensor scales by rho_min + 0.5^p
    h.set_densities(np.full(h.num_elements(0), 0.5), RHO_MIN, P)
    h.solve(gmt.ELASTIC, tol=1e-8)
    C_half = h.homogenize(gmt.ELASTIC)
    assert np.abs(C_half - (RHO_MIN + 0.5 ** P) * C_bin).max() <= 1e-7 * np.abs(C_bin).max()
    h.set_densities(None)
    h.solve(gmt.ELASTIC, tol=1e-8)
    assert np.abs(h.homogenize(gmt.ELASTIC) - C_bin).max() <= 1e-9 * np.abs(C_bin).max()


def test_bad_densities_are_rejected(gmt_lib):
    gmt = gmt_lib
    h = gmt.Hierarchy(_cell("octet16"))
    ne = h.num_elements(0)
    for rho, rmin in ((np.full(ne, 1.5), 1e-3), (np.full(ne, -0.1), 1e-3), (np.zeros(ne), 0.0)):
        with pytest.raises(gmt.GmtError) as e:
            h.set_densities(rho, rmin, P)
        assert e.value.status == gmt.ERR_ARG
