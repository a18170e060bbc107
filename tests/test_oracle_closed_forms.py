"""Pins for the oracle's cell solve and C^H (App. F): closed forms, bounds, invariants,
brute force. Fixtures are written in tests/golden/closed_forms.txt with their sources."""
import numpy as np
import pytest

from oracle import fe, solve
from paper_2604_26518_b300 import lattices as L

E, NU = 1.0, 0.3
LAM, MU = fe.lame(E, NU)


def test_fully_solid_cell_returns_C0():
    vox = np.ones((8, 8, 8), dtype=np.uint8)
    out = solve.solve_cell(vox, "elastic", E, NU)
    assert np.abs(out["F"]).max() == 0.0          # f = 0 for a uniform cell
    np.testing.assert_allclose(out["CH"], fe.elastic_C0(E, NU), atol=1e-13)
    outh = solve.solve_cell(vox, "heat", k=1.0)
    np.testing.assert_allclose(outh["CH"], np.eye(3), atol=1e-13)


@pytest.mark.parametrize("layers", [[0, 1], [0, 1, 2, 4, 5], [3]])
def test_void_laminate_plane_stress(layers):
    n = 8
    vox = L.laminate_z(n, layers)
    phi = len(layers) / n
    C = solve.solve_cell(vox, "elastic", E, NU)["CH"]
    expect = np.zeros((6, 6))
    expect[0, 0] = expect[1, 1] = phi * E / (1 - NU ** 2)
    expect[0, 1] = expect[1, 0] = phi * E * NU / (1 - NU ** 2)
    expect[5, 5] = phi * MU
    np.testing.assert_allclose(C, expect, atol=1e-10)
    kap = solve.solve_cell(vox, "heat", k=1.0)["CH"]
    np.testing.assert_allclose(kap, np.diag([phi, phi, 0.0]), atol=1e-10)


def _backus(phis, scales):
    """Exact effective stiffness of isotropic layers normal to z (layered-medium averages)."""
    C = [s * fe.elastic_C0(E, NU) for s in scales]
    avg = lambda f: sum(p * f(c) for p, c in zip(phis, C))
    inv33 = 1.0 / avg(lambda c: 1.0 / c[2, 2])
    r13 = avg(lambda c: c[0, 2] / c[2, 2])
    out = np.zeros((6, 6))
    out[2, 2] = inv33
    out[0, 2] = out[2, 0] = out[1, 2] = out[2, 1] = r13 * inv33
    out[0, 0] = out[1, 1] = avg(lambda c: c[0, 0] - c[0, 2] ** 2 / c[2, 2]) + r13 ** 2 * inv33
    out[0, 1] = out[1, 0] = avg(lambda c: c[0, 1] - c[0, 2] ** 2 / c[2, 2]) + r13 ** 2 * inv33
    out[3, 3] = out[4, 4] = 1.0 / avg(lambda c: 1.0 / c[3, 3])
    out[5, 5] = avg(lambda c: c[5, 5])
    return out


def test_two_phase_laminate_series_parallel():
    n = 8
    vox = np.ones((n, n, n), dtype=np.uint8)
    coef = np.ones((n, n, n))
    coef[:3] = 0.2                                 # 3 soft layers, 5 stiff layers
    phis, scales = [3 / 8, 5 / 8], [0.2, 1.0]
    kap = solve.solve_cell(vox, "heat", k=1.0, coef=coef)["CH"]
    par = sum(p * s for p, s in zip(phis, scales))
    ser = 1.0 / sum(p / s for p, s in zip(phis, scales))
    np.testing.assert_allclose(kap, np.diag([par, par, ser]), atol=1e-10)
    C = solve.solve_cell(vox, "elastic", E, NU, coef=coef)["CH"]
    np.testing.assert_allclose(C, _backus(phis, scales), atol=1e-10)


def test_rods_along_x_uniaxial():
    n = 8
    vox = L.rods_x(n, 2, 2, 2)
    phi = vox.mean()
    C = solve.solve_cell(vox, "elastic", E, NU)["CH"]
    expect = np.zeros((6, 6))
    expect[0, 0] = phi * E
    np.testing.assert_allclose(C, expect, atol=1e-10)
    kap = solve.solve_cell(vox, "heat", k=1.0)["CH"]
    np.testing.assert_allclose(kap, np.diag([phi, 0, 0]), atol=1e-10)


@pytest.mark.parametrize("n,seed", [(4, 1), (6, 2), (8, 3)])
def test_brute_force_matches_cg(n, seed):
    rng = np.random.default_rng(seed)
    vox = L.random_binary(n, 0.55, rng)
    for kind in ("elastic", "heat"):
        out = solve.solve_cell(vox, kind, E, NU, tol=1e-13)
        Ub, Cb = solve.brute_force(vox, kind, E, NU)
        scale = np.abs(Cb).max()
        assert np.abs(out["CH"] - Cb).max() <= 1e-10 * scale
        err = solve.energy_norm_error(out["K"], out["U"], Ub, out["Ke"], out["x0"],
                                      out["level"], out["D"])
        assert err.max() < 1e-8


@pytest.fixture(scope="module")
def gyroid16():
    # fixed level-set threshold (not the exact-count rule, whose tie-breaking by linear
    # index can break the cyclic symmetry of the voxel set)
    vox = (L.gyroid_field(16) < -0.45).astype(np.uint8)
    assert (np.transpose(vox, (1, 2, 0)) == vox).all()
    return vox, solve.solve_cell(vox, "elastic", E, NU), solve.solve_cell(vox, "heat", k=1.0)


def test_gyroid_bounds_and_symmetry(gyroid16):
    vox, el, th = gyroid16
    C, kap = el["CH"], th["CH"]
    phi = vox.mean()
    assert el["res"].max() <= 1e-12 and th["res"].max() <= 1e-12
    np.testing.assert_allclose(C, C.T, atol=1e-12)
    assert np.linalg.eigvalsh(C).min() > -1e-12
    # Voigt bound (exact for FE): phi*C0 - C^H is positive semidefinite
    assert np.linalg.eigvalsh(phi * fe.elastic_C0(E, NU) - C).min() > -1e-12
    assert np.linalg.eigvalsh(phi * np.eye(3) - kap).min() > -1e-12
    # gyroid is invariant under the cyclic permutation x->y->z of the voxel-centre grid
    s = np.abs(C).max()
    assert abs(C[0, 0] - C[1, 1]) < 1e-9 * s and abs(C[1, 1] - C[2, 2]) < 1e-9 * s
    assert abs(C[0, 1] - C[1, 2]) < 1e-9 * s and abs(C[0, 1] - C[0, 2]) < 1e-9 * s
    assert abs(C[3, 3] - C[4, 4]) < 1e-9 * s and abs(C[4, 4] - C[5, 5]) < 1e-9 * s
    assert abs(kap[0, 0] - kap[1, 1]) < 1e-9 and abs(kap[1, 1] - kap[2, 2]) < 1e-9
    # mixed form equals the energy form at convergence
    mixed = solve.homogenize_mixed(el["level"], el["U"], el["Ke"], el["x0"], 3)
    assert np.abs(mixed - C).max() < 1e-10 * s
    # Hashin-Shtrikman upper bound for a void phase (soft: voxel FE is stiffer)
    kHS = 2 * phi / (3 - phi)
    assert kap[0, 0] <= kHS * 1.25


def test_roll_and_scaling_invariance(gyroid16):
    vox, el, _ = gyroid16
    rolled = np.roll(vox, shift=(3, 5, 1), axis=(0, 1, 2))
    C2 = solve.solve_cell(rolled, "elastic", E, NU)["CH"]
    assert np.abs(C2 - el["CH"]).max() < 1e-10
    C3 = solve.solve_cell(vox, "elastic", 2.5, NU)["CH"]
    assert np.abs(C3 - 2.5 * el["CH"]).max() < 1e-10


def test_rotation_permutes_tensor(gyroid16):
    vox, el, _ = gyroid16
    # swap x and y axes of the voxel field (array axes are [z, y, x])
    sw = np.ascontiguousarray(np.swapaxes(vox, 1, 2))
    C2 = solve.solve_cell(sw, "elastic", E, NU)["CH"]
    perm = [1, 0, 2, 4, 3, 5]                      # xx<->yy, yz<->xz, xy fixed
    assert np.abs(C2 - el["CH"][np.ix_(perm, perm)]).max() < 1e-10


def test_ebe_apply_and_chunked_energy_match_assembled(gyroid16):
    vox, el, _ = gyroid16
    rng = np.random.default_rng(5)
    U = rng.standard_normal(el["F"].shape)
    np.testing.assert_allclose(solve.apply_ebe(el["level"], el["Ke"], U, 3, chunk=257),
                               el["K"] @ U, atol=1e-12)
    C = solve.homogenize_chunked(el["level"], el["U"], el["Ke"], el["x0"], 3, chunk=300)
    np.testing.assert_allclose(C, el["CH"], atol=1e-14)
