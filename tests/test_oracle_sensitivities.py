"""Pins of the oracle's inverse-homogenization sensitivities (App. F.3).

dC^H / d rho_e of the SIMP model C_e = (rho_min + rho_e^p) C0 at rho_e = 1 is p times the
derivative of C^H with respect to a scalar stiffness factor s_e of element e. C^H is the
minimum of the cell energy over periodic fields, so that derivative is the element's
energy at the minimiser (no field-derivative term): it is checked here by central finite
differences of brute-force (dense pseudo-inverse) solves with s_e = 1 +- h, which share no
step with the energy formula. The sum over elements returns p C^H exactly. At intermediate densities rho_e in (0, 1)
the derivative with respect to rho_e itself is checked by central finite differences of
brute-force solves with the coefficients rho_min + rho^p.
"""
import numpy as np
import pytest

from oracle import fe, solve
from oracle.grid import Level
from paper_2604_26518_b300 import lattices


def _cell(n, seed):
    rng = np.random.default_rng(seed)
    vox = lattices.largest_component(lattices.random_binary(n, 0.6, rng))
    assert vox.any()
    return vox


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_sensitivity_matches_finite_difference(kind):
    vox = _cell(4, 11)
    Ke, x0, D, NC, C0 = fe.physics(kind, 1.0, 0.3, 1.0)
    lev = Level(vox.astype(bool))
    U, _ = solve.brute_force(vox, kind)
    p = 3.0
    sens = solve.sensitivities(lev, U, Ke, x0, D, p)
    rng = np.random.default_rng(5)
    h = 1e-5
    for e in rng.choice(lev.num_elements, size=3, replace=False):
        coef = np.ones(vox.shape)
        coef.reshape(-1)[lev.elem_lin[e]] = 1.0 + h
        _, Cp = solve.brute_force(vox, kind, coef=coef)
        coef.reshape(-1)[lev.elem_lin[e]] = 1.0 - h
        _, Cm = solve.brute_force(vox, kind, coef=coef)
        fd = p * (Cp - Cm) / (2 * h)
        assert np.abs(sens[e] - fd).max() <= 1e-6 * max(np.abs(sens[e]).max(), 1e-3), (e, sens[e], fd)


def test_sensitivities_sum_to_p_times_CH():
    vox = lattices.tpms_network("gyroid", 8, 0.4)
    Ke, x0, D, NC, C0 = fe.physics("elastic", 1.0, 0.3, 1.0)
    lev = Level(vox.astype(bool))
    U, CH = solve.brute_force(vox, "elastic")
    sens = solve.sensitivities(lev, U, Ke, x0, D, 2.5)
    assert np.allclose(sens.sum(axis=0), 2.5 * CH, rtol=1e-12, atol=1e-14)
    assert np.allclose(sens, np.transpose(sens, (0, 2, 1)))


def test_solid_cell_sensitivity_is_uniform():
    # fully solid: u = 0, every element carries x0^T K0 x0 = C0 (unit element volume)
    vox = np.ones((4, 4, 4), dtype=np.uint8)
    Ke, x0, D, NC, C0 = fe.physics("elastic", 1.0, 0.3, 1.0)
    lev = Level(vox.astype(bool))
    U = np.zeros((lev.num_nodes * D, NC))
    sens = solve.sensitivities(lev, U, Ke, x0, D, 3.0)
    assert np.allclose(sens, 3.0 / 64.0 * C0[None], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_simp_sensitivity_at_intermediate_densities(kind):
    vox = _cell(4, 12)
    Ke, x0, D, NC, C0 = fe.physics(kind, 1.0, 0.3, 1.0)
    lev = Level(vox.astype(bool))
    rng = np.random.default_rng(21)
    rho = rng.uniform(0.2, 0.95, lev.num_elements)
    rho_min, p = 1e-3, 3.0
    U, C = solve.brute_force(vox, kind, coef=solve.simp_coef(lev, rho, rho_min, p))
    sens = solve.sensitivities(lev, U, Ke, x0, D, p, rho=rho)
    h = 1e-5
    for e in rng.choice(lev.num_elements, size=3, replace=False):
        r = rho.copy()
        r[e] += h
        _, Cp = solve.brute_force(vox, kind, coef=solve.simp_coef(lev, r, rho_min, p))
        r[e] -= 2 * h
        _, Cm = solve.brute_force(vox, kind, coef=solve.simp_coef(lev, r, rho_min, p))
        fd = (Cp - Cm) / (2 * h)
        assert np.abs(sens[e] - fd).max() <= 1e-6 * max(np.abs(sens[e]).max(), 1e-4), (e, sens[e], fd)
    # the sum rule with coefficients: sum_e rho_e^(1-p) s_e / p * dC/drho_e = C^H
    s_e = rho_min + rho ** p
    back = (s_e / (p * rho ** (p - 1.0)))[:, None, None] * sens
    assert np.allclose(back.sum(axis=0), C, rtol=1e-11, atol=1e-14)


def test_simp_coefficients_of_uniform_density_scale_the_tensor():
    """A uniform density rho on every element scales C^H by rho_min + rho^p exactly
    (the system K u = f scales as a whole, u is unchanged)."""
    vox = lattices.tpms_network("gyroid", 8, 0.4)
    lev = Level(vox.astype(bool))
    base = solve.solve_cell(vox, "elastic")["CH"]
    rho = np.full(lev.num_elements, 0.7)
    C = solve.solve_cell(vox, "elastic", coef=solve.simp_coef(lev, rho, 1e-3, 3.0))["CH"]
    assert np.allclose(C, (1e-3 + 0.7 ** 3) * base, rtol=1e-9, atol=1e-14)
