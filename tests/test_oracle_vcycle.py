"""Pins for the oracle V-cycle (Alg. 1 with damped block-Jacobi / Chebyshev smoothing)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fe, galerkin, grid, solve, vcycle
from paper_2604_26518_b300 import lattices as L


def _setup(vox, kind, levels=None):
    lv = grid.hierarchy(vox, levels)
    Ke, x0, D, NC, C0 = fe.physics(kind)
    K1 = solve.assemble(lv[0], Ke, D)
    F = solve.cancel_rounding(solve.load(lv[0], Ke, x0, D), solve.gross_load_norm(lv[0], Ke, x0, D))
    Ks, Ps = galerkin.galerkin_hierarchy(lv, K1, D)
    return lv, Ke, x0, D, K1, F, Ks, Ps


def _lmax(Ks, D):
    out = []
    for K in Ks[:-1]:
        A = vcycle.block_diag_inverse(K, D) @ K
        out.append(float(np.max(np.abs(spla.eigs(A, k=1, which="LM", return_eigenvectors=False)))))
    return out


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_vcycles_converge_to_cg_solution(kind, smoother):
    vox = L.tpms_network("gyroid", 16, 0.3)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, kind)
    kw = {}
    if smoother == "chebyshev":
        kw = {"cheb_lmax": _lmax(Ks, D)}
    vc = vcycle.VCycle(Ks, Ps, D, smoother=smoother, **kw)
    U = np.zeros_like(F)
    fn = np.linalg.norm(F, axis=0)
    hist = []
    for it in range(60):
        U = vc.cycle(F, U)
        hist.append((np.linalg.norm(F - K1 @ U, axis=0) / fn).max())
        if hist[-1] < 1e-11:
            break
    assert hist[-1] < 1e-11
    rate = (hist[-1] / hist[0]) ** (1.0 / (len(hist) - 1))
    assert rate < 0.86                # well under the paper's GMG reference (App. D.2)
    ref = solve.solve_cell(vox, kind)
    U = solve.gauge(U, D)
    C = solve.homogenize(lv[0], U, Ke, x0, D)
    assert np.abs(C - ref["CH"]).max() < 1e-9 * np.abs(ref["CH"]).max()


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_vcycle_operator_is_symmetric(smoother):
    vox = L.tpms_network("schwarz_p", 8, 0.4)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, "elastic", levels=2)
    kw = {"cheb_lmax": _lmax(Ks, D)} if smoother == "chebyshev" else {}
    vc = vcycle.VCycle(Ks, Ps, D, nu_pre=2, nu_post=2, smoother=smoother, **kw)
    rng = np.random.default_rng(0)
    a = solve.gauge(rng.standard_normal((K1.shape[0], 1)), D)
    b = solve.gauge(rng.standard_normal((K1.shape[0], 1)), D)
    ba = vc.cycle(a)
    bb = vc.cycle(b)
    lhs, rhs = float(b[:, 0] @ ba[:, 0]), float(a[:, 0] @ bb[:, 0])
    assert abs(lhs - rhs) < 1e-10 * max(abs(lhs), 1.0)


def test_coarsest_solve_is_zero_mean_solution():
    vox = L.tpms_network("gyroid", 8, 0.4)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, "elastic", levels=2)
    A = vcycle.coarsest_matrix(Ks[-1], D)
    rng = np.random.default_rng(1)
    f = solve.gauge(rng.standard_normal((Ks[-1].shape[0], 2)), D)
    u = np.linalg.solve(A, f)
    assert np.abs(Ks[-1] @ u - f).max() < 1e-10 * np.abs(f).max()
    assert np.abs(u.reshape(-1, D, 2).mean(axis=0)).max() < 1e-12 * np.abs(u).max()
