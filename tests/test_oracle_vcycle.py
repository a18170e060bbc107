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


# ---------------------------------------------------------------- 8-colour Gauss-Seidel
def test_same_colour_nodes_are_decoupled():
    vox = L.tpms_network("diamond", 16, 0.35)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, "elastic")
    for lev, K in zip(lv[:-1], Ks[:-1]):
        xyz = lev.node_xyz()
        col = (xyz[:, 0] & 1) + 2 * (xyz[:, 1] & 1) + 4 * (xyz[:, 2] & 1)
        Kc = K.tocoo()
        a, b = Kc.row // D, Kc.col // D
        off = (a != b) & (np.abs(Kc.data) > 0)
        assert not np.any(col[a[off]] == col[b[off]])


def test_gs8_sweep_equals_nodewise_block_gauss_seidel():
    """With omega = 1 the colour-by-colour sweep is block Gauss-Seidel over the nodes in
    colour order (written here as a plain loop solving each node's D x D block)."""
    vox = L.tpms_network("gyroid", 8, 0.4)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, "elastic", 2)
    vc = vcycle.VCycle(Ks, Ps, D, omega=1.0, smoother="gs8", levels=lv)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(F.shape)
    got = vc.smooth(0, u0, F, 1)
    K = Ks[0].toarray()
    xyz = lv[0].node_xyz()
    col = (xyz[:, 0] & 1) + 2 * (xyz[:, 1] & 1) + 4 * (xyz[:, 2] & 1)
    u = u0.copy()
    for c in range(8):
        for n in np.nonzero(col == c)[0]:
            rows = slice(n * D, n * D + D)
            r = F[rows] - K[rows] @ u
            u[rows] += np.linalg.solve(K[rows, rows], r)
    assert np.abs(got - u).max() <= 1e-12 * np.abs(u).max()


# ---------------------------------------------------------------- W- and F-cycles
def test_two_level_cycles_coincide():
    vox = L.tpms_network("schwarz_p", 16, 0.3)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, "elastic", 2)
    outs = [vcycle.VCycle(Ks, Ps, D, kind=k).cycle(F) for k in ("V", "W", "F")]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_three_level_w_cycle_is_v_with_two_coarse_cycles():
    """On three levels the W-cycle's coarse correction is two level-1 cycles (the second
    starting from the first), each ending in the exact coarsest solve; written out here from
    the assembled matrices with the smoother formula, not through VCycle.cycle."""
    vox = L.tpms_network("gyroid", 16, 0.3)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, "elastic", 3)
    vc = vcycle.VCycle(Ks, Ps, D, kind="W")
    Di = [vcycle.block_diag_inverse(K, D) for K in Ks[:-1]]
    Ainv = np.linalg.inv(vcycle.coarsest_matrix(Ks[-1], D))

    def jac(l, u, f, n):
        for _ in range(n):
            u = u + 0.6 * (Di[l] @ (f - Ks[l] @ u))
        return u

    def two_grid(l, f, u):
        u = jac(l, u, f, 2)
        uc = Ainv @ (Ps[l].T @ (f - Ks[l] @ u))
        return jac(l, u + Ps[l] @ uc, f, 2)

    u = jac(0, np.zeros_like(F), F, 2)
    fc = Ps[0].T @ (F - Ks[0] @ u)
    uc = two_grid(1, fc, np.zeros_like(fc))
    uc = two_grid(1, fc, uc)
    expect = jac(0, u + Ps[0] @ uc, F, 2)
    got = vc.cycle(F)
    assert np.abs(got - expect).max() <= 1e-12 * np.abs(expect).max()
    # F on three levels: F-cycle then V-cycle on level 1 = the same two two-grid cycles
    assert np.abs(vcycle.VCycle(Ks, Ps, D, kind="F").cycle(F) - expect).max() <= 1e-12 * np.abs(expect).max()


@pytest.mark.parametrize("kind", ["W", "F"])
def test_w_and_f_cycles_contract_at_least_as_well_as_v(kind):
    vox = L.tpms_network("gyroid", 32, 0.3)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, "elastic", 4)
    fn = np.linalg.norm(F, axis=0)

    def rate(k):
        vc = vcycle.VCycle(Ks, Ps, D, kind=k)
        U = np.zeros_like(F)
        for _ in range(6):
            U = vc.cycle(F, U)
        return (np.linalg.norm(F - Ks[0] @ U, axis=0) / fn).max()

    assert rate(kind) <= rate("V") * 1.0001


# ---------------------------------------------------------------- Chebyshev closed form
def _cheb_T(k: int, x: np.ndarray) -> np.ndarray:
    """T_k(x) from its closed forms: cos(k arccos x) on |x| <= 1, sign(x)^k cosh(k arccosh|x|)
    outside (not from the three-term recurrence the smoother uses)."""
    x = np.asarray(x, dtype=np.float64)
    inside = np.abs(x) <= 1.0
    out = np.empty_like(x)
    out[inside] = np.cos(k * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** k * np.cosh(k * np.arccosh(np.abs(xo)))
    return out


@pytest.mark.parametrize("D", [1, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_chebyshev_smoother_matches_closed_form_damping(D, k):
    """The Chebyshev semi-iteration of degree k on D^-1 K over [a, b] multiplies the error's
    component along each eigenvector of D^-1 K (eigenvalue lam) by
        T_k((theta - lam) / delta) / T_k(theta / delta),   theta = (b+a)/2, delta = (b-a)/2.
    K is a random SPD matrix with a chosen spectrum; the eigenpairs of D^-1 K (D its D x D
    block diagonal) come from a dense eigendecomposition. Eigenvalues lie both inside [a, b]
    and below a (where the damping is weak), so a wrong interval end, recurrence coefficient
    or dropped rho' rho factor changes the per-eigenvalue ratio."""
    import scipy.sparse as sp
    rng = np.random.default_rng(100 + 10 * D + k)
    n = 12 * D
    # eigenvalues: a few below a = lmax/ratio, the rest spread over [a, lmax]
    lmax, ratio, upper = 3.0, 30.0, 1.1
    a_lo = lmax / ratio
    lam = np.concatenate([rng.uniform(0.2 * a_lo, 0.9 * a_lo, 3),
                          rng.uniform(a_lo, lmax, n - 4), [lmax]])
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * lam) @ Q.T                            # SPD with spectrum lam
    K = sp.csr_matrix(A)
    Dinv = vcycle.block_diag_inverse(K, D).toarray()
    # D^-1 K is similar to the symmetric D^-1/2 K D^-1/2: real eigenpairs (w, V)
    w, V = np.linalg.eig(Dinv @ A)
    w, V = w.real, V.real
    lm = float(w.max())
    vc = vcycle.VCycle([K, sp.identity(1, format="csr")], [None], D, smoother="chebyshev",
                       cheb_lmax=[lm], cheb_ratio=ratio, cheb_upper=upper)
    u_star = rng.standard_normal((n, 2))
    f = A @ u_star
    u0 = rng.standard_normal((n, 2))
    got = vc.smooth(0, u0, f, k)
    b, a = upper * lm, lm / ratio
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    damp = _cheb_T(k, (theta - w) / delta) / _cheb_T(k, np.array([theta / delta]))[0]
    e0 = np.linalg.solve(V, u0 - u_star)           # error in the eigenbasis of D^-1 K
    expect = u_star + V @ (damp[:, None] * e0)
    assert np.abs(got - expect).max() <= 1e-12 * np.abs(expect).max()
    # the spectrum has eigenvalues below a (weakly damped) and inside [a, b], where the
    # damping is at most 1 / T_k(theta/delta)
    inside = (w >= a) & (w <= b)
    assert inside.sum() >= n // 2 and (w < a).sum() >= 1
    assert np.all(np.abs(damp[inside]) <= 1.0 / _cheb_T(k, np.array([theta / delta]))[0] + 1e-12)


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_injected_corrections_follow_the_error_propagation_form(kind):
    """Alg. 2's injected coarse start, pinned by the textbook error propagation of the cycle:
    on three levels, starting level 1's coarse unknown from x instead of zero changes the
    cycle's output by S0_post P0 S1_post (I - P1 A2 P1^T K1) S1_pre x, S = (I - w D^-1 K)^nu
    the damped-Jacobi error propagators and A2 the exact coarsest solve; an entry at the
    coarsest level changes nothing, and corrections that are all None give Alg. 1 exactly."""
    vox = L.tpms_network("gyroid", 16, 0.3)
    lv, Ke, x0, D, K1, F, Ks, Ps = _setup(vox, kind, levels=3)
    vc = vcycle.VCycle(Ks, Ps, D, nu_pre=1, nu_post=1, nu_coarse=2)
    rng = np.random.default_rng(11)
    x = rng.standard_normal((Ks[1].shape[0], F.shape[1]))
    base = vc.cycle(F)
    assert np.array_equal(vc.cycle(F, e=[None, None, None]), base)
    assert np.array_equal(vc.cycle(F, e=[None, None, rng.standard_normal((Ks[2].shape[0], F.shape[1]))]), base)

    def S(l, v, nu):
        Di = vcycle.block_diag_inverse(Ks[l], D)
        for _ in range(nu):
            v = v - 0.6 * (Di @ (Ks[l] @ v))
        return v
    d = S(1, x, 2)
    d = d - Ps[1] @ (vc.Ainv @ (Ps[1].T @ (Ks[1] @ d)))
    d = S(1, d, 2)
    d = S(0, Ps[0] @ d, 1)
    got = vc.cycle(F, e=[None, x, None]) - base
    assert np.abs(got - d).max() <= 1e-9 * np.abs(d).max(), np.abs(got - d).max() / np.abs(d).max()
    assert np.abs(d).max() > 1e-3 * np.abs(base).max()     # the injection is not negligible
