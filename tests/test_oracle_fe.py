"""Pins for the oracle's element matrices (App. F.1, F.2)."""
import numpy as np
import pytest

from oracle import fe

# 1D integrals on [0,1] with N0 = 1-t, N1 = t (textbook closed forms)
M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])          # int Na Nb
K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])               # int Na' Nb'
G1 = np.array([[-0.5, -0.5], [0.5, 0.5]])               # int Na' Nb (a differentiated)


def _grad_integral(i, a, j, b):
    """int over the unit cube of d_i N_a d_j N_b, as a product of 1D integrals."""
    la, lb = fe.LOCAL[a], fe.LOCAL[b]
    v = 1.0
    for d in range(3):
        if d == i and d == j:
            v *= K1[la[d], lb[d]]
        elif d == i:
            v *= G1[la[d], lb[d]]
        elif d == j:
            v *= G1[lb[d], la[d]]
        else:
            v *= M1[la[d], lb[d]]
    return v


def _elastic_Ke_tensor_product(E, nu):
    lam, mu = fe.lame(E, nu)
    K = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            for i in range(3):
                for j in range(3):
                    v = lam * _grad_integral(i, a, j, b) + mu * _grad_integral(j, a, i, b)
                    if i == j:
                        v += mu * sum(_grad_integral(k, a, k, b) for k in range(3))
                    K[3 * a + i, 3 * b + j] = v
    return K


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (2.5, 0.0), (0.7, 0.45)])
def test_elastic_Ke_matches_tensor_product_integrals(E, nu):
    # Independent route: closed-form 1D integrals of the bilinear form
    # lambda div u div v + 2 mu eps(u):eps(v), instead of Gauss quadrature of B^T C0 B.
    np.testing.assert_allclose(fe.elastic_Ke(E, nu), _elastic_Ke_tensor_product(E, nu),
                               rtol=0, atol=1e-14)


def test_heat_Ke_textbook_values():
    # Q1 Laplacian on the unit cube: 1/3 on the diagonal, 0 along edges, -1/12 across face
    # and body diagonals.
    K = fe.heat_Ke(1.0)
    for a in range(8):
        for b in range(8):
            h = int(np.abs(fe.LOCAL[a] - fe.LOCAL[b]).sum())
            expect = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[h]
            assert abs(K[a, b] - expect) < 1e-15


def test_elastic_Ke_kernel_and_symmetry():
    K = fe.elastic_Ke(1.0, 0.3)
    np.testing.assert_allclose(K, K.T, atol=1e-15)
    w = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(w) < 1e-12) == 6 and w.min() > -1e-13
    X = fe.LOCAL.astype(float)
    for d in range(3):                      # translations
        t = np.zeros(24)
        t[d::3] = 1.0
        assert np.abs(K @ t).max() < 1e-14
    for (i, j) in [(0, 1), (0, 2), (1, 2)]:  # infinitesimal rotations
        r = np.zeros(24)
        r[i::3] = -X[:, j]
        r[j::3] = X[:, i]
        assert np.abs(K @ r).max() < 1e-14


def test_x0_energy_is_C0_and_load_equals_direct_integral():
    E, nu = 1.0, 0.3
    K, X = fe.elastic_Ke(E, nu), fe.elastic_x0()
    np.testing.assert_allclose(X.T @ K @ X, fe.elastic_C0(E, nu), atol=1e-14)
    np.testing.assert_allclose(K @ X, fe.element_load_direct(E, nu), atol=1e-14)
    Kh, Xh = fe.heat_Ke(2.0), fe.heat_x0()
    np.testing.assert_allclose(Xh.T @ Kh @ Xh, 2.0 * np.eye(3), atol=1e-14)
    np.testing.assert_allclose(Kh @ Xh, fe.heat_load_direct(2.0), atol=1e-14)
    assert np.abs(Kh.sum(axis=1)).max() < 1e-15


def test_C0_closed_form():
    C = fe.elastic_C0(1.0, 0.3)
    assert abs(C[0, 0] - 1.346153846153846) < 1e-12
    assert abs(C[0, 1] - 0.576923076923077) < 1e-12
    assert abs(C[3, 3] - 0.384615384615385) < 1e-12
