"""Hex8 element matrices on the unit voxel (App. F.1, F.2) — oracle, test infrastructure.

Local node a = (a_x, a_y, a_z) in {0,1}^3 has index a_x + 2 a_y + 4 a_z. Element degrees
of freedom are ordered (node a, component i) -> 3 a + i for elasticity and a for heat.

Elasticity (App. F.1): K_e = int_{[0,1]^3} B^T C0 B dV, integrated with the 2x2x2
Gauss-Legendre rule (exact for this polynomial integrand). Voigt order is
(xx, yy, zz, yz, xz, xy) with engineering shear strains, as the six unit macro-strain
modes of App. F.1 are written.

Heat (App. F.2): K_e^th = int grad(N)^T kappa0 grad(N) dV.

The macroscopic modes: the paper writes x0 = K_e^{-1} f_e, which is not defined because
K_e is singular. Reading used here: x0 is the element-local nodal vector of the affine
field u(x) = E_m x (E_m the symmetric strain tensor of Voigt mode m, shear entries 1/2),
or T(x) = e_i . x for heat. K_e x0 equals int B^T C0 eps_m dV = f_e (App. F.1), and any
rigid-motion difference from another choice is annihilated by K_e.
"""
from __future__ import annotations

import numpy as np

GAUSS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))
LOCAL = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int64)


def shape_values(xi):
    """Trilinear shape functions N_a at point xi in [0,1]^3."""
    out = np.ones(8)
    for a in range(8):
        for d in range(3):
            out[a] *= xi[d] if LOCAL[a, d] else (1.0 - xi[d])
    return out


def shape_gradients(xi):
    """dN_a/dx_d at xi, shape (8, 3)."""
    g = np.zeros((8, 3))
    for a in range(8):
        for d in range(3):
            v = 1.0 if LOCAL[a, d] else -1.0
            for e in range(3):
                if e != d:
                    v *= xi[e] if LOCAL[a, e] else (1.0 - xi[e])
            g[a, d] = v
    return g


def lame(E: float, nu: float):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elastic_C0(E: float, nu: float) -> np.ndarray:
    """Isotropic 6x6 Voigt stiffness, engineering shear (C44 = mu)."""
    lam, mu = lame(E, nu)
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2.0 * mu
        C[3 + i, 3 + i] = mu
    return C


def strain_matrix(xi) -> np.ndarray:
    """B (6 x 24): Voigt engineering strain of the element displacement at xi."""
    g = shape_gradients(xi)
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = g[a]
        c = 3 * a
        B[0, c + 0] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 1] = gz
        B[3, c + 2] = gy
        B[4, c + 0] = gz
        B[4, c + 2] = gx
        B[5, c + 0] = gy
        B[5, c + 1] = gx
    return B


def gauss_points():
    for qz in GAUSS:
        for qy in GAUSS:
            for qx in GAUSS:
                yield np.array([qx, qy, qz]), 1.0 / 8.0


def elastic_Ke(E: float, nu: float) -> np.ndarray:
    """K_e = sum_q w_q B_q^T C0 B_q (24 x 24), App. F.1."""
    C = elastic_C0(E, nu)
    K = np.zeros((24, 24))
    for xi, w in gauss_points():
        B = strain_matrix(xi)
        K += w * B.T @ C @ B
    return K


def heat_Ke(k: float) -> np.ndarray:
    """K_e^th = sum_q w_q grad(N)_q k grad(N)_q^T (8 x 8), App. F.2."""
    K = np.zeros((8, 8))
    for xi, w in gauss_points():
        g = shape_gradients(xi)
        K += w * k * g @ g.T
    return K


def voigt_strain_tensor(m: int) -> np.ndarray:
    """Symmetric strain tensor of unit Voigt mode m (engineering shear -> 1/2 entries)."""
    E = np.zeros((3, 3))
    if m < 3:
        E[m, m] = 1.0
    else:
        i, j = {3: (1, 2), 4: (0, 2), 5: (0, 1)}[m]
        E[i, j] = E[j, i] = 0.5
    return E


def elastic_x0() -> np.ndarray:
    """Nodal values of the six affine modes on the unit element, shape (24, 6)."""
    X = np.zeros((24, 6))
    for m in range(6):
        Em = voigt_strain_tensor(m)
        for a in range(8):
            X[3 * a:3 * a + 3, m] = Em @ LOCAL[a].astype(np.float64)
    return X


def heat_x0() -> np.ndarray:
    """Nodal values of T0^(i) = e_i . x on the unit element, shape (8, 3)."""
    return LOCAL.astype(np.float64).copy()


def element_load_direct(E: float, nu: float) -> np.ndarray:
    """f_e = int B^T C0 eps_bar dV for the six unit strain modes (24 x 6), App. F.1,
    integrated directly (not through x0) — used to pin f_e = K_e x0."""
    C = elastic_C0(E, nu)
    F = np.zeros((24, 6))
    for xi, w in gauss_points():
        B = strain_matrix(xi)
        F += w * B.T @ C
    return F


def heat_load_direct(k: float) -> np.ndarray:
    """F_e^th = int B_th^T k I dV (8 x 3), App. F.2."""
    F = np.zeros((8, 3))
    for xi, w in gauss_points():
        F += w * k * shape_gradients(xi)
    return F


def physics(kind: str, E: float = 1.0, nu: float = 0.3, k: float = 1.0):
    """(K_e, x0, dofs per node, number of load cases, base tensor) for 'elastic' / 'heat'."""
    if kind == "elastic":
        return elastic_Ke(E, nu), elastic_x0(), 3, 6, elastic_C0(E, nu)
    if kind == "heat":
        return heat_Ke(k), heat_x0(), 1, 3, k * np.eye(3)
    raise ValueError(kind)
