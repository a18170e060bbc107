"""Assembled FE system, CG solve and homogenized tensor — oracle, test infrastructure.

Definitions (paper): the discrete cell problem K u = f (eq. linear_system, Sec. 3.1) with
K = sum_e A_e^T K_e A_e over active elements and periodic node identification (Sec. 4.6
"Matrix-Free EBE Formulation"), f = sum_e A_e^T K_e x0 (App. F.1 f_e = int B^T C0 eps).
Sign reading: the weak form of App. F.1 puts a minus on the right-hand side; solving
K u = +f gives u = -chi, so the total field is x0 - u, which is what the C^H formula of
App. F.1 uses. Both readings give the same C^H.

C^H (App. F.1, reading of the index-free formula):
    C^H_IJ = 1/|Omega| sum_e s_e (x0^I - u_e^I)^T K_e (x0^J - u_e^J),  |Omega| = N^3.
kappa^H (App. F.2) is the same expression with the thermal matrices.
Relative residual (Sec. 5 metrics): r = ||f - K u||_2 / ||f||_2 per load case.
Gauge (Sec. 3.1, Sec. 4.5): the zero-mean constraint, applied as a hard projection
(subtract the mean over active nodes per component and load case).
Sensitivities (App. F.3): the per-element energies above, scaled by p / |Omega|.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fe
from .grid import Level


def element_dofs(level: Level, D: int) -> np.ndarray:
    en = level.element_nodes()
    if D == 1:
        return en
    return (en[:, :, None] * D + np.arange(D)[None, None, :]).reshape(en.shape[0], 8 * D)


def assemble(level: Level, Ke: np.ndarray, D: int, coef: np.ndarray | None = None):
    """Global K (CSR, ndof x ndof) = sum_e s_e A_e^T K_e A_e."""
    dofs = element_dofs(level, D)
    ne, m = dofs.shape
    s = np.ones(ne) if coef is None else coef.reshape(-1)[level.elem_lin]
    rows = np.repeat(dofs, m, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, m)).reshape(-1)
    vals = (s[:, None] * Ke.reshape(1, -1)).reshape(-1)
    ndof = level.num_nodes * D
    return sp.csr_matrix(sp.coo_matrix((vals, (rows, cols)), shape=(ndof, ndof)))


def load(level: Level, Ke: np.ndarray, x0: np.ndarray, D: int, coef=None) -> np.ndarray:
    """f = sum_e s_e A_e^T (K_e x0), shape (ndof, cases)."""
    dofs = element_dofs(level, D)
    s = np.ones(dofs.shape[0]) if coef is None else coef.reshape(-1)[level.elem_lin]
    fe_ = Ke @ x0
    F = np.zeros((level.num_nodes * D, x0.shape[1]))
    np.add.at(F, dofs.reshape(-1), (s[:, None, None] * fe_[None, :, :]).reshape(-1, x0.shape[1]))
    return F


def gross_load_norm(level: Level, Ke: np.ndarray, x0: np.ndarray, D: int, coef=None):
    """sqrt(sum_e ||s_e K_e x0||^2) per case: the load's size before nodal cancellation."""
    s = np.ones(level.num_elements) if coef is None else coef.reshape(-1)[level.elem_lin]
    fe_ = Ke @ x0
    return np.sqrt(np.sum(s ** 2) * np.sum(fe_ ** 2, axis=0))


def cancel_rounding(F: np.ndarray, gross: np.ndarray, rel: float = 1e-12) -> np.ndarray:
    """A load case whose assembled norm is at most rel * its gross norm is exactly zero in
    exact arithmetic (e.g. a uniform cell); set it to zero so that the relative residual
    is not taken against rounding noise."""
    F = F.copy()
    F[:, np.linalg.norm(F, axis=0) <= rel * gross] = 0.0
    return F


def gauge(U: np.ndarray, D: int) -> np.ndarray:
    """Subtract the mean over active nodes, per component and load case."""
    n = U.shape[0] // D
    V = U.reshape(n, D, -1)
    return (V - V.mean(axis=0, keepdims=True)).reshape(U.shape)


def cg(K, F: np.ndarray, tol: float = 1e-12, maxiter: int = 200000):
    """Jacobi-preconditioned conjugate gradients from u = 0, independently per column,
    until ||f - K u|| <= tol ||f||. Returns (U, iterations per column)."""
    F = np.asarray(F, dtype=np.float64)
    U = np.zeros_like(F)
    dinv = 1.0 / K.diagonal()
    R = F.copy()
    fn = np.linalg.norm(F, axis=0)
    done = fn == 0.0
    Z = dinv[:, None] * R
    P = Z.copy()
    rz = np.einsum("ij,ij->j", R, Z)
    iters = np.zeros(F.shape[1], dtype=np.int64)
    for it in range(maxiter):
        rn = np.linalg.norm(R, axis=0)
        done |= rn <= tol * np.where(fn > 0, fn, 1.0)
        if done.all():
            break
        KP = K @ P
        pkp = np.einsum("ij,ij->j", P, KP)
        alpha = np.where(done, 0.0, rz / np.where(pkp != 0, pkp, 1.0))
        U += alpha * P
        R -= alpha * KP
        Z = dinv[:, None] * R
        rz_new = np.einsum("ij,ij->j", R, Z)
        beta = np.where(done, 0.0, rz_new / np.where(rz != 0, rz, 1.0))
        P = Z + beta * P
        rz = rz_new
        iters += ~done
    return U, iters


def apply_ebe(level: Level, Ke: np.ndarray, U: np.ndarray, D: int, chunk: int = 65536):
    """K U = sum_e A_e^T K_e A_e U (Sec. 4.6 EBE form) without assembling K, in element
    chunks; for cells too large for an assembled matrix."""
    en = level.element_nodes()
    out = np.zeros_like(U)
    for s in range(0, en.shape[0], chunk):
        nodes = en[s:s + chunk]
        dofs = nodes if D == 1 else (nodes[:, :, None] * D + np.arange(D)).reshape(nodes.shape[0], -1)
        Y = np.einsum("rc,ecm->erm", Ke, U[dofs])
        np.add.at(out, dofs.reshape(-1), Y.reshape(-1, U.shape[1]))
    return out


def homogenize_chunked(level: Level, U, Ke, x0, D, chunk: int = 65536) -> np.ndarray:
    """homogenize() evaluated in element chunks (same definition, bounded memory)."""
    en = level.element_nodes()
    C = np.zeros((x0.shape[1], x0.shape[1]))
    for s in range(0, en.shape[0], chunk):
        nodes = en[s:s + chunk]
        dofs = nodes if D == 1 else (nodes[:, :, None] * D + np.arange(D)).reshape(nodes.shape[0], -1)
        W = x0[None, :, :] - U[dofs]
        C += np.einsum("eri,erj->ij", W, np.einsum("rc,ecm->erm", Ke, W))
    return C / float(level.n ** 3)


def relative_residual(K, F: np.ndarray, U: np.ndarray) -> np.ndarray:
    """r_m = ||f_m - K u_m|| / ||f_m|| per load case (0 where f_m = 0 and u_m solves)."""
    R = F - K @ U
    fn = np.linalg.norm(F, axis=0)
    rn = np.linalg.norm(R, axis=0)
    return np.where(fn > 0, rn / np.where(fn > 0, fn, 1.0), rn)


def homogenize(level: Level, U: np.ndarray, Ke: np.ndarray, x0: np.ndarray, D: int,
               coef=None) -> np.ndarray:
    """C^H_IJ = 1/N^3 sum_e s_e (x0^I - u_e^I)^T K_e (x0^J - u_e^J) (App. F.1 / F.2)."""
    dofs = element_dofs(level, D)
    s = np.ones(dofs.shape[0]) if coef is None else coef.reshape(-1)[level.elem_lin]
    W = x0[None, :, :] - U[dofs]                      # (ne, 8D, cases)
    KW = np.einsum("rc,ecm->erm", Ke, W)
    C = np.einsum("e,eri,erj->ij", s, W, KW)
    return C / float(level.n ** 3)


def homogenize_mixed(level: Level, U, Ke, x0, D, coef=None) -> np.ndarray:
    """Mixed form 1/N^3 sum_e s_e (x0^I)^T K_e (x0^J - u_e^J); equals C^H at convergence."""
    dofs = element_dofs(level, D)
    s = np.ones(dofs.shape[0]) if coef is None else coef.reshape(-1)[level.elem_lin]
    W = x0[None, :, :] - U[dofs]
    KW = np.einsum("rc,ecm->erm", Ke, W)
    return np.einsum("e,ri,erj->ij", s, x0, KW) / float(level.n ** 3)


def element_energies(level: Level, U, Ke, x0, D, coef=None) -> np.ndarray:
    """Per-element contributions (ne, cases, cases) to N^3 C^H, in canonical element order."""
    dofs = element_dofs(level, D)
    s = np.ones(dofs.shape[0]) if coef is None else coef.reshape(-1)[level.elem_lin]
    W = x0[None, :, :] - U[dofs]
    KW = np.einsum("rc,ecm->erm", Ke, W)
    return np.einsum("e,eri,erj->eij", s, W, KW)


def simp_coef(level: Level, rho: np.ndarray, rho_min: float, p: float) -> np.ndarray:
    """Dense N^3 element coefficients s_e = rho_min + rho_e^p of the SIMP interpolation
    C_e = (rho_min + rho_e^p) C0 (App. F.3), for densities rho given per active element in
    canonical element order; inactive voxels get 0 (they are not part of the mesh)."""
    N = level.active.shape[0]
    coef = np.zeros(N ** 3)
    coef[level.elem_lin] = rho_min + np.asarray(rho, dtype=np.float64) ** p
    return coef.reshape(level.active.shape)


def sensitivities(level: Level, U, Ke, x0, D, p: float, rho=None) -> np.ndarray:
    """Inverse-homogenization sensitivities (App. F.3) of the SIMP model
    C_e = (rho_min + rho_e^p) C0, per active element:
        dC^H_IJ / d rho_e = p rho_e^(p-1) / |Omega| (x0^I - u_e^I)^T K0 (x0^J - u_e^J),
    u the solution for the current densities; rho None means the binary design (rho_e = 1).
    Shape (ne, cases, cases), canonical element order, |Omega| = N^3."""
    N = level.active.shape[0]
    fac = np.full(level.num_elements, float(p)) if rho is None else \
        p * np.asarray(rho, dtype=np.float64) ** (p - 1.0)
    return fac[:, None, None] / float(N) ** 3 * element_energies(level, U, Ke, x0, D)


def solve_cell(vox: np.ndarray, kind: str = "elastic", E: float = 1.0, nu: float = 0.3,
               k: float = 1.0, tol: float = 1e-12, coef=None):
    """Full oracle solve of one cell: returns dict with U (gauged), C^H, residuals."""
    Ke, x0, D, NC, C0 = fe.physics(kind, E, nu, k)
    lev = Level(vox.astype(bool))
    K = assemble(lev, Ke, D, coef)
    F = cancel_rounding(load(lev, Ke, x0, D, coef), gross_load_norm(lev, Ke, x0, D, coef))
    U, iters = cg(K, F, tol=tol)
    U = gauge(U, D)
    C = homogenize(lev, U, Ke, x0, D, coef)
    return {"U": U, "CH": C, "res": relative_residual(K, F, U), "iters": iters,
            "K": K, "F": F, "level": lev, "Ke": Ke, "x0": x0, "D": D, "NC": NC, "C0": C0}


def brute_force(vox: np.ndarray, kind: str = "elastic", E=1.0, nu=0.3, k=1.0, coef=None):
    """Dense pseudo-inverse solve (symmetric eigendecomposition, cut-off 1e-10 lambda_max)
    for tiny cells; returns (U gauged, C^H)."""
    Ke, x0, D, NC, C0 = fe.physics(kind, E, nu, k)
    lev = Level(vox.astype(bool))
    K = assemble(lev, Ke, D, coef).toarray()
    F = cancel_rounding(load(lev, Ke, x0, D, coef), gross_load_norm(lev, Ke, x0, D, coef))
    w, V = np.linalg.eigh(K)
    keep = w > 1e-10 * w.max()
    U = V[:, keep] @ ((V[:, keep].T @ F) / w[keep, None])
    U = gauge(U, D)
    return U, homogenize(lev, U, Ke, x0, D, coef)


def energy_norm_error(K, U_test: np.ndarray, U_ref: np.ndarray, Ke, x0, level, D) -> np.ndarray:
    """Per case ||u_test - u_ref||_K / ||x0 - u_ref||_K (K-seminorm, blind to null modes)."""
    E = U_test - U_ref
    num = np.sqrt(np.maximum(np.einsum("ij,ij->j", E, K @ E), 0.0))
    C = homogenize(level, U_ref, Ke, x0, D) * float(level.n ** 3)
    den = np.sqrt(np.maximum(np.diag(C), 1e-300))
    return num / den
