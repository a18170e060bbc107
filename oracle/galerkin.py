"""Global prolongation and Galerkin coarse operators — oracle, test infrastructure.

Sec. 3.2 ("Operator Consistency"): K^(l+1) = R K^(l) P with R = P^T. The prolongation is
the matrix of App. E.2's weighted gather u_f(i) = sum_k W_ik u_c(I_ik), expanded over the D
components of each node (P (x) I_D). The coarse operators are formed globally here, as a
sparse triple product, so that the library's element-local construction (Sec. 4.6,
K_c = R_loc K_patch P_loc) can be checked against the global definition.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import Level, transfer_stencil


def prolongation(fine: Level, coarse: Level, D: int):
    idx, w = transfer_stencil(fine, coarse)
    nf, nc = fine.num_nodes, coarse.num_nodes
    rows, cols, vals = [], [], []
    for k in range(8):
        nz = idx[:, k] >= 0
        r = np.nonzero(nz)[0]
        for c in range(D):
            rows.append(r * D + c)
            cols.append(idx[nz, k] * D + c)
            vals.append(w[nz, k])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix(sp.coo_matrix((vals, (rows, cols)), shape=(nf * D, nc * D)))


def galerkin_hierarchy(levels, K1, D: int):
    """[K_1, K_2, ..., K_L] with K_{l+1} = P_l^T K_l P_l, and the list of P_l."""
    Ks, Ps = [K1], []
    for l in range(len(levels) - 1):
        P = prolongation(levels[l], levels[l + 1], D)
        Ps.append(P)
        Ks.append(sp.csr_matrix(P.T @ Ks[-1] @ P))
    return Ks, Ps
