"""Shared test helpers: oracle hierarchies for a cell and GPU<->oracle field conversion."""
import numpy as np

from oracle import fe, galerkin, grid, solve


def oracle_setup(vox, kind, levels):
    lv = grid.hierarchy(vox, levels)
    Ke, x0, D, M, C0 = fe.physics(kind)
    K1 = solve.assemble(lv[0], Ke, D)
    F = solve.cancel_rounding(solve.load(lv[0], Ke, x0, D), solve.gross_load_norm(lv[0], Ke, x0, D))
    Ks, Ps = galerkin.galerkin_hierarchy(lv, K1, D)
    return dict(levels=lv, Ke=Ke, x0=x0, D=D, M=M, K=K1, F=F, Ks=Ks, Ps=Ps)


def to_np(t, D, M):
    return t.detach().cpu().numpy().reshape(-1, M)


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
