"""Sparse periodic GMG hierarchy — oracle, test infrastructure.

Follows Sec. 4.1 ("Domain Discretization", "Solver-Aligned Hierarchy Construction") and
App. E.1/E.2 of the paper:
  * level-1 active elements are the solid voxels;
  * each node carries an 8-bit octant mask: bit o (o = o_x + 2 o_y + 4 o_z) is set when the
    voxel (p - o) mod N is active, i.e. the element that has node p as its local vertex o;
  * active nodes are the vertex union of the active elements (eq. gmgcoarsenode);
  * a coarse element is active when any of its 8 children is active;
  * transfer stencil of an active fine node x_f: coarse neighbours (floor(x_f/2) + o_k) mod
    N_c with trilinear weights prod_d (1 - |xi_d - o_{k,d}|), xi = (x_f mod 2)/2.

Canonical node order at every level: increasing linear index x + N y + N^2 z.
Voxel arrays are indexed [z, y, x].
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(o & 1, (o >> 1) & 1, (o >> 2) & 1) for o in range(8)]


def choose_levels(n: int, coarsest_max: int = 8) -> int:
    """Level count: the smallest L whose coarsest grid is at most `coarsest_max` per side,
    keeping every non-coarsest level divisible by 4 (N % 2^L == 0 for L >= 2).
    The paper uses L=5 for 64^3-256^3 and L=6 at 512^3 (App. A); this reading picks L from N
    so the coarsest direct solve stays small."""
    if n % 4 != 0 or n <= 0:
        raise ValueError("resolution must be a positive multiple of 4")
    L = 1
    while (n >> (L - 1)) > coarsest_max and n % (1 << (L + 1)) == 0:
        L += 1
    return L


def node_masks(active: np.ndarray) -> np.ndarray:
    """8-bit octant mask of every node site of a periodic grid of element flags."""
    act = active.astype(bool)
    mask = np.zeros(act.shape, dtype=np.uint8)
    for o, (ox, oy, oz) in enumerate(OFFSETS):
        # rolled[p] = act[p - o]
        rolled = np.roll(act, shift=(oz, oy, ox), axis=(0, 1, 2))
        mask |= (rolled.astype(np.uint8) << o)
    return mask


def coarsen(active: np.ndarray) -> np.ndarray:
    """Coarse element active iff any of its 8 children is active."""
    n = active.shape[0] // 2
    return active.reshape(n, 2, n, 2, n, 2).astype(bool).any(axis=(1, 3, 5))


class Level:
    """One level: element flags, node masks, canonical node list and rank map."""

    def __init__(self, active: np.ndarray):
        self.n = active.shape[0]
        self.active = active.astype(bool)
        self.mask = node_masks(self.active)
        flat = self.mask.reshape(-1)
        self.node_lin = np.nonzero(flat)[0]                      # canonical order
        self.rank = np.full(flat.size, -1, dtype=np.int64)
        self.rank[self.node_lin] = np.arange(self.node_lin.size)
        self.elem_lin = np.nonzero(self.active.reshape(-1))[0]

    @property
    def num_nodes(self) -> int:
        return int(self.node_lin.size)

    @property
    def num_elements(self) -> int:
        return int(self.elem_lin.size)

    def node_xyz(self) -> np.ndarray:
        n = self.n
        lin = self.node_lin
        return np.stack([lin % n, (lin // n) % n, lin // (n * n)], axis=1).astype(np.int64)

    def elem_xyz(self) -> np.ndarray:
        n = self.n
        lin = self.elem_lin
        return np.stack([lin % n, (lin // n) % n, lin // (n * n)], axis=1).astype(np.int64)

    def node_mask_list(self) -> np.ndarray:
        return self.mask.reshape(-1)[self.node_lin]

    def element_nodes(self) -> np.ndarray:
        """(num_elements, 8) canonical node ranks of each active element's vertices."""
        n = self.n
        xyz = self.elem_xyz()
        out = np.empty((xyz.shape[0], 8), dtype=np.int64)
        for a, (ax, ay, az) in enumerate(OFFSETS):
            x = (xyz[:, 0] + ax) % n
            y = (xyz[:, 1] + ay) % n
            z = (xyz[:, 2] + az) % n
            out[:, a] = self.rank[x + n * y + n * n * z]
        assert (out >= 0).all()
        return out


def hierarchy(vox: np.ndarray, levels: int | None = None):
    """List of Level objects, finest first."""
    n = vox.shape[0]
    L = choose_levels(n) if levels is None else int(levels)
    if n % (1 << (L - 1)) != 0:
        raise ValueError("resolution not divisible by 2^(L-1)")
    out = [Level(vox.astype(bool))]
    for _ in range(1, L):
        out.append(Level(coarsen(out[-1].active)))
    return out


def transfer_stencil(fine: Level, coarse: Level):
    """App. E.2 stencil tuples: for every active fine node (canonical order) the 8 coarse
    neighbour ranks and weights. Zero-weight slots hold index -1 and weight 0."""
    nf, nc = fine.n, coarse.n
    xyz = fine.node_xyz()
    idx = np.full((xyz.shape[0], 8), -1, dtype=np.int64)
    wts = np.zeros((xyz.shape[0], 8))
    base = xyz // 2
    xi = (xyz % 2) / 2.0
    for k, o in enumerate(OFFSETS):
        w = np.ones(xyz.shape[0])
        for d in range(3):
            w *= 1.0 - np.abs(xi[:, d] - o[d])
        cx = (base[:, 0] + o[0]) % nc
        cy = (base[:, 1] + o[1]) % nc
        cz = (base[:, 2] + o[2]) % nc
        r = coarse.rank[cx + nc * cy + nc * nc * cz]
        nz = w != 0.0
        if (r[nz] < 0).any():
            raise AssertionError("nonzero transfer weight onto an inactive coarse node")
        idx[nz, k] = r[nz]
        wts[nz, k] = w[nz]
    return idx, wts
