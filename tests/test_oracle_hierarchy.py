"""Pins for the oracle's sparse hierarchy (Sec. 4.1), transfers (App. E) and Galerkin
coarse operators (Sec. 3.2, Sec. 4.6)."""
import itertools

import numpy as np
import pytest

from oracle import fe, galerkin, grid, solve
from paper_2604_26518_b300 import lattices as L


def test_level_count_rule():
    table = {4: 1, 8: 1, 12: 2, 16: 2, 20: 2, 32: 3, 48: 4, 64: 4, 96: 5, 128: 5,
             256: 6, 512: 7}
    for n, levels in table.items():
        assert grid.choose_levels(n) == levels, n
    with pytest.raises(ValueError):
        grid.choose_levels(30)


@pytest.mark.parametrize("seed", [0, 1])
def test_masks_and_coarsening_brute_force(seed):
    n = 8
    vox = L.random_binary(n, 0.3, np.random.default_rng(seed))
    mask = grid.node_masks(vox)
    for z, y, x in itertools.product(range(n), repeat=3):
        m = 0
        for o in range(8):
            ox, oy, oz = o & 1, (o >> 1) & 1, (o >> 2) & 1
            if vox[(z - oz) % n, (y - oy) % n, (x - ox) % n]:
                m |= 1 << o
        assert mask[z, y, x] == m
    c = grid.coarsen(vox)
    for Z, Y, X in itertools.product(range(n // 2), repeat=3):
        assert c[Z, Y, X] == vox[2 * Z:2 * Z + 2, 2 * Y:2 * Y + 2, 2 * X:2 * X + 2].any()
    lev = grid.Level(vox)
    # active nodes = vertex union of active elements
    verts = set()
    for (x, y, z) in lev.elem_xyz():
        for o in range(8):
            verts.add((x + (o & 1)) % n + n * ((y + ((o >> 1) & 1)) % n)
                      + n * n * ((z + ((o >> 2) & 1)) % n))
    assert sorted(verts) == lev.node_lin.tolist()


@pytest.mark.parametrize("n", [8, 16])
def test_transfer_stencil_properties(n):
    vox = L.tpms_network("diamond", n, 0.25)
    levels = grid.hierarchy(vox, levels=2)
    f, c = levels
    idx, w = grid.transfer_stencil(f, c)
    np.testing.assert_array_equal(w.sum(axis=1), 1.0)          # partition of unity
    assert set(np.unique(w)) <= {0.0, 0.125, 0.25, 0.5, 1.0}
    xyz = f.node_xyz()
    odd = (xyz % 2).sum(axis=1)
    np.testing.assert_array_equal((idx >= 0).sum(axis=1), 2 ** odd)
    # trilinear weights reproduce the fine coordinate from unwrapped coarse positions
    rec = np.zeros_like(xyz, dtype=float)
    for k, o in enumerate(grid.OFFSETS):
        rec += w[:, k:k + 1] * 2.0 * (xyz // 2 + np.array(o))
    np.testing.assert_array_equal(rec, xyz.astype(float))


def _local_galerkin(levels, Ke, D):
    """Element-local Galerkin (Sec. 4.6): each coarse element's matrix is
    sum over active children of P_loc^T K_child P_loc, then assembled."""
    n_l = len(levels)
    mats = {tuple(e): Ke for e in levels[0].elem_xyz()}
    out = []
    for l in range(1, n_l):
        fine, coarse = levels[l - 1], levels[l]
        new = {}
        for E in coarse.elem_xyz():
            Kc = np.zeros((8 * D, 8 * D))
            for c in range(8):
                child = tuple((2 * E + np.array(grid.OFFSETS[c])) % fine.n)
                if child not in mats:
                    continue
                P = np.zeros((8 * D, 8 * D))
                for a in range(8):               # child's local vertex a
                    pos = np.array(grid.OFFSETS[c]) + np.array(grid.OFFSETS[a])   # in [0,2]^3
                    for b in range(8):           # coarse local vertex b
                        wt = np.prod(1.0 - np.abs(pos / 2.0 - np.array(grid.OFFSETS[b])))
                        for i in range(D):
                            P[a * D + i, b * D + i] = wt
                Kc += P.T @ mats[child] @ P
            new[tuple(E)] = Kc
        mats = new
        ne = coarse.num_elements
        Kg = np.zeros((coarse.num_nodes * D,) * 2)
        en = coarse.element_nodes()
        for e, E in enumerate(coarse.elem_xyz()):
            dofs = (en[e][:, None] * D + np.arange(D)[None, :]).reshape(-1)
            Kg[np.ix_(dofs, dofs)] += new[tuple(E)]
        out.append(Kg)
    return out


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_galerkin_global_equals_element_local(kind):
    vox = L.tpms_network("gyroid", 8, 0.35)
    levels = grid.hierarchy(vox, levels=3)
    Ke, x0, D, NC, _ = fe.physics(kind)
    K1 = solve.assemble(levels[0], Ke, D)
    Ks, Ps = galerkin.galerkin_hierarchy(levels, K1, D)
    local = _local_galerkin(levels, Ke, D)
    for l in range(1, 3):
        G = Ks[l].toarray()
        np.testing.assert_allclose(G, local[l - 1], atol=1e-12 * np.abs(G).max())
        np.testing.assert_allclose(G, G.T, atol=1e-13 * np.abs(G).max())
        for d in range(D):
            t = np.zeros(G.shape[0])
            t[d::D] = 1.0
            assert np.abs(G @ t).max() < 1e-12 * np.abs(G).max()
