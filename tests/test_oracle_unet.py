"""Pins of the initializer network's oracle (oracle/unet.py) against what fixes it
independently: dense periodic convolutions (torch conv3d) on full grids, the adjoint
relation between the up and down convolutions, the symmetry of the neighbour tables,
central finite differences of the loss, and the closed form of AdamW's first step."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet
from paper_2604_26518_b300 import lattices


def _full_xyz(n):
    lin = np.arange(n ** 3)
    return np.stack([lin % n, (lin // n) % n, lin // (n * n)], axis=1)


def _dense_weight(W):
    """[27][cin][cout] -> conv3d weight [cout][cin][kz][ky][kx] with t = kz*9 + ky*3 + kx."""
    return W.permute(2, 1, 0).reshape(W.shape[2], W.shape[1], 3, 3, 3)


def _grid_tensor(x, n):
    """(n^3, c) in canonical order (x fastest) -> [1][c][z][y][x]."""
    return x.T.reshape(1, x.shape[1], n, n, n)


def test_same_level_conv_on_full_grid_is_periodic_conv3d():
    n, ci, co = 6, 3, 4
    g = torch.Generator().manual_seed(1)
    x = torch.randn(n ** 3, ci, generator=g, dtype=torch.float64)
    W = torch.randn(27, ci, co, generator=g, dtype=torch.float64)
    b = torch.randn(co, generator=g, dtype=torch.float64)
    z = unet.conv(x, unet.same_table(n, _full_xyz(n)), W, b)
    ref = F.conv3d(F.pad(_grid_tensor(x, n), (1, 1, 1, 1, 1, 1), mode="circular"),
                   _dense_weight(W), b)
    assert torch.allclose(_grid_tensor(z, n), ref, rtol=1e-12, atol=1e-12)


def test_down_conv_on_full_grid_is_strided_periodic_conv3d():
    nf, ci, co = 8, 2, 3
    g = torch.Generator().manual_seed(2)
    x = torch.randn(nf ** 3, ci, generator=g, dtype=torch.float64)
    W = torch.randn(27, ci, co, generator=g, dtype=torch.float64)
    z = unet.conv(x, unet.down_table(nf, _full_xyz(nf), _full_xyz(nf // 2)), W, None)
    ref = F.conv3d(F.pad(_grid_tensor(x, nf), (1, 1, 1, 1, 1, 1), mode="circular"),
                   _dense_weight(W), stride=2)
    assert torch.allclose(_grid_tensor(z, nf // 2), ref, rtol=1e-12, atol=1e-12)


@pytest.fixture(scope="module")
def graph():
    return unet.Graph(lattices.tpms_network("gyroid", 32, 0.25))


def test_up_conv_is_adjoint_of_down_conv(graph):
    g = torch.Generator().manual_seed(3)
    for l in range(2):
        ci, co = 3, 5
        W = torch.randn(27, ci, co, generator=g, dtype=torch.float64)
        y = torch.randn(graph.n[l + 1], ci, generator=g, dtype=torch.float64)
        x = torch.randn(graph.n[l], co, generator=g, dtype=torch.float64)
        up = unet.conv(y, graph.up[l], W, None)                          # coarse -> fine
        down = unet.conv(x, graph.down[l], W.transpose(1, 2), None)      # fine -> coarse
        assert abs(float((up * x).sum() - (y * down).sum())) <= 1e-10 * float(
            (up * x).abs().sum())


def test_tables_are_mutually_consistent(graph):
    for l in range(3):
        tab = graph.same[l]
        n, t = np.nonzero(tab >= 0)
        assert (graph.same[l][tab[n, t], 26 - t] == n).all()
        assert (tab[:, 13] == np.arange(tab.shape[0])).all()       # centre tap
    for l in range(2):
        q, t = np.nonzero(graph.down[l] >= 0)
        assert (graph.up[l][graph.down[l][q, t], t] == q).all()
        f, t = np.nonzero(graph.up[l] >= 0)
        assert (graph.down[l][graph.up[l][f, t], t] == f).all()
        # every active fine node has at least one coarse parent (conservative coarsening)
        assert ((graph.up[l] >= 0).sum(axis=1) >= 1).all()
        # a fine node of parity class c (odd axes = set bits of c) can only have parents
        # under the 2^popcount(c) taps that are 0 on its even axes and +-1 on its odd ones
        xyz = graph.levels[l].node_xyz()
        cls = (xyz[:, 0] & 1) + 2 * (xyz[:, 1] & 1) + 4 * (xyz[:, 2] & 1)
        for c in range(8):
            taps = np.nonzero((graph.up[l][cls == c] >= 0).any(axis=0))[0]
            allowed = [t for t, d in enumerate(unet.TAPS)
                       if all((d[a] != 0) == bool((c >> a) & 1) for a in range(3))]
            assert set(taps) <= set(allowed) and len(allowed) == 2 ** bin(c).count("1")


def test_input_features_are_octant_bits(graph):
    m = graph.levels[0].node_mask_list().astype(int)
    bits = graph.x0.numpy().astype(int)
    assert (bits @ (1 << np.arange(8)) == m).all()


def test_gradient_matches_central_differences(graph):
    rows = unet.layers(3, widths=(2, 3, 4))
    p = lattices.unet_init(rows, seed=5).astype(np.float64)
    p[np.random.default_rng(0).random(p.size) < 0.3] += 0.05        # non-zero biases too
    rng = np.random.default_rng(1)
    u = rng.normal(size=(graph.n[0], 3))
    loss, grad = unet.loss_and_grad(graph, p, rows, u, scale=2.0)
    assert loss > 0
    offs = np.cumsum([0] + [27 * r[4] * r[5] + r[5] for r in rows])
    picks = [int(offs[i] + rng.integers(0, offs[i + 1] - offs[i])) for i in range(len(rows))]
    picks += [int(offs[i + 1] - 1) for i in range(len(rows))]           # a bias of each layer
    h = 1e-6
    for k in picks:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (unet.loss_and_grad(graph, pp, rows, u, 2.0)[0] -
              unet.loss_and_grad(graph, pm, rows, u, 2.0)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1e-3, abs(grad).max()), (k, fd, grad[k])


def test_adamw_first_step_closed_form():
    # after one step the bias-corrected moments are g and g^2, so each parameter moves by
    # lr * (g / (|g| + eps) + wd * p)
    rng = np.random.default_rng(2)
    p, g = rng.normal(size=100), rng.normal(size=100)
    lr, wd, eps = 1e-3, 0.01, 1e-8
    q, m, v = unet.adamw_step(p, g, np.zeros(100), np.zeros(100), 1, lr, 0.9, 0.999, eps, wd)
    assert np.allclose(q, p - lr * (g / (np.abs(g) + eps) + wd * p), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps the step at lr * sign(g) (without decay) at every step
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    gc = np.array([1.0, -2.0, 0.5, 3.0])
    for s in range(1, 6):
        p1, m, v = unet.adamw_step(p, gc, m, v, s, lr, 0.9, 0.999, 0.0, 0.0)
        assert np.allclose(p1 - p, -lr * np.sign(gc), rtol=1e-12, atol=0)
        p = p1


def test_library_layer_table_matches_oracle():
    from paper_2604_26518_b300 import gmt
    for cout in (18, 3):
        assert [tuple(r) for r in gmt.unet_layers(cout)] == unet.layers(cout)
        assert gmt.unet_param_count(cout) == unet.param_count(unet.layers(cout))
    assert 1.5e6 < gmt.unet_param_count(18) < 2.5e6


def test_energy_loss_gradient_matches_central_differences(graph):
    from oracle import fe
    from oracle import solve as osolve
    Ke, _, D, _, _ = fe.physics("heat", 1.0, 0.3, 1.0)
    K = osolve.assemble(graph.levels[0], Ke, D)
    rows = unet.layers(3, widths=(2, 3, 4))
    p = lattices.unet_init(rows, seed=6).astype(np.float64)
    rng = np.random.default_rng(3)
    u = rng.normal(size=(graph.n[0], 3))
    loss, grad = unet.loss_and_grad(graph, p, rows, u, 1.5, K=K)
    # a zero network output leaves e = -u: the loss is exactly 1
    z = np.zeros_like(p)
    assert abs(unet.loss_and_grad(graph, z, rows, u, 1.5, K=K)[0] - 1.0) < 1e-12
    offs = np.cumsum([0] + [27 * r[4] * r[5] + r[5] for r in rows])
    picks = [int(offs[i] + rng.integers(0, offs[i + 1] - offs[i])) for i in range(len(rows))]
    h = 1e-6
    for k in picks:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (unet.loss_and_grad(graph, pp, rows, u, 1.5, K=K)[0] -
              unet.loss_and_grad(graph, pm, rows, u, 1.5, K=K)[0]) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1e-3, abs(grad).max()), (k, fd, grad[k])
