"""Parity of the learned initializer's CUDA path (gmt_netgraph_*, gmt_unet_*) with the
float64 oracle network (oracle/unet.py): neighbour tables bit-exact, forward output,
loss and every parameter's gradient within FP32 accumulation error, and the AdamW update."""
import numpy as np
import pytest
import torch

from oracle import unet as ounet
from paper_2604_26518_b300 import gmt, lattices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cell():
    vox = lattices.tpms_network("gyroid", 32, 0.25)
    h = gmt.Hierarchy(vox)
    return vox, h, gmt.NetGraph(h), ounet.Graph(vox)


def test_tables_bit_exact(cell):
    _, _, G, O = cell
    assert G.n == O.n
    for l in range(3):
        same, down, up = G.tables(l)
        assert np.array_equal(same.cpu().numpy(), O.same[l])
        if l < 2:
            assert np.array_equal(down.cpu().numpy(), O.down[l])
            assert np.array_equal(up.cpu().numpy(), O.up[l])


def test_netgraph_needs_three_levels():
    h = gmt.Hierarchy(lattices.tpms_network("gyroid", 16, 0.3))
    assert h.levels < 3
    with pytest.raises(gmt.GmtError):
        gmt.NetGraph(h)


def _segments(rows):
    offs = np.cumsum([0] + [27 * r[4] * r[5] + r[5] for r in rows])
    return [(int(offs[i]), int(offs[i + 1])) for i in range(len(rows))]


@pytest.mark.parametrize("cout", [18, 3])
def test_forward_loss_and_gradient_parity(cell, cout):
    _, _, G, O = cell
    rows = ounet.layers(cout)
    p = lattices.unet_init(rows, seed=11 + cout)
    p[_segments(rows)[3][1] - 64:_segments(rows)[3][1]] = 0.1   # non-zero biases in a layer
    net = gmt.UNet(cout, torch.tensor(p))
    scale = 1.7
    y_gpu = net.forward(G, scale).cpu().numpy()
    y_ref = scale * ounet.forward(O, torch.tensor(p.astype(np.float64)), rows).numpy()
    assert np.abs(y_gpu - y_ref).max() <= 1e-4 * np.abs(y_ref).max()
    u = np.random.default_rng(cout).normal(size=(O.n[0], cout)) * scale
    loss_g, grad_g = net.gradient(G, torch.tensor(u), scale)
    loss_r, grad_r = ounet.loss_and_grad(O, p, rows, u, scale)
    assert abs(loss_g - loss_r) <= 1e-5 * loss_r
    grad_g = grad_g.cpu().numpy().astype(np.float64)
    # FP32 sums of up to 27 * 128 terms per value through eleven layers, and relu masks
    # that may differ where a pre-activation lies within FP32 rounding of zero: 1e-3 of the
    # layer's largest gradient entry (measured: at most 4.1e-4)
    for i, (a, b) in enumerate(_segments(rows)):
        ref = np.abs(grad_r[a:b]).max()
        assert ref > 0, i
        err = np.abs(grad_g[a:b] - grad_r[a:b]).max()
        assert err <= 1e-3 * ref, (i, err, ref)
    # the parameters did not change
    assert np.array_equal(net.params().cpu().numpy(), p)


def test_adamw_step_parity(cell):
    _, _, G, O = cell
    rows = ounet.layers(18)
    p = lattices.unet_init(rows, seed=3)
    net = gmt.UNet(18, torch.tensor(p))
    u = torch.tensor(np.random.default_rng(4).normal(size=(O.n[0], 18)))
    m = np.zeros(p.size)
    v = np.zeros(p.size)
    q = p.astype(np.float64)
    hp = dict(lr=2e-3, beta1=0.9, beta2=0.99, eps=1e-8, weight_decay=0.05)
    for step in (1, 2):
        _, g = net.gradient(G, u, 1.0)                       # gradient at the current params
        loss = net.train_step(G, u.cuda(), 1.0, **hp)
        assert np.isfinite(loss)
        q, m, v = ounet.adamw_step(q, g.cpu().numpy().astype(np.float64), m, v, step,
                                   hp["lr"], hp["beta1"], hp["beta2"], hp["eps"],
                                   hp["weight_decay"])
        got = net.params().cpu().numpy().astype(np.float64)
        assert np.abs(got - q).max() <= 1e-6 * max(1.0, np.abs(q).max()), step
