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


def test_energy_loss_and_gradient_parity(cell):
    from oracle import fe
    from oracle import solve as osolve
    _, h, G, O = cell
    rows = ounet.layers(18)
    p = lattices.unet_init(rows, seed=21)
    net = gmt.UNet(18, torch.tensor(p))
    with pytest.raises(gmt.GmtError):            # the energy loss needs a prepared material
        gmt.Hierarchy(lattices.tpms_network("gyroid", 32, 0.25)) and net.gradient(
            G, torch.zeros(O.n[0], 18), 1.0, loss=gmt.LOSS_ENERGY, hier=None)
    h.prepare(gmt.ELASTIC, E=1.0, nu=0.3)
    Ke, _, D, _, _ = fe.physics("elastic", 1.0, 0.3)
    K = osolve.assemble(O.levels[0], Ke, D)
    u = np.random.default_rng(8).normal(size=(O.n[0], 18))
    scale = 0.7
    loss_g, grad_g = net.gradient(G, torch.tensor(u), scale, loss=gmt.LOSS_ENERGY, hier=h)
    loss_r, grad_r = ounet.loss_and_grad(O, p, rows, u, scale, K=K)
    # K applied in FP32 on the device: relative 1e-5 on the loss
    assert abs(loss_g - loss_r) <= 1e-5 * loss_r, (loss_g, loss_r)
    grad_g = grad_g.cpu().numpy().astype(np.float64)
    for i, (a, b) in enumerate(_segments(rows)):
        ref = np.abs(grad_r[a:b]).max()
        err = np.abs(grad_g[a:b] - grad_r[a:b]).max()
        assert err <= 1e-3 * ref, (i, err, ref)


def test_training_lowers_energy_error_and_warm_start_keeps_accuracy():
    """Train on 16 seeded 32^3 cells (energy loss, AdamW), then on held-out cells: the
    prediction's energy-norm error is below the zero start's (which is 1 by definition), the
    solve from it reaches the tolerance, and C^H equals the zero-start result; the V-cycle
    counts of both starts are printed (the plain cycles are the fallback and decide convergence)."""
    fams = ("gyroid", "schwarz_p", "diamond", "plate_gyroid", "bcc", "octet")
    rows = ounet.layers(18)
    net = gmt.UNet(18, torch.tensor(lattices.unet_init(rows, seed=0)))
    scale = 0.04 * 32
    data = []
    for i in range(16):
        h = gmt.Hierarchy(lattices.mixed_cell(500 + i, 32, families=fams)[0])
        _, u, _ = h.solve(gmt.ELASTIC, tol=1e-6)
        data.append((h, gmt.NetGraph(h), u.reshape(h.num_nodes(0), 18).contiguous()))
    epochs = 12
    losses = []
    for ep in range(epochs):
        for i in np.random.default_rng(ep).permutation(len(data)):
            h, g, u = data[i]
            lr = 1e-3 * 0.5 * (1 + np.cos(np.pi * len(losses) / (epochs * len(data))))
            losses.append(net.train_step(g, u, scale, lr=lr, loss=gmt.LOSS_ENERGY, hier=h))
    first, last = np.mean(losses[:16]), np.mean(losses[-16:])
    assert last < 0.5 * first, (first, last)
    for i in range(3):
        h = gmt.Hierarchy(lattices.mixed_cell(900 + i, 32, families=fams)[0])
        st0, u_ref, i0 = h.solve(gmt.ELASTIC, tol=1e-6)
        CH0 = h.homogenize(gmt.ELASTIC)
        g = gmt.NetGraph(h)
        pred = net.forward(g, scale)
        err, _ = net.gradient(g, u_ref.reshape(-1, 18), scale, loss=gmt.LOSS_ENERGY, hier=h)
        assert err < 0.9, err
        st1, _, i1 = h.solve(gmt.ELASTIC, tol=1e-5, u0=pred)
        assert st1 == gmt.OK and max(i1.rel_residual[:6]) <= 1e-5
        CH1 = h.homogenize(gmt.ELASTIC)
        assert np.abs(CH1 - CH0).max() <= 1e-4 * np.abs(CH0).max()
        _, _, iz = h.solve(gmt.ELASTIC, tol=1e-5)
        print(f"held-out cell {i}: energy error of the prediction {err:.3f}, "
              f"V-cycles from zero {iz.inner_total}, from the prediction {i1.inner_total}")


@pytest.mark.parametrize("cout", [18, 3])
def test_tensor_core_forward_parity(cell, cout):
    """gmt_unet_set_tensor_cores: every layer as a tcgen05 implicit-GEMM gather convolution
    (FP16 operands, FP32 accumulation in tensor memory). The prediction matches the float64
    oracle within FP16 operand rounding through twelve layers; switching back gives the FP32
    forward bit for bit, and the gradient (training) stays the FP32 one."""
    _, _, G, O = cell
    rows = ounet.layers(cout)
    p = lattices.unet_init(rows, seed=21 + cout)
    p[_segments(rows)[3][1] - 64:_segments(rows)[3][1]] = 0.1
    net = gmt.UNet(cout, torch.tensor(p))
    scale = 1.3
    y32 = net.forward(G, scale).cpu().numpy()
    u = torch.tensor(np.random.default_rng(5).normal(size=(O.n[0], cout)) * scale)
    loss32, grad32 = net.gradient(G, u, scale)
    net.tensor_cores(True)
    ytc = net.forward(G, scale).cpu().numpy()
    y_ref = scale * ounet.forward(O, torch.tensor(p.astype(np.float64)), rows).numpy()
    err = np.abs(ytc - y_ref).max()
    # FP16 rounding of every operand (unit roundoff 4.9e-4) through twelve layers
    assert err <= 1e-2 * np.abs(y_ref).max(), (err, np.abs(y_ref).max())
    assert not np.array_equal(ytc, y32)           # the tensor-core path did run
    loss_tc, grad_tc = net.gradient(G, u, scale)  # training stays FP32
    assert loss_tc == loss32 and torch.equal(grad_tc, grad32)
    net.tensor_cores(False)
    assert np.array_equal(net.forward(G, scale).cpu().numpy(), y32)
