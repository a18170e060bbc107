"""Learned-initializer network — oracle, test infrastructure (never on the product path).

The paper's method starts the V-cycles from a learned prediction of the fine-level field
(Sec. 4.2-4.3, Alg. 2). The network here is a sparse 3D convolutional U-Net over levels
0-2 of the node hierarchy of Sec. 4.1, written plainly in float64 PyTorch:

  * activations are [node][channel] over the canonical active nodes of a level;
  * every convolution has 27 taps d_t = (dx, dy, dz), t = (dz+1)*9 + (dy+1)*3 + (dx+1);
      same-level  z[n] = b + sum_t W[t]^T x[node at p_n + d_t]          (periodic wrap)
      down l->l+1 z[q] = b + sum_t W[t]^T x[fine node at 2 q + d_t]
      up l+1->l   z[p] = b + sum_t W[t]^T x[coarse node q with p = 2 q + d_t]
    where a neighbour that is not an active node contributes zero (down and up follow the
    parent/child relation of the trilinear transfer of App. E.2);
  * y = relu(z + skip), twelve layers (the list in `layers`);
  * input: the 8 octant-mask bits of each fine node; output: the field divided by `scale`;
  * losses: the mean over nodes and channels of (y - u / scale)^2, or the relative energy
    norm (e^T K e) / (u^T K u) of the error e = scale y - u summed over the load cases,
    with the assembled level-0 stiffness K (oracle/solve.py);
  * gradients by torch autograd; AdamW of Loshchilov and Hutter (decoupled weight decay,
    bias-corrected moments) written out in `adamw_step`.

Tables come from dense index maps of the oracle hierarchy (`grid.hierarchy`), not from the
library. Parameters: per layer W [27][cin][cout] then b [cout], layers in order.
"""
from __future__ import annotations

import numpy as np
import torch

from . import grid

TAPS = [(t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1) for t in range(27)]   # (dx, dy, dz)
SAME, DOWN, UP = 0, 1, 2
IN_CH = 8


def layers(cout: int, widths=(32, 64, 128)):
    """Rows (kind, output level, input activation, skip activation, cin, cout); activation
    0 is the input, activation i+1 the output of layer i; every layer but the last has relu."""
    w0, w1, w2 = widths
    return [(SAME, 0, 0, -1, IN_CH, w0), (SAME, 0, 1, -1, w0, w0),
            (DOWN, 1, 2, -1, w0, w1), (SAME, 1, 3, -1, w1, w1),
            (DOWN, 2, 4, -1, w1, w2), (SAME, 2, 5, -1, w2, w2), (SAME, 2, 6, -1, w2, w2),
            (UP, 1, 7, 4, w2, w1), (SAME, 1, 8, -1, w1, w1),
            (UP, 0, 9, 2, w1, w0), (SAME, 0, 10, -1, w0, w0), (SAME, 0, 11, -1, w0, cout)]


def param_count(rows) -> int:
    return sum(27 * r[4] * r[5] + r[5] for r in rows)


def split_params(p: torch.Tensor, rows):
    """Views (W [27][cin][cout], b [cout]) of a flat parameter vector."""
    out, off = [], 0
    for r in rows:
        nw = 27 * r[4] * r[5]
        out.append((p[off:off + nw].view(27, r[4], r[5]), p[off + nw:off + nw + r[5]]))
        off += nw + r[5]
    assert off == p.numel()
    return out


# ------------------------------------------------------------------ tables
def _index_map(n: int, xyz: np.ndarray) -> np.ndarray:
    m = -np.ones((n, n, n), dtype=np.int64)         # [x, y, z]
    m[xyz[:, 0], xyz[:, 1], xyz[:, 2]] = np.arange(xyz.shape[0])
    return m


def same_table(n: int, xyz: np.ndarray) -> np.ndarray:
    m = _index_map(n, xyz)
    tab = np.empty((xyz.shape[0], 27), dtype=np.int64)
    for t, (dx, dy, dz) in enumerate(TAPS):
        tab[:, t] = m[(xyz[:, 0] + dx) % n, (xyz[:, 1] + dy) % n, (xyz[:, 2] + dz) % n]
    return tab


def down_table(nf: int, xyz_f: np.ndarray, xyz_c: np.ndarray) -> np.ndarray:
    """Coarse node q -> fine node at 2 q + d_t."""
    m = _index_map(nf, xyz_f)
    tab = np.empty((xyz_c.shape[0], 27), dtype=np.int64)
    for t, (dx, dy, dz) in enumerate(TAPS):
        tab[:, t] = m[(2 * xyz_c[:, 0] + dx) % nf, (2 * xyz_c[:, 1] + dy) % nf,
                      (2 * xyz_c[:, 2] + dz) % nf]
    return tab


def up_table(nf: int, xyz_f: np.ndarray, xyz_c: np.ndarray) -> np.ndarray:
    """Fine node p -> coarse node q with p = 2 q + d_t (mod the fine side), or -1."""
    m = _index_map(nf // 2, xyz_c)
    tab = -np.ones((xyz_f.shape[0], 27), dtype=np.int64)
    for t, d in enumerate(TAPS):
        a = (xyz_f - np.array(d)[None, :]) % nf
        even = (a % 2 == 0).all(axis=1)
        q = a[even] // 2
        tab[even, t] = m[q[:, 0], q[:, 1], q[:, 2]]
    return tab


class Graph:
    """Node lists, tables and input features of levels 0-2 of a voxel cell."""

    def __init__(self, vox: np.ndarray):
        H = grid.hierarchy(vox)
        if len(H) < 3:
            raise ValueError("the network needs at least 3 levels")
        self.levels = H[:3]
        xyz = [lv.node_xyz() for lv in self.levels]
        ns = [lv.n for lv in self.levels]
        self.n = [x.shape[0] for x in xyz]
        self.same = [same_table(ns[l], xyz[l]) for l in range(3)]
        self.down = [down_table(ns[l], xyz[l], xyz[l + 1]) for l in range(2)]
        self.up = [up_table(ns[l], xyz[l], xyz[l + 1]) for l in range(2)]
        masks = self.levels[0].node_mask_list().astype(np.int64)
        self.x0 = torch.tensor(((masks[:, None] >> np.arange(8)[None, :]) & 1).astype(np.float64))

    def table(self, kind: int, lvl_out: int) -> np.ndarray:
        if kind == SAME:
            return self.same[lvl_out]
        if kind == DOWN:
            return self.down[lvl_out - 1]
        return self.up[lvl_out]


# ------------------------------------------------------------------ network
def conv(x: torch.Tensor, tab: np.ndarray, W: torch.Tensor, b: torch.Tensor | None):
    """z[n] = b + sum_t W[t]^T x[tab[n, t]] (missing neighbours, tab < 0, add nothing)."""
    xp = torch.cat([x, torch.zeros((1, x.shape[1]), dtype=x.dtype)], dim=0)
    idx = torch.as_tensor(np.where(tab < 0, x.shape[0], tab))
    z = torch.zeros((tab.shape[0], W.shape[2]), dtype=x.dtype)
    for t in range(27):
        z = z + xp[idx[:, t]] @ W[t]
    return z if b is None else z + b


def forward(g: Graph, params: torch.Tensor, rows):
    """Output activation (n0, cout) for a flat parameter vector."""
    P = split_params(params, rows)
    acts = [g.x0]
    for i, (kind, lo, a_in, skip, _, _) in enumerate(rows):
        z = conv(acts[a_in], g.table(kind, lo), P[i][0], P[i][1])
        if skip >= 0:
            z = z + acts[skip]
        acts.append(torch.relu(z) if i + 1 < len(rows) else z)
    return acts[-1]


def loss_and_grad(g: Graph, params: np.ndarray, rows, u: np.ndarray, scale: float, K=None):
    """(loss, gradient) in float64 for the canonical target field u (n0, cout): the mean
    squared error, or with K (scipy sparse, (n0 D) x (n0 D), node-major) the relative energy
    norm of the error."""
    p = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    y = forward(g, p, rows)
    ut = torch.as_tensor(np.asarray(u, dtype=np.float64).reshape(y.shape))
    if K is None:
        loss = ((y - ut / scale) ** 2).mean()
    else:
        Kc = K.tocoo()
        Kt = torch.sparse_coo_tensor(np.vstack([Kc.row, Kc.col]), Kc.data, Kc.shape)
        ncase = y.shape[1] * y.shape[0] // K.shape[0]        # M load cases
        e = (scale * y - ut).reshape(K.shape[0], ncase)
        uu = ut.reshape(K.shape[0], ncase)
        loss = (e * torch.sparse.mm(Kt, e)).sum() / (uu * torch.sparse.mm(Kt, uu)).sum()
    loss.backward()
    return float(loss.detach()), p.grad.numpy().copy()


def adamw_step(p, grad, m, v, step, lr, beta1, beta2, eps, weight_decay):
    """One AdamW update (bias-corrected moments, weight decay decoupled from the gradient),
    in float64; returns (p, m, v) after the step (`step` counts from 1)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    p = p - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * p)
    return p, m, v
