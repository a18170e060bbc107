"""Full-size 512^3 gyroid (phi 0.20), elasticity and heat conduction: the benchmark's 512^3
cell, solved with the schedule its autotuner picks there (nu 1, coarse nu 2, FP16 coarse
stencils), checked where the FP64 oracle can follow at 30 M nodes (an assembled solve of
2e8 unknowns is out of its reach; the 128^3 test checks the whole-field identities):
- canonical numbering (Sec. 4.1): the library's node list is the oracle's, node for node;
- the matrix-free operator (Sec. 4.6): the library's FP64 and FP32 K u at sampled nodes,
  interior and surface, against the oracle's sum over each node's active incident elements
  of K_e times the same field;
- the residual (Sec. 5 metric r): at every sampled node the oracle's f_n - (K u)_n of the
  library's converged field is below tol * ||f_m|| for every case m, a bound that any
  field meeting the global criterion satisfies node by node, with ||f_m|| exact from the
  histogram of node masks;
- C^H: symmetric, positive definite and below the Voigt bound phi C0."""
import numpy as np
import pytest

from oracle import fe, grid
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu
TOL = 1e-5
N = 512


def _mask_tables(Ke, x0, D):
    """Per octant mask: the node's load f (D x M) = sum over set bits a of (K_e x0)[a] with
    FP64 rounding cancelled below 1e-12 of the gross sum, and the (a, d) element blocks."""
    fe_ = Ke @ x0                                   # (8D, M)
    F = np.zeros((256, D, fe_.shape[1]))
    for mk in range(256):
        acc = np.zeros((D, fe_.shape[1]))
        gross = np.zeros((D, fe_.shape[1]))
        for a in range(8):
            if mk >> a & 1:
                acc += fe_[a * D:(a + 1) * D]
                gross += np.abs(fe_[a * D:(a + 1) * D])
        acc[np.abs(acc) <= 1e-12 * gross] = 0.0
        F[mk] = acc
    return F


def _oracle_Ku(Ke, D, masks, U27):
    """(K u)_n = sum over active incident elements e = n - a (bit a of the node's mask) of
    K_e[rows of local vertex a] u_e, u_e's vertex b being the neighbour at offset b - a;
    also the row scale sum |K_e| |u| for the FP32 tolerance. U27: (S, 27, D, M)."""
    S, _, _, M = U27.shape
    Ku = np.zeros((S, D, M))
    scale = np.zeros((S, D, M))
    for a, (ax, ay, az) in enumerate(grid.OFFSETS):
        on = ((masks >> a) & 1).astype(np.float64)[:, None, None]
        for b, (bx, by, bz) in enumerate(grid.OFFSETS):
            d = (bx - ax + 1) + 3 * (by - ay + 1) + 9 * (bz - az + 1)
            blk = Ke[a * D:(a + 1) * D, b * D:(b + 1) * D]          # (D, D)
            Ku += on * np.einsum("ij,sjm->sim", blk, U27[:, d])
            scale += on * np.einsum("ij,sjm->sim", np.abs(blk), np.abs(U27[:, d]))
    return Ku, scale


@pytest.fixture(scope="module")
def cell512():
    vox = L.tpms_network("gyroid", N, 0.20)
    return vox, grid.Level(vox)


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_full_size_512_sampled_parity(gmt_lib, cell512, kind):
    import torch
    gmt = gmt_lib
    vox, lev = cell512
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    Ke, x0, D, M, C0 = fe.physics(kind)
    opts = gmt.default_options(nu_coarse=2, coarse_fp16=1)
    opts.nu_pre = opts.nu_post = 1
    h = gmt.Hierarchy(torch.from_numpy(vox).cuda(), opts)
    st, u, info = h.solve(ph, tol=TOL)
    assert st == gmt.OK and max(info.as_dict()["rel_residual"][:M]) <= TOL

    # canonical numbering, node for node
    n = h.num_nodes(0)
    assert n == lev.num_nodes
    xyz, mk = h.node_coords(0)
    xyz = xyz.cpu().numpy().astype(np.int64)
    lin = xyz[:, 0] + N * xyz[:, 1] + N * N * xyz[:, 2]
    assert np.array_equal(lin, lev.node_lin)
    masks_all = lev.mask.reshape(-1)[lev.node_lin]
    assert np.array_equal(mk.cpu().numpy(), masks_all)
    del xyz, lin

    # sampled nodes: uniform, surface (partial masks) and the two ends of the numbering
    rng = np.random.default_rng(512)
    surface = np.nonzero(masks_all != 255)[0]
    ranks = np.unique(np.concatenate([rng.choice(n, 3000, replace=False),
                                      rng.choice(surface, 3000, replace=False), [0, n - 1]]))
    masks = masks_all[ranks].astype(np.int64)
    lin = lev.node_lin[ranks]
    x, y, z = lin % N, (lin // N) % N, lin // (N * N)
    nbr = np.empty((ranks.size, 27), dtype=np.int64)
    for d in range(27):
        dx, dy, dz = d % 3 - 1, (d // 3) % 3 - 1, d // 9 - 1
        nbr[:, d] = lev.rank[((x + dx) % N) + N * ((y + dy) % N) + N * N * ((z + dz) % N)]
    idx = torch.from_numpy(np.maximum(nbr, 0)).cuda()
    U27 = u[idx].cpu().numpy()                                   # (S, 27, D, M)
    U27[nbr < 0] = 0.0
    Ku, scale = _oracle_Ku(Ke, D, masks, U27)
    # every neighbour an active element reaches is an active node
    for a, (ax, ay, az) in enumerate(grid.OFFSETS):
        for b, (bx, by, bz) in enumerate(grid.OFFSETS):
            d = (bx - ax + 1) + 3 * (by - ay + 1) + 9 * (bz - az + 1)
            assert (nbr[(masks >> a & 1) == 1, d] >= 0).all()

    sel = torch.from_numpy(ranks).cuda()
    y64 = h.apply(0, u, gmt.FP64)[sel].cpu().numpy()
    y32 = h.apply(0, u, gmt.FP32)[sel].cpu().numpy()
    assert (np.abs(y64 - Ku) <= 1e-12 * scale + 1e-300).all()
    assert (np.abs(y32 - Ku) <= 2e-6 * scale + 1e-300).all()

    # the node-by-node residual bound from the global criterion
    Ftab = _mask_tables(Ke, x0, D)
    counts = np.bincount(masks_all, minlength=256).astype(np.float64)
    fnorm = np.sqrt(np.einsum("k,kim->m", counts, Ftab ** 2))   # ||f_m||_2 over all nodes
    r = Ftab[masks] - Ku                                          # (S, D, M)
    rn = np.sqrt((r ** 2).sum(axis=1))                            # (S, M)
    assert (rn <= TOL * fnorm[None, :] * (1 + 1e-9)).all(), (rn / fnorm).max()
    # the load itself is large at the surface: the bound is not met trivially
    assert (np.sqrt((Ftab[masks] ** 2).sum(axis=1)) > TOL * fnorm).any()

    CH = h.homogenize(ph)
    phi = vox.mean()
    assert np.abs(CH - CH.T).max() < 1e-12 * np.abs(CH).max()
    assert np.linalg.eigvalsh(CH).min() > 0
    assert np.linalg.eigvalsh(phi * C0 - CH).min() > -1e-9
    h.free()
