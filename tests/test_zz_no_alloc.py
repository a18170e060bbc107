"""The allocation-free C^H entry point (gmt_homogenize_dense_noalloc) against the regular
one (gmt_homogenize) on the same field, twice in a row, and against the FP64 oracle on
small and odd cell sides.

Callers that cannot allocate device memory (their memory manager owns the device, a fixed
memory budget, or no room for an allocation's implicit synchronisation) use this call: it
takes the field on the dense periodic node grid and writes C^H into the caller's device
buffer, using only a fixed working array inside the library. This file is collected last so
that a failure here does not stop the other tests from running first."""
import numpy as np
import pytest
import torch

from oracle import grid, solve
from paper_2604_26518_b300 import lattices as L

pytestmark = pytest.mark.gpu
REL = 2e-7   # the tolerance the float-float C^H path is held to elsewhere in the tests


def _dense(h, u, n, C):
    xyz, _ = h.node_coords(0)
    xyz = xyz.long()
    dense = torch.zeros((n, n, n, C), dtype=torch.float64, device="cuda")
    dense[xyz[:, 2], xyz[:, 1], xyz[:, 0]] = u.reshape(-1, C)
    return dense.contiguous()


@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_noalloc_homogenize_matches_regular_entry_point(gmt_lib, kind):
    gmt = gmt_lib
    n = 32
    vox = L.tpms_network("gyroid", n, 0.3)
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    D, M = (3, 6) if kind == "elastic" else (1, 3)
    h = gmt.Hierarchy(vox)
    st, u, info = h.solve(ph, tol=1e-5)
    ref = h.homogenize(ph, u=u)
    dense = _dense(h, u, n, D * M)
    vox_dev = torch.from_numpy(vox).cuda()
    for _ in range(2):
        out = gmt.homogenize_dense_noalloc(vox_dev, n, ph, u_dense=dense)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= REL * np.abs(ref).max(), (got, ref)
        np.testing.assert_array_equal(got, got.T)


@pytest.mark.parametrize("n", [5, 7, 17])
@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_noalloc_homogenize_matches_oracle_on_odd_sides(gmt_lib, kind, n):
    """Sides that are not multiples of 4 (and tiny ones) exercise the periodic wrap of the
    dense node grid; the field is the oracle's own converged FP64 solution, and C^H is held
    to the oracle's energy average of that field at FP64 rounding."""
    gmt = gmt_lib
    rng = np.random.default_rng(700 + n)
    vox = L.largest_component(L.random_binary(n, 0.55, rng))
    ref = solve.solve_cell(vox, kind)
    D, M = (3, 6) if kind == "elastic" else (1, 3)
    xyz = ref["level"].node_xyz()
    dense = np.zeros((n, n, n, D * M))
    dense[xyz[:, 2], xyz[:, 1], xyz[:, 0]] = ref["U"].reshape(-1, D * M)
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    vox_dev = torch.from_numpy(np.ascontiguousarray(vox)).cuda()
    u_dev = torch.from_numpy(dense.reshape(-1)).cuda()
    for _ in range(2):
        got = gmt.homogenize_dense_noalloc(vox_dev, n, ph, u_dense=u_dev).cpu().numpy()
        assert np.abs(got - ref["CH"]).max() <= 1e-12 * np.abs(ref["CH"]).max(), (got, ref["CH"])


def test_noalloc_rejects_oversized_cells(gmt_lib):
    gmt = gmt_lib
    vox = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    u = torch.zeros(4 ** 3 * 18, dtype=torch.float64, device="cuda")
    out = torch.zeros((6, 6), dtype=torch.float64, device="cuda")
    st = gmt.lib().gmt_homogenize_dense_noalloc(vox.data_ptr(), 513, gmt.ELASTIC, 1.0, 0.3, 1.0,
                                               u.data_ptr(), out.data_ptr(), None)
    assert st == gmt.ERR_ARG and b"512" in gmt.lib().gmt_last_error()
