"""The allocation-free C^H entry point (gmt_homogenize_dense_noalloc) against the regular
one (gmt_homogenize) on the same field, twice in a row.

Callers that cannot allocate device memory (their memory manager owns the device, a fixed
memory budget, or no room for an allocation's implicit synchronisation) use this call: it
takes the field on the dense periodic node grid and writes C^H into the caller's device
buffer, using only a fixed working array inside the library. This file is collected last so
that a failure here does not stop the other tests from running first."""
import numpy as np
import pytest
import torch

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


def test_noalloc_rejects_oversized_cells(gmt_lib):
    gmt = gmt_lib
    vox = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    u = torch.zeros(4 ** 3 * 18, dtype=torch.float64, device="cuda")
    with pytest.raises(gmt.GmtError) as e:
        gmt.homogenize_dense_noalloc(vox, 513, gmt.ELASTIC, u_dense=u)
    assert e.value.status == gmt.ERR_ARG and "512" in str(e.value)
