"""Parity of gmt_sensitivities (App. F.3) with the oracle's sensitivities of the same field:
the library's field of a config-1 gyroid (32^3, 3 levels) is handed to the oracle, which
evaluates p / N^3 (x0 - u_e)^T K0 (x0 - u_e) per element in canonical element order."""
import numpy as np
import pytest

from oracle import solve
from paper_2604_26518_b300 import lattices as L
from helpers import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gyroid32_oracle():
    vox = L.tpms_network("gyroid", 32, 0.30)
    return vox, {k: solve.solve_cell(vox, k, tol=1e-8) for k in ("elastic", "heat")}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["elastic", "heat"])
def test_sensitivities_match_oracle(gmt_lib, gyroid32_oracle, precision, kind):
    gmt = gmt_lib
    vox, refs = gyroid32_oracle
    ref = refs[kind]
    prec = gmt.FP64 if precision == "fp64" else gmt.FP32
    h = gmt.Hierarchy(vox, gmt.default_options(precision=prec, levels=3))
    ph = gmt.ELASTIC if kind == "elastic" else gmt.HEAT
    st, u, _ = h.solve(ph, tol=1e-5)
    D, M = ref["D"], ref["NC"]
    U = to_np(u, D, M)
    p = 3.0
    sens = h.sensitivities(ph, p=p).cpu().numpy()          # stored solution
    expect = solve.sensitivities(ref["level"], U, ref["Ke"], ref["x0"], D, p)
    assert sens.shape == expect.shape == (ref["level"].num_elements, M, M)
    scale = np.abs(expect).max()
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert np.abs(sens - expect).max() <= tol * scale
    # the same through an explicit field, and the sum rule against the library's C^H
    sens_u = h.sensitivities(ph, p=p, u=u).cpu().numpy()
    assert np.abs(sens_u - expect).max() <= (1e-12 if precision == "fp64" else 2e-6) * scale
    CH = h.homogenize(ph)
    # (the FP32 path rounds each element's energy once in FP32 before either sum)
    rule = 1e-10 if precision == "fp64" else 5e-7
    assert np.abs(sens.sum(axis=0) - p * CH).max() <= rule * p * np.abs(CH).max()


def test_sensitivities_need_positive_p(gmt_lib):
    gmt = gmt_lib
    h = gmt.Hierarchy(np.ones((8, 8, 8), dtype=np.uint8))
    h.solve(gmt.ELASTIC, tol=1e-5)
    with pytest.raises(gmt.GmtError):
        h.sensitivities(gmt.ELASTIC, p=0.0)
