"""The C-ABI library builds, loads and exports every symbol include/gmt.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes

from paper_2604_26518_b300 import build, gmt


def test_library_builds_and_exports_declared_symbols():
    build.build()
    L = ctypes.CDLL(gmt.LIB_PATH)
    names = gmt.declared_symbols()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares a signature for every exported entry point
    assert set(names) == set(gmt._SIGS), set(names) ^ set(gmt._SIGS)


def test_host_only_calls():
    L = gmt.lib()
    o = gmt.default_options()
    assert o.levels == 0 and o.coarsest_max == 8 and o.nu_pre == 1 and o.nu_coarse == 2
    assert o.precision == gmt.FP32
    assert L.gmt_status_string(gmt.ERR_RES).decode().startswith("unsupported")
    # argument errors are reported as statuses, not crashes (checked before any CUDA call)
    h = ctypes.c_void_p()
    st = L.gmt_build_hierarchy(None, 32, 0, None, None, ctypes.byref(h))
    assert st == gmt.ERR_ARG
    buf = (ctypes.c_uint8 * 8)()
    st = L.gmt_build_hierarchy(buf, 30, 0, None, None, ctypes.byref(h))
    assert st == gmt.ERR_RES and b"multiple of 4" in L.gmt_last_error()
    assert L.gmt_num_levels(None) == 0


def test_trace_category_names():
    from paper_2604_26518_b300 import gmt
    L = gmt.lib()
    names = [L.gmt_trace_name(c).decode() for c in range(gmt.TRACE_CATEGORIES)]
    assert len(set(names)) == gmt.TRACE_CATEGORIES and all(names)
    assert {"smooth_l0", "setup_hierarchy", "setup_operators", "setup_coarse_inverse"} <= set(names)
    assert L.gmt_trace_name(gmt.TRACE_CATEGORIES).decode() == ""
    assert L.gmt_trace_name(-1).decode() == ""


def test_noalloc_binding_rejects_bad_tensors_before_the_library():
    """The allocation-free entry point's binding checks dtype, size, shape and contiguity of
    every tensor (and that they are on CUDA) before calling the library, so that a short or
    mistyped field can never reach the kernel."""
    import pytest
    import torch
    n = 8
    vox = torch.zeros(n ** 3, dtype=torch.uint8)
    good = torch.zeros(n ** 3 * 18, dtype=torch.float64)
    with pytest.raises(ValueError, match="u_dense must have"):
        gmt.homogenize_dense_noalloc(vox, n, gmt.ELASTIC, u_dense=good[:-1])
    with pytest.raises(ValueError, match="u_dense must be torch.float64"):
        gmt.homogenize_dense_noalloc(vox, n, gmt.ELASTIC, u_dense=good.float())
    with pytest.raises(ValueError, match="u_dense must have"):        # heat: D*M = 3
        gmt.homogenize_dense_noalloc(vox, n, gmt.HEAT, u_dense=good)
    with pytest.raises(ValueError, match="contiguous"):
        gmt.homogenize_dense_noalloc(vox, n, gmt.ELASTIC,
                                     u_dense=torch.zeros(n ** 3 * 36, dtype=torch.float64)[::2])
    with pytest.raises(ValueError, match="voxels must have"):
        gmt.homogenize_dense_noalloc(vox[:-1], n, gmt.ELASTIC, u_dense=good)
    with pytest.raises(ValueError, match="voxels must be torch.uint8"):
        gmt.homogenize_dense_noalloc(vox.int(), n, gmt.ELASTIC, u_dense=good)
    with pytest.raises(ValueError, match="out must have shape"):
        gmt.homogenize_dense_noalloc(vox, n, gmt.ELASTIC, u_dense=good,
                                     out=torch.zeros((36,), dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA tensor"):
        gmt.homogenize_dense_noalloc(vox, n, gmt.ELASTIC, u_dense=good)
    # the library's own checks: null pointers and an oversized cell are statuses
    L = gmt.lib()
    assert L.gmt_homogenize_dense_noalloc(None, n, 0, 1.0, 0.3, 1.0, None, None, None) == gmt.ERR_ARG
    buf = (ctypes.c_uint8 * 8)()
    assert L.gmt_homogenize_dense_noalloc(buf, 513, 0, 1.0, 0.3, 1.0, buf, buf, None) == gmt.ERR_ARG
    assert b"512" in L.gmt_last_error()
