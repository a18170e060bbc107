"""Python binding of libgmt.so (C ABI in include/gmt.h).

Argument marshalling only: every computation runs in the library's CUDA kernels. Device
buffers are torch CUDA tensors (torch supplies device memory and the current stream); the
library receives raw pointers and sizes. There is no CPU fallback: if the library or a CUDA
device is missing, every call raises.

Field layout (canonical): float64 tensor of shape (nodes, D, M), D = 3 components and
M = 6 Voigt load cases for elasticity, D = 1 and M = 3 for heat conduction; node order is
increasing x + N*y + N^2*z over active nodes of the level.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgmt.so")

ELASTIC, HEAT = 0, 1
FP64, FP32, BF16 = 0, 1, 2
JACOBI, CHEBYSHEV, GS8 = 0, 1, 2
CYCLE_V, CYCLE_W, CYCLE_F = 0, 1, 2

OK, ERR_ARG, ERR_RES, ERR_EMPTY, ERR_OOM, ERR_CUDA, NOT_CONVERGED, DIVERGED, ERR_STATE = range(9)


class Options(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("coarsest_max", ctypes.c_int),
        ("smoother", ctypes.c_int),
        ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("cheb_ratio", ctypes.c_double),
        ("cheb_upper", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("krylov", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("max_inner", ctypes.c_int),
        ("max_outer", ctypes.c_int),
        ("cycle", ctypes.c_int),
        ("fp64_fallback", ctypes.c_int),
        ("nu_coarse", ctypes.c_int),
        ("graphs", ctypes.c_int),
        ("coarse_fp16", ctypes.c_int),
        ("warm_sweeps", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("outer", ctypes.c_int),
        ("inner_total", ctypes.c_int),
        ("cases", ctypes.c_int),
        ("rel_residual", ctypes.c_double * 6),
        ("t_setup_ms", ctypes.c_double),
        ("t_solve_ms", ctypes.c_double),
        ("fp64_fallback", ctypes.c_int),
    ]

    def as_dict(self):
        return {"outer": self.outer, "cycles": self.inner_total,
                "rel_residual": list(self.rel_residual)[: self.cases],
                "t_setup_ms": self.t_setup_ms, "t_solve_ms": self.t_solve_ms,
                "fp64_fallback": self.fp64_fallback}


class GmtError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status} ({message})")
        self.status = status


class AdamW(ctypes.Structure):
    """gmt_adamw: AdamW hyper-parameters of gmt_unet_train_step."""
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("weight_decay", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_L = ctypes.c_int64

_SIGS = {
    "gmt_default_options": (None, [ctypes.POINTER(Options)]),
    "gmt_status_string": (ctypes.c_char_p, [_I]),
    "gmt_last_error": (ctypes.c_char_p, []),
    "gmt_build_hierarchy": (_I, [_P, _I, _I, ctypes.POINTER(Options), _P, ctypes.POINTER(_P)]),
    "gmt_free_hierarchy": (None, [_P]),
    "gmt_set_stream": (_I, [_P, _P]),
    "gmt_set_options": (_I, [_P, ctypes.POINTER(Options)]),
    "gmt_num_levels": (_I, [_P]),
    "gmt_level_res": (_I, [_P, _I]),
    "gmt_num_nodes": (_L, [_P, _I]),
    "gmt_num_elements": (_L, [_P, _I]),
    "gmt_num_bricks": (_L, [_P, _I]),
    "gmt_device_bytes": (_L, [_P]),
    "gmt_node_coords": (_I, [_P, _I, _P, _P]),
    "gmt_element_coords": (_I, [_P, _I, _P, _P]),
    "gmt_transfer_stencil": (_I, [_P, _I, _P, _P]),
    "gmt_prepare": (_I, [_P, _I, _D, _D, _D]),
    "gmt_apply": (_I, [_P, _I, _I, _P, _P]),
    "gmt_smooth": (_I, [_P, _I, _I, _P, _P, _I, _I]),
    "gmt_restrict": (_I, [_P, _I, _I, _P, _P]),
    "gmt_prolong": (_I, [_P, _I, _I, _P, _P]),
    "gmt_coarse_solve": (_I, [_P, _P, _P]),
    "gmt_vcycle": (_I, [_P, _I, _P, _P, _I]),
    "gmt_vcycle_batch": (_I, [_P, _I, _P, _P, _I]),
    "gmt_vcycle_inject": (_I, [_P, _I, _P, _P, _I, _P, _I]),
    "gmt_solve_batch": (_I, [_P, _I, _I, _D, _D, _D, _D, _P, _P, _P, _P]),
    "gmt_autotune": (_I, [_P, _I, _D, _D, _D, _D, ctypes.POINTER(Options), _P]),
    "gmt_lambda_max": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "gmt_solve": (_I, [_P, _I, _D, _D, _D, _D, _P, _P, ctypes.POINTER(Info)]),
    "gmt_homogenize": (_I, [_P, _I, _D, _D, _D, _P, _P]),
    "gmt_sensitivities": (_I, [_P, _I, _D, _D, _D, _D, _P, _P]),
    "gmt_set_densities": (_I, [_P, _P, _I, _D, _D]),
    "gmt_residual": (_I, [_P, _I, _P, _P]),
    "gmt_trace_enable": (_I, [_P, _I]),
    "gmt_trace_query": (_I, [_P, _I, ctypes.POINTER(_L), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gmt_trace_name": (ctypes.c_char_p, [_I]),
    "gmt_launch_count": (_L, []),
    "gmt_homogenize_dense_noalloc": (_I, [_P, _I, _I, _D, _D, _D, _P, _P, _P]),
    "gmt_release_cached_memory": (None, []),
    "gmt_cached_bytes": (_L, []),
    "gmt_unet_param_count": (_L, [_I, _P]),
    "gmt_unet_layers": (_I, [_I, _P, _P]),
    "gmt_unet_create": (_I, [_I, _P, _P, ctypes.POINTER(_P)]),
    "gmt_unet_free": (None, [_P]),
    "gmt_unet_num_params": (_L, [_P]),
    "gmt_unet_get_params": (_I, [_P, _P]),
    "gmt_unet_set_params": (_I, [_P, _P]),
    "gmt_unet_set_tensor_cores": (_I, [_P, _I]),
    "gmt_netgraph_build": (_I, [_P, ctypes.POINTER(_P)]),
    "gmt_netgraph_free": (None, [_P]),
    "gmt_netgraph_nodes": (_L, [_P, _I]),
    "gmt_netgraph_tables": (_I, [_P, _I, _P, _P, _P]),
    "gmt_unet_forward": (_I, [_P, _P, _D, _P]),
    "gmt_unet_gradient": (_I, [_P, _P, _P, _I, _P, _D, _P, ctypes.POINTER(_D)]),
    "gmt_unet_train_step": (_I, [_P, _P, _P, _I, _P, _D, ctypes.POINTER(AdamW),
                                 ctypes.POINTER(_D)]),
}

TRACE_CATEGORIES = 16
AUTOTUNE_CANDIDATES = 13


def release_cached_memory():
    """Return the library's cached, unused device blocks to the driver."""
    lib().gmt_release_cached_memory()


def cached_bytes() -> int:
    return int(lib().gmt_cached_bytes())


def launch_count() -> int:
    """Kernels launched through the library by this process so far."""
    return int(lib().gmt_launch_count())


def lib():
    """Load libgmt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2604_26518_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    lib().gmt_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _check(st: int, where: str, allow=(OK,)):
    if st not in allow:
        msg = lib().gmt_last_error().decode() or lib().gmt_status_string(st).decode()
        raise GmtError(st, where, msg)
    return st


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libgmt needs a CUDA device; none is available")
    return torch


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Hierarchy:
    """Sparse periodic GMG hierarchy of one voxel cell (gmt_build_hierarchy)."""

    def __init__(self, voxels, options: Options | None = None, stream=None):
        torch = _torch()
        self._h = _P()
        L = lib()
        if isinstance(voxels, np.ndarray):
            vox = np.ascontiguousarray(voxels, dtype=np.uint8)
            n = vox.shape[0]
            if vox.shape != (n, n, n):
                raise ValueError(f"voxels must be a cube, got shape {vox.shape}")
            src, on_dev, self._keep = vox.ctypes.data, 0, vox
        else:
            vox = voxels.contiguous()
            if vox.dtype != torch.uint8 or vox.dim() != 3 or len(set(vox.shape)) != 1:
                raise ValueError(f"voxels must be a uint8 cube, got {vox.dtype} {tuple(vox.shape)}")
            n = vox.shape[0]
            src, on_dev, self._keep = vox.data_ptr(), int(vox.is_cuda), vox
        self.n = int(n)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opts = options if options is not None else default_options()
        st = L.gmt_build_hierarchy(src, self.n, on_dev, ctypes.byref(opts),
                                   self.stream.cuda_stream, ctypes.byref(self._h))
        _check(st, "gmt_build_hierarchy")
        self._keep = None
        self.physics = None

    # ---------------------------------------------------------------- lifetime
    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gmt_free_hierarchy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # ---------------------------------------------------------------- sizes
    @property
    def levels(self) -> int:
        return lib().gmt_num_levels(self._h)

    def level_res(self, l: int) -> int:
        return lib().gmt_level_res(self._h, l)

    def num_nodes(self, l: int = 0) -> int:
        return int(lib().gmt_num_nodes(self._h, l))

    def num_elements(self, l: int = 0) -> int:
        return int(lib().gmt_num_elements(self._h, l))

    def num_bricks(self, l: int = 0) -> int:
        return int(lib().gmt_num_bricks(self._h, l))

    def device_bytes(self) -> int:
        return int(lib().gmt_device_bytes(self._h))

    def set_options(self, options: Options):
        _check(lib().gmt_set_options(self._h, ctypes.byref(options)), "gmt_set_options")

    # ---------------------------------------------------------------- geometry export
    def node_coords(self, l: int = 0):
        torch = _torch()
        n = self.num_nodes(l)
        xyz = torch.empty((n, 3), dtype=torch.int32, device="cuda")
        m = torch.empty((n,), dtype=torch.uint8, device="cuda")
        _check(lib().gmt_node_coords(self._h, l, _ptr(xyz), _ptr(m)), "gmt_node_coords")
        return xyz, m

    def element_coords(self, l: int = 0):
        torch = _torch()
        n = self.num_elements(l)
        xyz = torch.empty((n, 3), dtype=torch.int32, device="cuda")
        c = torch.empty((n,), dtype=torch.uint8, device="cuda")
        _check(lib().gmt_element_coords(self._h, l, _ptr(xyz), _ptr(c)), "gmt_element_coords")
        return xyz, c

    def transfer_stencil(self, l: int = 0):
        torch = _torch()
        n = self.num_nodes(l)
        idx = torch.empty((n, 8), dtype=torch.int32, device="cuda")
        w = torch.empty((n, 8), dtype=torch.float64, device="cuda")
        _check(lib().gmt_transfer_stencil(self._h, l, _ptr(idx), _ptr(w)), "gmt_transfer_stencil")
        return idx, w

    # ---------------------------------------------------------------- operators
    def prepare(self, physics=ELASTIC, E=1.0, nu=0.3, k=1.0):
        _check(lib().gmt_prepare(self._h, physics, E, nu, k), "gmt_prepare")
        self.physics = physics

    def _dm(self):
        return (3, 6) if self.physics == ELASTIC else (1, 3)

    def _field(self, l, x):
        torch = _torch()
        D, M = self._dm()
        n = self.num_nodes(l)
        if x is None:
            return torch.zeros((n, D, M), dtype=torch.float64, device="cuda")
        x = torch.as_tensor(x, dtype=torch.float64, device="cuda").contiguous()
        if x.numel() != n * D * M:   # the library reads exactly n * D * M values
            raise ValueError(f"level-{l} field has {x.numel()} values, expected {n * D * M}")
        return x.view(n, D, M)

    def apply(self, level, u, precision=FP64):
        u = self._field(level, u)
        y = self._field(level, None)
        _check(lib().gmt_apply(self._h, level, precision, _ptr(u), _ptr(y)), "gmt_apply")
        return y

    def smooth(self, level, f, u=None, sweeps=1, precision=FP64):
        f = self._field(level, f)
        zero = u is None
        u = self._field(level, u).clone()
        _check(lib().gmt_smooth(self._h, level, precision, _ptr(f), _ptr(u), sweeps, int(zero)),
               "gmt_smooth")
        return u

    def restrict(self, level, r, precision=FP64):
        r = self._field(level, r)
        fc = self._field(level + 1, None)
        _check(lib().gmt_restrict(self._h, level, precision, _ptr(r), _ptr(fc)), "gmt_restrict")
        return fc

    def prolong(self, level, uc, uf=None, precision=FP64):
        uc = self._field(level + 1, uc)
        uf = self._field(level, uf).clone()
        _check(lib().gmt_prolong(self._h, level, precision, _ptr(uc), _ptr(uf)), "gmt_prolong")
        return uf

    def coarse_solve(self, f):
        f = self._field(self.levels - 1, f)
        u = self._field(self.levels - 1, None)
        _check(lib().gmt_coarse_solve(self._h, _ptr(f), _ptr(u)), "gmt_coarse_solve")
        return u

    def vcycle(self, f, u=None, precision=FP64, corrections=None):
        """One V-cycle on K_0 u = f (gmt_vcycle). corrections: per-level starting fields
        of the coarse unknowns (Alg. 2's injected corrections, gmt_vcycle_inject), a list
        of `levels` entries, each None or a level-l field; entry 0 is not used."""
        f = self._field(0, f)
        zero = u is None
        u = self._field(0, u).clone()
        if corrections is None:
            _check(lib().gmt_vcycle(self._h, precision, _ptr(f), _ptr(u), int(zero)),
                   "gmt_vcycle")
            return u
        if len(corrections) != self.levels:
            raise ValueError(f"{len(corrections)} corrections for {self.levels} levels")
        es = [None if (l == 0 or c is None) else self._field(l, c)
              for l, c in enumerate(corrections)]
        ep = (_P * self.levels)(*[_ptr(x) for x in es])
        _check(lib().gmt_vcycle_inject(self._h, precision, _ptr(f), _ptr(u), int(zero), ep,
                                       self.levels), "gmt_vcycle_inject")
        return u

    def lambda_max(self, level):
        out = ctypes.c_double()
        _check(lib().gmt_lambda_max(self._h, level, ctypes.byref(out)), "gmt_lambda_max")
        return out.value

    # ---------------------------------------------------------------- solve
    def solve(self, physics=ELASTIC, E=1.0, nu=0.3, k=1.0, tol=1e-5, u0=None, want_field=True,
              allow_not_converged=False):
        self.physics = physics
        u0t = None if u0 is None else self._field(0, u0)
        out = self._field(0, None) if want_field else None
        info = Info()
        allow = (OK, NOT_CONVERGED, DIVERGED) if allow_not_converged else (OK,)
        st = lib().gmt_solve(self._h, physics, E, nu, k, tol, _ptr(u0t), _ptr(out),
                             ctypes.byref(info))
        _check(st, "gmt_solve", allow)
        return st, out, info

    def autotune(self, physics=ELASTIC, E=1.0, nu=0.3, k=1.0, tol=1e-5):
        """gmt_autotune: solve once per candidate schedule and keep the fastest. Returns the
        chosen Options (also set on the hierarchy) and each candidate's time in ms."""
        self.physics = physics
        best = Options()
        times = np.zeros(AUTOTUNE_CANDIDATES, dtype=np.float64)
        _check(lib().gmt_autotune(self._h, physics, E, nu, k, tol, ctypes.byref(best),
                                  times.ctypes.data_as(ctypes.c_void_p)), "gmt_autotune")
        return best, times

    def homogenize(self, physics=ELASTIC, E=1.0, nu=0.3, k=1.0, u=None):
        self.physics = physics
        D, M = self._dm()
        CH = np.zeros((M, M), dtype=np.float64)
        ut = None if u is None else self._field(0, u)
        _check(lib().gmt_homogenize(self._h, physics, E, nu, k, _ptr(ut),
                                    CH.ctypes.data_as(ctypes.c_void_p)), "gmt_homogenize")
        return CH

    def set_densities(self, rho=None, rho_min=1e-3, p=3.0):
        """SIMP element densities (gmt_set_densities): rho per level-0 element in canonical
        element order (numpy or torch float64, host or device), or None for the binary
        design. C_e = (rho_min + rho_e^p) C0."""
        if rho is None:
            _check(lib().gmt_set_densities(self._h, None, 0, 0.0, 0.0), "gmt_set_densities")
            return
        ne = self.num_elements(0)
        if isinstance(rho, np.ndarray):
            r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
            if r.size != ne:
                raise ValueError(f"{r.size} densities for {ne} elements")
            ptr, dev, keep = r.ctypes.data, 0, r
        else:
            torch = _torch()
            r = rho.to(torch.float64).contiguous().reshape(-1)
            if r.numel() != ne:
                raise ValueError(f"{r.numel()} densities for {ne} elements")
            ptr, dev, keep = r.data_ptr(), int(r.is_cuda), r
        _check(lib().gmt_set_densities(self._h, ptr, dev, float(rho_min), float(p)),
               "gmt_set_densities")
        del keep

    def sensitivities(self, physics=ELASTIC, E=1.0, nu=0.3, k=1.0, p=3.0, u=None):
        """dC^H / d rho_e per solid element (SIMP penalisation p), a device tensor
        [n_elems][M][M] in canonical element order (gmt_sensitivities)."""
        torch = _torch()
        self.physics = physics
        D, M = self._dm()
        out = torch.empty((self.num_elements(0), M, M), dtype=torch.float64, device="cuda")
        ut = None if u is None else self._field(0, u)
        _check(lib().gmt_sensitivities(self._h, physics, E, nu, k, p, _ptr(ut), _ptr(out)),
               "gmt_sensitivities")
        return out

    # ---------------------------------------------------------------- tracing
    def trace(self, on=True, brackets_only=False):
        """Enable (and reset) the library's launch tracer; brackets_only records only the
        whole-V-cycle category, without per-launch events inside the cycles."""
        mode = (2 if brackets_only else 1) if on else 0
        _check(lib().gmt_trace_enable(self._h, mode), "gmt_trace_enable")

    def trace_totals(self):
        """{category: (launches, device ms, algorithmic bytes)} since trace(True)."""
        out = {}
        for c in range(TRACE_CATEGORIES):
            n, ms, b = _L(), _D(), _D()
            _check(lib().gmt_trace_query(self._h, c, ctypes.byref(n), ctypes.byref(ms),
                                         ctypes.byref(b)), "gmt_trace_query")
            out[lib().gmt_trace_name(c).decode()] = (n.value, ms.value, b.value)
        return out

    def residual(self, u, precision=FP32):
        D, M = self._dm()
        u = self._field(0, u)
        out = np.zeros(M, dtype=np.float64)
        _check(lib().gmt_residual(self._h, precision, _ptr(u), out.ctypes.data_as(ctypes.c_void_p)),
               "gmt_residual")
        return out


UNET_WIDTHS = (32, 64, 128)
LOSS_MSE, LOSS_ENERGY = 0, 1


BATCH_MAX = 64


def vcycle_batch(hierarchies, fs, us=None):
    """One FP32 V-cycle on each hierarchy at once (gmt_vcycle_batch): returns the fields
    u_i = V-cycle(f_i) (from zero, or from us[i]), each bitwise the one Hierarchy.vcycle
    returns at FP32 precision. The hierarchies share the material, options and stream."""
    n = len(hierarchies)
    if not 1 <= n <= BATCH_MAX or len(fs) != n or (us is not None and len(us) != n):
        raise ValueError(f"batch of {n} hierarchies with {len(fs)} loads (1..{BATCH_MAX})")
    f = [h._field(0, x) for h, x in zip(hierarchies, fs)]
    u = [h._field(0, None if us is None else x).clone() for h, x in
         zip(hierarchies, us if us is not None else [None] * n)]
    hp = (_P * n)(*[h._h for h in hierarchies])
    fp = (_P * n)(*[_ptr(x) for x in f])
    up = (_P * n)(*[_ptr(x) for x in u])
    _check(lib().gmt_vcycle_batch(hp, n, fp, up, int(us is None)), "gmt_vcycle_batch")
    return u


def solve_batch(hierarchies, physics=ELASTIC, E=1.0, nu=0.3, k=1.0, tol=1e-5, u0s=None,
                want_fields=True, allow_not_converged=False):
    """Solve the cells of several hierarchies together (gmt_solve_batch): every result is
    bitwise Hierarchy.solve's for that cell, while the V-cycles of all cells share their
    launches. Returns a list of (status, field or None, Info) per hierarchy."""
    torch = _torch()
    n = len(hierarchies)
    if not 1 <= n <= BATCH_MAX or (u0s is not None and len(u0s) != n):
        raise ValueError(f"batch of {n} hierarchies (1..{BATCH_MAX})")
    for h in hierarchies:
        h.physics = physics
    u0t = [None if (u0s is None or x is None) else h._field(0, x)
           for h, x in zip(hierarchies, u0s if u0s is not None else [None] * n)]
    outs = [h._field(0, None) if want_fields else None for h in hierarchies]
    infos = (Info * n)()
    stats = (ctypes.c_int * n)()
    hp = (_P * n)(*[h._h for h in hierarchies])
    u0p = (_P * n)(*[_ptr(x) for x in u0t]) if u0s is not None else None
    outp = (_P * n)(*[_ptr(x) for x in outs]) if want_fields else None
    st = lib().gmt_solve_batch(hp, n, physics, E, nu, k, tol, u0p, outp, infos, stats)
    allow = (OK, NOT_CONVERGED, DIVERGED) if allow_not_converged else (OK,)
    _check(st, "gmt_solve_batch", allow)
    torch.cuda.synchronize()
    return [(int(stats[i]), outs[i], infos[i]) for i in range(n)]


def unet_layers(out_channels: int, widths=UNET_WIDTHS):
    """Layer table of the initializer network (gmt_unet_layers): rows of (kind, output
    level, input activation, skip activation, cin, cout); kind 0 same-level, 1 down, 2 up."""
    w = (ctypes.c_int * 3)(*widths)
    out = (ctypes.c_int32 * 72)()
    _check(lib().gmt_unet_layers(int(out_channels), ctypes.addressof(w), ctypes.addressof(out)),
           "gmt_unet_layers")
    return [tuple(out[6 * i:6 * i + 6]) for i in range(12)]


def unet_param_count(out_channels: int, widths=UNET_WIDTHS) -> int:
    w = (ctypes.c_int * 3)(*widths)
    return int(lib().gmt_unet_param_count(int(out_channels), ctypes.addressof(w)))


class NetGraph:
    """Neighbour tables and input features of a hierarchy for the initializer network
    (gmt_netgraph_build); needs at least 3 levels."""

    def __init__(self, hier: "Hierarchy"):
        self._g = _P()
        _check(lib().gmt_netgraph_build(hier._h, ctypes.byref(self._g)), "gmt_netgraph_build")
        self.n = [int(lib().gmt_netgraph_nodes(self._g, l)) for l in range(3)]

    def tables(self, level: int):
        """(same, down, up) int32 tables of a level (down and up None at level 2)."""
        torch = _torch()
        n = self.n[level]
        same = torch.empty((n, 27), dtype=torch.int32, device="cuda")
        down = up = None
        if level < 2:
            down = torch.empty((self.n[level + 1], 27), dtype=torch.int32, device="cuda")
            up = torch.empty((n, 27), dtype=torch.int32, device="cuda")
        _check(lib().gmt_netgraph_tables(self._g, level, _ptr(same), _ptr(down), _ptr(up)),
               "gmt_netgraph_tables")
        return same, down, up

    def free(self):
        if self._g:
            lib().gmt_netgraph_free(self._g)
            self._g = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class UNet:
    """The learned initializer (gmt_unet_*): a sparse 3D convolutional U-Net that predicts
    the canonical fine field of a cell from its octant masks. `params`: float32 tensor of
    the initial parameters (the caller draws them)."""

    def __init__(self, out_channels: int, params, widths=UNET_WIDTHS):
        torch = _torch()
        self.out_channels = int(out_channels)
        self.widths = tuple(widths)
        p = params.detach().to(device="cuda", dtype=torch.float32).contiguous()
        w = (ctypes.c_int * 3)(*self.widths)
        self._n = _P()
        _check(lib().gmt_unet_create(self.out_channels, ctypes.addressof(w), _ptr(p),
                                     ctypes.byref(self._n)), "gmt_unet_create")
        self.num_params = int(lib().gmt_unet_num_params(self._n))

    def params(self):
        torch = _torch()
        out = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        _check(lib().gmt_unet_get_params(self._n, _ptr(out)), "gmt_unet_get_params")
        return out

    def set_params(self, p):
        torch = _torch()
        p = p.detach().to(device="cuda", dtype=torch.float32).contiguous()
        _check(lib().gmt_unet_set_params(self._n, _ptr(p)), "gmt_unet_set_params")

    def tensor_cores(self, on: bool = True):
        """Inference on the tensor cores (FP16 operands, FP32 accumulation); training stays
        FP32 (gmt_unet_set_tensor_cores)."""
        _check(lib().gmt_unet_set_tensor_cores(self._n, int(bool(on))), "gmt_unet_set_tensor_cores")

    def forward(self, graph: NetGraph, scale: float):
        """Predicted canonical field, float64 (n0, cout) on the device (gmt_unet_forward)."""
        torch = _torch()
        u = torch.empty((graph.n[0], self.out_channels), dtype=torch.float64, device="cuda")
        _check(lib().gmt_unet_forward(self._n, graph._g, float(scale), _ptr(u)), "gmt_unet_forward")
        return u

    def gradient(self, graph: NetGraph, target, scale: float, loss=LOSS_MSE,
                 hier: "Hierarchy | None" = None):
        """(loss, gradient) against a canonical target field (gmt_unet_gradient); the energy
        loss needs the graph's hierarchy with the material prepared."""
        torch = _torch()
        t = target.detach().to(device="cuda", dtype=torch.float64).contiguous()
        g = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        out = _D()
        _check(lib().gmt_unet_gradient(self._n, graph._g, hier._h if hier else None, int(loss),
                                       _ptr(t), float(scale), _ptr(g), ctypes.byref(out)),
               "gmt_unet_gradient")
        return float(out.value), g

    def train_step(self, graph: NetGraph, target, scale: float, lr=1e-3, beta1=0.9,
                   beta2=0.999, eps=1e-8, weight_decay=1e-4, loss=LOSS_MSE,
                   hier: "Hierarchy | None" = None) -> float:
        """One AdamW step on one cell; returns the loss before the update. `target`: device
        float64 canonical field."""
        hp = AdamW(lr, beta1, beta2, eps, weight_decay)
        out = _D()
        _check(lib().gmt_unet_train_step(self._n, graph._g, hier._h if hier else None, int(loss),
                                         _ptr(target), float(scale), ctypes.byref(hp),
                                         ctypes.byref(out)), "gmt_unet_train_step")
        return float(out.value)

    def free(self):
        if self._n:
            lib().gmt_unet_free(self._n)
            self._n = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _noalloc_check(name: str, t, dtype, numel: int, shape=None):
    """Reject, before any library call, a tensor the allocation-free kernel would read or
    write out of bounds: wrong dtype, wrong size or shape, or non-contiguous. (The device
    is checked afterwards, once for all arguments.)"""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} values, got {t.numel()}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def homogenize_dense_noalloc(voxels, res: int, physics=ELASTIC, E=1.0, nu=0.3, k=1.0,
                             u_dense=None, out=None, stream=None):
    """C^H of a nodal field on the dense periodic node grid without any device allocation
    in the library (gmt_homogenize_dense_noalloc). voxels: contiguous CUDA uint8 tensor with
    N^3 values (x fastest); u_dense: contiguous CUDA float64 tensor with N^3 * D * M values
    (node site major); out: contiguous CUDA float64 (M, M) tensor, created if omitted (by
    torch, outside the library). Every tensor is checked (dtype, size, contiguity, device)
    before the library is called; the library itself rejects N > 512."""
    import torch
    if physics not in (ELASTIC, HEAT):
        raise ValueError(f"unknown physics {physics}")
    D, M = (3, 6) if physics == ELASTIC else (1, 3)
    res = int(res)
    n3 = res ** 3 if res > 0 else 0
    _noalloc_check("voxels", voxels, torch.uint8, n3)
    _noalloc_check("u_dense", u_dense, torch.float64, n3 * D * M)
    if out is not None:
        _noalloc_check("out", out, torch.float64, M * M, shape=(M, M))
    for name, t in (("voxels", voxels), ("u_dense", u_dense), ("out", out)):
        if t is not None and not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    torch = _torch()
    if out is None:
        out = torch.empty((M, M), dtype=torch.float64, device=voxels.device)
    if voxels.device != u_dense.device or out.device != voxels.device:
        raise ValueError("voxels, u_dense and out must be on the same CUDA device")
    s = stream if stream is not None else torch.cuda.current_stream(voxels.device)
    st = lib().gmt_homogenize_dense_noalloc(_ptr(voxels), res, physics, E, nu, k, _ptr(u_dense),
                                            _ptr(out), s.cuda_stream)
    _check(st, "gmt_homogenize_dense_noalloc")
    return out


def declared_symbols(header: str | None = None):
    """Function names declared in include/gmt.h."""
    import re
    if header is None:
        header = os.path.join(os.path.dirname(_HERE), "include", "gmt.h")
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gmt_[a-z_0-9]+)\s*\(", text)))
