"""Python binding of libvarsim (include/varsim.h): the GB300 (sm_103a)
Green's-function thermal solver with leakage and conductivity variation.

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch provides device memory and the current stream. Importing works
without a GPU (so the C ABI can be inspected); any call that needs the library
raises if libvarsim.so is missing -- there is no CPU fallback.

Maps are float32 CUDA tensors [n, n] (row-major, x fastest), power in W per
cell, temperatures in K above ambient.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

__all__ = [
    "VS_OK", "VS_ERR_INVALID_ARG", "VS_ERR_CUDA", "VS_ERR_OOM", "VS_ERR_NO_CONVERGENCE",
    "VS_ERR_RUNAWAY", "VS_ERR_NONFINITE", "VS_ERR_TIMEOUT", "VarsimError", "Stack", "Grid",
    "KernelOpts", "SolveParams", "Kernel", "Plan", "lib", "lib_path", "solve_steady",
    "solve_batch", "solve_batch_host", "HostPlan", "solve_transient", "hankel_radial", "EXPORTS",
    "solve_steady_noalloc",
    "tc_transform", "VS_PREC_FP32", "VS_PREC_BF16_SPLIT", "VS_ENGINE_AUTO",
    "VS_ENGINE_STREAMED", "VS_ENGINE_CLUSTER", "Model", "WarmPlan",
    "warm_features", "warm_target", "warm_apply", "VS_WARM_FIRST", "VS_WARM_PREDICT",
    "VS_WARM_SOLVE", "VS_WARM_ALL", "VS_LEAK_LAGGED", "VS_LEAK_IMPLICIT", "VS_MAX_WINDOW",
    "VS_CF_CONV", "VS_CF_IMPULSE", "solve_closed_form", "VS_COND_LINEAR", "VS_COND_KIRCHHOFF",
]

VS_OK, VS_ERR_INVALID_ARG, VS_ERR_CUDA, VS_ERR_OOM = 0, 1, 2, 3
VS_ERR_NO_CONVERGENCE, VS_ERR_RUNAWAY, VS_ERR_NONFINITE, VS_ERR_TIMEOUT = 4, 5, 6, 7
VS_PREC_FP32, VS_PREC_BF16_SPLIT = 0, 1
VS_ENGINE_AUTO, VS_ENGINE_STREAMED, VS_ENGINE_CLUSTER = 0, 1, 2
VS_WARM_FIRST, VS_WARM_PREDICT, VS_WARM_SOLVE, VS_WARM_ALL = 1, 2, 4, 7
VS_LEAK_LAGGED, VS_LEAK_IMPLICIT, VS_MAX_WINDOW = 0, 1, 256
VS_CF_CONV, VS_CF_IMPULSE = 0, 1
VS_COND_LINEAR, VS_COND_KIRCHHOFF = 0, 1
VS_STOP_UPDATE, VS_STOP_ESTIMATE = 0, 1
VS_MAX_LAYERS = 8

EXPORTS = [
    "vs_make_kernel", "vs_free_kernel", "vs_kernel_n", "vs_kernel_spectrum", "vs_kernel_radial",
    "vs_hankel_radial", "vs_solve_steady", "vs_plan_create", "vs_plan_run", "vs_plan_info",
    "vs_plan_launches", "vs_plan_free", "vs_solve_batch", "vs_solve_transient",
    "vs_status_string", "vs_last_error", "vs_version", "vs_solve_steady_noalloc",
    "vs_tc_transform", "vs_model_create", "vs_free_model", "vs_model_nparams",
    "vs_model_get_params", "vs_model_set_params", "vs_model_forward", "vs_model_loss_grad",
    "vs_model_train", "vs_model_save", "vs_model_load", "vs_warm_features", "vs_warm_target",
    "vs_warm_apply", "vs_solve_batch_host", "vs_host_plan_create", "vs_host_plan_run",
    "vs_host_plan_free", "vs_model_shape", "vs_warm_plan_create",
    "vs_warm_plan_run", "vs_warm_plan_launches", "vs_warm_plan_info", "vs_warm_plan_free",
    "vs_solve_transient_ex", "vs_solve_closed_form", "vs_plan_create_shaped", "vs_plan_shape",
    "vs_model_forward_tc",
]

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.path.join(_HERE, "libvarsim.so")


class VarsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class _Stack(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("thickness_m", C.c_double * VS_MAX_LAYERS),
                ("kappa_W_mK", C.c_double * VS_MAX_LAYERS), ("h_conv_W_m2K", C.c_double),
                ("heat_cap_J_m2K", C.c_double), ("spreader_layer", C.c_int),
                ("spreader_side_m", C.c_double)]


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int), ("die_m", C.c_double)]


class _KernelOpts(C.Structure):
    _fields_ = [("quad_nodes", C.c_int), ("rel_tol", C.c_double), ("dt_s", C.c_double)]


VS_MAX_LEAK_POINTS = 16


class _SolveParams(C.Structure):
    _fields_ = [("beta_per_K", C.c_double), ("alpha_per_K", C.c_double), ("tol_K", C.c_double),
                ("max_iter", C.c_int), ("precision", C.c_int), ("engine", C.c_int),
                ("conductivity", C.c_int), ("eta", C.c_double), ("t_amb_K", C.c_double),
                ("leak_points", C.c_int), ("leak_theta_K", C.c_double * VS_MAX_LEAK_POINTS),
                ("leak_g", C.c_double * VS_MAX_LEAK_POINTS), ("stop_rule", C.c_int)]


class _SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("residual_K", C.c_double),
                ("mu_W", C.c_double), ("fell_back", C.c_int)]


class _TransientOpts(C.Structure):
    _fields_ = [("window", C.c_int), ("leakage", C.c_int)]


class _BatchItem(C.Structure):
    _fields_ = [("k", C.c_void_p), ("p_dyn", C.c_void_p), ("p_leak0", C.c_void_p),
                ("s_kappa", C.c_void_p), ("theta", C.c_void_p), ("theta_init", C.c_void_p)]


_lib = None


def lib():
    """The loaded libvarsim (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libvarsim.so not found at %s: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    L = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.c_int, C.POINTER(C.c_double)
    sig = {
        "vs_make_kernel": (ip, [C.POINTER(_Stack), C.POINTER(_Grid), C.POINTER(_KernelOpts),
                                C.POINTER(vp), vp]),
        "vs_free_kernel": (None, [vp]),
        "vs_kernel_n": (ip, [vp]),
        "vs_kernel_spectrum": (ip, [vp, dp]),
        "vs_kernel_radial": (ip, [vp, dp, C.POINTER(ip)]),
        "vs_hankel_radial": (ip, [C.POINTER(_Stack), C.POINTER(_Grid), ip, vp, vp, ip, vp]),
        "vs_solve_steady": (ip, [vp, vp, vp, vp, C.POINTER(_SolveParams), vp,
                                 C.POINTER(_SolveInfo), vp]),
        "vs_solve_steady_noalloc": (ip, [vp, vp, vp, vp, C.POINTER(_SolveParams), vp,
                                         C.POINTER(_SolveInfo), vp]),
        "vs_plan_create": (ip, [C.POINTER(_BatchItem), ip, C.POINTER(_SolveParams),
                                C.POINTER(vp), vp]),
        "vs_plan_create_shaped": (ip, [C.POINTER(_BatchItem), ip, C.POINTER(_SolveParams), ip,
                                       C.POINTER(vp), vp]),
        "vs_plan_shape": (ip, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_double)]),
        "vs_plan_run": (ip, [vp, vp]),
        "vs_plan_info": (ip, [vp, C.POINTER(_SolveInfo), vp]),
        "vs_plan_launches": (ip, [vp]),
        "vs_plan_free": (None, [vp]),
        "vs_solve_batch": (ip, [C.POINTER(_BatchItem), ip, C.POINTER(_SolveParams),
                                C.POINTER(_SolveInfo), vp]),
        "vs_solve_batch_host": (ip, [vp, ip, vp, vp, vp, vp, C.POINTER(_SolveParams),
                                     C.POINTER(_SolveInfo), ip, vp]),
        "vs_host_plan_create": (ip, [vp, ip, ip, C.POINTER(_SolveParams), ip, C.POINTER(vp)]),
        "vs_host_plan_run": (ip, [vp, vp, vp, vp, vp, C.POINTER(_SolveInfo), vp]),
        "vs_host_plan_free": (None, [vp]),
        "vs_solve_transient": (ip, [vp, ip, vp, vp, vp, C.POINTER(_SolveParams), vp,
                                    C.POINTER(_SolveInfo), vp]),
        "vs_solve_transient_ex": (ip, [vp, ip, vp, vp, vp, C.POINTER(_SolveParams),
                                       C.POINTER(_TransientOpts), vp, C.POINTER(_SolveInfo), vp]),
        "vs_solve_closed_form": (ip, [vp, ip, vp, vp, vp, C.POINTER(_SolveParams), ip, vp,
                                      vp, vp]),
        "vs_tc_transform": (ip, [vp, vp, ip, ip, ip, vp]),
        "vs_model_create": (ip, [ip, ip, C.c_ulonglong, C.POINTER(vp)]),
        "vs_free_model": (None, [vp]),
        "vs_model_nparams": (C.c_longlong, [vp]),
        "vs_model_get_params": (ip, [vp, vp]),
        "vs_model_set_params": (ip, [vp, vp]),
        "vs_model_forward": (ip, [vp, vp, vp, ip, vp]),
        "vs_model_forward_tc": (ip, [vp, vp, vp, ip, vp]),
        "vs_model_loss_grad": (ip, [vp, vp, vp, ip, C.POINTER(C.c_double), vp, vp]),
        "vs_model_train": (ip, [vp, vp, vp, ip, ip, ip, C.c_float, C.c_ulonglong,
                                C.POINTER(C.c_double), vp]),
        "vs_model_save": (ip, [vp, C.c_char_p]),
        "vs_model_load": (ip, [C.c_char_p, C.POINTER(vp)]),
        "vs_warm_features": (ip, [vp, vp, vp, ip, ip, ip, vp, vp]),
        "vs_warm_target": (ip, [vp, vp, ip, ip, ip, vp, vp]),
        "vs_warm_apply": (ip, [vp, vp, ip, ip, ip, vp, vp]),
        "vs_model_shape": (ip, [vp, C.POINTER(ip), C.POINTER(ip)]),
        "vs_warm_plan_create": (ip, [vp, ip, vp, vp, vp, vp, vp, vp, vp, C.POINTER(_SolveParams),
                                     C.POINTER(vp), vp]),
        "vs_warm_plan_run": (ip, [vp, ip, vp]),
        "vs_warm_plan_launches": (ip, [vp]),
        "vs_warm_plan_info": (ip, [vp, C.POINTER(_SolveInfo), ip, C.POINTER(ip), vp]),
        "vs_warm_plan_free": (None, [vp]),
        "vs_status_string": (C.c_char_p, [ip]),
        "vs_last_error": (C.c_char_p, []),
        "vs_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int, what: str, ok=(VS_OK,)):
    if rc not in ok:
        L = lib()
        raise VarsimError(rc, "%s: %s: %s" % (what, L.vs_status_string(rc).decode(),
                                              L.vs_last_error().decode()))
    return rc


def _stream(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t, n: Optional[int] = None, name: str = "map", allow_none=False):
    import torch
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError("%s must be a float32 CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n is not None and tuple(t.shape[-2:]) != (n, n):
        raise ValueError("%s must be [..., %d, %d], got %s" % (name, n, n, tuple(t.shape)))
    return t.data_ptr()


@dataclass
class Stack:
    """Layer stack, top (source) layer first; SI units. spreader_layer > 0
    makes layers spreader_layer.. a spreader of side spreader_side_m wider
    than the die (vs_stack)."""
    thickness_m: Sequence[float] = (0.5e-3, 0.02e-3, 3.5e-3)
    kappa_W_mK: Sequence[float] = (130.0, 4.0, 400.0)
    h_conv_W_m2K: float = 2.0e4
    heat_cap_J_m2K: float = 1.63e6 * 0.5e-3
    spreader_layer: int = 0
    spreader_side_m: float = 0.0

    def _c(self) -> _Stack:
        s = _Stack()
        s.n_layers = len(self.thickness_m)
        for i, (t, k) in enumerate(zip(self.thickness_m, self.kappa_W_mK)):
            s.thickness_m[i] = t
            s.kappa_W_mK[i] = k
        s.h_conv_W_m2K = self.h_conv_W_m2K
        s.heat_cap_J_m2K = self.heat_cap_J_m2K
        s.spreader_layer = self.spreader_layer
        s.spreader_side_m = self.spreader_side_m
        return s


@dataclass
class Grid:
    n: int
    die_m: float

    def _c(self) -> _Grid:
        return _Grid(self.n, self.die_m)


@dataclass
class KernelOpts:
    quad_nodes: int = 256
    rel_tol: float = 1e-13
    dt_s: float = 0.0


@dataclass
class SolveParams:
    beta_per_K: float = 0.0275
    alpha_per_K: float = 0.3 * 1.3 / 318.15
    tol_K: float = 1e-4
    max_iter: int = 50
    precision: int = 0
    engine: int = 0
    conductivity: int = 0                 # VS_COND_LINEAR or VS_COND_KIRCHHOFF (eta, t_amb_K)
    eta: float = 0.0
    t_amb_K: float = 0.0
    leak_table: Optional[Sequence] = None  # [(theta_K, g), ...]: piecewise-linear leakage
    stop_rule: int = 0                    # VS_STOP_UPDATE or VS_STOP_ESTIMATE

    def _c(self) -> _SolveParams:
        c = _SolveParams(self.beta_per_K, self.alpha_per_K, self.tol_K, self.max_iter,
                         self.precision, self.engine, self.conductivity, self.eta, self.t_amb_K,
                         len(self.leak_table) if self.leak_table else 0)
        for i, (x, g) in enumerate(self.leak_table or ()):
            if i >= VS_MAX_LEAK_POINTS:
                break
            c.leak_theta_K[i] = x
            c.leak_g[i] = g
        c.stop_rule = self.stop_rule
        return c


def _info(i: _SolveInfo) -> dict:
    return {"status": i.status, "iterations": i.iterations, "residual_K": i.residual_K,
            "mu_W": i.mu_W, "fell_back": i.fell_back}


class Kernel:
    """Green's function of one (stack, grid) built on the GPU (vs_make_kernel)."""

    def __init__(self, stack: Stack, grid: Grid, opts: Optional[KernelOpts] = None, stream=None):
        L = lib()
        o = opts or KernelOpts()
        h = C.c_void_p()
        self.stack, self.grid, self.opts = stack, grid, o
        _check(L.vs_make_kernel(C.byref(stack._c()), C.byref(grid._c()),
                                C.byref(_KernelOpts(o.quad_nodes, o.rel_tol, o.dt_s)),
                                C.byref(h), _stream(stream)), "vs_make_kernel")
        self.handle = h.value

    @property
    def n(self) -> int:
        return lib().vs_kernel_n(self.handle)

    def spectrum(self):
        """FP64 cosine-basis kernel K[p][q] as a numpy array."""
        import numpy as np
        out = np.empty((self.n, self.n), dtype=np.float64)
        _check(lib().vs_kernel_spectrum(self.handle, out.ctypes.data_as(C.POINTER(C.c_double))),
               "vs_kernel_spectrum")
        return out

    def radial(self):
        """Top-layer radial table G1(cell*sqrt(m)), m = 0..m_max (numpy)."""
        import numpy as np
        m = C.c_int()
        _check(lib().vs_kernel_radial(self.handle, None, C.byref(m)), "vs_kernel_radial")
        out = np.empty(m.value + 1, dtype=np.float64)
        _check(lib().vs_kernel_radial(self.handle, out.ctypes.data_as(C.POINTER(C.c_double)),
                                      C.byref(m)), "vs_kernel_radial")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().vs_free_kernel(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hankel_radial(stack: Stack, grid: Grid, r, quad_nodes: int = 256, stream=None):
    """G1(r) for float64 CUDA radii r (vs_hankel_radial)."""
    import torch
    if r.dtype != torch.float64 or not r.is_cuda or not r.is_contiguous():
        raise TypeError("r must be a contiguous float64 CUDA tensor")
    out = torch.empty_like(r)
    _check(lib().vs_hankel_radial(C.byref(stack._c()), C.byref(grid._c()), quad_nodes,
                                  r.data_ptr(), out.data_ptr(), r.numel(), _stream(stream)),
           "vs_hankel_radial")
    return out


_SOLVE_OK = (VS_OK, VS_ERR_NO_CONVERGENCE, VS_ERR_RUNAWAY, VS_ERR_NONFINITE)


def solve_steady(kernel: Kernel, p_dyn, p_leak0, s_kappa=None, params: Optional[SolveParams] = None,
                 theta=None, stream=None):
    """One steady map. Returns (theta, info dict); raises on argument/CUDA errors."""
    import torch
    n = kernel.n
    prm = params or SolveParams()
    if theta is None:
        theta = torch.empty_like(p_dyn)
    info = _SolveInfo()
    _check(lib().vs_solve_steady(kernel.handle, _ptr(p_dyn, n, "p_dyn"),
                                 _ptr(p_leak0, n, "p_leak0"),
                                 _ptr(s_kappa, n, "s_kappa", allow_none=True), C.byref(prm._c()),
                                 _ptr(theta, n, "theta"), C.byref(info), _stream(stream)),
           "vs_solve_steady", ok=_SOLVE_OK)
    return theta, _info(info)


def tc_transform(x, inverse: bool = False, stream=None):
    """Split-precision tensor-core DCT-II (or its inverse) along the last axis
    of a float32 CUDA tensor [rows, n] (vs_tc_transform)."""
    import torch
    n = x.shape[-1]
    rows = x.numel() // n
    out = torch.empty_like(x)
    _check(lib().vs_tc_transform(_ptr(x, None, "x"), out.data_ptr(), rows, n, int(inverse),
                                 _stream(stream)), "vs_tc_transform")
    return out


def solve_steady_noalloc(kernel: Kernel, p_dyn, p_leak0, s_kappa=None,
                         params: Optional[SolveParams] = None, theta=None, stream=None):
    """vs_solve_steady_noalloc: same as solve_steady, but the library makes no
    device allocation (scratch is a fixed device array; n <= 512; calls that
    overlap on the GPU race). `theta` should be preallocated by callers that
    cannot allocate."""
    import torch
    n = kernel.n
    prm = params or SolveParams()
    if theta is None:
        theta = torch.empty_like(p_dyn)
    info = _SolveInfo()
    _check(lib().vs_solve_steady_noalloc(kernel.handle, _ptr(p_dyn, n, "p_dyn"),
                                         _ptr(p_leak0, n, "p_leak0"),
                                         _ptr(s_kappa, n, "s_kappa", allow_none=True),
                                         C.byref(prm._c()), _ptr(theta, n, "theta"),
                                         C.byref(info), _stream(stream)),
           "vs_solve_steady_noalloc", ok=_SOLVE_OK)
    return theta, _info(info)


class Plan:
    """A batched solve over many maps (vs_plan_*). One launch per run; with the
    cluster engine, one launch per distinct grid size (`launches`)."""

    def __init__(self, items, params: Optional[SolveParams] = None, stream=None, shape: int = 0):
        """items: sequence of (Kernel, p_dyn, p_leak0, s_kappa or None, theta
        [, theta_init or None]). shape: 0 = tuned or cached launch shape, else
        forced (vs_plan_create_shaped)."""
        prm = params or SolveParams()
        arr = (_BatchItem * len(items))()
        self._keep = []
        for i, item in enumerate(items):
            k, pd, pl, sk, th = item[:5]
            ti = item[5] if len(item) > 5 else None
            n = k.n
            arr[i] = _BatchItem(k.handle, _ptr(pd, n, "p_dyn"), _ptr(pl, n, "p_leak0"),
                                _ptr(sk, n, "s_kappa", allow_none=True), _ptr(th, n, "theta"),
                                _ptr(ti, n, "theta_init", allow_none=True))
            self._keep.append(item)
        h = C.c_void_p()
        _check(lib().vs_plan_create_shaped(arr, len(items), C.byref(prm._c()), int(shape),
                                           C.byref(h), _stream(stream)), "vs_plan_create_shaped")
        self.handle = h.value
        self.n_items = len(items)

    def shape(self) -> dict:
        """The launch shape and the candidates the autotuner timed (vs_plan_shape)."""
        sh, nt = C.c_int(), C.c_int()
        cs, ms = (C.c_int * 8)(), (C.c_double * 8)()
        _check(lib().vs_plan_shape(self.handle, C.byref(sh), C.byref(nt), cs, ms), "vs_plan_shape")
        return {"shape": sh.value, "timed": {cs[i]: ms[i] for i in range(nt.value)}}

    def run(self, stream=None):
        _check(lib().vs_plan_run(self.handle, _stream(stream)), "vs_plan_run")

    def info(self, stream=None):
        arr = (_SolveInfo * self.n_items)()
        rc = lib().vs_plan_info(self.handle, arr, _stream(stream))
        _check(rc, "vs_plan_info", ok=_SOLVE_OK)
        return [_info(a) for a in arr]

    @property
    def launches(self) -> int:
        return lib().vs_plan_launches(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().vs_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(items, params: Optional[SolveParams] = None, stream=None):
    """Create a plan, run it once, return the per-map info list."""
    p = Plan(items, params, stream)
    try:
        p.run(stream)
        return p.info(stream)
    finally:
        p.close()


def _host_ptr(t, n: int, count: int, name: str, allow_none=False):
    import torch
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32:
        raise TypeError("%s must be a float32 CPU tensor" % name)
    if not t.is_contiguous() or tuple(t.shape) != (count, n, n):
        raise ValueError("%s must be contiguous [%d, %d, %d], got %s"
                         % (name, count, n, n, tuple(t.shape)))
    return t.data_ptr()


def solve_batch_host(kernel: Kernel, p_dyn, p_leak0, s_kappa=None, theta=None,
                     params: Optional[SolveParams] = None, chunk_maps: int = 0, stream=None):
    """vs_solve_batch_host: host (CPU) tensors [count, n, n] in and out; the
    copies overlap the solve chunk by chunk (use pinned tensors for overlap).
    Returns (theta, info list)."""
    import torch
    n, count = kernel.n, p_dyn.shape[0]
    prm = params or SolveParams()
    if theta is None:
        theta = torch.empty((count, n, n), dtype=torch.float32, pin_memory=p_dyn.is_pinned())
    info = (_SolveInfo * count)()
    _check(lib().vs_solve_batch_host(kernel.handle, count, _host_ptr(p_dyn, n, count, "p_dyn"),
                                     _host_ptr(p_leak0, n, count, "p_leak0"),
                                     _host_ptr(s_kappa, n, count, "s_kappa", allow_none=True),
                                     _host_ptr(theta, n, count, "theta"), C.byref(prm._c()), info,
                                     int(chunk_maps), _stream(stream)),
           "vs_solve_batch_host", ok=_SOLVE_OK)
    return theta, [_info(i) for i in info]


class HostPlan:
    """vs_host_plan_*: the host-memory batch solve as a reusable object (streams,
    device buffer slots and chunk plans made once); run() takes host (CPU)
    tensors [count, n, n] and returns (theta, info list)."""

    def __init__(self, kernel: Kernel, count: int, with_s: bool = True,
                 params: Optional[SolveParams] = None, chunk_maps: int = 0):
        self.kernel, self.count, self.with_s = kernel, count, bool(with_s)
        prm = params or SolveParams()
        h = C.c_void_p()
        _check(lib().vs_host_plan_create(kernel.handle, count, int(self.with_s), C.byref(prm._c()),
                                         int(chunk_maps), C.byref(h)), "vs_host_plan_create")
        self.handle = h.value

    def run(self, p_dyn, p_leak0, s_kappa=None, theta=None, stream=None):
        import torch
        n, count = self.kernel.n, self.count
        if theta is None:
            theta = torch.empty((count, n, n), dtype=torch.float32, pin_memory=p_dyn.is_pinned())
        info = (_SolveInfo * count)()
        _check(lib().vs_host_plan_run(self.handle, _host_ptr(p_dyn, n, count, "p_dyn"),
                                      _host_ptr(p_leak0, n, count, "p_leak0"),
                                      _host_ptr(s_kappa, n, count, "s_kappa", allow_none=True),
                                      _host_ptr(theta, n, count, "theta"), info, _stream(stream)),
               "vs_host_plan_run", ok=_SOLVE_OK)
        return theta, [_info(i) for i in info]

    def close(self):
        if getattr(self, "handle", None):
            lib().vs_host_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_transient(kernel: Kernel, p_dyn_trace, p_leak0, s_kappa=None,
                    params: Optional[SolveParams] = None, theta_trace=None, stream=None,
                    window: int = 0, leakage: int = VS_LEAK_LAGGED):
    """Transient over the trace [n_steps, n, n]; returns (theta_trace, info).
    window: 0 untruncated, K >= 1 step responses settled from age K on;
    leakage: VS_LEAK_LAGGED or VS_LEAK_IMPLICIT (vs_solve_transient_ex)."""
    import torch
    n = kernel.n
    prm = params or SolveParams()
    steps = p_dyn_trace.shape[0]
    if theta_trace is None:
        theta_trace = torch.empty_like(p_dyn_trace)
    info = _SolveInfo()
    opts = _TransientOpts(window, leakage)
    _check(lib().vs_solve_transient_ex(kernel.handle, steps, _ptr(p_dyn_trace, n, "p_dyn_trace"),
                                       _ptr(p_leak0, n, "p_leak0"),
                                       _ptr(s_kappa, n, "s_kappa", allow_none=True),
                                       C.byref(prm._c()), C.byref(opts),
                                       _ptr(theta_trace, n, "theta_trace"),
                                       C.byref(info), _stream(stream)),
           "vs_solve_transient_ex", ok=_SOLVE_OK)
    return theta_trace, _info(info)


def solve_closed_form(kernel: Kernel, p_dyn, p_leak0, s_kappa=None,
                      params: Optional[SolveParams] = None, mode: int = VS_CF_CONV,
                      theta=None, stream=None, info: bool = True):
    """One-shot closed form (vs_solve_closed_form) of maps [B, n, n]; returns
    (theta, infos) -- infos is None with info=False (no synchronisation)."""
    import torch
    n = kernel.n
    prm = params or SolveParams()
    B = p_dyn.shape[0]
    if theta is None:
        theta = torch.empty_like(p_dyn)
    arr = (_SolveInfo * B)() if info else None
    _check(lib().vs_solve_closed_form(kernel.handle, B, _ptr(p_dyn, n, "p_dyn"),
                                      _ptr(p_leak0, n, "p_leak0"),
                                      _ptr(s_kappa, n, "s_kappa", allow_none=True),
                                      C.byref(prm._c()), mode, _ptr(theta, n, "theta"),
                                      C.cast(arr, C.c_void_p) if info else None, _stream(stream)),
           "vs_solve_closed_form", ok=_SOLVE_OK)
    return theta, ([_info(a) for a in arr] if info else None)


# --------------------------------------------------------------------------
# Learned warm start (vs_model_*, vs_warm_*)
# --------------------------------------------------------------------------

class Model:
    """The warm-start U-Net (vs_model_create); parameters live on the GPU."""

    def __init__(self, base_channels: int = 16, resolution: int = 64, seed: int = 1,
                 _handle=None):
        if _handle is not None:
            self.handle = _handle
        else:
            h = C.c_void_p()
            _check(lib().vs_model_create(base_channels, resolution, seed, C.byref(h)),
                   "vs_model_create")
            self.handle = h.value
        self.base_channels = base_channels
        self.resolution = resolution

    @classmethod
    def load(cls, path: str):
        h = C.c_void_p()
        _check(lib().vs_model_load(path.encode(), C.byref(h)), "vs_model_load")
        c, r = C.c_int(), C.c_int()
        _check(lib().vs_model_shape(h, C.byref(c), C.byref(r)), "vs_model_shape")
        return cls(c.value, r.value, _handle=h.value)

    def save(self, path: str):
        _check(lib().vs_model_save(self.handle, path.encode()), "vs_model_save")

    @property
    def nparams(self) -> int:
        return int(lib().vs_model_nparams(self.handle))

    def get_params(self):
        import numpy as np
        out = np.empty(self.nparams, dtype=np.float32)
        _check(lib().vs_model_get_params(self.handle, out.ctypes.data), "vs_model_get_params")
        return out

    def set_params(self, p):
        import numpy as np
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.size == self.nparams
        _check(lib().vs_model_set_params(self.handle, a.ctypes.data), "vs_model_set_params")

    def forward(self, x, stream=None, tensor_cores: bool = False):
        """y = net(x); tensor_cores: the convolutions as tcgen05 implicit GEMMs
        (BF16 activations, vs_model_forward_tc), as the warm plan runs them."""
        import torch
        y = torch.empty(x.shape[0], 1, self.resolution, self.resolution, device=x.device)
        fn = lib().vs_model_forward_tc if tensor_cores else lib().vs_model_forward
        _check(fn(self.handle, _ptr(x, None, "x"), y.data_ptr(), x.shape[0], _stream(stream)),
               "vs_model_forward")
        return y

    def loss_grad(self, x, t, stream=None):
        import numpy as np
        loss = C.c_double()
        g = np.empty(self.nparams, dtype=np.float32)
        _check(lib().vs_model_loss_grad(self.handle, _ptr(x, None, "x"), _ptr(t, None, "t"),
                                        x.shape[0], C.byref(loss), g.ctypes.data,
                                        _stream(stream)), "vs_model_loss_grad")
        return loss.value, g

    def train(self, x, t, epochs: int = 8, batch: int = 64, lr: float = 1e-3, seed: int = 7,
              stream=None) -> float:
        loss = C.c_double()
        _check(lib().vs_model_train(self.handle, _ptr(x, None, "x"), _ptr(t, None, "t"),
                                    x.shape[0], epochs, batch, lr, seed, C.byref(loss),
                                    _stream(stream)), "vs_model_train")
        return loss.value

    def close(self):
        if getattr(self, "handle", None):
            lib().vs_free_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def warm_features(theta1, p_leak0, s_kappa, resolution: int, stream=None):
    import torch
    B, n = theta1.shape[0], theta1.shape[-1]
    x = torch.empty(B, 3, resolution, resolution, device=theta1.device)
    _check(lib().vs_warm_features(_ptr(theta1, n, "theta1"), _ptr(p_leak0, n, "p_leak0"),
                                  _ptr(s_kappa, n, "s", allow_none=True), B, n, resolution,
                                  x.data_ptr(), _stream(stream)), "vs_warm_features")
    return x


def warm_target(theta_star, theta1, resolution: int, stream=None):
    import torch
    B, n = theta1.shape[0], theta1.shape[-1]
    t = torch.empty(B, 1, resolution, resolution, device=theta1.device)
    _check(lib().vs_warm_target(_ptr(theta_star, n, "theta_star"), _ptr(theta1, n, "theta1"), B,
                                n, resolution, t.data_ptr(), _stream(stream)), "vs_warm_target")
    return t


def warm_apply(theta1, y, out=None, stream=None):
    import torch
    B, n = theta1.shape[0], theta1.shape[-1]
    R = y.shape[-1]
    if out is None:
        out = torch.empty_like(theta1)
    _check(lib().vs_warm_apply(_ptr(theta1, n, "theta1"), _ptr(y, None, "y"), B, n, R,
                               out.data_ptr(), _stream(stream)), "vs_warm_apply")
    return out


class WarmPlan:
    """Warm-started batched solve of maps [B, n, n] with one kernel
    (vs_warm_plan_*): a one-iteration solve gives the first iterate theta1;
    the network predicts the remaining correction at reduced resolution; the
    batched solve starts from theta_init = theta1 + correction. Maps that do
    not converge from the warm start are solved again from theta_0 = 0 when
    `info(fallback=True)` is read."""

    def __init__(self, kernel: Kernel, p_dyn, p_leak0, s_kappa, theta, model: Model,
                 params: Optional[SolveParams] = None, stream=None):
        import torch
        prm = params or SolveParams()
        n = kernel.n
        self.B, self.stream = p_dyn.shape[0], stream
        self.theta1 = torch.empty_like(p_dyn)
        self.theta_init = torch.empty_like(p_dyn)
        self._keep = (kernel, p_dyn, p_leak0, s_kappa, theta, model)
        h = C.c_void_p()
        _check(lib().vs_warm_plan_create(
            kernel.handle, self.B, _ptr(p_dyn, n, "p_dyn"), _ptr(p_leak0, n, "p_leak0"),
            _ptr(s_kappa, n, "s_kappa", allow_none=True), _ptr(theta, n, "theta"),
            _ptr(self.theta1, n, "theta1"), _ptr(self.theta_init, n, "theta_init"),
            model.handle, C.byref(prm._c()), C.byref(h), _stream(stream)), "vs_warm_plan_create")
        self.handle = h.value
        self.fallbacks = 0

    @property
    def launches(self) -> int:
        return lib().vs_warm_plan_launches(self.handle)

    def run(self, stream=None, stages: int = VS_WARM_ALL):
        st = stream if stream is not None else self.stream
        _check(lib().vs_warm_plan_run(self.handle, stages, _stream(st)), "vs_warm_plan_run")

    def info(self, fallback: bool = True):
        arr = (_SolveInfo * self.B)()
        fell = (C.c_int * self.B)()
        rc = lib().vs_warm_plan_info(self.handle, arr, int(fallback), fell, _stream(self.stream))
        _check(rc, "vs_warm_plan_info", ok=_SOLVE_OK)
        infos = [_info(a) for a in arr]
        self.fallbacks = 0
        for i in range(self.B):
            if fell[i]:
                infos[i]["fell_back"] = True
                self.fallbacks += 1
        return infos

    def close(self):
        if getattr(self, "handle", None):
            lib().vs_warm_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
