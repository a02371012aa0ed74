"""Python binding of the hj C ABI (include/hj.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels
of libhj_gb300.so.  There is no CPU fallback.  If the library is missing or
no CUDA device is present, the calls raise.

The module-level functions carry the C names (hj_grid_create, hj_solve, ...).
`Grid` and `solve_batch` are thin conveniences over them, and they accept
numpy arrays and torch CUDA tensors for the value field.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhj_gb300.so")

HJ_OK, HJ_ERR_ARG, HJ_ERR_OOM, HJ_ERR_CUDA = 0, 1, 2, 3
HJ_ERR_NOT_CONVERGED, HJ_ERR_STATE, HJ_ERR_ABORTED, HJ_ERR_DIVERGED = 4, 5, 6, 7
HJ_DRIFT, HJ_QUAD_Z, HJ_QUAD_X4 = 0, 1, 2
HJ_FIRST, HJ_ENO2, HJ_WENO5 = 1, 2, 5
HJ_CLAMP_VI, HJ_CLAMP_MONOTONE = 0, 1
HJ_COLD, HJ_WARM = 0, 1
HJ_ORDER_FIFO, HJ_ORDER_SHORTEST = 0, 1
HJ_MAX_DIM = 4

STATUS_NAMES = {0: "HJ_OK", 1: "HJ_ERR_ARG", 2: "HJ_ERR_OOM", 3: "HJ_ERR_CUDA",
                4: "HJ_ERR_NOT_CONVERGED", 5: "HJ_ERR_STATE", 6: "HJ_ERR_ABORTED",
                7: "HJ_ERR_DIVERGED"}
MODELS = {"drift": HJ_DRIFT, "quad_z": HJ_QUAD_Z, "quad_x4": HJ_QUAD_X4}


class HJError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class hj_solve_opts(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("tol", ctypes.c_double), ("check_dt", ctypes.c_double),
                ("max_steps", ctypes.c_longlong), ("fixed_steps", ctypes.c_longlong),
                ("max_wall_ms", ctypes.c_double), ("clamp", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("band", ctypes.c_double),
                ("autotune", ctypes.c_int), ("band_margin", ctypes.c_int),
                ("local_tol", ctypes.c_double), ("local_margin", ctypes.c_int)]


class hj_solve_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("t", ctypes.c_double),
                ("residual", ctypes.c_double), ("dt", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("converged", ctypes.c_int),
                ("windows", ctypes.c_longlong), ("stepped", ctypes.c_double)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.POINTER
_vp, _i, _d, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong


class hj_request(ctypes.Structure):
    _fields_ = [("ndim", _i), ("n", _i * HJ_MAX_DIM), ("lo", _d * HJ_MAX_DIM),
                ("hi", _d * HJ_MAX_DIM), ("model", _i), ("params", _d * 8), ("nparams", _i),
                ("d_lo", _d * HJ_MAX_DIM), ("d_hi", _d * HJ_MAX_DIM), ("nd", _i),
                ("con_ball", _i), ("con_a", _d * HJ_MAX_DIM), ("con_b", _d * HJ_MAX_DIM),
                ("mode", _i), ("key", _ll), ("opts", hj_solve_opts), ("coarse_n", _i),
                ("coarse_n2", _i), ("coarse_scheme", _i)]


class hj_server_stats(ctypes.Structure):
    _fields_ = [("submitted", _ll), ("admitted", _ll), ("completed", _ll), ("failed", _ll),
                ("rejected", _ll), ("warm_starts", _ll), ("cold_starts", _ll),
                ("evictions", _ll), ("rounds", _ll), ("bytes_in_use", _ll),
                ("peak_bytes", _ll), ("active", _ll), ("queued", _ll), ("p50_ms", _d),
                ("p99_ms", _d), ("updates", _d), ("busy_ms", _d), ("translated_starts", _ll)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}

# C signatures: name -> (restype, argtypes)
SIGNATURES = {
    "hj_default_opts": (None, [_P(hj_solve_opts)]),
    "hj_grid_create": (_i, [_P(_vp), _i, _P(_i), _P(_d), _P(_d), _vp]),
    "hj_grid_destroy": (None, [_vp]),
    "hj_set_stream": (_i, [_vp, _vp]),
    "hj_set_dynamics": (_i, [_vp, _i, _P(_d), _i]),
    "hj_set_constraint": (_i, [_vp, _P(_d), _P(_d)]),
    "hj_set_constraint_ball": (_i, [_vp, _P(_d), _d]),
    "hj_set_constraint_field": (_i, [_vp, _vp, _i]),
    "hj_set_disturbance_bound": (_i, [_vp, _P(_d), _P(_d), _i]),
    "hj_set_disturbance_field": (_i, [_vp, _vp, _vp, _i, _i]),
    "hj_solve": (_i, [_vp, _i, _P(hj_solve_opts), _P(hj_solve_stats)]),
    "hj_solve_batch": (_i, [_P(_vp), _i, _P(_i), _P(hj_solve_opts), _i, _P(hj_solve_stats),
                            _P(_i)]),
    "hj_prolong": (_i, [_vp, _vp]),
    "hj_translate": (_i, [_vp, _vp, _P(_d)]),
    "hj_set_jit": (None, [_i]),
    "hj_jit_kernels": (_ll, []),
    "hj_jit_pending": (_ll, []),
    "hj_jit_check": (_i, [_i, _P(_i), _i, _i, _i]),
    "hj_jit_check_tiles": (_i, [_i, _P(_i), _i, _i, _i]),
    "hj_jit_check_resources": (_i, [_i, _P(_i), _i, _i, _i, ctypes.c_uint, _P(_i), _P(_i)]),
    "hj_jit_check_group": (_i, [_i, _P(_i), _P(_i), _P(_i), _P(_i)]),
    "hj_set_launch_shape": (_i, [_vp, _i, _i]),
    "hj_set_allocator": (_i, [_vp, _vp, _vp]),
    "hj_get_launch_shape": (_i, [_vp, _P(_i), _P(_i)]),
    "hj_set_value": (_i, [_vp, _vp, _i]),
    "hj_get_value": (_i, [_vp, _vp, _i]),
    "hj_query_value": (_i, [_vp, _i, _P(_d), _P(_d)]),
    "hj_query_gradient": (_i, [_vp, _i, _P(_d), _P(_d)]),
    "hj_safety_filter": (_i, [_P(_vp), _i, _P(_i), _P(_i), _i, _i, ctypes.c_longlong, _vp, _vp,
                              _d, _vp, _vp, _vp, _i]),
    "hj_alpha": (_i, [_vp, _P(_d)]),
    "hj_autotune": (_i, [_vp, _i, _P(_i)]),
    "hj_grid_points": (_ll, [_vp]),
    "hj_last_error": (ctypes.c_char_p, []),
    "hj_kernel_launches": (ctypes.c_ulonglong, []),
    "hj_server_create": (_i, [_P(_vp), _ll, _i, _vp]),
    "hj_server_destroy": (None, [_vp]),
    "hj_server_submit": (_i, [_vp, _P(hj_request), _P(_ll)]),
    "hj_server_poll": (_i, [_vp, _ll, _P(_i), _P(_i), _P(hj_solve_stats)]),
    "hj_server_wait": (_i, [_vp, _ll, _d, _P(_i), _P(hj_solve_stats)]),
    "hj_server_get_value": (_i, [_vp, _ll, _vp, _i]),
    "hj_server_release": (_i, [_vp, _ll]),
    "hj_server_cancel": (_i, [_vp, _ll]),
    "hj_server_get_stats": (_i, [_vp, _P(hj_server_stats)]),
    "hj_server_set_policy": (_i, [_vp, _i, _ll]),
    "hj_server_set_translated_starts": (_i, [_vp, _i]),
    "hj_solve_fixed_static": (_i, [_i, _P(_i), _P(_d), _P(_d), _i, _P(_d), _i, _P(_d), _P(_d),
                                   _i, _P(_d), _P(_d), _i, _i, _d, _ll, _i, _vp, _vp]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libhj_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libhj_gb300.so is not built: run paper_2101_05916_gb300.build.build() "
                "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def hj_last_error() -> str:
    m = lib().hj_last_error()
    return m.decode() if m else ""


def _check(status: int) -> int:
    if status != HJ_OK:
        raise HJError(status, hj_last_error())
    return status


def _darr(vals: Sequence[float]):
    a = (ctypes.c_double * max(1, len(vals)))()
    for i, v in enumerate(vals):
        a[i] = float(v)
    return a


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


# ---------------------------------------------------------------- C names

def hj_default_opts() -> hj_solve_opts:
    o = hj_solve_opts()
    lib().hj_default_opts(ctypes.byref(o))
    return o


def hj_grid_create(n: Sequence[int], lo: Sequence[float], hi: Sequence[float], stream=None) -> int:
    h = ctypes.c_void_p()
    nd = len(n)
    na = (ctypes.c_int * nd)(*[int(v) for v in n])
    _check(lib().hj_grid_create(ctypes.byref(h), nd, na, _darr(lo), _darr(hi),
                                _stream_handle(stream)))
    return h.value


def hj_grid_destroy(g: int) -> None:
    lib().hj_grid_destroy(g)


def hj_set_stream(g: int, stream) -> None:
    _check(lib().hj_set_stream(g, _stream_handle(stream)))


def hj_set_dynamics(g: int, model, params: Sequence[float]) -> None:
    m = MODELS[model] if isinstance(model, str) else int(model)
    _check(lib().hj_set_dynamics(g, m, _darr(params), len(params)))


def hj_set_constraint(g: int, box_lo: Sequence[float], box_hi: Sequence[float]) -> None:
    _check(lib().hj_set_constraint(g, _darr(box_lo), _darr(box_hi)))


def hj_set_constraint_ball(g: int, centre: Sequence[float], radius: float) -> None:
    _check(lib().hj_set_constraint_ball(g, _darr(centre), float(radius)))


def hj_set_constraint_field(g: int, l) -> None:
    """Constraint as its margin l on the grid: numpy array with one value per
    node (host), or a flat float32 CUDA tensor of npts values."""
    npts = lib().hj_grid_points(g)
    try:
        import torch
        if isinstance(l, torch.Tensor):
            if l.numel() != npts:
                raise ValueError("l must hold one value per node")
            _check(lib().hj_set_constraint_field(g, l.data_ptr(), 1))
            return
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(l, dtype=np.float32)
    if a.size != npts:
        raise ValueError("l must hold one value per node")
    _check(lib().hj_set_constraint_field(g, a.ctypes.data, 0))


def hj_set_disturbance_bound(g: int, d_lo: Sequence[float], d_hi: Sequence[float]) -> None:
    _check(lib().hj_set_disturbance_bound(g, _darr(d_lo), _darr(d_hi), len(d_lo)))


def hj_set_disturbance_field(g: int, d_lo, d_hi) -> None:
    """State-dependent disturbance box: d_lo, d_hi of shape (nd,) + grid shape
    (numpy, host) or flat float32 CUDA tensors of nd * npts values."""
    try:
        import torch
        if isinstance(d_lo, torch.Tensor):
            npts = lib().hj_grid_points(g)
            nd = d_lo.numel() // npts
            _check(lib().hj_set_disturbance_field(g, d_lo.data_ptr(), d_hi.data_ptr(), nd, 1))
            return
    except ImportError:  # pragma: no cover
        pass
    lo = np.ascontiguousarray(d_lo, dtype=np.float32)
    hi = np.ascontiguousarray(d_hi, dtype=np.float32)
    npts = lib().hj_grid_points(g)
    nd = lo.size // npts
    if lo.size != nd * npts or hi.size != lo.size:
        raise ValueError("field must hold nd * npts values")
    _check(lib().hj_set_disturbance_field(g, lo.ctypes.data, hi.ctypes.data, nd, 0))


def make_opts(scheme: int = HJ_WENO5, cfl: float = 0.5, dt: float = 0.0, tol: float = 1e-4,
              check_dt: float = 0.1, max_steps: int = 1000000, fixed_steps: int = 0,
              max_wall_ms: float = 0.0, clamp: int = HJ_CLAMP_VI,
              use_graph: bool = True, band: float = 0.0,
              autotune: bool = False, band_margin: int = 0, local_tol: float = 0.0,
              local_margin: int = 1) -> hj_solve_opts:
    return hj_solve_opts(scheme, cfl, dt, tol, check_dt, max_steps, fixed_steps, max_wall_ms,
                         clamp, 1 if use_graph else 0, band, 1 if autotune else 0, band_margin,
                         local_tol, local_margin)


def hj_solve(g: int, mode: int = HJ_COLD, opts: Optional[hj_solve_opts] = None,
             raise_on_error: bool = True):
    """Returns (status, stats dict)."""
    st = hj_solve_stats()
    rc = lib().hj_solve(g, int(mode), ctypes.byref(opts) if opts is not None else None,
                        ctypes.byref(st))
    if raise_on_error and rc not in (HJ_OK, HJ_ERR_NOT_CONVERGED):
        raise HJError(rc, hj_last_error())
    return rc, st.as_dict()


def hj_solve_batch(grids: Sequence[int], modes: Sequence[int],
                   opts: Optional[Sequence[hj_solve_opts]] = None):
    """Returns (first status, per-grid statuses, per-grid stats dicts)."""
    n = len(grids)
    ga = (ctypes.c_void_p * n)(*grids)
    ma = (ctypes.c_int * n)(*[int(m) for m in modes])
    if opts is None:
        oa, oc = None, 0
    else:
        oa = (hj_solve_opts * len(opts))(*opts)
        oc = len(opts)
    sa = (hj_solve_stats * n)()
    ra = (ctypes.c_int * n)()
    rc = lib().hj_solve_batch(ga, n, ma, oa, oc, sa, ra)
    if rc not in (HJ_OK, HJ_ERR_NOT_CONVERGED) and all(r == HJ_OK for r in ra):
        raise HJError(rc, hj_last_error())
    return rc, list(ra), [s.as_dict() for s in sa]


def hj_prolong(coarse: int, fine: int) -> None:
    _check(lib().hj_prolong(coarse, fine))


def _field_ptr(buf, npts: int, writable: bool):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor of npts floats."""
    try:
        import torch
        if isinstance(buf, torch.Tensor):
            if buf.dtype != torch.float32 or not buf.is_contiguous() or buf.numel() != npts:
                raise ValueError("need a contiguous float32 tensor of %d values" % npts)
            return buf.data_ptr(), 1 if buf.is_cuda else 0, buf
    except ImportError:  # pragma: no cover
        pass
    a = np.asarray(buf)
    if a.dtype != np.float32 or not a.flags.c_contiguous or a.size != npts:
        raise ValueError("need a C-contiguous float32 array of %d values" % npts)
    if writable and not a.flags.writeable:
        raise ValueError("array is read-only")
    return a.ctypes.data, 0, a


def hj_set_value(g: int, src) -> None:
    npts = lib().hj_grid_points(g)
    if isinstance(src, np.ndarray) and src.dtype != np.float32:
        src = np.ascontiguousarray(src, dtype=np.float32)
    ptr, dev, keep = _field_ptr(src, npts, False)
    _check(lib().hj_set_value(g, ptr, dev))
    del keep


def hj_get_value(g: int, dst) -> None:
    npts = lib().hj_grid_points(g)
    ptr, dev, keep = _field_ptr(dst, npts, True)
    _check(lib().hj_get_value(g, ptr, dev))
    del keep


def _points(xs, ndim):
    a = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, ndim)
    return a, a.ctypes.data_as(_P(_d))


def hj_query_value(g: int, xs, ndim: int) -> np.ndarray:
    a, p = _points(xs, ndim)
    out = np.zeros(a.shape[0])
    _check(lib().hj_query_value(g, a.shape[0], p, out.ctypes.data_as(_P(_d))))
    return out


def hj_query_gradient(g: int, xs, ndim: int) -> np.ndarray:
    a, p = _points(xs, ndim)
    out = np.zeros_like(a)
    _check(lib().hj_query_gradient(g, a.shape[0], p, out.ctypes.data_as(_P(_d))))
    return out


def hj_safety_filter(grids, axes, ctrl_index, states, u_perf, level: float = 0.0):
    """Safety filter over decomposed subsystem grids (see hj.h).  grids:
    Grid objects or handles; axes[k]: state index of each axis of grid k;
    ctrl_index[k]: control driven by grid k (-1: none).  states (nq,
    state_dim) and u_perf (nq, ctrl_dim): numpy (host) or float64 CUDA
    tensors.  Returns (u, w, active) of the same kind."""
    hs = [g.handle if hasattr(g, "handle") else g for g in grids]
    k = len(hs)
    ax = np.zeros((k, HJ_MAX_DIM), dtype=np.int32)
    for i, a in enumerate(axes):
        ax[i, :len(a)] = a
    ci = np.ascontiguousarray(ctrl_index, dtype=np.int32)
    harr = (_vp * k)(*hs)
    try:
        import torch
        if isinstance(states, torch.Tensor):
            nq, sd = states.shape
            cd = u_perf.shape[1]
            u = torch.empty_like(u_perf)
            w = torch.empty(nq, dtype=torch.float64, device=states.device)
            act = torch.empty(nq, dtype=torch.int32, device=states.device)
            _check(lib().hj_safety_filter(harr, k, ax.ctypes.data_as(_P(_i)),
                                          ci.ctypes.data_as(_P(_i)), sd, cd, nq,
                                          states.data_ptr(), u_perf.data_ptr(), float(level),
                                          u.data_ptr(), w.data_ptr(), act.data_ptr(), 1))
            return u, w, act
    except ImportError:  # pragma: no cover
        pass
    x = np.ascontiguousarray(states, dtype=np.float64)
    up = np.ascontiguousarray(u_perf, dtype=np.float64)
    nq, sd = x.shape
    cd = up.shape[1]
    u = np.empty_like(up)
    w = np.empty(nq, dtype=np.float64)
    act = np.empty(nq, dtype=np.int32)
    _check(lib().hj_safety_filter(harr, k, ax.ctypes.data_as(_P(_i)), ci.ctypes.data_as(_P(_i)),
                                  sd, cd, nq, x.ctypes.data, up.ctypes.data, float(level),
                                  u.ctypes.data, w.ctypes.data, act.ctypes.data, 0))
    return u, w, act


def hj_set_jit(enable: bool) -> None:
    lib().hj_set_jit(1 if enable else 0)


def hj_jit_kernels() -> int:
    return int(lib().hj_jit_kernels())


def hj_jit_pending() -> int:
    return int(lib().hj_jit_pending())


def hj_jit_check(n: Sequence[int], model, scheme: int, threads: int = 256) -> None:
    """Compile the shape-specialised stage source for this grid shape, model
    and scheme with NVRTC (no device needed); raises HJError on failure."""
    m = MODELS[model] if isinstance(model, str) else int(model)
    arr = (_i * len(n))(*[int(v) for v in n])
    _check(lib().hj_jit_check(len(n), arr, m, int(scheme), int(threads)))


def hj_jit_check_resources(n: Sequence[int], model, scheme: int, threads: int = 256,
                           con_axes: Sequence[int] = (0,)):
    """(registers per thread, spill-store bytes per thread), the largest over
    the three shape-specialised stage kernels, from ptxas through NVRTC (no
    device needed), with a box constraint on the axes con_axes."""
    m = MODELS[model] if isinstance(model, str) else int(model)
    arr = (_i * len(n))(*[int(v) for v in n])
    mask = 0
    for a in con_axes:
        mask |= 1 << int(a)
    regs, spill = _i(), _i()
    _check(lib().hj_jit_check_resources(len(n), arr, m, int(scheme), int(threads), mask,
                                        ctypes.byref(regs), ctypes.byref(spill)))
    return regs.value, spill.value


def hj_jit_check_tiles(n: Sequence[int], model, scheme: int, tile_rows: int) -> None:
    """The same for the row-tile stage kernels of tile_rows lines per block."""
    m = MODELS[model] if isinstance(model, str) else int(model)
    arr = (_i * len(n))(*[int(v) for v in n])
    _check(lib().hj_jit_check_tiles(len(n), arr, m, int(scheme), int(tile_rows)))


def hj_jit_check_group(grids) -> None:
    """Compile the group kernels of a batch with NVRTC (no device needed);
    grids: a list of (shape, model, scheme)."""
    k = len(grids)
    nd = (_i * k)(*[len(sh) for sh, _, _ in grids])
    shapes = (_i * (4 * k))()
    for j, (sh, _, _) in enumerate(grids):
        for i, v in enumerate(sh):
            shapes[4 * j + i] = int(v)
    models = (_i * k)(*[MODELS[m] if isinstance(m, str) else int(m) for _, m, _ in grids])
    schemes = (_i * k)(*[int(s) for _, _, s in grids])
    _check(lib().hj_jit_check_group(k, nd, shapes, models, schemes))


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)
_allocator_keepalive = None


def hj_set_allocator(alloc=None, free=None, user=None) -> None:
    """hj_set_allocator with ctypes function pointers (_ALLOC_FN, _FREE_FN)
    or None for both; the caller keeps the function objects alive."""
    a = ctypes.cast(alloc, ctypes.c_void_p) if alloc is not None else None
    f = ctypes.cast(free, ctypes.c_void_p) if free is not None else None
    _check(lib().hj_set_allocator(a, f, user))


def use_torch_allocator(on: bool = True) -> None:
    """Route the device allocations of grids, servers and batches created
    from now on through PyTorch's caching allocator (hj_set_allocator), so
    that they share its pool; on=False restores cudaMalloc / cudaFree."""
    global _allocator_keepalive
    if not on:
        _check(lib().hj_set_allocator(None, None, None))
        return
    import torch

    def _alloc(nbytes, device, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), int(device))
        except Exception:  # out of memory: the library reports HJ_ERR_OOM
            return None

    def _free(ptr, device, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _check(lib().hj_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p),
                                  None))
    # the library keeps the function pointers; the old ones must outlive the
    # objects created under them
    _allocator_keepalive = (a, f, _allocator_keepalive)


def hj_set_launch_shape(g: int, threads: int = 256, tile_rows: int = 0) -> None:
    _check(lib().hj_set_launch_shape(g, int(threads), int(tile_rows)))


def hj_get_launch_shape(g: int):
    """(threads per block of the flat mapping, tile_rows) of the grid."""
    t, r = ctypes.c_int(), ctypes.c_int()
    _check(lib().hj_get_launch_shape(g, ctypes.byref(t), ctypes.byref(r)))
    return t.value, r.value


def hj_jit_wait(timeout_s: float = 120.0) -> bool:
    """Wait until no shape-specialised compile is running (True) or the
    timeout passed (False)."""
    import time
    t0 = time.perf_counter()
    while hj_jit_pending() > 0:
        if time.perf_counter() - t0 > timeout_s:
            return False
        time.sleep(0.01)
    return True


class SafetyFilter:
    """hj_safety_filter with its grid, axis and control arguments marshalled
    once, for a control loop that filters a few host states per call: each
    call only copies the states in and the controls out."""

    def __init__(self, grids, axes, ctrl_index, state_dim: int, ctrl_dim: int,
                 max_states: int = 1):
        hs = [g.handle if hasattr(g, "handle") else g for g in grids]
        self._k = len(hs)
        self._h = (_vp * self._k)(*hs)
        ax = np.zeros((self._k, HJ_MAX_DIM), dtype=np.int32)
        for i, a in enumerate(axes):
            ax[i, :len(a)] = a
        self._ax = ax
        self._axp = ax.ctypes.data_as(_P(_i))
        self._ci = np.ascontiguousarray(ctrl_index, dtype=np.int32)
        self._cip = self._ci.ctypes.data_as(_P(_i))
        self._sd, self._cd = int(state_dim), int(ctrl_dim)
        self._u = np.empty((max_states, ctrl_dim), dtype=np.float64)
        self._w = np.empty(max_states, dtype=np.float64)
        self._a = np.empty(max_states, dtype=np.int32)
        self._fn = lib().hj_safety_filter

    def __call__(self, states: np.ndarray, u_perf: np.ndarray, level: float = 0.0):
        """states (nq, state_dim), u_perf (nq, ctrl_dim): C-contiguous float64
        host arrays with nq <= max_states.  Returns views (u, w, active) of
        buffers that the next call overwrites."""
        nq = states.shape[0]
        if nq > self._w.shape[0]:
            raise ValueError("more states than max_states")
        rc = self._fn(self._h, self._k, self._axp, self._cip, self._sd, self._cd, nq,
                      states.ctypes.data, u_perf.ctypes.data, float(level),
                      self._u.ctypes.data, self._w.ctypes.data, self._a.ctypes.data, 0)
        if rc != HJ_OK:
            raise HJError(rc, hj_last_error())
        return self._u[:nq], self._w[:nq], self._a[:nq]


def hj_autotune(g: int, scheme: int = HJ_WENO5) -> int:
    t = ctypes.c_int()
    _check(lib().hj_autotune(g, int(scheme), ctypes.byref(t)))
    return t.value


def hj_alpha(g: int, ndim: int) -> np.ndarray:
    out = (ctypes.c_double * ndim)()
    _check(lib().hj_alpha(g, out))
    return np.array(out[:])


def hj_solve_fixed_static(spec, W, mode: int = HJ_COLD, scheme: int = HJ_WENO5,
                          dt: float = 0.0, steps: int = 1, clamp: int = HJ_CLAMP_VI,
                          stream=None) -> None:
    """Allocation-free fixed-horizon solve of a box-constrained problem into the
    caller's device tensor W (float32, spec.npts values)."""
    if spec.con_kind != "box":
        raise ValueError("the allocation-free entry point takes box constraints")
    nd = len(spec.n)
    na = (ctypes.c_int * nd)(*[int(v) for v in spec.n])
    m = MODELS[spec.model]
    ptr, dev, keep = _field_ptr(W, int(np.prod(spec.n)), True)
    if not dev:
        raise ValueError("W must be device memory")
    import torch
    if W.device.index is not None and W.device.index != torch.cuda.current_device():
        raise ValueError("W lives on cuda:%d but cuda:%d is current"
                         % (W.device.index, torch.cuda.current_device()))
    _check(lib().hj_solve_fixed_static(nd, na, _darr(spec.lo), _darr(spec.hi), m,
                                       _darr(spec.params), len(spec.params), _darr(spec.d_lo),
                                       _darr(spec.d_hi), len(spec.d_lo), _darr(spec.con_a),
                                       _darr(spec.con_b), int(mode), int(scheme), float(dt),
                                       int(steps), int(clamp), ptr, _stream_handle(stream)))
    del keep


def make_request(spec, mode: int = HJ_COLD, key: int = 0, coarse_n: int = 0,
                 coarse_n2: int = 0, coarse_scheme: int = 0, **opts) -> hj_request:
    """An hj_request for a workloads.ProblemSpec (coarse_n > 0: coarse
    initialisation; coarse_n2: an intermediate level; coarse_scheme: the
    scheme of the coarse levels)."""
    r = hj_request()
    r.coarse_n = int(coarse_n)
    r.coarse_n2 = int(coarse_n2)
    r.coarse_scheme = int(coarse_scheme)
    r.ndim = spec.ndim
    for i in range(spec.ndim):
        r.n[i] = int(spec.n[i])
        r.lo[i] = float(spec.lo[i])
        r.hi[i] = float(spec.hi[i])
    r.model = MODELS[spec.model]
    for i, v in enumerate(spec.params):
        r.params[i] = float(v)
    r.nparams = len(spec.params)
    r.nd = len(spec.d_lo)
    for i in range(r.nd):
        r.d_lo[i] = float(spec.d_lo[i])
        r.d_hi[i] = float(spec.d_hi[i])
    r.con_ball = 0 if spec.con_kind == "box" else 1
    for i, v in enumerate(spec.con_a):
        r.con_a[i] = float(v)
    for i, v in enumerate(spec.con_b):
        r.con_b[i] = float(v)
    r.mode = int(mode)
    r.key = int(key)
    r.opts = make_opts(**opts)
    return r


def hj_server_create(budget_bytes: int, max_active: int = 64, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().hj_server_create(ctypes.byref(h), int(budget_bytes), int(max_active),
                                  _stream_handle(stream)))
    return h.value


def hj_server_destroy(s: int) -> None:
    lib().hj_server_destroy(s)


def hj_server_submit(s: int, req: hj_request) -> int:
    t = ctypes.c_longlong()
    _check(lib().hj_server_submit(s, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def hj_server_poll(s: int, ticket: int):
    """(done, status, stats dict)."""
    done, res, st = ctypes.c_int(), ctypes.c_int(), hj_solve_stats()
    _check(lib().hj_server_poll(s, ticket, ctypes.byref(done), ctypes.byref(res),
                                ctypes.byref(st)))
    return bool(done.value), res.value, st.as_dict()


def hj_server_wait(s: int, ticket: int, timeout_ms: float = 0.0):
    """(status, stats dict); raises HJError on timeout."""
    res, st = ctypes.c_int(), hj_solve_stats()
    _check(lib().hj_server_wait(s, ticket, float(timeout_ms), ctypes.byref(res),
                                ctypes.byref(st)))
    return res.value, st.as_dict()


def hj_server_get_value(s: int, ticket: int, dst) -> None:
    ptr, dev, keep = _field_ptr(dst, int(np.asarray(dst.shape).prod()) if hasattr(dst, "shape")
                                else len(dst), True)
    _check(lib().hj_server_get_value(s, ticket, ptr, dev))
    del keep


def hj_server_release(s: int, ticket: int) -> None:
    _check(lib().hj_server_release(s, ticket))


def hj_server_cancel(s: int, ticket: int) -> None:
    _check(lib().hj_server_cancel(s, ticket))


def hj_server_set_policy(s: int, order: int = HJ_ORDER_FIFO, max_active_nodes: int = 0) -> None:
    _check(lib().hj_server_set_policy(s, int(order), int(max_active_nodes)))


def hj_server_set_translated_starts(s: int, enable: bool) -> None:
    _check(lib().hj_server_set_translated_starts(s, 1 if enable else 0))


def hj_server_get_stats(s: int) -> Dict:
    st = hj_server_stats()
    _check(lib().hj_server_get_stats(s, ctypes.byref(st)))
    return st.as_dict()


def hj_grid_points(g: int) -> int:
    return int(lib().hj_grid_points(g))


def hj_kernel_launches() -> int:
    return int(lib().hj_kernel_launches())


# ------------------------------------------------------------ conveniences

class Grid:
    """Owns one hj_grid handle."""

    def __init__(self, n: Sequence[int], lo: Sequence[float], hi: Sequence[float], stream=None):
        self.n = tuple(int(v) for v in n)
        self.ndim = len(self.n)
        self.handle = hj_grid_create(self.n, lo, hi, stream)

    @classmethod
    def from_spec(cls, spec, stream=None) -> "Grid":
        """Grid, dynamics, disturbance box and constraint of a workloads.ProblemSpec."""
        g = cls(spec.n, spec.lo, spec.hi, stream)
        hj_set_dynamics(g.handle, spec.model, spec.params)
        hj_set_disturbance_bound(g.handle, spec.d_lo, spec.d_hi)
        if spec.con_kind == "box":
            hj_set_constraint(g.handle, spec.con_a, spec.con_b)
        else:
            hj_set_constraint_ball(g.handle, spec.con_a, spec.con_b[0])
        g.spec = spec
        return g

    def set_disturbance_bound(self, d_lo, d_hi) -> None:
        hj_set_disturbance_bound(self.handle, d_lo, d_hi)

    def set_disturbance_field(self, d_lo, d_hi) -> None:
        hj_set_disturbance_field(self.handle, d_lo, d_hi)

    def set_constraint_field(self, l) -> None:
        hj_set_constraint_field(self.handle, l)

    def solve(self, mode: int = HJ_COLD, **kw) -> Dict:
        rc, st = hj_solve(self.handle, mode, make_opts(**kw))
        st["status"] = rc
        return st

    def value(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float32)
        hj_get_value(self.handle, out)
        return out

    def value_into(self, tensor) -> None:
        hj_get_value(self.handle, tensor)

    def set_value(self, src) -> None:
        hj_set_value(self.handle, src)

    def query_value(self, xs) -> np.ndarray:
        return hj_query_value(self.handle, xs, self.ndim)

    def query_gradient(self, xs) -> np.ndarray:
        return hj_query_gradient(self.handle, xs, self.ndim)

    def alpha(self) -> np.ndarray:
        return hj_alpha(self.handle, self.ndim)

    def set_launch_shape(self, threads: int = 256, tile_rows: int = 0) -> None:
        hj_set_launch_shape(self.handle, threads, tile_rows)

    def launch_shape(self):
        return hj_get_launch_shape(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            hj_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve_batch(grids: List[Grid], modes: Sequence[int], **kw):
    opts = [make_opts(**kw)] if not isinstance(kw.get("per_grid"), list) else kw["per_grid"]
    return hj_solve_batch([g.handle for g in grids], modes, opts)


def prolong(coarse: Grid, fine: Grid) -> None:
    hj_prolong(coarse.handle, fine.handle)


def hj_translate(src: int, dst: int, shift: Sequence[float]) -> None:
    _check(lib().hj_translate(src, dst, _darr(shift)))


def translate(src: Grid, dst: Grid, shift: Sequence[float]) -> None:
    hj_translate(src.handle, dst.handle, shift)


def cfl_steps(check_dt: float, dt: float) -> int:
    return max(1, int(math.ceil(check_dt / dt - 1e-9)))
