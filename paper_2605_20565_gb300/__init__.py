"""GB300 octree Lagrangian-Eulerian coupling: host-cell search in a 2:1-balanced linear
octree, trilinear / Peskin-4 / Roma-3 interpolation and adjoint force spreading.

This module is a thin ``ctypes`` binding of the C ABI in ``include/octtrack.h``; every
function has the name of the C entry point it calls and only marshals arguments (PyTorch
tensors give device pointers and the current stream).  All computation runs in the CUDA
library ``libocttrack.so``; there is no CPU fallback: without the compiled library (build
it with ``__graft_entry__.build()``) every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = [
    "OT_TRILINEAR", "OT_PESKIN4", "OT_ROMA3", "OT_BINARY", "OT_LEARNED", "OT_SORTED", "OT_ATOMIC",
    "OT_ROOT_LINEAR", "OT_ROOT_MLP", "OT_DEV_OUTSIDE", "OT_DEV_STENCIL", "OT_DEV_REFINED_CAP", "OT_DEV_WINDOW",
    "OtError", "Octree", "Batch", "library_path", "ot_octree_build", "ot_octree_from_leaves", "ot_octree_info",
    "ot_octree_copy_leaves", "ot_octree_set_map_level", "ot_octree_get_map_level", "ot_octree_centres", "ot_octree_destroy", "ot_index_train", "ot_index_get_stats", "ot_index_get_root_params",
    "ot_index_mlp_grad", "ot_locate", "ot_interpolate", "ot_interpolate_f64", "ot_interpolate_workspace_size",
    "ot_field_mean_workspace_size", "ot_spread_workspace_size",
    "ot_spread", "ot_spread_f64", "ot_batch_create", "ot_batch_autotune", "ot_ibm_mdf", "ot_points_morton_order", "ot_field_fourier", "ot_body_sums", "ot_octree_set_periodic",
    "ot_octree_build_mates", "ot_octree_has_mates", "ot_octree_mates_bytes", "ot_octree_build_mates_in", "ot_field_subtract_mean", "ot_batch_run", "ot_batch_destroy", "ot_advect_ab2",
    "ot_last_error", "ot_launch_count", "ot_marker_force",
]

OT_TRILINEAR, OT_PESKIN4, OT_ROMA3 = 1, 2, 3
OT_BINARY, OT_LEARNED = 0, 1
OT_SORTED, OT_ATOMIC = 0, 1
OT_ROOT_LINEAR, OT_ROOT_MLP = 0, 1
OT_DEV_OUTSIDE, OT_DEV_STENCIL, OT_DEV_REFINED_CAP, OT_DEV_WINDOW = 1, 2, 4, 8

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libocttrack.so")
_lib = None
_lock = threading.Lock()


class OtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def library_path() -> str:
    return _LIB_PATH


class _Sphere(C.Structure):
    _fields_ = [("c", C.c_double * 3), ("r", C.c_double), ("shell", C.c_double)]


class _BuildParams(C.Structure):
    _fields_ = [("lmin", C.c_int), ("lmax", C.c_int), ("balance_full", C.c_int)]


class _IndexParams(C.Structure):
    _fields_ = [("root", C.c_int), ("n_leaf_models", C.c_int), ("n_mid_models", C.c_int), ("epochs", C.c_int),
                ("batch", C.c_int), ("lr", C.c_float), ("seed", C.c_uint64), ("steps", C.c_int),
                ("h_init", C.c_void_p)]


class _IndexStats(C.Structure):
    _fields_ = [("mean_window", C.c_double), ("max_window", C.c_int64), ("empty_models", C.c_int64),
                ("fallbacks", C.c_uint64), ("final_loss", C.c_float), ("mean_probes", C.c_double)]


class _Group(C.Structure):
    _fields_ = [("kernel", C.c_int), ("d_x", C.c_void_p), ("d_y", C.c_void_p), ("d_z", C.c_void_p),
                ("n", C.c_int64), ("d_u", C.c_void_p), ("d_host", C.c_void_p)]


class _Launch(C.Structure):
    _fields_ = [("block", C.c_int), ("tile", C.c_int), ("blocks_per_sm", C.c_int), ("order_level", C.c_int),
                ("tri_tile", C.c_int), ("tri_blocks_per_sm", C.c_int), ("tri_records", C.c_int)]

    _names = ("block", "tile", "blocks_per_sm", "order_level", "tri_tile", "tri_blocks_per_sm", "tri_records")

    @classmethod
    def of(cls, d: dict):
        return cls(*(int(d.get(k, 0)) for k in cls._names))

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k in self._names}


class _TuneResult(C.Structure):
    _fields_ = [("launch", _Launch), ("map_level", C.c_int), ("ms", C.c_float), ("tried", C.c_int)]


def _L():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(the CUDA library is required; there is no CPU fallback)")
            lib = C.CDLL(_LIB_PATH)
            P, i64, i32, st = C.c_void_p, C.c_int64, C.c_int, C.c_int
            sigs = {
                "ot_status_string": (C.c_char_p, [i32]),
                "ot_launch_count": (C.c_uint64, []),
                "ot_octree_build": (st, [P, i32, P, P, P]),
                "ot_octree_from_leaves": (st, [P, P, i64, i32, P, P]),
                "ot_octree_info": (st, [P, P, P, P]),
                "ot_octree_leaves": (st, [P, P, P, P]),
                "ot_octree_copy_leaves": (st, [P, P, P, P]),
                "ot_octree_centres": (st, [P, P, P]),
                "ot_octree_set_map_level": (st, [P, i32, P]),
                "ot_octree_get_map_level": (st, [P, P]),
                "ot_octree_destroy": (st, [P]),
                "ot_index_train": (st, [P, P, P]),
                "ot_index_get_stats": (st, [P, P, i32]),
                "ot_index_get_root_params": (st, [P, P]),
                "ot_index_mlp_grad": (st, [P, P, P, i64, P, P, P]),
                "ot_locate": (st, [P, P, P, P, i64, i32, P, P, P]),
                "ot_interpolate": (st, [P, i32, P, P, P, i64, P, i32, P, P, P, P, C.c_size_t, P]),
                "ot_interpolate_f64": (st, [P, i32, P, P, P, i64, P, i32, P, P, P, P, C.c_size_t, P]),
                "ot_interpolate_workspace_size": (st, [P, i32, i32, P]),
                "ot_field_mean_workspace_size": (st, [P, P]),
                "ot_spread_workspace_size": (st, [P, i32, i64, P]),
                "ot_spread": (st, [P, i32, i32, P, P, P, P, P, i64, P, P, C.c_size_t, P]),
                "ot_spread_f64": (st, [P, i32, i32, P, P, P, P, P, i64, P, P, C.c_size_t, P]),
                "ot_batch_create": (st, [P, P, i32, P, i32, P, P, P]),
                "ot_batch_autotune": (st, [P, P, i32, P, i32, i32, i32, P, P]),
                "ot_ibm_mdf_workspace_size": (st, [P, i32, i64, i32, P]),
                "ot_points_order_workspace_size": (st, [i64, P]),
                "ot_field_fourier": (st, [P, i32, P, P, P, P, P]),
                "ot_body_sums": (st, [P, P, P, P, P, C.c_float, i64, P, i32, P, C.c_double, P, P, P]),
                "ot_octree_set_periodic": (st, [P, i32]),
                "ot_octree_build_mates": (st, [P, i32, P]),
                "ot_octree_has_mates": (st, [P, P]),
                "ot_octree_mates_bytes": (st, [P, P]),
                "ot_octree_build_mates_in": (st, [P, P, C.c_size_t, P]),
                "ot_field_subtract_mean": (st, [P, P, P, P, C.c_size_t, P]),
                "ot_points_morton_order": (st, [P, P, P, i64, i32, P, P, C.c_size_t, P]),
                "ot_ibm_mdf": (st, [P, i32, P, P, P, P, P, i64, C.c_float, C.c_float, i32, P, P, P, P, C.c_size_t, P]),
                "ot_batch_run": (st, [P, P]),
                "ot_batch_destroy": (st, [P]),
                "ot_advect_ab2": (st, [P, P, P, P, P, i64, C.c_float, C.c_float, C.c_float, i32, i32, P]),
                "ot_marker_force": (st, [P, P, i64, C.c_float, P, P]),
                "ot_last_error": (st, [P, P, i32, P]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        raise OtError(status, _L().ot_status_string(status).decode())


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


class Octree:
    """Owner of an ``ot_octree*`` handle (destroyed with the object)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ot_octree_destroy(self._h)
            self._h = None

    @property
    def info(self):
        return ot_octree_info(self)


class Batch:
    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep  # tensors the captured graph points to

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ot_batch_destroy(self._h)
            self._h = None


# --- octree -------------------------------------------------------------------------------

def ot_octree_build(spheres, lmin: int, lmax: int, balance_full: int = 1, stream=None) -> Octree:
    """spheres: (n, 5) rows (cx, cy, cz, r, shell)."""
    sp = np.ascontiguousarray(np.asarray(spheres, np.float64).reshape(-1, 5))
    arr = (_Sphere * max(1, sp.shape[0]))()
    for i, row in enumerate(sp):
        arr[i].c[0], arr[i].c[1], arr[i].c[2] = row[0], row[1], row[2]
        arr[i].r, arr[i].shell = row[3], row[4]
    prm = _BuildParams(lmin, lmax, balance_full)
    h = C.c_void_p()
    _check(_L().ot_octree_build(arr, sp.shape[0], C.byref(prm), _stream(stream), C.byref(h)))
    return Octree(h)


def ot_octree_from_leaves(keys, levels, balance_full: int = 1, stream=None) -> Octree:
    """keys: CUDA int64 tensor holding the uint64 anchor keys; levels: CUDA uint8 tensor."""
    torch = _torch()
    h = C.c_void_p()
    _check(_L().ot_octree_from_leaves(_dptr(keys, torch.int64, "keys"), _dptr(levels, torch.uint8, "levels"),
                                      keys.numel(), balance_full, _stream(stream), C.byref(h)))
    return Octree(h)


def ot_octree_info(tree: Octree):
    n, a, b = C.c_int64(), C.c_int(), C.c_int()
    _check(_L().ot_octree_info(tree.handle, C.byref(n), C.byref(a), C.byref(b)))
    return n.value, a.value, b.value


def ot_octree_copy_leaves(tree: Octree, stream=None):
    """(keys int64 tensor, levels uint8 tensor) on the current CUDA device."""
    torch = _torch()
    n, _, _ = ot_octree_info(tree)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    lev = torch.empty(n, dtype=torch.uint8, device="cuda")
    _check(_L().ot_octree_copy_leaves(tree.handle, _dptr(keys), _dptr(lev), _stream(stream)))
    return keys, lev


def ot_octree_set_map_level(tree: Octree, level: int, stream=None):
    _check(_L().ot_octree_set_map_level(tree.handle, level, _stream(stream)))


def ot_octree_get_map_level(tree: Octree) -> int:
    v = C.c_int()
    _check(_L().ot_octree_get_map_level(tree.handle, C.byref(v)))
    return v.value


def ot_octree_centres(tree: Octree, out=None, stream=None):
    torch = _torch()
    n, _, _ = ot_octree_info(tree)
    if out is None:
        out = torch.empty((3, n), dtype=torch.float64, device="cuda")
    _check(_L().ot_octree_centres(tree.handle, _dptr(out, torch.float64, "out"), _stream(stream)))
    return out


def ot_octree_destroy(tree: Octree):
    if tree._h:
        _check(_L().ot_octree_destroy(tree._h))
        tree._h = None


# --- learned index ------------------------------------------------------------------------

def ot_index_train(tree: Octree, root: int = OT_ROOT_MLP, n_leaf_models: int = 4096, epochs: int = 4,
                   batch: int = 65536, lr: float = 1e-3, seed: int = 0, n_mid_models: int = 0, steps: int = 0,
                   init=None, stream=None):
    """init: 97 MLP parameters to start from (e.g. ot_index_get_root_params of the previous tree)."""
    import numpy as np
    h = None if init is None else np.ascontiguousarray(np.asarray(init, dtype=np.float32).reshape(97))
    prm = _IndexParams(root, n_leaf_models, n_mid_models, epochs, batch, lr, seed, steps,
                       None if h is None else h.ctypes.data_as(C.c_void_p))
    _check(_L().ot_index_train(tree.handle, C.byref(prm), _stream(stream)))


def ot_index_get_root_params(tree: Octree):
    import numpy as np
    h = np.empty(97, np.float32)
    _check(_L().ot_index_get_root_params(tree.handle, h.ctypes.data_as(C.c_void_p)))
    return h


def ot_index_get_stats(tree: Octree, reset: bool = False) -> dict:
    s = _IndexStats()
    _check(_L().ot_index_get_stats(tree.handle, C.byref(s), int(reset)))
    return {"mean_window": s.mean_window, "max_window": s.max_window, "empty_models": s.empty_models,
            "fallbacks": s.fallbacks, "final_loss": s.final_loss, "mean_probes": s.mean_probes}


def ot_index_mlp_grad(params, x, t, stream=None):
    """Loss and gradient (97 floats) of the root network's MSE loss on samples (x, t)."""
    torch = _torch()
    g = torch.empty(97, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(_L().ot_index_mlp_grad(_dptr(params, torch.float32, "params"), _dptr(x, torch.float32, "x"),
                                  _dptr(t, torch.float32, "t"), x.numel(), _dptr(g), _dptr(loss),
                                  _stream(stream)))
    return g, loss


# --- locate / interpolate / spread --------------------------------------------------------

def _xyz(x, y, z):
    torch = _torch()
    n = x.numel()
    if y.numel() != n or z.numel() != n:
        raise ValueError("x, y, z must have the same length")
    return n, _dptr(x, torch.float64, "x"), _dptr(y, torch.float64, "y"), _dptr(z, torch.float64, "z")


def ot_locate(tree: Octree, x, y, z, search: int = OT_BINARY, host=None, n_miss=None, stream=None):
    torch = _torch()
    n, px, py, pz = _xyz(x, y, z)
    if host is None:
        host = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(_L().ot_locate(tree.handle, px, py, pz, n, search, _dptr(host, torch.int32, "host"),
                          _dptr(n_miss, torch.int64, "n_miss"), _stream(stream)))
    return host


def ot_interpolate_workspace_size(tree: Octree, kernel: int, fp64: bool = False) -> int:
    """Bytes of workspace ot_interpolate (fp64=False) or ot_interpolate_f64 needs."""
    b = C.c_size_t()
    _check(_L().ot_interpolate_workspace_size(tree.handle, kernel, int(fp64), C.byref(b)))
    return b.value


def _interp(fn, dtype, tree, kernel, x, y, z, field, search, host_in, u, host_out, workspace, stream):
    torch = _torch()
    n, px, py, pz = _xyz(x, y, z)
    if u is None:
        u = torch.empty((3, n), dtype=dtype, device="cuda")
    if workspace is None:
        need = ot_interpolate_workspace_size(tree, kernel, dtype == torch.float64)
        workspace = torch.empty(need, dtype=torch.uint8, device="cuda") if need else None
    have = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(fn(tree.handle, kernel, px, py, pz, n, _dptr(host_in, torch.int32, "host_in"), search,
              _dptr(field, dtype, "field"), _dptr(u, dtype, "u"), _dptr(host_out, torch.int32, "host_out"),
              _dptr(workspace, None, "workspace"), have, _stream(stream)))
    return u


def ot_interpolate(tree: Octree, kernel: int, x, y, z, field, search: int = OT_BINARY, host_in=None, u=None,
                   host_out=None, workspace=None, stream=None):
    """field: (N, 4) float32; returns u (3, n) float32.  workspace: a CUDA uint8 tensor of
    ot_interpolate_workspace_size bytes (allocated here when None)."""
    torch = _torch()
    return _interp(_L().ot_interpolate, torch.float32, tree, kernel, x, y, z, field, search, host_in, u, host_out,
                   workspace, stream)


def ot_interpolate_f64(tree: Octree, kernel: int, x, y, z, field, search: int = OT_BINARY, host_in=None, u=None,
                       host_out=None, workspace=None, stream=None):
    """field: (N, 4) float64; returns u (3, n) float64."""
    torch = _torch()
    return _interp(_L().ot_interpolate_f64, torch.float64, tree, kernel, x, y, z, field, search, host_in, u,
                   host_out, workspace, stream)


def ot_spread_workspace_size(tree: Octree, kernel: int, n: int) -> int:
    b = C.c_size_t()
    _check(_L().ot_spread_workspace_size(tree.handle, kernel, n, C.byref(b)))
    return b.value


def _spread(fn, dtype, tree, kernel, mode, x, y, z, F, f, dV, workspace, stream):
    torch = _torch()
    n, px, py, pz = _xyz(x, y, z)
    have = 0
    if mode == OT_SORTED and workspace is None:
        workspace = torch.empty(max(1, ot_spread_workspace_size(tree, kernel, n)), dtype=torch.uint8, device="cuda")
    if workspace is not None:
        have = workspace.numel() * workspace.element_size()  # the real size; the library checks it
    _check(fn(tree.handle, kernel, mode, px, py, pz, _dptr(F, dtype, "F"), _dptr(dV, dtype, "dV"), n,
              _dptr(f, dtype, "f"), _dptr(workspace, None, "workspace"), have, _stream(stream)))
    return f


def ot_spread(tree: Octree, kernel: int, mode: int, x, y, z, F, f, dV=None, workspace=None, stream=None):
    """F: (3, n) float32; f: (N, 4) float32, accumulated in place."""
    torch = _torch()
    return _spread(_L().ot_spread, torch.float32, tree, kernel, mode, x, y, z, F, f, dV, workspace, stream)


def ot_spread_f64(tree: Octree, kernel: int, mode: int, x, y, z, F, f, dV=None, workspace=None, stream=None):
    torch = _torch()
    return _spread(_L().ot_spread_f64, torch.float64, tree, kernel, mode, x, y, z, F, f, dV, workspace, stream)


# --- batch ----------------------------------------------------------------------------------

def _groups(groups):
    torch = _torch()
    arr = (_Group * len(groups))()
    for i, g in enumerate(groups):
        n, px, py, pz = _xyz(g["x"], g["y"], g["z"])
        arr[i].kernel = g["kernel"]
        arr[i].d_x, arr[i].d_y, arr[i].d_z = px, py, pz
        arr[i].n = n
        arr[i].d_u = _dptr(g["u"], torch.float32, "u")
        arr[i].d_host = _dptr(g.get("host"), torch.int32, "host")
    return arr


def ot_batch_create(tree: Octree, groups, field, search: int = OT_BINARY, launch: dict | None = None,
                    stream=None) -> Batch:
    """groups: list of dicts {kernel, x, y, z, u, host (optional)}; tensors stay referenced."""
    torch = _torch()
    arr = _groups(groups)
    keep = [field] + list(groups)
    lp = None
    if launch:
        lp = _Launch.of(launch)
    h = C.c_void_p()
    _check(_L().ot_batch_create(tree.handle, arr, len(groups), _dptr(field, torch.float32, "field"), search,
                                C.byref(lp) if lp is not None else None, _stream(stream), C.byref(h)))
    keep.append(tree)
    return Batch(h, keep)


def ot_batch_autotune(tree: Octree, groups, field, search: int = OT_BINARY, tune_map_level: bool = True,
                      reps: int = 3, stream=None) -> dict:
    """Fastest launch shape (and level-map level) for a batch over these groups; the octree is
    left at the chosen level map.  Returns {launch: {block, tile, blocks_per_sm, order_level,
    tri_tile, tri_blocks_per_sm}, map_level, ms, tried}."""
    torch = _torch()
    r = _TuneResult()
    _check(_L().ot_batch_autotune(tree.handle, _groups(groups), len(groups), _dptr(field, torch.float32, "field"),
                                  search, int(tune_map_level), reps, _stream(stream), C.byref(r)))
    return {"launch": r.launch.as_dict(), "map_level": r.map_level, "ms": r.ms, "tried": r.tried}


def ot_ibm_mdf(tree: Octree, kernel: int, x, y, z, U, u, rho: float, dt: float, n_iter: int, dV=None,
               slip: bool = False, stream=None):
    """Multi-direct forcing in place on u ((N, 4) float32: u* in, corrected u out); returns
    (f (N, 4) total force, slip (n_iter + 1,) float32 tensor or None)."""
    torch = _torch()
    n, px, py, pz = _xyz(x, y, z)
    nl = ot_octree_info(tree)[0]
    b = C.c_size_t()
    _check(_L().ot_ibm_mdf_workspace_size(tree.handle, kernel, n, n_iter, C.byref(b)))
    ws = torch.empty(b.value + 256, dtype=torch.uint8, device=u.device)
    off = (-ws.data_ptr()) % 256
    f = torch.empty((nl, 4), dtype=torch.float32, device=u.device)
    sl = torch.empty(n_iter + 1, dtype=torch.float32, device=u.device) if slip else None
    _check(_L().ot_ibm_mdf(tree.handle, kernel, px, py, pz, _dptr(U, torch.float32, "U"),
                           _dptr(dV, torch.float32, "dV"), n, rho, dt, n_iter, _dptr(u, torch.float32, "u"),
                           _dptr(f), _dptr(sl), C.c_void_p(ws.data_ptr() + off), b.value, _stream(stream)))
    return f, sl


def ot_field_fourier(tree: Octree, wave, amp, phase, field=None, stream=None):
    """(N, 4) float32 field sum_m amp_m cos(2 pi wave_m . c + phase_m) at the leaf centres c.
    wave: (M, 3) integers; amp: (M, 3); phase: (M,) radians."""
    import numpy as np
    torch = _torch()
    w = np.ascontiguousarray(np.asarray(wave).reshape(-1, 3), dtype=np.int32)
    a = np.ascontiguousarray(np.asarray(amp, dtype=np.float64).reshape(-1, 3))
    p = np.ascontiguousarray(np.asarray(phase, dtype=np.float64).reshape(-1))
    if field is None:
        field = torch.empty((ot_octree_info(tree)[0], 4), dtype=torch.float32, device="cuda")
    _check(_L().ot_field_fourier(tree.handle, w.shape[0], w.ctypes.data_as(C.c_void_p), a.ctypes.data_as(C.c_void_p),
                                 p.ctypes.data_as(C.c_void_p), _dptr(field, torch.float32, "field"), _stream(stream)))
    return field


def ot_octree_set_periodic(tree: Octree, periodic: bool = True):
    _check(_L().ot_octree_set_periodic(tree.handle, int(periodic)))


def ot_octree_build_mates(tree: Octree, enable: bool = True, stream=None):
    """Builds (or, with enable=False, frees) the octree's level-mate table: 256 bytes per leaf
    of device memory; trilinear queries and batches made afterwards read their level-mates
    from it (bit-identical results)."""
    _check(_L().ot_octree_build_mates(tree.handle, int(enable), _stream(stream)))


def ot_octree_mates_bytes(tree: Octree) -> int:
    v = C.c_size_t()
    _check(_L().ot_octree_mates_bytes(tree.handle, C.byref(v)))
    return v.value


def ot_octree_build_mates_in(tree: Octree, buffer, stream=None):
    """Builds the level-mate table in the caller's buffer (a CUDA uint8 tensor of at least
    ot_octree_mates_bytes(tree) bytes), which the octree then references (kept alive here)."""
    torch = _torch()
    if not (isinstance(buffer, torch.Tensor) and buffer.is_cuda and buffer.dtype == torch.uint8
            and buffer.is_contiguous()):
        raise OtError(-1, "buffer must be a contiguous CUDA uint8 tensor")
    _check(_L().ot_octree_build_mates_in(tree.handle, C.c_void_p(buffer.data_ptr()), buffer.numel(),
                                         _stream(stream)))
    tree.keep_mates = buffer


def ot_octree_has_mates(tree: Octree) -> bool:
    v = C.c_int()
    _check(_L().ot_octree_has_mates(tree.handle, C.byref(v)))
    return bool(v.value)


def ot_field_mean_workspace_size(tree: Octree) -> int:
    b = C.c_size_t()
    _check(_L().ot_field_mean_workspace_size(tree.handle, C.byref(b)))
    return b.value


def ot_field_subtract_mean(tree: Octree, field, mean=None, workspace=None, stream=None):
    """Subtracts the volume-weighted mean of field ((N, 4) float32, in place); returns the mean
    (3 float64).  workspace: a CUDA uint8 tensor of ot_field_mean_workspace_size bytes."""
    torch = _torch()
    if mean is None:
        mean = torch.empty(3, dtype=torch.float64, device=field.device)
    if workspace is None:
        workspace = torch.empty(ot_field_mean_workspace_size(tree), dtype=torch.uint8, device=field.device)
    _check(_L().ot_field_subtract_mean(tree.handle, _dptr(field, torch.float32, "field"), _dptr(mean),
                                       _dptr(workspace, None, "workspace"),
                                       workspace.numel() * workspace.element_size(), _stream(stream)))
    return mean


def ot_body_sums(x, y, z, v, start, xb, scale: float, dV=None, w: float = 1.0, stream=None):
    """Per-body (lin, ang) float64 tensors (n_bodies, 3): scale sum v w and scale sum (X - x_b) x v w.
    start: int64 tensor (n_bodies + 1) of marker offsets; xb: float64 tensor (n_bodies, 3)."""
    torch = _torch()
    n, px, py, pz = _xyz(x, y, z)
    nb = xb.shape[0]
    lin = torch.empty((nb, 3), dtype=torch.float64, device=x.device)
    ang = torch.empty((nb, 3), dtype=torch.float64, device=x.device)
    _check(_L().ot_body_sums(px, py, pz, _dptr(v, torch.float32, "v"), _dptr(dV, torch.float32, "dV"), w, n,
                             _dptr(start, torch.int64, "start"), nb, _dptr(xb.contiguous(), torch.float64, "xb"),
                             float(scale), _dptr(lin), _dptr(ang), _stream(stream)))
    return lin, ang


def ot_points_morton_order(x, y, z, level: int = 8, stream=None):
    """int32 permutation putting the points in Morton (Z-curve) order of their level cells."""
    torch = _torch()
    n, px, py, pz = _xyz(x, y, z)
    b = C.c_size_t()
    _check(_L().ot_points_order_workspace_size(n, C.byref(b)))
    ws = torch.empty(max(1, b.value), dtype=torch.uint8, device=x.device)
    perm = torch.empty(n, dtype=torch.int32, device=x.device)
    _check(_L().ot_points_morton_order(px, py, pz, n, level, _dptr(perm), _dptr(ws), b.value, _stream(stream)))
    return perm


def ot_batch_run(batch: Batch, stream=None):
    _check(_L().ot_batch_run(batch._h, _stream(stream)))


def ot_batch_destroy(batch: Batch):
    if batch._h:
        _check(_L().ot_batch_destroy(batch._h))
        batch._h = None


# --- advection / diagnostics ----------------------------------------------------------------

def ot_advect_ab2(x, v, a_prev, v_prev, u, tau: float, re_coef: float, dt: float, first: bool,
                  periodic: bool = False, stream=None):
    """x: (3, n) float64; v, a_prev, v_prev, u: (3, n) float32 (updated in place)."""
    torch = _torch()
    n = x.shape[1]
    _check(_L().ot_advect_ab2(_dptr(x, torch.float64, "x"), _dptr(v, torch.float32, "v"),
                              _dptr(a_prev, torch.float32, "a_prev"), _dptr(v_prev, torch.float32, "v_prev"),
                              _dptr(u, torch.float32, "u"), n, tau, re_coef, dt, int(first), int(periodic),
                              _stream(stream)))


def ot_marker_force(u, dt: float, F=None, U=None, stream=None):
    """F = (U - u) / dt for markers (u, U: (3, n) float32; U None: markers at rest)."""
    torch = _torch()
    n = u.shape[1]
    if F is None:
        F = torch.empty_like(u)
    _check(_L().ot_marker_force(_dptr(U, torch.float32, "U"), _dptr(u, torch.float32, "u"), n, dt,
                                _dptr(F, torch.float32, "F"), _stream(stream)))
    return F


def ot_last_error(tree: Octree, clear: bool = True, stream=None) -> int:
    bits = C.c_uint()
    _check(_L().ot_last_error(tree.handle, C.byref(bits), int(clear), _stream(stream)))
    return bits.value


def ot_launch_count() -> int:
    return int(_L().ot_launch_count())
