"""FP64 CPU oracle for the octree Lagrangian-Eulerian coupling path.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The product package never imports this module,
and this module imports nothing from the product package.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over independent points,
compiled with ``-ffp-contract=off``).  This file only compiles it on first use and
marshals numpy arrays.  Each wrapper names the passage of the paper it follows; see the
header of ``oracle.c`` for which functions are pinned and how.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OT_TRILINEAR, OT_PESKIN4, OT_ROMA3 = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (next to it) when missing or stale."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int, C.c_double
            sig = {
                "or_num_threads": (i32, []),
                "or_morton": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint32]),
                "or_unmorton": (None, [C.c_uint64, P, P, P]),
                "or_upper_bound": (i64, [P, i64, C.c_uint64]),
                "or_octree_build": (i64, [P, i32, i32, i32, i32, P, P]),
                "or_free": (None, [P]),
                "or_count_unbalanced": (i64, [P, P, i64, i32]),
                "or_leaf_centres": (None, [P, P, i64, P]),
                "or_locate_ub": (None, [P, P, i64, P, P, P, i64, P]),
                "or_locate_brute": (None, [P, P, i64, P, P, P, i64, P]),
                "or_phi_peskin4": (dbl, [dbl]),
                "or_phi_roma3": (dbl, [dbl]),
                "or_phi_array": (None, [i32, P, i64, P]),
                "or_interp_delta": (i64, [P, P, i64, i32, i32, P, P, P, P, i64, P]),
                "or_spread_delta": (i64, [P, P, i64, i32, i32, P, P, P, P, P, i64, P]),
                "or_interp_trilinear": (None, [P, P, i64, P, P, P, P, P, i64, P]),
                "or_mlp_forward1": (dbl, [P, dbl]),
                "or_mlp_loss_grad": (dbl, [P, P, P, i64, P]),
                "or_advect_ab2": (None, [P, P, P, P, P, i64, dbl, dbl, dbl, i32, i32]),
                "or_ibm_mdf": (i64, [P, P, i64, i32, i32, P, P, P, P, P, P, i64, dbl, dbl, i32, P, P, P]),
                "or_body_sums": (None, [P, P, P, P, P, dbl, i64, P, i32, P, dbl, P, P]),
                "or_interp_delta_p": (i64, [P, P, i64, i32, i32, P, P, P, P, i64, P, i32]),
                "or_spread_delta_p": (i64, [P, P, i64, i32, i32, P, P, P, P, P, i64, P, i32]),
                "or_interp_trilinear_p": (None, [P, P, i64, P, P, P, P, P, i64, P, i32]),
                "or_field_mean": (None, [P, i64, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    """Host threads the OpenMP loops use."""
    return int(_L().or_num_threads())


# --- Morton keys (Sec. 3.1-3.2: leaves sorted in Z-order) -------------------------------

def morton(x: int, y: int, z: int) -> int:
    return int(_L().or_morton(x, y, z))


def unmorton(key: int):
    a, b, c = C.c_uint32(), C.c_uint32(), C.c_uint32()
    _L().or_unmorton(C.c_uint64(key), C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


# --- Octree (Sec. 3.1 refinement + 2:1 balance; Sec. 3.3 auxiliary IBM forest) ----------

def octree_build(spheres, lmin: int, lmax: int, full: int = 1):
    """Leaves (keys uint64, levels uint8) of the tree refined within w of each sphere surface
    (rows cx, cy, cz, r, w) from level lmin to lmax, then 2:1 balanced."""
    s = _c(np.asarray(spheres, dtype=np.float64).reshape(-1, 5), np.float64)
    kp, lp = C.c_void_p(), C.c_void_p()
    n = _L().or_octree_build(_p(s), s.shape[0], lmin, lmax, full, C.byref(kp), C.byref(lp))
    keys = np.ctypeslib.as_array(C.cast(kp, C.POINTER(C.c_uint64)), shape=(n,)).copy()
    lev = np.ctypeslib.as_array(C.cast(lp, C.POINTER(C.c_uint8)), shape=(n,)).copy()
    _L().or_free(kp)
    _L().or_free(lp)
    return keys, lev


def count_unbalanced(keys, levels, full: int = 1) -> int:
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    return int(_L().or_count_unbalanced(_p(k), _p(l), k.size, full))


def leaf_centres(keys, levels) -> np.ndarray:
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    out = np.empty((k.size, 3), np.float64)
    _L().or_leaf_centres(_p(k), _p(l), k.size, _p(out))
    return out


# --- Host-cell search (Algorithm 1, Sec. 3.2) -------------------------------------------

def _pts(x, y, z):
    return _c(x, np.float64), _c(y, np.float64), _c(z, np.float64)


def locate_ub(keys, levels, x, y, z) -> np.ndarray:
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    x, y, z = _pts(x, y, z)
    out = np.empty(x.size, np.int32)
    _L().or_locate_ub(_p(k), _p(l), k.size, _p(x), _p(y), _p(z), x.size, _p(out))
    return out


def locate_brute(keys, levels, x, y, z) -> np.ndarray:
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    x, y, z = _pts(x, y, z)
    out = np.empty(x.size, np.int32)
    _L().or_locate_brute(_p(k), _p(l), k.size, _p(x), _p(y), _p(z), x.size, _p(out))
    return out


# --- Delta kernels and IBM interpolation / spreading (Sec. 2.2) --------------------------

def phi(kernel: int, r) -> np.ndarray:
    r = _c(r, np.float64)
    out = np.empty_like(r)
    _L().or_phi_array(kernel, _p(r), r.size, _p(out))
    return out


def interp_delta(keys, levels, lmax, kernel, field, x, y, z, periodic: bool = False):
    """u (3, n) and the count of skipped stencil cells.  field: (N, 4) float64.  periodic: the
    stencil wraps around the unit cube."""
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    f = _c(field, np.float64).reshape(-1, 4)
    x, y, z = _pts(x, y, z)
    u = np.empty((3, x.size), np.float64)
    bad = _L().or_interp_delta_p(_p(k), _p(l), k.size, lmax, kernel, _p(f), _p(x), _p(y), _p(z), x.size, _p(u),
                                 int(periodic))
    return u, int(bad)


def spread_delta(keys, levels, lmax, kernel, x, y, z, F, dV=None, f=None, periodic: bool = False):
    """f (N, 4) accumulated in place (zeros when f is None) and the skipped-cell count."""
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    x, y, z = _pts(x, y, z)
    F = _c(F, np.float64).reshape(3, -1)
    if f is None:
        f = np.zeros((k.size, 4), np.float64)
    assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == (k.size, 4)
    dvp = None
    if dV is not None:
        dV = _c(dV, np.float64)
        dvp = _p(dV)
    bad = _L().or_spread_delta_p(_p(k), _p(l), k.size, lmax, kernel, _p(x), _p(y), _p(z), _p(F), dvp, x.size, _p(f),
                                 int(periodic))
    return f, int(bad)


def interp_trilinear(keys, levels, field, x, y, z, host, periodic: bool = False):
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    f = _c(field, np.float64).reshape(-1, 4)
    x, y, z = _pts(x, y, z)
    h = _c(host, np.int32)
    u = np.empty((3, x.size), np.float64)
    _L().or_interp_trilinear_p(_p(k), _p(l), k.size, _p(f), _p(x), _p(y), _p(z), _p(h), x.size, _p(u),
                               int(periodic))
    return u


def field_mean(levels, field) -> np.ndarray:
    """Volume-weighted mean over the unit cube of a cell field (N, 4): (3,)."""
    l = _c(levels, np.uint8)
    f = _c(field, np.float64).reshape(-1, 4)
    m = np.empty(3, np.float64)
    _L().or_field_mean(_p(l), l.size, _p(f), _p(m))
    return m


def ibm_mdf(keys, levels, lmax, kernel, u_star, X, U, rho, dt, n_iter, dV=None):
    """Multi-direct forcing (Sec. 2.2): (u (N, 4), f (N, 4), slip (n_iter + 1,), skipped cells).
    X, U: (3, nm) marker positions and prescribed velocities; u_star: (N, 4)."""
    k, l = _c(keys, np.uint64), _c(levels, np.uint8)
    us = _c(u_star, np.float64).reshape(-1, 4)
    x, y, z = _pts(*np.asarray(X, np.float64))
    Uc = _c(U, np.float64).reshape(3, -1)
    dvp = None
    if dV is not None:
        dV = _c(dV, np.float64)
        dvp = _p(dV)
    u = np.empty_like(us)
    f = np.empty_like(us)
    slip = np.empty(n_iter + 1, np.float64)
    bad = _L().or_ibm_mdf(_p(k), _p(l), k.size, lmax, kernel, _p(us), _p(x), _p(y), _p(z), _p(Uc), dvp, x.size,
                          rho, dt, n_iter, _p(u), _p(f), _p(slip))
    return u, f, slip, int(bad)


def body_sums(X, v, start, xb, scale, dV=None, w=1.0):
    """Per-body (lin, ang), each (nb, 3): scale * sum v w and scale * sum (X - x_b) x v w over
    the markers start[b] .. start[b+1]-1 (Sec. 2.3)."""
    x, y, z = _pts(*np.asarray(X, np.float64))
    vv = _c(v, np.float64).reshape(3, -1)
    st = _c(start, np.int64)
    xbc = _c(xb, np.float64).reshape(-1, 3)
    nb = xbc.shape[0]
    dvp = None
    if dV is not None:
        dV = _c(dV, np.float64)
        dvp = _p(dV)
    lin = np.empty((nb, 3))
    ang = np.empty((nb, 3))
    _L().or_body_sums(_p(x), _p(y), _p(z), _p(vv), dvp, float(w), x.size, _p(st), nb, _p(xbc), float(scale),
                      _p(lin), _p(ang))
    return lin, ang


# --- Learned-index root network (1 -> 32 ReLU -> 1) ------------------------------------

MLP_H = 32
MLP_NPARAM = 3 * MLP_H + 1


def mlp_forward(params, xin) -> np.ndarray:
    prm = _c(params, np.float64)
    return np.array([_L().or_mlp_forward1(_p(prm), float(v)) for v in np.asarray(xin, np.float64)])


def mlp_loss_grad(params, xin, tgt):
    prm = _c(params, np.float64)
    x, t = _c(xin, np.float64), _c(tgt, np.float64)
    g = np.empty(MLP_NPARAM, np.float64)
    loss = _L().or_mlp_loss_grad(_p(prm), _p(x), _p(t), x.size, _p(g))
    return float(loss), g


# --- Point-particle advection (Sec. 2.3.2) ----------------------------------------------

def advect_ab2(state: dict, u, tau: float, re_coef: float, dt: float, first: bool, periodic: bool = False):
    """Advance state {'x','v','a_prev','v_prev'} (each (3, n) float64, in place) one step."""
    u = _c(u, np.float64).reshape(3, -1)
    for key in ("x", "v", "a_prev", "v_prev"):
        a = state[key]
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _L().or_advect_ab2(_p(state["x"]), _p(state["v"]), _p(state["a_prev"]), _p(state["v_prev"]), _p(u),
                       u.shape[1], tau, re_coef, dt, int(first), int(periodic))
    return state
