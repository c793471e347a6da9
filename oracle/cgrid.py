"""ctypes front end of the C oracle (``tsdf_oracle.c``): fusion and ray bounds.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The C library is compiled with gcc on first use (``-ffp-contract=off``, no
fast-math) into ``oracle/_build/``; :func:`build` does it explicitly.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

STATUS_MISS, STATUS_BOUNDED, STATUS_FALLBACK = 0, 1, 2


def build(force=False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liborc.so")
    srcs = [os.path.join(_HERE, "tsdf_oracle.c"), os.path.join(_HERE, "orc_impl.h")]
    if force or not os.path.exists(out) or any(os.path.getmtime(s) > os.path.getmtime(out) for s in srcs):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
                               "-fsigned-char", "-shared", "-fPIC", srcs[0], "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = C.CDLL(build())
            _LIB.orc_dda_sequence_f64.restype = C.c_int64
            _LIB.orc_dda_sequence_f32.restype = C.c_int64
            _LIB.orc_half_from_float.restype = C.c_uint16
            _LIB.orc_half_from_float.argtypes = [C.c_float]
            _LIB.orc_float_from_half.restype = C.c_float
            _LIB.orc_float_from_half.argtypes = [C.c_uint16]
    return _LIB


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f(a):
    return np.ascontiguousarray(a, np.float32)


def _origin(grid):
    return np.ascontiguousarray(np.asarray(grid.origin, np.float64))


def integrate_projective(grid, views, mode="f32", V=None, W=None, vox=None):
    """Per-voxel projective TSDF fusion (Eq. 3, Alg. 2 projective form).

    mode "f64": FP64 reference; "f32": fp32-exact mode.  ``grid.dtype`` "f16"
    stores V as IEEE half (returned as uint16 bits).  V/W: initial state
    (default: V = -1, W = 0, Sec. A.1), shaped like the grid or like ``vox``.
    Returns (V, W).
    """
    f16 = grid.dtype == "f16"
    shape = grid.shape_zyx if vox is None else (len(vox),)
    if V is None:
        if f16:
            V = np.full(shape, 0xBC00, np.uint16)  # -1.0 in half
        else:
            V = np.full(shape, -1.0, np.float64 if mode == "f64" else np.float32)
    else:
        V = np.array(V, np.uint16 if f16 else (np.float64 if mode == "f64" else np.float32), copy=True)
    W = np.zeros(shape, np.uint8) if W is None else np.array(W, np.uint8, copy=True)
    vox_a = None if vox is None else np.ascontiguousarray(vox, np.int64)
    fn = lib().orc_integrate_projective_f64 if mode == "f64" else lib().orc_integrate_projective_f32
    dep, K, P = _f(views.depth), _f(views.K), _f(views.c2w)
    fn(C.c_int(grid.nx), C.c_int(grid.ny), C.c_int(grid.nz), _p(_origin(grid)), C.c_double(grid.voxel_size),
       C.c_double(grid.trunc), _p(dep), C.c_int(dep.shape[0]), C.c_int(dep.shape[1]), C.c_int(dep.shape[2]),
       _p(K), _p(P), _p(vox_a), C.c_int64(0 if vox is None else len(vox)), _p(V), _p(W), C.c_int(int(f16)))
    return V, W


def integrate_raycast(grid, views):
    """Alg. 2 as printed (march every training ray), FP64."""
    V = np.full(grid.shape_zyx, -1.0, np.float64)
    W = np.zeros(grid.shape_zyx, np.uint8)
    dep, K, P = _f(views.depth), _f(views.K), _f(views.c2w)
    lib().orc_integrate_raycast_f64(C.c_int(grid.nx), C.c_int(grid.ny), C.c_int(grid.nz), _p(_origin(grid)),
                                    C.c_double(grid.voxel_size), C.c_double(grid.trunc), _p(dep),
                                    C.c_int(dep.shape[0]), C.c_int(dep.shape[1]), C.c_int(dep.shape[2]),
                                    _p(K), _p(P), _p(V), _p(W))
    return V, W


def integrate_raycast_batched(grid, views, mode="f32", V=None, W=None):
    """Alg. 2 as printed with each view's rays applied together (reading R27).

    mode "f64": FP64 reference (sums in FP64); "f32": fp32-exact mode (binary32
    rays and walk, fixed-point sums in 2^-32 units, FP64 update rounded once).
    ``grid.dtype`` "f16" stores V as IEEE half (uint16 bits), rounded once per view.
    V/W: initial state (default V = -1, W = 0).  Returns (V, W)."""
    f16 = grid.dtype == "f16"
    if V is None:
        V = np.full(grid.shape_zyx, 0xBC00, np.uint16) if f16 else \
            np.full(grid.shape_zyx, -1.0, np.float64 if mode == "f64" else np.float32)
    else:
        V = np.array(V, np.uint16 if f16 else (np.float64 if mode == "f64" else np.float32), copy=True)
    W = np.zeros(grid.shape_zyx, np.uint8) if W is None else np.array(W, np.uint8, copy=True)
    fn = lib().orc_integrate_raycast_batched_f64 if mode == "f64" else lib().orc_integrate_raycast_batched_f32
    dep, K, P = _f(views.depth), _f(views.K), _f(views.c2w)
    fn(C.c_int(grid.nx), C.c_int(grid.ny), C.c_int(grid.nz), _p(_origin(grid)), C.c_double(grid.voxel_size),
       C.c_double(grid.trunc), _p(dep), C.c_int(dep.shape[0]), C.c_int(dep.shape[1]), C.c_int(dep.shape[2]),
       _p(K), _p(P), _p(V), _p(W), C.c_int(int(f16)))
    return V, W


def _grid_values(V, f16):
    if f16:
        return np.ascontiguousarray(V, np.uint16)
    return np.ascontiguousarray(V, np.float32)


def ray_bounds(grid, V, rays_o, rays_d, bp, mode="f32"):
    """Alg. 1 per ray + the adaptive count of Sec. 3.4.

    V: normalised TSDF as float32 (or uint16 half bits when grid.dtype == "f16").
    Returns dict of t_n, t_f, n, t_zero, status, steps.
    """
    f16 = grid.dtype == "f16"
    Vg = _grid_values(V, f16)
    o, d = _f(rays_o).reshape(-1, 3), _f(rays_d).reshape(-1, 3)
    N = len(o)
    dt = np.float64 if mode == "f64" else np.float32
    out = dict(t_n=np.empty(N, dt), t_f=np.empty(N, dt), n=np.empty(N, np.int32), t_zero=np.empty(N, dt),
               status=np.empty(N, np.uint8), steps=np.empty(N, np.int32))
    fn = lib().orc_ray_bounds_f64 if mode == "f64" else lib().orc_ray_bounds_f32
    fn(C.c_int(grid.nx), C.c_int(grid.ny), C.c_int(grid.nz), _p(_origin(grid)), C.c_double(grid.voxel_size),
       C.c_double(grid.trunc), _p(Vg), C.c_int(int(f16)), _p(o), _p(d), C.c_int64(N),
       C.c_double(bp.d_s), C.c_double(bp.t_near), C.c_double(bp.t_far), C.c_double(bp.step),
       C.c_int(bp.nb_radius), C.c_int(bp.m_confirm), C.c_int(bp.n_max), C.c_int(bp.n_fallback),
       _p(out["t_n"]), _p(out["t_f"]), _p(out["n"]), _p(out["t_zero"]), _p(out["status"]), _p(out["steps"]))
    return out


def dda_sequence(grid, o, d, t_near, t_far, mode="f64", cap=100000):
    """Voxels (i, j, k) and entry parameters visited by the Alg. 1 voxel walk."""
    xyz = np.empty((cap, 3), np.int32)
    t = np.empty(cap, np.float64 if mode == "f64" else np.float32)
    fn = lib().orc_dda_sequence_f64 if mode == "f64" else lib().orc_dda_sequence_f32
    n = fn(C.c_int(grid.nx), C.c_int(grid.ny), C.c_int(grid.nz), _p(_origin(grid)), C.c_double(grid.voxel_size),
           _p(_f(o)), _p(_f(d)), C.c_double(t_near), C.c_double(t_far), _p(xyz), _p(t), C.c_int64(cap))
    return xyz[:n].copy(), t[:n].copy()


def inside_mask(grid, V, radius, mode="f32"):
    """Alg. 1's far-phase test ("all neighbours < 0") evaluated at every voxel."""
    f16 = grid.dtype == "f16"
    out = np.empty(grid.shape_zyx, np.uint8)
    fn = lib().orc_inside_mask_f64 if mode == "f64" else lib().orc_inside_mask_f32
    fn(C.c_int(grid.nx), C.c_int(grid.ny), C.c_int(grid.nz), _p(_grid_values(V, f16)), C.c_int(int(f16)),
       C.c_int(radius), _p(out))
    return out


def half_from_float(x):
    return np.array([lib().orc_half_from_float(float(v)) for v in np.ravel(x)], np.uint16).reshape(np.shape(x))


def float_from_half(h):
    return np.array([lib().orc_float_from_half(int(v)) for v in np.ravel(h)], np.float32).reshape(np.shape(h))


def clip_rays(grid, rays_o, rays_d, t_near, t_far, mode="f64"):
    """[t0, t_end] = [t_near, t_far] intersected with the grid box, per ray."""
    o, d = _f(rays_o).reshape(-1, 3), _f(rays_d).reshape(-1, 3)
    N = len(o)
    dt = np.float64 if mode == "f64" else np.float32
    t0, te, ok = np.empty(N, dt), np.empty(N, dt), np.empty(N, np.uint8)
    fn = lib().orc_clip_rays_f64 if mode == "f64" else lib().orc_clip_rays_f32
    fn(C.c_int(grid.nx), C.c_int(grid.ny), C.c_int(grid.nz), _p(_origin(grid)), C.c_double(grid.voxel_size),
       _p(o), _p(d), C.c_int64(N), C.c_double(t_near), C.c_double(t_far), _p(t0), _p(te), _p(ok))
    return t0, te, ok.astype(bool)
