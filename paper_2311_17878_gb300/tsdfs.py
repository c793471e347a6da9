"""Thin Python binding of ``libtsdfs.so`` (the C ABI in ``include/tsdfs.h``).

The functions named like the C entry points marshal torch tensors (device
memory) and the current torch CUDA stream into the C calls, nothing more:
every step of the path runs in the library's kernels.  The small helper
classes at the bottom allocate outputs and workspaces with torch.

There is no fallback: if ``libtsdfs.so`` is missing or fails to load, every
call raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsdfs.so")
_LIB = None
_LOCK = threading.Lock()

TSDFS_OK, TSDFS_E_INVALID, TSDFS_E_CUDA, TSDFS_E_WORKSPACE, TSDFS_E_UNSUPPORTED, TSDFS_E_DEVICE = 0, -1, -2, -3, -4, -5
TSDFS_F32, TSDFS_F16 = 0, 1
TSDFS_MISS, TSDFS_BOUNDED, TSDFS_FALLBACK = 0, 1, 2
TSDFS_ARCH_TINY, TSDFS_ARCH_ROOM = 0, 1
TSDFS_PREC_F32, TSDFS_PREC_BF16, TSDFS_PREC_F16, TSDFS_PREC_BF16X2 = 0, 1, 2, 3
TSDFS_NETKERNEL_SERIAL, TSDFS_NETKERNEL_PIPELINED = 1, 2
TSDFS_BACKWARD_SIMT, TSDFS_BACKWARD_GEMM = 1, 2
TSDFS_OPACITY_NEUS, TSDFS_OPACITY_VOLSDF = 0, 1
TSDFS_DEV_SAMPLES_OVERFLOW, TSDFS_DEV_MARCH_CAP, TSDFS_DEV_TIMEOUT, TSDFS_DEV_NONFINITE = 1, 2, 4, 8

EXPORTS = ["tsdfs_last_error", "tsdfs_sync_status", "tsdfs_grid_init", "tsdf_integrate", "tsdfs_inside_mask_words",
           "tsdfs_inside_mask", "tsdfs_bounds_workspace_size", "tsdf_ray_bounds", "tsdfs_render_workspace_size",
           "render_rays", "tsdfs_hier_workspace_size", "render_rays_hier", "render_rays_hier96", "tsdfs_backward_workspace_size",
           "render_rays_backward", "tsdfs_packed_size", "tsdfs_pack_mlp", "tsdfs_sdf_param_count",
           "tsdfs_rgb_param_count", "tsdf_ray_bounds_noalloc", "tsdf_ray_bounds_noalloc_max_rays",
           "tsdf_recovery_bounds", "tsdf_recovery_merge", "tsdfs_check_mlp", "tsdfs_adaptive_counts_workspace_size",
           "tsdf_adaptive_counts", "tsdfs_hier_bounded_workspace_size", "render_rays_hier_bounded",
           "tsdfs_autotune_bounds", "tsdfs_set_bounds_launch_shape", "tsdfs_bounds_launch_shape",
           "tsdfs_set_network_kernel", "tsdfs_network_kernel", "tsdfs_set_test_limits",
           "tsdfs_loss_f64_workspace_size", "tsdfs_loss_f64", "tsdfs_autotune_network", "tsdfs_l2_read_probe",
           "tsdfs_raycast_workspace_size", "tsdf_integrate_raycast", "tsdfs_profile", "tsdfs_profile_read",
           "tsdfs_set_backward_kernel", "tsdfs_backward_kernel", "tsdfs_set_backward_chunk",
           "tsdfs_backward_chunk_samples", "tsdfs_train_workspace_size", "render_rays_train",
           "render_rays_backward_kept"]


class TsdfsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tsdfs error {code}: {msg}")
        self.code = code


class tsdfs_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("origin", C.c_float * 3),
                ("voxel_size", C.c_float), ("trunc", C.c_float), ("dtype", C.c_int32), ("tsdf", C.c_void_p),
                ("weight", C.c_void_p)]


class tsdfs_bounds_params(C.Structure):
    _fields_ = [("d_s", C.c_float), ("t_near", C.c_float), ("t_far", C.c_float), ("step", C.c_float),
                ("nb_radius", C.c_int32), ("m_confirm", C.c_int32), ("n_max", C.c_int32), ("n_fallback", C.c_int32)]


class tsdfs_mlp(C.Structure):
    _fields_ = [("arch", C.c_int32), ("precision", C.c_int32), ("sdf_w", C.c_void_p), ("rgb_w", C.c_void_p),
                ("packed", C.c_void_p), ("center", C.c_float * 3), ("scale", C.c_float), ("inv_s", C.c_float),
                ("beta", C.c_float), ("alpha_eps", C.c_float), ("opacity", C.c_int32)]


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2311_17878_gb300.build`")
            L = C.CDLL(LIB_PATH)
            L.tsdfs_last_error.restype = C.c_char_p
            for name in ["tsdfs_bounds_workspace_size", "tsdfs_render_workspace_size", "tsdfs_hier_workspace_size",
                         "tsdfs_backward_workspace_size", "tsdfs_train_workspace_size", "tsdfs_packed_size", "tsdfs_adaptive_counts_workspace_size",
                         "tsdfs_hier_bounded_workspace_size", "tsdfs_raycast_workspace_size",
                         "tsdfs_loss_f64_workspace_size"]:
                getattr(L, name).restype = C.c_size_t
            for name in ["tsdfs_inside_mask_words", "tsdfs_sdf_param_count", "tsdfs_rgb_param_count",
                         "tsdfs_backward_chunk_samples", "tsdfs_train_workspace_size", "render_rays_train",
           "render_rays_backward_kept"]:
                getattr(L, name).restype = C.c_int64
            L.tsdfs_bounds_workspace_size.argtypes = [C.c_int64]
            L.tsdfs_render_workspace_size.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
            L.tsdfs_hier_workspace_size.argtypes = [C.c_void_p, C.c_int64]
            L.tsdfs_adaptive_counts_workspace_size.argtypes = [C.c_int64]
            L.tsdfs_raycast_workspace_size.argtypes = [C.c_void_p]
            L.tsdfs_hier_bounded_workspace_size.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int64]
            L.tsdfs_backward_workspace_size.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
            L.tsdfs_train_workspace_size.argtypes = [C.c_void_p, C.c_int64, C.c_int64]
            L.tsdfs_packed_size.argtypes = [C.c_int32]
            L.tsdfs_sdf_param_count.argtypes = [C.c_int32]
            L.tsdfs_rgb_param_count.argtypes = [C.c_int32]
            _LIB = L
    return _LIB


def _p(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc):
    if rc != TSDFS_OK:
        raise TsdfsError(rc, lib().tsdfs_last_error().decode())


def _cuda(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


# ----------------------------------------------------------------------------
# same-name wrappers of the C entry points
# ----------------------------------------------------------------------------
def tsdfs_last_error() -> str:
    return lib().tsdfs_last_error().decode()


def tsdfs_sync_status():
    bits = C.c_uint32(0)
    rc = lib().tsdfs_sync_status(_stream(), C.byref(bits))
    if rc not in (TSDFS_OK, TSDFS_E_DEVICE):
        _check(rc)
    return rc, bits.value


def tsdfs_grid_init(grid: "Grid"):
    _check(lib().tsdfs_grid_init(C.byref(grid.c), _stream()))


def tsdfs_raycast_workspace_size(grid: "Grid") -> int:
    return int(lib().tsdfs_raycast_workspace_size(C.byref(grid.c)))


def tsdf_integrate_raycast(grid: "Grid", depth, K, c2w, workspace):
    _cuda(depth, torch.float32, "depth"), _cuda(K, torch.float32, "K"), _cuda(c2w, torch.float32, "c2w")
    nv, H, W = depth.shape
    _check(lib().tsdf_integrate_raycast(C.byref(grid.c), _p(depth), C.c_int32(nv), C.c_int32(H), C.c_int32(W), _p(K),
                                        _p(c2w), _p(workspace), C.c_size_t(workspace.numel()), _stream()))


def tsdf_integrate(grid: "Grid", depth, K, c2w):
    _cuda(depth, torch.float32, "depth"), _cuda(K, torch.float32, "K"), _cuda(c2w, torch.float32, "c2w")
    nv, H, W = depth.shape
    _check(lib().tsdf_integrate(C.byref(grid.c), _p(depth), C.c_int32(nv), C.c_int32(H), C.c_int32(W), _p(K),
                                _p(c2w), _stream()))


def tsdfs_inside_mask_words(grid: "Grid") -> int:
    return int(lib().tsdfs_inside_mask_words(C.byref(grid.c)))


def tsdfs_inside_mask(grid: "Grid", nb_radius: int, mask_bits):
    _cuda(mask_bits, torch.int32, "mask_bits")
    _check(lib().tsdfs_inside_mask(C.byref(grid.c), C.c_int32(nb_radius), _p(mask_bits), _stream()))


def tsdfs_bounds_workspace_size(n_rays: int) -> int:
    return int(lib().tsdfs_bounds_workspace_size(C.c_int64(n_rays)))


def tsdf_ray_bounds(grid: "Grid", inside_mask, ray_o, ray_d, params: tsdfs_bounds_params, t_n, t_f, n_samples,
                    offsets, t_zero, status, workspace):
    n = ray_o.shape[0]
    _check(lib().tsdf_ray_bounds(C.byref(grid.c), _p(inside_mask), _p(ray_o), _p(ray_d), C.c_int64(n),
                                 C.byref(params), _p(t_n), _p(t_f), _p(n_samples), _p(offsets), _p(t_zero),
                                 _p(status), _p(workspace), C.c_size_t(workspace.numel() if workspace is not None else 0),
                                 _stream()))


def tsdf_ray_bounds_noalloc_max_rays() -> int:
    L = lib()
    L.tsdf_ray_bounds_noalloc_max_rays.restype = C.c_int64
    return int(L.tsdf_ray_bounds_noalloc_max_rays())


def tsdf_ray_bounds_noalloc(grid: "Grid", inside_mask, ray_o, ray_d, params: tsdfs_bounds_params, t_n, t_f,
                            n_samples, offsets, t_zero, status):
    """tsdf_ray_bounds for callers that cannot allocate device memory: no
    workspace argument; the library's own fixed device scratch is used."""
    n = ray_o.shape[0]
    _check(lib().tsdf_ray_bounds_noalloc(C.byref(grid.c), _p(inside_mask), _p(ray_o), _p(ray_d), C.c_int64(n),
                                         C.byref(params), _p(t_n), _p(t_f), _p(n_samples), _p(offsets), _p(t_zero),
                                         _p(status), _stream()))


def tsdf_recovery_bounds(grid: "Grid", ray_o, ray_d, params: tsdfs_bounds_params, tau, wsum, status, t_n2, t_f2, n2,
                         offsets2, status2, workspace):
    n = ray_o.shape[0]
    _check(lib().tsdf_recovery_bounds(C.byref(grid.c), _p(ray_o), _p(ray_d), C.c_int64(n), C.byref(params),
                                      C.c_float(tau), _p(wsum), _p(status), _p(t_n2), _p(t_f2), _p(n2), _p(offsets2),
                                      _p(status2), _p(workspace),
                                      C.c_size_t(workspace.numel() if workspace is not None else 0), _stream()))


def tsdf_recovery_merge(status2, rgb2, depth2, wsum2, normal2, rgb, depth, wsum, normal):
    n = status2.shape[0]
    _check(lib().tsdf_recovery_merge(C.c_int64(n), _p(status2), _p(rgb2), _p(depth2), _p(wsum2), _p(normal2), _p(rgb),
                                     _p(depth), _p(wsum), _p(normal), _stream()))


def tsdfs_render_workspace_size(mlp: "Mlp", n_rays: int, max_samples: int) -> int:
    return int(lib().tsdfs_render_workspace_size(C.byref(mlp.c), C.c_int64(n_rays), C.c_int64(max_samples)))


def render_rays(mlp: "Mlp", ray_o, ray_d, t_n, t_f, offsets, status, max_samples, rgb, depth, wsum, normal, eik,
                workspace):
    n = ray_o.shape[0]
    _check(lib().render_rays(C.byref(mlp.c), _p(ray_o), _p(ray_d), _p(t_n), _p(t_f), _p(offsets), _p(status),
                             C.c_int64(n), C.c_int64(max_samples), _p(rgb), _p(depth), _p(wsum), _p(normal), _p(eik),
                             _p(workspace), C.c_size_t(workspace.numel()), _stream()))


def tsdfs_hier_workspace_size(mlp: "Mlp", n_rays: int) -> int:
    return int(lib().tsdfs_hier_workspace_size(C.byref(mlp.c), C.c_int64(n_rays)))


def render_rays_hier(mlp: "Mlp", grid: "Grid", ray_o, ray_d, n_coarse, n_fine, t_near, t_far, rgb, depth, wsum, normal,
                     workspace):
    n = ray_o.shape[0]
    _check(lib().render_rays_hier(C.byref(mlp.c), C.byref(grid.c), _p(ray_o), _p(ray_d), C.c_int64(n),
                                  C.c_int(n_coarse), C.c_int(n_fine), C.c_float(t_near), C.c_float(t_far), _p(rgb),
                                  _p(depth), _p(wsum), _p(normal), _p(workspace), C.c_size_t(workspace.numel()),
                                  _stream()))


def render_rays_hier96(mlp: "Mlp", grid: "Grid", ray_o, ray_d, t_near, t_far, rgb, depth, wsum, normal, workspace):
    n = ray_o.shape[0]
    _check(lib().render_rays_hier96(C.byref(mlp.c), C.byref(grid.c), _p(ray_o), _p(ray_d), C.c_int64(n),
                                    C.c_float(t_near), C.c_float(t_far), _p(rgb), _p(depth), _p(wsum), _p(normal),
                                    _p(workspace), C.c_size_t(workspace.numel()), _stream()))


def tsdfs_autotune_bounds(grid: "Grid", inside_mask, ray_o, ray_d, p, t_n, t_f, n_samples, offsets, t_zero, status,
                          workspace, reps=3):
    """Time the march's candidate launch shapes on these rays and keep the fastest; returns
    (block, blocks_per_sm, ms per launch)."""
    n = ray_o.shape[0]
    best = C.c_float(0.0)
    _check(lib().tsdfs_autotune_bounds(C.byref(grid.c), _p(inside_mask), _p(ray_o), _p(ray_d), C.c_int64(n),
                                       C.byref(p), _p(t_n), _p(t_f), _p(n_samples), _p(offsets), _p(t_zero),
                                       _p(status), _p(workspace), C.c_size_t(workspace.numel()), C.c_int32(reps),
                                       C.byref(best), _stream()))
    b, s = tsdfs_bounds_launch_shape()
    return b, s, best.value


def tsdfs_set_bounds_launch_shape(block=0, blocks_per_sm=0):
    _check(lib().tsdfs_set_bounds_launch_shape(C.c_int32(block), C.c_int32(blocks_per_sm)))


def tsdfs_set_network_kernel(precision, kernel):
    """Process-wide choice of the tensor-core network kernel for a 16-bit precision."""
    _check(lib().tsdfs_set_network_kernel(C.c_int32(precision), C.c_int32(kernel)))


def tsdfs_set_backward_kernel(kind):
    """Process-wide choice of render_rays_backward's implementation (TSDFS_BACKWARD_*)."""
    _check(lib().tsdfs_set_backward_kernel(C.c_int32(kind)))


def tsdfs_backward_kernel() -> int:
    return int(lib().tsdfs_backward_kernel())


def tsdfs_set_backward_chunk(samples=0):
    """Samples per chunk of the layer-major backward (0: the default, 16 GiB of activations)."""
    _check(lib().tsdfs_set_backward_chunk(C.c_int64(samples)))


def tsdfs_backward_chunk_samples(mlp: "Mlp", max_samples) -> int:
    rc = int(lib().tsdfs_backward_chunk_samples(C.byref(mlp.c), C.c_int64(max_samples)))
    _check(min(rc, 0))
    return rc


def tsdfs_loss_f64_workspace_size(n_rays, max_samples) -> int:
    return int(lib().tsdfs_loss_f64_workspace_size(C.c_int64(n_rays), C.c_int64(max_samples)))


def tsdfs_loss_f64(mlp: "Mlp", sdf_w64, rgb_w64, ray_o, ray_d, t_n, t_f, offsets, status, max_samples, g_rgb, g_depth,
                   g_eik, loss, workspace):
    """FP64 functional of the bounded render (the finite-difference harness); `loss` is a
    one-element float64 device tensor."""
    n = ray_o.shape[0]
    _check(lib().tsdfs_loss_f64(C.byref(mlp.c), _p(sdf_w64), _p(rgb_w64), _p(ray_o), _p(ray_d), _p(t_n), _p(t_f),
                                _p(offsets), _p(status), C.c_int64(n), C.c_int64(max_samples), _p(g_rgb), _p(g_depth),
                                _p(g_eik), _p(loss), _p(workspace), C.c_size_t(workspace.numel()), _stream()))


def tsdfs_l2_read_probe(buf, reps=20):
    """Milliseconds of `reps` streaming reads of the device tensor `buf` (kept in L2);
    returns the achieved read bandwidth in GB/s."""
    sink = torch.zeros(1, dtype=torch.int32, device=buf.device)
    ms = C.c_float(0.0)
    nbytes = buf.numel() * buf.element_size()
    _check(lib().tsdfs_l2_read_probe(_p(buf), C.c_size_t(nbytes), C.c_int32(reps), _p(sink), C.byref(ms), _stream()))
    return reps * nbytes / (ms.value / 1e3) / 1e9


def tsdfs_set_test_limits(spin_limit=0, march_step_cap=0, withhold_chunk=-1):
    """Test-only limits of the failure paths (0, 0, -1: normal operation)."""
    _check(lib().tsdfs_set_test_limits(C.c_uint32(spin_limit), C.c_int32(march_step_cap), C.c_int32(withhold_chunk)))


def tsdfs_network_kernel(precision) -> int:
    rc = int(lib().tsdfs_network_kernel(C.c_int32(precision)))
    _check(min(rc, 0))
    return rc


def tsdfs_bounds_launch_shape():
    b, s = C.c_int32(0), C.c_int32(0)
    _check(lib().tsdfs_bounds_launch_shape(C.byref(b), C.byref(s)))
    return b.value, s.value


def tsdfs_adaptive_counts_workspace_size(n_rays: int) -> int:
    return int(lib().tsdfs_adaptive_counts_workspace_size(C.c_int64(n_rays)))


def tsdf_adaptive_counts(t_n, t_f, status, n_mean, n_min, n_max, n_fallback, n_samples, offsets, mean_len, workspace):
    n = t_n.shape[0]
    _check(lib().tsdf_adaptive_counts(_p(t_n), _p(t_f), _p(status), C.c_int64(n), C.c_float(n_mean), C.c_int32(n_min),
                                      C.c_int32(n_max), C.c_int32(n_fallback), _p(n_samples), _p(offsets),
                                      _p(mean_len), _p(workspace), C.c_size_t(workspace.numel()), _stream()))


def tsdfs_hier_bounded_workspace_size(mlp: "Mlp", n_rays: int, n_fine: int, max_coarse: int) -> int:
    return int(lib().tsdfs_hier_bounded_workspace_size(C.byref(mlp.c), C.c_int64(n_rays), C.c_int32(n_fine),
                                                       C.c_int64(max_coarse)))


def render_rays_hier_bounded(mlp: "Mlp", ray_o, ray_d, t_n, t_f, offsets, status, n_fine, max_coarse, rgb, depth, wsum,
                             normal, workspace):
    n = ray_o.shape[0]
    _check(lib().render_rays_hier_bounded(C.byref(mlp.c), _p(ray_o), _p(ray_d), _p(t_n), _p(t_f), _p(offsets),
                                          _p(status), C.c_int64(n), C.c_int32(n_fine), C.c_int64(max_coarse), _p(rgb),
                                          _p(depth), _p(wsum), _p(normal), _p(workspace),
                                          C.c_size_t(workspace.numel()), _stream()))


def tsdfs_backward_workspace_size(mlp: "Mlp", n_rays: int, max_samples: int) -> int:
    return int(lib().tsdfs_backward_workspace_size(C.byref(mlp.c), C.c_int64(n_rays), C.c_int64(max_samples)))


def render_rays_backward(mlp: "Mlp", ray_o, ray_d, t_n, t_f, offsets, status, max_samples, d_rgb, d_depth, d_eik,
                         d_sdf_w, d_rgb_w, workspace):
    n = ray_o.shape[0]
    _check(lib().render_rays_backward(C.byref(mlp.c), _p(ray_o), _p(ray_d), _p(t_n), _p(t_f), _p(offsets),
                                      _p(status), C.c_int64(n), C.c_int64(max_samples), _p(d_rgb), _p(d_depth),
                                      _p(d_eik), _p(d_sdf_w), _p(d_rgb_w), _p(workspace),
                                      C.c_size_t(workspace.numel()), _stream()))


def tsdfs_train_workspace_size(mlp: "Mlp", n_rays: int, max_samples: int) -> int:
    return int(lib().tsdfs_train_workspace_size(C.byref(mlp.c), C.c_int64(n_rays), C.c_int64(max_samples)))


def render_rays_train(mlp: "Mlp", ray_o, ray_d, t_n, t_f, offsets, status, max_samples, rgb, depth, wsum, normal, eik,
                      workspace):
    """render_rays with the layer-major FP32 networks, keeping records and activations in
    `workspace` for render_rays_backward_kept."""
    n = ray_o.shape[0]
    _check(lib().render_rays_train(C.byref(mlp.c), _p(ray_o), _p(ray_d), _p(t_n), _p(t_f), _p(offsets), _p(status),
                                   C.c_int64(n), C.c_int64(max_samples), _p(rgb), _p(depth), _p(wsum), _p(normal),
                                   _p(eik), _p(workspace), C.c_size_t(workspace.numel()), _stream()))


def render_rays_backward_kept(mlp: "Mlp", ray_o, ray_d, t_n, t_f, offsets, status, max_samples, d_rgb, d_depth, d_eik,
                              d_sdf_w, d_rgb_w, workspace):
    n = ray_o.shape[0]
    _check(lib().render_rays_backward_kept(C.byref(mlp.c), _p(ray_o), _p(ray_d), _p(t_n), _p(t_f), _p(offsets),
                                           _p(status), C.c_int64(n), C.c_int64(max_samples), _p(d_rgb), _p(d_depth),
                                           _p(d_eik), _p(d_sdf_w), _p(d_rgb_w), _p(workspace),
                                           C.c_size_t(workspace.numel()), _stream()))


def tsdfs_packed_size(arch: int) -> int:
    return int(lib().tsdfs_packed_size(C.c_int32(arch)))


def tsdfs_pack_mlp(mlp: "Mlp", packed):
    _check(lib().tsdfs_pack_mlp(C.byref(mlp.c), _p(packed), _stream()))


def tsdfs_check_mlp(mlp: "Mlp"):
    _check(lib().tsdfs_check_mlp(C.byref(mlp.c), _stream()))


def tsdfs_sdf_param_count(arch: int) -> int:
    return int(lib().tsdfs_sdf_param_count(C.c_int32(arch)))


def tsdfs_rgb_param_count(arch: int) -> int:
    return int(lib().tsdfs_rgb_param_count(C.c_int32(arch)))


# ----------------------------------------------------------------------------
# allocation helpers (torch memory only)
# ----------------------------------------------------------------------------
def _bytes(n, device):
    return torch.empty(max(int(n), 1), dtype=torch.uint8, device=device)


@dataclass
class GridSpecLike:
    """Grid geometry (the fields of ``tsdfs_grid`` besides the arrays)."""
    nx: int
    ny: int
    nz: int
    origin: tuple
    voxel_size: float
    trunc: float
    dtype: str = "f32"


class Grid:
    """A TSDF grid in device memory (V, W) and its ``tsdfs_grid`` descriptor."""

    def __init__(self, spec, device="cuda", V=None, W=None):
        self.spec = spec
        shape = (spec.nz, spec.ny, spec.nx)
        f16 = spec.dtype == "f16"
        if V is None:
            V = torch.empty(shape, dtype=torch.float16 if f16 else torch.float32, device=device)
        if W is None:
            W = torch.empty(shape, dtype=torch.uint8, device=device)
        self.V, self.W = V.contiguous(), W.contiguous()
        self.c = tsdfs_grid(spec.nx, spec.ny, spec.nz, (C.c_float * 3)(*spec.origin), spec.voxel_size, spec.trunc,
                            TSDFS_F16 if f16 else TSDFS_F32, self.V.data_ptr(), self.W.data_ptr())

    def init(self):
        tsdfs_grid_init(self)
        return self

    def integrate(self, depth, K, c2w):
        tsdf_integrate(self, depth, K, c2w)
        return self

    def integrate_raycast(self, depth, K, c2w, workspace=None):
        """Alg. 2 as printed (every pixel's ray marched), each view's rays applied together."""
        ws = workspace if workspace is not None else _bytes(tsdfs_raycast_workspace_size(self), self.V.device)
        tsdf_integrate_raycast(self, depth, K, c2w, ws)
        return self

    def save(self, path):
        """Checkpoint of the fused volume: geometry header plus V and W (V in its storage
        type), so later sessions render novel views without fusing again."""
        sp = self.spec
        header = np.array([sp.nx, sp.ny, sp.nz, *sp.origin, sp.voxel_size, sp.trunc], np.float64)
        np.savez(path, header=header, dtype=np.array(sp.dtype), V=self.V.cpu().numpy(), W=self.W.cpu().numpy())

    @classmethod
    def load(cls, path, device="cuda"):
        z = np.load(path)
        h = z["header"]
        spec = GridSpecLike(int(h[0]), int(h[1]), int(h[2]), (float(h[3]), float(h[4]), float(h[5])), float(h[6]),
                            float(h[7]), str(z["dtype"]))
        return cls(spec, device=device, V=torch.as_tensor(z["V"]).to(device), W=torch.as_tensor(z["W"]).to(device))

    def inside_mask(self, nb_radius):
        bits = torch.empty(tsdfs_inside_mask_words(self), dtype=torch.int32, device=self.V.device)
        tsdfs_inside_mask(self, nb_radius, bits)
        return bits


def bounds_params(bp) -> tsdfs_bounds_params:
    return tsdfs_bounds_params(bp.d_s, bp.t_near, bp.t_far, bp.step, bp.nb_radius, bp.m_confirm, bp.n_max,
                               bp.n_fallback)


class Bounds:
    """Outputs of ``tsdf_ray_bounds`` for a batch of rays (device tensors)."""

    def __init__(self, n, device="cuda"):
        self.t_n = torch.empty(n, dtype=torch.float32, device=device)
        self.t_f = torch.empty(n, dtype=torch.float32, device=device)
        self.n = torch.empty(n, dtype=torch.int32, device=device)
        self.offsets = torch.empty(n + 1, dtype=torch.int32, device=device)
        self.t_zero = torch.empty(n, dtype=torch.float32, device=device)
        self.status = torch.empty(n, dtype=torch.uint8, device=device)
        self.workspace = _bytes(tsdfs_bounds_workspace_size(n), device)

    def autotune(self, grid: Grid, rays_o, rays_d, bp, inside_mask=None, reps=3):
        """Pick the march's launch shape on these rays (tsdfs_autotune_bounds); fills the outputs."""
        p = bp if isinstance(bp, tsdfs_bounds_params) else bounds_params(bp)
        return tsdfs_autotune_bounds(grid, inside_mask, rays_o, rays_d, p, self.t_n, self.t_f, self.n, self.offsets,
                                     self.t_zero, self.status, self.workspace, reps)

    def compute(self, grid: Grid, rays_o, rays_d, bp, inside_mask=None):
        p = bp if isinstance(bp, tsdfs_bounds_params) else bounds_params(bp)
        tsdf_ray_bounds(grid, inside_mask, rays_o, rays_d, p, self.t_n, self.t_f, self.n, self.offsets, self.t_zero,
                        self.status, self.workspace)
        return self


class Mlp:
    """Network parameters on the device and their ``tsdfs_mlp`` descriptor.

    By default the parameters are copied from ``spec`` into new device tensors.  Given
    ``sdf_w`` / ``rgb_w`` (contiguous float32 device tensors of the packed parameter
    layout), the descriptor points at those tensors instead, without a copy; 16-bit
    precisions then pack them into a buffer of their own at construction, so a later
    change of the tensors needs :meth:`repack`."""

    def __init__(self, spec, precision=TSDFS_PREC_F32, device="cuda", sdf_w=None, rgb_w=None):
        self.spec = spec
        self.sdf_w = torch.tensor(spec.packed("sdf"), device=device) if sdf_w is None else \
            _param_tensor(sdf_w, tsdfs_sdf_param_count(spec.arch), "sdf_w")
        self.rgb_w = torch.tensor(spec.packed("rgb"), device=device) if rgb_w is None else \
            _param_tensor(rgb_w, tsdfs_rgb_param_count(spec.arch), "rgb_w")
        if self.sdf_w.device != self.rgb_w.device:
            raise ValueError("sdf_w and rgb_w must be on the same device")
        device = self.sdf_w.device
        self.packed = None
        self.precision = precision
        if precision != TSDFS_PREC_F32:
            self.packed = torch.zeros(max(tsdfs_packed_size(spec.arch), 1), dtype=torch.uint8, device=device)
        self.c = tsdfs_mlp(spec.arch, precision, self.sdf_w.data_ptr(), self.rgb_w.data_ptr(),
                           self.packed.data_ptr() if self.packed is not None else None,
                           (C.c_float * 3)(*spec.center), spec.scale, spec.inv_s, spec.beta, spec.alpha_eps,
                           spec.opacity)
        if precision != TSDFS_PREC_F32:
            tsdfs_pack_mlp(self, self.packed)

    def with_params(self, sdf_w, rgb_w):
        """The same networks (architecture, precision, constants) over the given
        parameter tensors, which the returned descriptor reads in place."""
        return Mlp(self.spec, self.precision, sdf_w=sdf_w, rgb_w=rgb_w)

    def repack(self):
        if self.packed is not None:
            tsdfs_pack_mlp(self, self.packed)


def _param_tensor(w, count, name):
    """A caller's parameter tensor, checked: float32, contiguous, on a CUDA device,
    `count` elements (the packed (W, b) layout of the network's layers)."""
    w = w.detach()
    if w.dtype != torch.float32 or not w.is_contiguous() or not w.is_cuda:
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if w.numel() != count:
        raise ValueError(f"{name} has {w.numel()} elements, the network has {count} parameters")
    return w


class RenderOut:
    def __init__(self, n, device="cuda"):
        self.rgb = torch.empty((n, 3), dtype=torch.float32, device=device)
        self.depth = torch.empty(n, dtype=torch.float32, device=device)
        self.wsum = torch.empty(n, dtype=torch.float32, device=device)
        self.normal = torch.empty((n, 3), dtype=torch.float32, device=device)
        self.eik = torch.empty(n, dtype=torch.float32, device=device)


class Renderer:
    """render_rays with a workspace sized for ``max_samples``."""

    def __init__(self, mlp: Mlp, n_rays, max_samples, device="cuda"):
        self.mlp = mlp
        self.max_samples = int(max_samples)
        self.out = RenderOut(n_rays, device)
        self.workspace = _bytes(tsdfs_render_workspace_size(mlp, n_rays, self.max_samples), device)

    def render(self, rays_o, rays_d, b: Bounds):
        o = self.out
        render_rays(self.mlp, rays_o, rays_d, b.t_n, b.t_f, b.offsets, b.status, self.max_samples, o.rgb, o.depth,
                    o.wsum, o.normal, o.eik, self.workspace)
        return o

    def autotune(self, rays_o, rays_d, b: Bounds, reps=3):
        """Pick the faster network kernel for this precision on these rays
        (tsdfs_autotune_network); returns (kernel, ms serial, ms pipelined)."""
        o = self.out
        ms = (C.c_float * 2)(-1.0, -1.0)
        rc = int(lib().tsdfs_autotune_network(C.byref(self.mlp.c), _p(rays_o), _p(rays_d), _p(b.t_n), _p(b.t_f),
                                              _p(b.offsets), _p(b.status), C.c_int64(rays_o.shape[0]),
                                              C.c_int64(self.max_samples), _p(o.rgb), _p(o.depth), _p(o.wsum),
                                              _p(o.normal), _p(self.workspace), C.c_size_t(self.workspace.numel()),
                                              C.c_int32(reps), ms, _stream()))
        _check(min(rc, 0))
        return rc, float(ms[0]), float(ms[1])


class Recovery:
    """The recovery pass of Sec. 4.5 for a batch of rays: rays whose weight sum
    after ``Renderer.render`` stays below ``tau`` are rendered again over the
    whole [t0, t_end] with ``n_fallback`` samples, and merged into ``out``."""

    def __init__(self, mlp: Mlp, n, n_fallback=96, device="cuda"):
        self.bounds = Bounds(n, device)
        self.render2 = Renderer(mlp, n, max(n * n_fallback, 1), device)

    def apply(self, grid: Grid, rays_o, rays_d, bp, tau, out: RenderOut, first: Bounds):
        p = bp if isinstance(bp, tsdfs_bounds_params) else bounds_params(bp)
        b = self.bounds
        tsdf_recovery_bounds(grid, rays_o, rays_d, p, tau, out.wsum, first.status, b.t_n, b.t_f, b.n, b.offsets,
                             b.status, b.workspace)
        o2 = self.render2.render(rays_o, rays_d, b)
        tsdf_recovery_merge(b.status, o2.rgb, o2.depth, o2.wsum, o2.normal, out.rgb, out.depth, out.wsum, out.normal)
        return out


class AdaptiveCounts:
    """Counts relative to the mean interval (tsdf_adaptive_counts) for the bounds
    of a batch: ``apply`` returns a ``Bounds`` view sharing the input's t_n, t_f and
    status with the new counts and offsets."""

    def __init__(self, n, device="cuda"):
        self.n = torch.empty(n, dtype=torch.int32, device=device)
        self.offsets = torch.empty(n + 1, dtype=torch.int32, device=device)
        self.mean_len = torch.empty(1, dtype=torch.float32, device=device)
        self.workspace = _bytes(tsdfs_adaptive_counts_workspace_size(n), device)

    def apply(self, b: Bounds, n_mean, n_min=2, n_max=64, n_fallback=64):
        tsdf_adaptive_counts(b.t_n, b.t_f, b.status, n_mean, n_min, n_max, n_fallback, self.n, self.offsets,
                             self.mean_len, self.workspace)
        out = Bounds.__new__(Bounds)
        out.t_n, out.t_f, out.status, out.t_zero = b.t_n, b.t_f, b.status, b.t_zero
        out.n, out.offsets, out.workspace = self.n, self.offsets, None
        return out


class HierBoundedRenderer:
    """Coarse + fine inside the TSDF bound (render_rays_hier_bounded): the bounds'
    counts are the coarse samples, ``n_fine`` inverse-CDF samples are added per ray."""

    def __init__(self, mlp: Mlp, n_rays, n_fine, max_coarse, device="cuda"):
        self.mlp = mlp
        self.n_fine, self.max_coarse = int(n_fine), int(max_coarse)
        self.out = RenderOut(n_rays, device)
        self.workspace = _bytes(tsdfs_hier_bounded_workspace_size(mlp, n_rays, self.n_fine, self.max_coarse), device)

    def render(self, rays_o, rays_d, b: Bounds):
        o = self.out
        render_rays_hier_bounded(self.mlp, rays_o, rays_d, b.t_n, b.t_f, b.offsets, b.status, self.n_fine,
                                 self.max_coarse, o.rgb, o.depth, o.wsum, o.normal, self.workspace)
        return o


class HierRenderer:
    """The hierarchical comparator: n_coarse uniform + n_fine inverse-CDF samples per ray (64 + 32 by default)."""

    def __init__(self, mlp: Mlp, n_rays, device="cuda", n_coarse=64, n_fine=32):
        self.mlp = mlp
        self.n_coarse, self.n_fine = int(n_coarse), int(n_fine)
        self.out = RenderOut(n_rays, device)
        self.workspace = _bytes(tsdfs_hier_workspace_size(mlp, n_rays), device)

    def render(self, grid: Grid, rays_o, rays_d, t_near, t_far):
        o = self.out
        render_rays_hier(self.mlp, grid, rays_o, rays_d, self.n_coarse, self.n_fine, t_near, t_far, o.rgb, o.depth,
                         o.wsum, o.normal, self.workspace)
        return o


class RenderFunction(torch.autograd.Function):
    """render_rays as a differentiable torch op over the packed fp32 parameters.

    forward(sdf_w, rgb_w, mlp, rays_o, rays_d, bounds, max_samples) -> (rgb, depth, eik)
    renders with ``mlp``'s architecture, precision and constants over the parameter
    tensors ``sdf_w`` / ``rgb_w`` themselves (read in place; 16-bit precisions pack them
    on every call), so an optimizer stepping those tensors changes the next render.
    With FP32 networks and the layer-major backward (the default) the forward is
    render_rays_train and the backward render_rays_backward_kept over the workspace the
    forward kept; otherwise the forward is render_rays and the backward calls
    render_rays_backward (FP32 networks, activations recomputed) at the same tensors.
    """

    @staticmethod
    def forward(ctx, sdf_w, rgb_w, mlp, rays_o, rays_d, b, max_samples):
        n = rays_o.shape[0]
        m = mlp.with_params(sdf_w, rgb_w)
        out = RenderOut(n, device=rays_o.device)
        ctx.b, ctx.max_samples = b, max_samples
        ctx.save_for_backward(rays_o, rays_d)
        if m.precision == TSDFS_PREC_F32 and tsdfs_backward_kernel() == TSDFS_BACKWARD_GEMM:
            ws = _bytes(tsdfs_train_workspace_size(m, n, max_samples), rays_o.device)
            render_rays_train(m, rays_o, rays_d, b.t_n, b.t_f, b.offsets, b.status, max_samples, out.rgb, out.depth,
                              out.wsum, out.normal, out.eik, ws)
            ctx.mlp, ctx.kept = m, ws
            return out.rgb, out.depth, out.eik
        ws = _bytes(tsdfs_render_workspace_size(m, n, max_samples), rays_o.device)
        render_rays(m, rays_o, rays_d, b.t_n, b.t_f, b.offsets, b.status, max_samples, out.rgb, out.depth,
                    out.wsum, out.normal, out.eik, ws)
        # the backward runs the FP32 networks over the same parameter tensors
        ctx.mlp = m if m.precision == TSDFS_PREC_F32 else Mlp(mlp.spec, TSDFS_PREC_F32, sdf_w=sdf_w, rgb_w=rgb_w)
        ctx.kept = None
        return out.rgb, out.depth, out.eik

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_eik):
        rays_o, rays_d = ctx.saved_tensors
        mlp, b, ms = ctx.mlp, ctx.b, ctx.max_samples
        n = rays_o.shape[0]
        d_sdf = torch.zeros_like(mlp.sdf_w)
        d_rgb = torch.zeros_like(mlp.rgb_w)
        gr = (g_rgb if g_rgb is not None else torch.zeros((n, 3), device=rays_o.device)).contiguous().float()
        gd = None if g_depth is None else g_depth.contiguous().float()
        ge = None if g_eik is None else g_eik.contiguous().float()
        if ctx.kept is not None:
            render_rays_backward_kept(mlp, rays_o, rays_d, b.t_n, b.t_f, b.offsets, b.status, ms, gr, gd, ge, d_sdf,
                                      d_rgb, ctx.kept)
            ctx.kept = None
        else:
            ws = _bytes(tsdfs_backward_workspace_size(mlp, n, ms), rays_o.device)
            render_rays_backward(mlp, rays_o, rays_d, b.t_n, b.t_f, b.offsets, b.status, ms, gr, gd, ge, d_sdf, d_rgb,
                                 ws)
        return d_sdf, d_rgb, None, None, None, None, None
