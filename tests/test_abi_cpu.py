"""The C-ABI library loads on a machine without a GPU, exports every entry
point that include/tsdfs.h declares, and rejects bad arguments on the host
(before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import torch

from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return T.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "tsdfs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("typedef",)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    assert set(T.EXPORTS) <= set(names)


def test_param_counts_match_architectures(L):
    for arch, spec in [(T.TSDFS_ARCH_TINY, synth.tiny_mlp()), (T.TSDFS_ARCH_ROOM, synth.room_mlp())]:
        assert T.tsdfs_sdf_param_count(arch) == spec.packed("sdf").size
        assert T.tsdfs_rgb_param_count(arch) == spec.packed("rgb").size
    assert T.tsdfs_sdf_param_count(7) == -1


def test_workspace_sizes_are_monotone(L):
    assert T.tsdfs_bounds_workspace_size(0) > 0
    assert T.tsdfs_bounds_workspace_size(10 ** 6) >= T.tsdfs_bounds_workspace_size(10)
    m = T.tsdfs_mlp()
    assert L.tsdfs_render_workspace_size(C.byref(m), 10, 1000) >= 1000 * 48
    assert L.tsdfs_hier_workspace_size(C.byref(m), 100) >= 100 * 96 * 48


def _grid_struct(nx=8):
    return T.tsdfs_grid(nx, nx, nx, (C.c_float * 3)(0, 0, 0), 0.1, 0.3, T.TSDFS_F32, 0x1000, 0x2000)


def test_invalid_arguments_fail_on_host(L):
    g = _grid_struct()
    p = T.tsdfs_bounds_params(0.1, 0.0, 10.0, 0.1, 2, 15, 32, 96)
    # NULL grid
    assert L.tsdf_ray_bounds(None, None, None, None, C.c_int64(0), C.byref(p), None, None, None, None, None, None,
                             None, C.c_size_t(0), None) == T.TSDFS_E_INVALID
    assert "grid" in T.tsdfs_last_error()
    # bad radius
    p.nb_radius = 9
    assert L.tsdf_ray_bounds(C.byref(g), None, None, None, C.c_int64(0), C.byref(p), None, None, None,
                             C.c_void_p(0x3000), None, None, C.c_void_p(0x4000), C.c_size_t(1 << 20),
                             None) == T.TSDFS_E_INVALID
    p.nb_radius = 2
    # workspace too small
    assert L.tsdf_ray_bounds(C.byref(g), None, C.c_void_p(8), C.c_void_p(8), C.c_int64(100), C.byref(p),
                             C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), None, C.c_void_p(8),
                             C.c_void_p(8), C.c_size_t(1), None) == T.TSDFS_E_WORKSPACE
    # bad grid geometry
    g.voxel_size = 0.0
    assert L.tsdfs_grid_init(C.byref(g), None) == T.TSDFS_E_INVALID
    g.voxel_size = 0.1
    g.dtype = 5
    assert L.tsdf_integrate(C.byref(g), None, 1, 4, 4, None, None, None) == T.TSDFS_E_INVALID
    # bad mlp
    m = T.tsdfs_mlp(9, 0, 8, 8, None, (C.c_float * 3)(0, 0, 0), 1.0, 64.0, 100.0, 1e-5)
    assert L.render_rays(C.byref(m), *([C.c_void_p(8)] * 7), C.c_int64(1), C.c_int64(1), *([C.c_void_p(8)] * 5),
                         C.c_void_p(8), C.c_size_t(1 << 20), None) == T.TSDFS_E_INVALID
    m.arch = 0
    m.precision = T.TSDFS_PREC_BF16
    assert L.render_rays(C.byref(m), *([C.c_void_p(8)] * 7), C.c_int64(1), C.c_int64(1), *([C.c_void_p(8)] * 5),
                         C.c_void_p(8), C.c_size_t(1 << 20), None) == T.TSDFS_E_INVALID  # packed is NULL
    # unknown opacity transform
    m.precision = 0
    m.opacity = 5
    assert L.render_rays(C.byref(m), *([C.c_void_p(8)] * 7), C.c_int64(1), C.c_int64(1), *([C.c_void_p(8)] * 5),
                         C.c_void_p(8), C.c_size_t(1 << 20), None) == T.TSDFS_E_INVALID
    assert "opacity" in T.tsdfs_last_error()
    m.opacity = T.TSDFS_OPACITY_VOLSDF
    # zero rays is a no-op that succeeds without touching the device
    m.precision = 0
    assert L.render_rays(C.byref(m), *([None] * 6), C.c_int64(0), C.c_int64(0), *([None] * 5), None, C.c_size_t(0),
                         None) == T.TSDFS_OK


def test_hier_counts_checked_on_host(L):
    g = _grid_struct()
    m = T.tsdfs_mlp(0, 0, 8, 8, None, (C.c_float * 3)(0, 0, 0), 1.0, 64.0, 100.0, 1e-5)
    v = C.c_void_p(8)
    ws = L.tsdfs_hier_workspace_size(C.byref(m), 100)
    for nc, nf in [(1, 8), (65, 8), (16, 0), (16, 33)]:
        assert L.render_rays_hier(C.byref(m), C.byref(g), v, v, C.c_int64(100), nc, nf, C.c_float(0.1),
                                  C.c_float(5.0), v, v, v, None, v, C.c_size_t(ws), None) == T.TSDFS_E_INVALID
        assert "sample counts" in T.tsdfs_last_error()
    # zero rays with valid counts succeed without the device
    assert L.render_rays_hier(C.byref(m), C.byref(g), None, None, C.c_int64(0), 16, 8, C.c_float(0.1), C.c_float(5.0),
                              None, None, None, None, None, C.c_size_t(0), None) == T.TSDFS_OK


def test_adaptive_counts_and_bounded_hier_arguments_fail_on_host(L):
    v = C.c_void_p(8)
    ws = T.tsdfs_adaptive_counts_workspace_size(100)
    args = lambda n_mean, n_min, n_max, n_fb, wsb=ws: (v, v, v, C.c_int64(100), C.c_float(n_mean), C.c_int32(n_min),
                                                       C.c_int32(n_max), C.c_int32(n_fb), v, v, None, v,
                                                       C.c_size_t(wsb), None)
    for bad in [(0.0, 1, 64, 96), (float("nan"), 1, 64, 96), (6.0, 0, 64, 96), (6.0, 9, 8, 96), (6.0, 1, 5000, 96),
                (6.0, 1, 64, -1)]:
        assert L.tsdf_adaptive_counts(*args(*bad)) == T.TSDFS_E_INVALID
    assert L.tsdf_adaptive_counts(*args(6.0, 1, 64, 96, 1)) == T.TSDFS_E_WORKSPACE
    # zero rays: offsets[0] = 0 is written on the stream (needs the device), so only the
    # workspace-size function is checked here
    assert T.tsdfs_adaptive_counts_workspace_size(0) > 0
    assert T.tsdfs_adaptive_counts_workspace_size(10 ** 6) > T.tsdfs_adaptive_counts_workspace_size(10)
    m = T.tsdfs_mlp(0, 0, 8, 8, None, (C.c_float * 3)(0, 0, 0), 1.0, 64.0, 100.0, 1e-5)
    wsh = L.tsdfs_hier_bounded_workspace_size(C.byref(m), C.c_int64(100), C.c_int32(8), C.c_int64(1000))
    assert wsh >= (1000 + 100 * 8) * 48
    hb = lambda n_fine, wsb=wsh, n=100: L.render_rays_hier_bounded(C.byref(m), v, v, v, v, v, v, C.c_int64(n),
                                                                  C.c_int32(n_fine), C.c_int64(1000), v, v, v, None,
                                                                  v, C.c_size_t(wsb), None)
    assert hb(-1) == T.TSDFS_E_INVALID and hb(33) == T.TSDFS_E_INVALID
    assert "fine" in T.tsdfs_last_error()
    assert hb(8, 16) == T.TSDFS_E_WORKSPACE
    assert hb(8, 0, 0) == T.TSDFS_OK


def test_network_kernel_choice(L):
    """Per-precision choice of the network kernel: both kernels for BF16 / FP16, the
    pipelined one only for BF16X2, nothing for FP32."""
    assert L.tsdfs_network_kernel(3) == 2
    assert L.tsdfs_set_network_kernel(3, 1) < 0
    assert L.tsdfs_set_network_kernel(0, 1) < 0 and L.tsdfs_network_kernel(0) < 0
    assert L.tsdfs_set_network_kernel(2, 7) < 0
    for prec in (1, 2):
        old = L.tsdfs_network_kernel(prec)
        assert old in (1, 2)
        assert L.tsdfs_set_network_kernel(prec, 2) == 0 and L.tsdfs_network_kernel(prec) == 2
        assert L.tsdfs_set_network_kernel(prec, 1) == 0 and L.tsdfs_network_kernel(prec) == 1
        assert L.tsdfs_set_network_kernel(prec, old) == 0


def test_backward_kernel_choice_and_workspace(L):
    """The layer-major backward is the default; the workspace follows the choice and the
    chunk (records of every sample plus the activations of one chunk)."""
    assert L.tsdfs_backward_kernel() == T.TSDFS_BACKWARD_GEMM
    assert L.tsdfs_set_backward_kernel(0) < 0 and L.tsdfs_set_backward_kernel(3) < 0
    assert L.tsdfs_set_backward_chunk(C.c_int64(-1)) < 0 and L.tsdfs_set_backward_chunk(C.c_int64(1 << 29)) < 0
    mlp = T.Mlp(synth.room_mlp(), device="cpu")
    size = lambda ms: T.tsdfs_backward_workspace_size(mlp, 1000, ms)
    try:
        big = size(200000)
        assert T.tsdfs_backward_chunk_samples(mlp, 200000) > 150000
        assert L.tsdfs_set_backward_chunk(C.c_int64(1000)) == 0
        assert T.tsdfs_backward_chunk_samples(mlp, 200000) == 1000
        assert T.tsdfs_backward_chunk_samples(mlp, 10) == 10
        small = size(200000)
        assert small < big
        # room: 4 SDF rows of every layer's padded input and output, the colour rows and
        # two work buffers make about 79 KB per sample of a chunk; records 80 B per sample
        per_sample = (small - size(1) - 199999 * 80) / 999
        assert 75e3 < per_sample < 85e3, per_sample
        assert size(500) < small
        assert L.tsdfs_set_backward_kernel(T.TSDFS_BACKWARD_SIMT) == 0
        assert L.tsdfs_backward_kernel() == T.TSDFS_BACKWARD_SIMT
        assert size(200000) != small
    finally:
        L.tsdfs_set_backward_chunk(C.c_int64(0))
        L.tsdfs_set_backward_kernel(T.TSDFS_BACKWARD_GEMM)


def test_bounds_launch_shape_arguments(L):
    for b, sm in [(16, 8), (96 + 1, 8), (512, 8), (128, 0), (128, 2000)]:
        assert L.tsdfs_set_bounds_launch_shape(C.c_int32(b), C.c_int32(sm)) == T.TSDFS_E_INVALID
    assert L.tsdfs_bounds_launch_shape(None, None) == T.TSDFS_E_INVALID
    v = C.c_void_p(8)
    p = T.tsdfs_bounds_params(0.1, 0.0, 10.0, 0.1, 2, 15, 32, 96)
    g = _grid_struct()
    assert L.tsdfs_autotune_bounds(C.byref(g), None, v, v, C.c_int64(10), C.byref(p), v, v, v, v, None, v, v,
                                   C.c_size_t(1 << 20), C.c_int32(0), None, None) == T.TSDFS_E_INVALID
    assert L.tsdfs_autotune_bounds(C.byref(g), None, v, v, C.c_int64(0), C.byref(p), v, v, v, v, None, v, v,
                                   C.c_size_t(1 << 20), C.c_int32(3), None, None) == T.TSDFS_E_INVALID


def test_raycast_fusion_arguments_fail_on_host(L):
    g = _grid_struct()
    v = C.c_void_p(8)
    ws = L.tsdfs_raycast_workspace_size(C.byref(g))
    assert ws >= 8 * 8 * 8 * 12
    call = lambda nv, H, W, wsb: L.tsdf_integrate_raycast(C.byref(g), v, C.c_int32(nv), C.c_int32(H), C.c_int32(W),
                                                         v, v, v, C.c_size_t(wsb), None)
    assert call(-1, 4, 4, ws) == T.TSDFS_E_INVALID
    assert call(1, 0, 4, ws) == T.TSDFS_E_INVALID
    assert call(1, 2048, 2048, ws) == T.TSDFS_E_INVALID and "2^21" in T.tsdfs_last_error()
    assert call(1, 4, 4, ws - 1) == T.TSDFS_E_WORKSPACE
    assert call(0, 4, 4, 0) == T.TSDFS_OK   # no views: nothing to do, no device touched
    g.weight = None
    assert call(1, 4, 4, ws) == T.TSDFS_E_INVALID


def test_recovery_arguments_fail_on_host(L):
    g = _grid_struct()
    p = T.tsdfs_bounds_params(0.1, 0.0, 10.0, 0.1, 2, 15, 32, 96)
    v = C.c_void_p(8)
    args = lambda tau, ws: (C.byref(g), v, v, C.c_int64(100), C.byref(p), C.c_float(tau), v, v, v, v, v, v, v, v,
                            C.c_size_t(ws), None)
    assert L.tsdf_recovery_bounds(None, v, v, C.c_int64(1), C.byref(p), C.c_float(0.9), *([v] * 8),
                                  C.c_size_t(1 << 20), None) == T.TSDFS_E_INVALID
    assert L.tsdf_recovery_bounds(*args(float("nan"), 1 << 20)) == T.TSDFS_E_INVALID
    assert "tau" in T.tsdfs_last_error()
    assert L.tsdf_recovery_bounds(*args(0.95, 1)) == T.TSDFS_E_WORKSPACE
    p.n_fallback = 5000
    assert L.tsdf_recovery_bounds(*args(0.95, 1 << 20)) == T.TSDFS_E_INVALID
    # merge: normal and normal2 both or neither; zero rays succeed without the device
    assert L.tsdf_recovery_merge(C.c_int64(4), v, v, v, v, None, v, v, v, v, None) == T.TSDFS_E_INVALID
    assert L.tsdf_recovery_merge(C.c_int64(-1), v, v, v, v, v, v, v, v, v, None) == T.TSDFS_E_INVALID
    assert L.tsdf_recovery_merge(C.c_int64(0), None, None, None, None, None, None, None, None, None, None) == T.TSDFS_OK


def test_grid_checkpoint_roundtrip(tmp_path):
    from paper_2311_17878_gb300 import synth
    for dtype, tdt in (("f32", torch.float32), ("f16", torch.float16)):
        spec = synth.GridSpec(7, 5, 3, (-0.5, 0.25, 1.0), 0.125, 0.375, dtype)
        g = T.Grid(spec, device="cpu", V=torch.linspace(-1, 1, 105).reshape(3, 5, 7).to(tdt),
                   W=torch.arange(105, dtype=torch.uint8).reshape(3, 5, 7))
        path = tmp_path / f"grid_{dtype}.npz"
        g.save(path)
        h = T.Grid.load(path, device="cpu")
        assert (h.spec.nx, h.spec.ny, h.spec.nz, h.spec.dtype) == (7, 5, 3, dtype)
        assert h.spec.origin == spec.origin and h.spec.voxel_size == spec.voxel_size and h.spec.trunc == spec.trunc
        assert torch.equal(h.V, g.V) and torch.equal(h.W, g.W) and h.V.dtype == tdt
        assert h.c.nx == 7 and h.c.dtype == (T.TSDFS_F16 if dtype == "f16" else T.TSDFS_F32)
