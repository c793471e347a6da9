"""GPU parity of the ray-casting fusion (tsdf_integrate_raycast: Alg. 2 as printed,
each view's rays applied together) against the oracle's fp32-exact mode: weights
and values bit for bit, in fp32 and half storage, on ragged grids, split into
several calls, and on two full-size views of the room."""
import numpy as np
import pytest
import torch

from oracle import cgrid
from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a.view(np.uint16)


def raycast_gpu(spec, views, splits=(None,)):
    g = T.Grid(spec).init()
    depth = dev(views.depth)
    K, P = dev(views.K), dev(views.c2w)
    ws = torch.empty(T.tsdfs_raycast_workspace_size(g), dtype=torch.uint8, device="cuda")
    bounds = [0] + [s for s in splits if s is not None] + [depth.shape[0]]
    for a, b in zip(bounds[:-1], bounds[1:]):
        g.integrate_raycast(depth[a:b].contiguous(), K[a:b].contiguous(), P[a:b].contiguous(), ws)
    torch.cuda.synchronize()
    rc, st = T.tsdfs_sync_status()
    assert rc == 0 and st == 0
    V = g.V.cpu().numpy()
    return (V.view(np.uint16) if spec.dtype == "f16" else V), g.W.cpu().numpy()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_tiny_raycast_bit_exact(dtype):
    wl = synth.tiny_workload()
    spec = synth.GridSpec(**{**wl.grid.__dict__, "dtype": dtype})
    Vg, Wg = raycast_gpu(spec, wl.views)
    V, W = cgrid.integrate_raycast_batched(spec, wl.views, "f32")
    assert np.array_equal(Wg, W)
    assert np.array_equal(bits(Vg), bits(V))
    assert (W > 0).mean() > 0.3


def test_ragged_grid_and_split_calls_bit_exact():
    """A 37 x 29 x 41 grid that covers part of the scene (rays enter through
    every face and leave through the far ones), views fused in three calls."""
    wl = synth.tiny_workload()
    spec = synth.GridSpec(37, 29, 41, (-0.61, -0.43, -0.7), 0.029, 0.087)
    Vg, Wg = raycast_gpu(spec, wl.views, splits=(3, 5))
    V, W = cgrid.integrate_raycast_batched(spec, wl.views, "f32")
    assert np.array_equal(Wg, W)
    assert np.array_equal(bits(Vg), bits(V))


def test_room_two_views_full_size_bit_exact():
    """Two 640x480 training views of the room into the 256^3 grid."""
    wl = synth.room_workload(n_views=2)
    Vg, Wg = raycast_gpu(wl.grid, wl.views)
    V, W = cgrid.integrate_raycast_batched(wl.grid, wl.views, "f32")
    assert np.array_equal(Wg, W)
    assert np.array_equal(bits(Vg), bits(V))
    assert W.max() > 1   # near the cameras several rays of a view cross one voxel
