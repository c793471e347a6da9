"""Pins of the oracle's ray-casting fusion with each view's rays applied together
(Alg. 2 as printed; reading R27):

* a single ray along +z onto a plane gives the closed form s = (o_z + D) - c_z on
  the voxel column it crosses, stops at the first s <= -D_T and leaves every
  other voxel unseen;
* a ray with no surface (D = +inf) writes s = D_T on every voxel it crosses;
* without weight saturation the batched update equals Alg. 2's one-ray-at-a-time
  running mean (the as-printed oracle) exactly;
* identical views saturate W at 255 and leave V unchanged;
* the fp32-exact mode agrees with FP64 within the rounding of its binary32
  ray arithmetic wherever both visit a voxel equally often."""
import numpy as np

from oracle import cgrid
from paper_2311_17878_gb300 import synth


def one_ray_views(depth, n_views=1, o=(0.0, 0.0, 0.0)):
    """A 1x1-pixel camera at o looking along +z (pixel centre on the optical axis)."""
    c2w = synth.look_at(o, (o[0], o[1], o[2] + 1.0), up=(0, -1, 0)).astype(np.float32).reshape(12)
    K = np.array([100.0, 100.0, 0.5, 0.5], np.float32)
    return synth.Views(np.tile(K, (n_views, 1)), np.tile(c2w, (n_views, 1)),
                       np.full((n_views, 1, 1), depth, np.float32), 1, 1)


def column_grid():
    # 8 x 8 x 32 voxels of 1/32 m from (-0.125, -0.125, 0.25); the camera at (1/64, 1/64, 0)
    # looks down the column of voxel (4, 4, *) through voxel centres in x and y
    vs = 1.0 / 32
    return synth.GridSpec(8, 8, 32, (-0.125, -0.125, 0.25), vs, 3 * vs)


def test_single_ray_plane_closed_form():
    grid = column_grid()
    o = (1.0 / 64, 1.0 / 64, 0.0)
    D = 0.75
    V, W = cgrid.integrate_raycast_batched(grid, one_ray_views(D, o=o), "f64")
    vs, T = grid.voxel_size, grid.trunc
    cz = grid.origin[2] + (np.arange(grid.nz) + 0.5) * vs
    s = np.clip((o[2] + D) - cz, -T, T)
    visited = np.zeros(grid.nz, bool)
    for k in range(grid.nz):   # the walk stops at the first s <= -D_T
        if s[k] <= -T:
            break
        visited[k] = True
    col_V, col_W = V[:, 4, 4], W[:, 4, 4]
    assert np.array_equal(col_W, visited.astype(np.uint8))
    assert np.max(np.abs(col_V[visited] - s[visited] / T)) < 1e-12
    assert np.all(col_V[~visited] == -1.0)
    others = np.ones(grid.shape_zyx, bool)
    others[:, 4, 4] = False
    assert np.all(W[others] == 0) and np.all(V[others] == -1.0)


def test_free_ray_writes_the_truncation():
    grid = column_grid()
    V, W = cgrid.integrate_raycast_batched(grid, one_ray_views(np.inf, o=(1.0 / 64, 1.0 / 64, 0.0)), "f64")
    assert np.all(W[:, 4, 4] == 1) and np.all(V[:, 4, 4] == 1.0)
    assert W.sum() == grid.nz


def test_batched_equals_the_running_mean_without_saturation():
    wl = synth.tiny_workload()
    Vb, Wb = cgrid.integrate_raycast_batched(wl.grid, wl.views, "f64")
    Vs, Ws = cgrid.integrate_raycast(wl.grid, wl.views)
    assert Wb.max() < 255
    assert np.array_equal(Wb, Ws)
    assert np.max(np.abs(Vb - Vs)) < 1e-12


def test_identical_views_saturate_the_weight():
    grid = column_grid()
    o = (1.0 / 64, 1.0 / 64, 0.0)
    V1, W1 = cgrid.integrate_raycast_batched(grid, one_ray_views(0.75, 1, o), "f64")
    V3, W3 = cgrid.integrate_raycast_batched(grid, one_ray_views(0.75, 300, o), "f64")
    seen = W1 > 0
    assert np.all(W3[seen] == 255) and np.all(W3[~seen] == 0)
    assert np.max(np.abs(V3[seen] - V1[seen])) < 1e-12


def test_fp32_exact_mode_tracks_fp64():
    wl = synth.tiny_workload()
    V64, W64 = cgrid.integrate_raycast_batched(wl.grid, wl.views, "f64")
    V32, W32 = cgrid.integrate_raycast_batched(wl.grid, wl.views, "f32")
    seen = W64 > 0
    # the binary32 walk may resolve a corner crossing the other way on a few rays
    assert (W32 != W64).sum() < 0.02 * seen.sum()
    same = seen & (W32 == W64)
    # s = v . (o + D v - c) in binary32: a few units of 2^-24 of the largest range, over D_T
    d_max = float(np.max(wl.views.depth[np.isfinite(wl.views.depth)]))
    bound = 8 * 2.0 ** -24 * d_max / wl.grid.trunc
    assert np.max(np.abs(V32[same] - V64[same])) <= bound
