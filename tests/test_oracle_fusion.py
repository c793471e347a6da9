"""Pins of the oracle's TSDF fusion (Eq. 3, Alg. 2 and its projective form).

Every check compares the oracle with something other than itself: a closed
form (a plane seen head-on), an invariance of the running weighted mean (view
order, repeated views), the truncation rule, a library conversion (numpy's
float16) or the independent ray-casting form of Alg. 2.
"""
import numpy as np
import pytest

from oracle import cgrid
from paper_2311_17878_gb300 import synth


class PlaneScene:
    """Solid half-space z >= d (the camera looks at it along +z)."""

    def __init__(self, d):
        self.d = d

    def ray_range(self, o, dirs):
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (self.d - o[:, 2]) / dirs[:, 2]
        return np.where(t > 0, t, np.inf)


def plane_setup(fx=1000.0, n=32, res=64):
    """Grid [-0.25, 0.25]^2 x [0.5, 1.0], plane z = 0.75, camera at the origin
    looking along +z with a narrow field of view (half-angle theta < 0.033 rad)."""
    vs = 0.5 / n
    grid = synth.GridSpec(n, n, n, (-0.25, -0.25, 0.5), vs, 3 * vs)
    scene = PlaneScene(0.75)
    c2w = synth.look_at((0, 0, 0), (0, 0, 1), up=(0, -1, 0))
    c = res / 2.0
    depth = synth.render_depth_maps(scene, [c2w], fx, fx, c, c, res, res)
    views = synth.Views(np.array([[fx, fx, c, c]], np.float32), c2w.astype(np.float32).reshape(1, 12), depth, res, res)
    return grid, scene, views


def centres(grid):
    o = np.asarray(grid.origin)
    k, j, i = np.meshgrid(np.arange(grid.nz), np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    return np.stack([o[0] + (i + 0.5) * grid.voxel_size, o[1] + (j + 0.5) * grid.voxel_size,
                     o[2] + (k + 0.5) * grid.voxel_size], -1)


def test_plane_head_on_closed_form():
    grid, scene, views = plane_setup()
    V, W = cgrid.integrate_projective(grid, views, "f64")
    c = centres(grid)
    # the frustum half-width at z is z * 32/1000: only voxels near the axis are seen
    seen = W > 0
    assert seen.sum() > 50
    T = grid.trunc
    s_true = np.clip(scene.d - c[..., 2], -T, T) / T
    band = seen & (scene.d - c[..., 2] > -T)
    # a pixel ray at angle theta from the axis: D = (d - o_z)/cos(theta) and
    # s - (d - z) = (D - rho)(1 - cos(theta)) + O(rho dtheta^2), |D - rho| <= D_T,
    # so |V - (d - z)/D_T| <= theta^2/2 + 1e-6 with theta <= 32*sqrt(2)/1000
    theta = 32 * np.sqrt(2) / 1000.0
    assert np.max(np.abs(V[band] - s_true[band])) < theta ** 2 / 2 + 1e-6
    # truncation: voxels more than D_T behind the surface are never updated (Alg. 2, s > -D_T)
    behind = (c[..., 2] - scene.d > T * 1.01) & (np.abs(c[..., 0]) < 0.01) & (np.abs(c[..., 1]) < 0.01)
    assert behind.any() and np.all(W[behind] == 0) and np.all(V[behind] == -1.0)
    # single view: weights are 0 or 1, values within [-1, 1]
    assert set(np.unique(W)) <= {0, 1}
    assert V.min() >= -1.0 and V.max() <= 1.0


def test_unseen_voxels_keep_initial_state():
    grid, scene, views = plane_setup()
    V, W = cgrid.integrate_projective(grid, views, "f64")
    c = centres(grid)
    # far off-axis voxels are outside the narrow frustum
    outside = (np.abs(c[..., 0]) > 0.05) | (np.abs(c[..., 1]) > 0.05)
    assert np.all(W[outside] == 0) and np.all(V[outside] == -1.0)


@pytest.mark.parametrize("reps", [3, 300])
def test_repeated_views_mean_and_weight_saturation(reps):
    wl = synth.tiny_workload()
    one = synth.Views(wl.views.K[:1], wl.views.c2w[:1], wl.views.depth[:1], 64, 64)
    many = synth.Views(np.repeat(one.K, reps, 0), np.repeat(one.c2w, reps, 0), np.repeat(one.depth, reps, 0), 64, 64)
    V1, W1 = cgrid.integrate_projective(wl.grid, one, "f64")
    Vn, Wn = cgrid.integrate_projective(wl.grid, many, "f64")
    # the running mean of identical samples is the sample; the weight saturates at 255
    assert np.array_equal(Wn, np.minimum(W1.astype(int) * reps, 255).astype(np.uint8))
    assert np.max(np.abs(Vn - V1)) < 1e-12


def test_view_order_invariance():
    wl = synth.tiny_workload()
    V, W = cgrid.integrate_projective(wl.grid, wl.views, "f64")
    perm = np.array([5, 2, 7, 0, 3, 6, 1, 4])
    pv = synth.Views(wl.views.K[perm], wl.views.c2w[perm], wl.views.depth[perm], 64, 64)
    Vp, Wp = cgrid.integrate_projective(wl.grid, pv, "f64")
    assert np.array_equal(W, Wp)
    assert np.max(np.abs(V - Vp)) < 1e-12


def test_mean_of_two_views_equals_average_of_single_views():
    wl = synth.tiny_workload()
    a = synth.Views(wl.views.K[:1], wl.views.c2w[:1], wl.views.depth[:1], 64, 64)
    b = synth.Views(wl.views.K[1:2], wl.views.c2w[1:2], wl.views.depth[1:2], 64, 64)
    ab = synth.Views(wl.views.K[:2], wl.views.c2w[:2], wl.views.depth[:2], 64, 64)
    Va, Wa = cgrid.integrate_projective(wl.grid, a, "f64")
    Vb, Wb = cgrid.integrate_projective(wl.grid, b, "f64")
    Vab, Wab = cgrid.integrate_projective(wl.grid, ab, "f64")
    both = (Wa == 1) & (Wb == 1)
    assert both.any()
    assert np.max(np.abs(Vab[both] - 0.5 * (Va[both] + Vb[both]))) < 1e-12
    only_a = (Wa == 1) & (Wb == 0)
    assert np.max(np.abs(Vab[only_a] - Va[only_a])) < 1e-12
    assert np.array_equal(Wab, (Wa + Wb).astype(np.uint8))


def test_raycast_form_agrees_with_projective_on_plane():
    grid, scene, views = plane_setup(fx=1000.0, res=128)
    Vp, Wp = cgrid.integrate_projective(grid, views, "f64")
    Vr, Wr = cgrid.integrate_raycast(grid, views)
    both = (Wp > 0) & (Wr > 0)
    assert both.sum() > 100
    # Ray casting evaluates v.(p* - c) for rays passing up to sqrt(3)/2 vs from
    # the centre: |V_ray - (d - z)/D_T| <= theta sqrt(3)/2 vs/D_T + theta^2/2;
    # the projective form is within theta^2/2 (see the closed-form test).
    theta = 64 * np.sqrt(2) / 1000.0
    bound = theta * np.sqrt(3) / 2 * grid.voxel_size / grid.trunc + theta ** 2
    assert np.max(np.abs(Vp[both] - Vr[both])) < bound


def test_fp32_exact_mode_close_to_fp64():
    wl = synth.tiny_workload()
    V64, W64 = cgrid.integrate_projective(wl.grid, wl.views, "f64")
    V32, W32 = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    assert np.array_equal(W32, W64)
    # fp32 error of s = D - v.(c - o): a few ulps of the range (~2 m) over D_T = 3/64 m
    bound = 8 * np.spacing(np.float32(2.5)) / wl.grid.trunc
    assert np.max(np.abs(V32.astype(np.float64) - V64)) < bound


def test_subset_matches_full_grid():
    wl = synth.tiny_workload()
    V, W = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    vox = synth.sub_sample(64 ** 3, 500, seed=11)
    Vs, Ws = cgrid.integrate_projective(wl.grid, wl.views, "f32", vox=vox)
    assert np.array_equal(Vs, V.reshape(-1)[vox]) and np.array_equal(Ws, W.reshape(-1)[vox])


def test_half_storage_is_rounded_fp32_result():
    wl = synth.tiny_workload()
    V32, W32 = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    g16 = synth.GridSpec(**{**wl.grid.__dict__, "dtype": "f16"})
    V16, W16 = cgrid.integrate_projective(g16, wl.views, "f32")
    assert np.array_equal(W16, W32)
    assert np.array_equal(V16, V32.astype(np.float16).view(np.uint16))


def test_half_conversions_match_numpy():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-1, 1, 3000), rng.uniform(-1e-4, 1e-4, 3000), rng.normal(0, 1e-6, 500),
                        np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65520.0, 6.1e-5, 5.96e-8, 2.98e-8])]).astype(np.float32)
    assert np.array_equal(cgrid.half_from_float(x), x.astype(np.float16).view(np.uint16))
    h = np.arange(0, 65536, dtype=np.uint32).astype(np.uint16)
    h = h[((h >> 10) & 0x1F) != 0x1F]   # finite values
    assert np.array_equal(cgrid.float_from_half(h), h.view(np.float16).astype(np.float32))
