"""Pins of the oracle's ray bounds (Alg. 1) and adaptive count (Sec. 3.4).

Checked against brute force (ray / voxel-box intersection for the voxel walk,
scipy's maximum filter for the neighbourhood test), closed forms (analytic
sphere and plane hits on their exact distance grids, a half-space where the
far bound is a known number of voxels) and theorems of the algorithm (the
near bound never passes the first hit on an exact distance grid).
"""
import numpy as np
import pytest
from scipy import ndimage

from oracle import cgrid
from paper_2311_17878_gb300 import synth


def fib_dirs(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = np.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def brute_voxels(grid, o, d, t_near, t_far):
    """All voxels whose box the ray segment [t0, t_end] crosses with positive
    length, sorted by entry parameter (FP64 slab tests over every voxel)."""
    o = o.astype(np.float64)
    d = d.astype(np.float64)
    lo_g, hi_g = grid.aabb
    n = np.array([grid.nx, grid.ny, grid.nz])
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = np.stack([i, j, k], -1).reshape(-1, 3)
    lo = lo_g + idx * grid.voxel_size
    hi = lo + grid.voxel_size
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - o) / d
        t2 = (hi - o) / d
    inside_slab = (o >= lo) & (o <= hi)
    lo_t = np.where(d == 0, np.where(inside_slab, -np.inf, np.inf), np.minimum(t1, t2))
    hi_t = np.where(d == 0, np.where(inside_slab, np.inf, -np.inf), np.maximum(t1, t2))
    tmin = np.max(lo_t, 1)
    tmax = np.min(hi_t, 1)
    ta = np.max(np.minimum((lo_g - o) / np.where(d == 0, np.inf, d), (hi_g - o) / np.where(d == 0, np.inf, d)))
    t0 = max(t_near, ta)
    entry = np.maximum(tmin, t0)
    exitp = np.minimum(tmax, t_far)
    keep = exitp - entry > 1e-9
    order = np.argsort(entry[keep], kind="stable")
    return idx[keep][order], entry[keep][order]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_voxel_walk_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = rng.integers(4, 9, 3)
    grid = synth.GridSpec(int(n[0]), int(n[1]), int(n[2]), tuple(rng.uniform(-1, 0, 3)), float(rng.uniform(0.1, 0.3)), 0.5)
    lo, hi = grid.aabb
    dirs = np.concatenate([fib_dirs(64), np.eye(3), -np.eye(3), [[1, 1, 0], [0, -1, 1], [1, 1, 1]]])
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    checked = 0
    for r, dv in enumerate(dirs):
        inside = rng.uniform() < 0.4
        o = rng.uniform(lo, hi) if inside else 0.5 * (lo + hi) - 3.0 * dv + rng.uniform(-0.2, 0.2, 3)
        o = o.astype(np.float32).astype(np.float64)
        d = dv.astype(np.float32).astype(np.float64)
        xyz, t = cgrid.dda_sequence(grid, o, d, 0.0, 100.0, "f64")
        bx, bt = brute_voxels(grid, o, d, 0.0, 100.0)
        assert np.array_equal(xyz, bx), (seed, r)
        assert np.allclose(t, bt, atol=1e-9)
        checked += len(bx) > 0
    assert checked > 40


def sphere_setup(trunc_vox=3):
    wl = synth.tiny_workload()
    grid = synth.GridSpec(64, 64, 64, (-0.5, -0.5, -0.5), 1 / 64, trunc_vox / 64)
    V = synth.analytic_tsdf(wl.scene, grid)
    return wl, grid, V


@pytest.mark.parametrize("mode", ["f32", "f64"])
def test_sphere_bounds_contain_first_hit_on_exact_grid(mode):
    """With an exact distance grid, the voxel containing the hit has its centre
    within sqrt(3)/2 vs <= D_s of the surface, so the near phase triggers at or
    before it (t_n <= t*), and every voxel before t* is outside the solid, so
    the far phase cannot confirm M inside voxels before t* (t_f >= t*).  Tab. 1's
    "failed to find surface" count is therefore 0."""
    wl, grid, V = sphere_setup()
    b = cgrid.ray_bounds(grid, V, wl.rays_o, wl.rays_d, wl.bounds, mode)
    o, d = wl.rays_o.astype(np.float64), wl.rays_d.astype(np.float64)
    t_star = synth.ray_sphere(o, d, (0, 0, 0), 0.5)
    hit = np.isfinite(t_star)
    assert hit.sum() > 500
    assert np.all(b["status"][hit] == 1)
    assert np.all(b["t_n"][hit] <= t_star[hit] + 1e-6)
    assert np.all(b["t_f"][hit] >= t_star[hit] - 1e-6)
    # near-bound tightness: the point at t_n is within D_s + sqrt(3)/2 vs of the
    # sphere and the sphere lies behind its tangent plane, so
    # t* - t_n <= (D_s + sqrt(3)/2 vs) / cos(theta)
    p = o + t_star[:, None] * d
    cos_t = -np.sum(d * p / 0.5, 1)
    vs = grid.voxel_size
    bound = (wl.bounds.d_s + np.sqrt(3) / 2 * vs) / np.maximum(cos_t, 1e-12) + 1e-6
    assert np.all((t_star - b["t_n"])[hit] <= bound[hit])


def test_sphere_zero_crossing_second_order():
    wl, grid, V = sphere_setup()
    b = cgrid.ray_bounds(grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f64")
    o, d = wl.rays_o.astype(np.float64), wl.rays_d.astype(np.float64)
    t_star = synth.ray_sphere(o, d, (0, 0, 0), 0.5)
    p = o + t_star[:, None] * d
    cos_t = -np.sum(d * p / 0.5, 1)
    vs = grid.voxel_size
    # inside the hull of the voxel-centre lattice (clamp-to-edge is first order outside it)
    interior = np.max(np.abs(np.nan_to_num(p, nan=1.0)), 1) < 0.5 - 1.5 * vs
    ok = np.isfinite(t_star) & (cos_t > 0.5) & interior
    assert ok.sum() > 300
    err = np.abs(b["t_zero"][ok] - t_star[ok])
    # trilinear interpolation of the sphere distance: error O(vs^2 / r); along the ray / cos(theta)
    assert np.all(err <= 2.0 * vs * vs / 0.5 / cos_t[ok])


def test_plane_zero_crossing_exact():
    """A linear distance field is reproduced exactly by trilinear interpolation,
    and the secant root of a linear function is exact."""
    n = np.array([0.3, -0.5, 0.81])
    n /= np.linalg.norm(n)
    dpl = 0.05
    vs = 1 / 32
    grid = synth.GridSpec(32, 32, 32, (-0.5, -0.5, -0.5), vs, 8 * vs)
    k, j, i = np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij")
    c = np.stack([-0.5 + (i + 0.5) * vs, -0.5 + (j + 0.5) * vs, -0.5 + (k + 0.5) * vs], -1)
    V = np.clip((c @ n - dpl) / grid.trunc, -1, 1).astype(np.float64)
    # keep the grid values exactly linear: no clamping anywhere in the grid
    assert np.abs(c @ n - dpl).max() < grid.trunc * 8
    grid = synth.GridSpec(32, 32, 32, (-0.5, -0.5, -0.5), vs, 2.0)
    V = ((c @ n - dpl) / 2.0).astype(np.float32)
    rng = np.random.default_rng(3)
    m = 200
    o = (n * 1.5 + rng.uniform(-0.15, 0.15, (m, 3))).astype(np.float32)
    target = rng.uniform(-0.2, 0.2, (m, 3))
    target -= np.outer(target @ n - dpl, n)
    dv = target - o
    dv = (dv / np.linalg.norm(dv, axis=1, keepdims=True)).astype(np.float32)
    bp = synth.BoundsParams(d_s=vs * 2.0 / 2.0, t_near=0.0, t_far=10.0, step=vs, n_max=64)
    bp.d_s = 0.02  # V <= 0.01 in normalised units
    b = cgrid.ray_bounds(grid, V, o, dv, bp, "f64")
    od, dd = o.astype(np.float64), dv.astype(np.float64)
    t_star = (dpl - od @ n) / (dd @ n)
    ok = b["status"] == 1
    assert ok.sum() > 150
    assert np.nanmax(np.abs(b["t_zero"][ok] - t_star[ok])) < 1e-5 * vs


def halfspace_grid(nx=64, solid_from=20, ny=8, nz=8):
    V = np.ones((nz, ny, nx), np.float32)
    V[:, :, solid_from:] = -0.5
    grid = synth.GridSpec(nx, ny, nz, (0.0, 0.0, 0.0), 0.125, 0.5)
    return grid, V


@pytest.mark.parametrize("mode", ["f32", "f64"])
def test_far_bound_half_space_closed_form(mode):
    """Ray along +x into a solid half-space starting at voxel 20: the near
    voxel is 20; with radius 2 the neighbourhood is all negative from voxel 22
    on; the 15th consecutive inside voxel is 36, so t_f is the entry of 37."""
    grid, V = halfspace_grid()
    o = np.array([[-1.0, 0.5, 0.5]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    for step, n_expect in [(0.125, 17), (0.25, 9), (0.3, 8), (0.01, 64)]:
        bp = synth.BoundsParams(d_s=0.125, t_near=0.0, t_far=100.0, step=step, n_max=64)
        b = cgrid.ray_bounds(grid, V, o, d, bp, mode)
        assert b["status"][0] == 1
        assert b["t_n"][0] == 1.0 + 20 * 0.125
        assert b["t_f"][0] == 1.0 + 37 * 0.125
        assert b["n"][0] == n_expect
        assert b["steps"][0] == 21 + 17


def test_thin_solid_never_confirms_far():
    """A solid slab 10 voxels thick never gives 15 consecutive inside voxels:
    t_f stays at the original far bound (the grid exit)."""
    grid, V = halfspace_grid()
    V[:, :, 30:] = 1.0
    o = np.array([[-1.0, 0.5, 0.5]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    bp = synth.BoundsParams(d_s=0.125, t_near=0.0, t_far=100.0, step=0.125, n_max=64)
    b = cgrid.ray_bounds(grid, V, o, d, bp, "f64")
    assert b["status"][0] == 1 and b["t_n"][0] == 3.5 and b["t_f"][0] == 1.0 + 64 * 0.125
    bp.t_far = 7.3
    b = cgrid.ray_bounds(grid, V, o, d, bp, "f64")
    assert b["t_f"][0] == 7.3


def test_miss_and_fallback():
    grid, V = halfspace_grid()
    bp = synth.BoundsParams(d_s=0.125, t_near=0.0, t_far=100.0, step=0.125, n_max=64, n_fallback=96)
    o = np.array([[-1.0, 5.0, 0.5], [-1.0, 0.5, 0.5], [2.0, 0.5, 0.5]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], np.float32)
    b = cgrid.ray_bounds(grid, np.ones_like(V), o, d, bp, "f64")
    assert b["status"][0] == 0 and b["n"][0] == 0
    assert b["status"][1] == 2 and b["n"][1] == 96 and b["t_n"][1] == 1.0 and b["t_f"][1] == 9.0
    assert b["status"][2] == 2 and b["t_n"][2] == 0.0 and b["t_f"][2] == 0.5
    # t_near beyond the box: miss
    bp.t_near = 20.0
    b = cgrid.ray_bounds(grid, V, o[1:2], d[1:2], bp, "f64")
    assert b["status"][0] == 0


@pytest.mark.parametrize("radius", [1, 2, 3])
def test_inside_mask_matches_scipy_filter(radius):
    rng = np.random.default_rng(5)
    V = -rng.uniform(0.0, 1.0, (12, 10, 14)).astype(np.float32)
    V[rng.uniform(size=V.shape) < 0.004] = 0.3
    V[0, 0, 0] = 0.0  # zero is not negative
    grid = synth.GridSpec(14, 10, 12, (0, 0, 0), 0.1, 0.3)
    m = cgrid.inside_mask(grid, V, radius)
    ref = ndimage.maximum_filter(V, size=2 * radius + 1, mode="constant", cval=-1.0) < 0
    assert np.array_equal(m.astype(bool), ref)
    assert ref.any() and not ref.all()


def test_fp32_and_fp64_bounds_agree_on_tiny():
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    b32 = cgrid.ray_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f32")
    b64 = cgrid.ray_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f64")
    assert np.array_equal(b32["status"], b64["status"])
    assert np.array_equal(b32["n"], b64["n"])
    assert np.array_equal(b32["steps"], b64["steps"])
    ok = b32["status"] > 0
    assert np.max(np.abs(b32["t_n"][ok] - b64["t_n"][ok])) < 1e-5
    assert np.max(np.abs(b32["t_f"][ok] - b64["t_f"][ok])) < 1e-5
