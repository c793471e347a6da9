"""Seeded synthetic inputs: scenes, cameras, rays, depth maps and MLP parameters.

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark.  It holds none of the method's arithmetic (no fusion, no marching,
no MLP evaluation, no compositing): only analytic scene geometry, camera
poses, ray directions, analytic depth maps and the seeded parameters of the
SDF / colour networks.  Everything is numpy float64 internally and handed out
as float32 arrays in the layouts the C ABI takes.

Scenes stand in for the paper's datasets (Sec. 4.1: Lobby, Garage, Replica),
which are not available:

* ``tiny``  -- analytic sphere r=0.5 in the unit cube, 8 pinhole views.
* ``room``  -- 8x6x3 m box room with 20 boxes and 4 thin (2 cm) partition
  plates, 100 pinhole views at 640x480 with N(0, 5 mm) range noise.
* ``large`` -- 20x20x4 m multi-room floor with 200 boxes and 40 plates.

Depth maps store the *range* along the unit ray through the pixel centre
(the depth of Eq. 2 with a unit direction).  Pixels that hit nothing hold +inf.
Cameras follow the OpenCV convention (x right, y down, z forward); ``c2w`` is
a row-major 3x4 matrix [R | o] whose columns of R are the camera axes in world
coordinates.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_SCENE, SEED_POSES, SEED_NOISE, SEED_MLP, SEED_RAYS, SEED_HELDOUT, SEED_TRAIN_RAYS = 0, 1, 2, 3, 4, 5, 6

ARCH_TINY, ARCH_ROOM = 0, 1


# ----------------------------------------------------------------------------
# cameras and rays
# ----------------------------------------------------------------------------
def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Row-major 3x4 camera-to-world matrix, OpenCV axes (x right, y down, z fwd)."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    c2w = np.zeros((3, 4))
    c2w[:, 0], c2w[:, 1], c2w[:, 2], c2w[:, 3] = right, down, fwd, eye
    return c2w


def yaw_pitch_pose(eye, yaw, pitch) -> np.ndarray:
    d = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch)])
    return look_at(eye, np.asarray(eye, np.float64) + d)


def pinhole_rays(c2w, fx, fy, cx, cy, width, height):
    """Unit rays through the pixel centres, row-major over (v, u).  float64."""
    u, v = np.meshgrid(np.arange(width) + 0.5, np.arange(height) + 0.5)
    dc = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], -1).reshape(-1, 3)
    d = dc @ np.asarray(c2w)[:, :3].T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(np.asarray(c2w)[:, 3], d.shape).copy()
    return o, d


def equirect_rays(center, width, height):
    """Equirectangular panorama rays, z up: lon = 2pi(u+1/2)/W - pi, lat = pi/2 - pi(v+1/2)/H."""
    u, v = np.meshgrid(np.arange(width) + 0.5, np.arange(height) + 0.5)
    lon = 2.0 * np.pi * u / width - np.pi
    lat = 0.5 * np.pi - np.pi * v / height
    d = np.stack([np.cos(lat) * np.sin(lon), np.cos(lat) * np.cos(lon), np.sin(lat)], -1).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(np.asarray(center, np.float64), d.shape).copy()
    return o, d


# ----------------------------------------------------------------------------
# analytic geometry (ray ranges and signed distances of the fixtures)
# ----------------------------------------------------------------------------
def _safe_inv(d):
    with np.errstate(divide="ignore"):
        inv = 1.0 / d
    return inv


def ray_sphere(o, d, center, r):
    """First positive hit of unit rays with a sphere, +inf if none."""
    oc = o - np.asarray(center)
    b = np.sum(oc * d, 1)
    c = np.sum(oc * oc, 1) - r * r
    disc = b * b - c
    t = np.full(len(o), np.inf)
    ok = disc >= 0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    t0, t1 = -b - sq, -b + sq
    t = np.where(ok & (t0 > 0), t0, np.where(ok & (t1 > 0), t1, np.inf))
    return t


def ray_boxes_entry(o, d, lo, hi):
    """Entry distance of rays (N) into axis-aligned boxes (B); +inf if missed or behind."""
    inv = _safe_inv(d)[:, None, :]
    with np.errstate(invalid="ignore"):
        t1 = (lo[None] - o[:, None, :]) * inv
        t2 = (hi[None] - o[:, None, :]) * inv
    t1 = np.nan_to_num(t1, nan=-np.inf)
    t2 = np.nan_to_num(t2, nan=np.inf)
    tmin = np.max(np.minimum(t1, t2), axis=2)
    tmax = np.min(np.maximum(t1, t2), axis=2)
    hit = (tmax >= tmin) & (tmin > 0)
    return np.where(hit, tmin, np.inf)


def ray_box_exit(o, d, lo, hi):
    """Exit distance of rays starting inside one axis-aligned box."""
    inv = _safe_inv(d)
    with np.errstate(invalid="ignore"):
        t1 = (lo[None] - o) * inv
        t2 = (hi[None] - o) * inv
    t1 = np.nan_to_num(t1, nan=-np.inf)
    t2 = np.nan_to_num(t2, nan=np.inf)
    return np.min(np.maximum(t1, t2), axis=1)


def sdf_boxes(x, lo, hi):
    """Signed distance (N, B) of points to axis-aligned boxes (negative inside)."""
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    q = np.abs(x[:, None, :] - c[None]) - h[None]
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=2)
    inside = np.minimum(np.max(q, axis=2), 0.0)
    return outside + inside


@dataclass
class SphereScene:
    center: tuple = (0.0, 0.0, 0.0)
    radius: float = 0.5
    albedo: tuple = (0.8, 0.5, 0.3)

    def ray_range(self, o, d):
        return ray_sphere(o, d, self.center, self.radius)

    def sdf(self, x):
        return np.linalg.norm(x - np.asarray(self.center), axis=1) - self.radius


@dataclass
class BoxRoomScene:
    """Axis-aligned room (inward-facing walls) with boxes and thin plates.

    Solid space is the outside of the room plus every box and plate.
    """
    room_lo: np.ndarray
    room_hi: np.ndarray
    box_lo: np.ndarray          # (B, 3): boxes and plates together
    box_hi: np.ndarray
    albedo: np.ndarray          # (B + 6, 3): boxes/plates, then walls -x,+x,-y,+y,-z,+z
    n_plates: int = 0

    def ray_range(self, o, d, return_id=False):
        t_box = ray_boxes_entry(o, d, self.box_lo, self.box_hi) if len(self.box_lo) else np.full((len(o), 0), np.inf)
        t_wall = ray_box_exit(o, d, self.room_lo, self.room_hi)
        t_best = np.min(t_box, axis=1) if t_box.shape[1] else np.full(len(o), np.inf)
        use_wall = t_wall < t_best
        t = np.where(use_wall, t_wall, t_best)
        if not return_id:
            return t
        ids = np.argmin(t_box, axis=1) if t_box.shape[1] else np.zeros(len(o), np.int64)
        # which wall: the axis/side achieving the exit
        p = o + t_wall[:, None] * d
        dist = np.stack([p[:, 0] - self.room_lo[0], self.room_hi[0] - p[:, 0],
                         p[:, 1] - self.room_lo[1], self.room_hi[1] - p[:, 1],
                         p[:, 2] - self.room_lo[2], self.room_hi[2] - p[:, 2]], 1)
        wall = np.argmin(np.abs(dist), axis=1)
        ids = np.where(use_wall, len(self.box_lo) + wall, ids)
        return t, ids

    def sdf(self, x):
        d_room = np.min(np.concatenate([x - self.room_lo[None], self.room_hi[None] - x], 1), axis=1)
        # exact distance outside the room box for points beyond the walls
        q = np.maximum(np.maximum(self.room_lo[None] - x, x - self.room_hi[None]), 0.0)
        out = np.linalg.norm(q, axis=1)
        d_room = np.where(out > 0, -out, d_room)
        if len(self.box_lo):
            d_box = np.min(sdf_boxes(x, self.box_lo, self.box_hi), axis=1)
            return np.minimum(d_room, d_box)
        return d_room

    def albedo_at(self, ids):
        return self.albedo[ids]


def make_box_room(seed, room_lo, room_hi, n_boxes, n_plates, plate_thick=0.02, plate_len=(1.0, 3.0),
                  box_side=(0.2, 1.5), interior_walls=()):
    rng = np.random.default_rng(seed)
    room_lo = np.asarray(room_lo, np.float64)
    room_hi = np.asarray(room_hi, np.float64)
    lo, hi = [], []
    for (wlo, whi) in interior_walls:
        lo.append(np.asarray(wlo, np.float64))
        hi.append(np.asarray(whi, np.float64))
    for _ in range(n_boxes):
        s = rng.uniform(box_side[0], box_side[1], 3)
        s[2] = min(s[2], room_hi[2] - room_lo[2] - 0.05)
        c = rng.uniform(room_lo[:2] + s[:2] / 2 + 0.01, room_hi[:2] - s[:2] / 2 - 0.01)
        lo.append(np.array([c[0] - s[0] / 2, c[1] - s[1] / 2, room_lo[2]]))
        hi.append(np.array([c[0] + s[0] / 2, c[1] + s[1] / 2, room_lo[2] + s[2]]))
    for _ in range(n_plates):
        length = rng.uniform(*plate_len)
        along_x = rng.uniform() < 0.5
        ext = np.array([length, plate_thick]) if along_x else np.array([plate_thick, length])
        c = rng.uniform(room_lo[:2] + ext / 2 + 0.05, room_hi[:2] - ext / 2 - 0.05)
        lo.append(np.array([c[0] - ext[0] / 2, c[1] - ext[1] / 2, room_lo[2]]))
        hi.append(np.array([c[0] + ext[0] / 2, c[1] + ext[1] / 2, room_hi[2]]))
    lo = np.array(lo).reshape(-1, 3)
    hi = np.array(hi).reshape(-1, 3)
    albedo = rng.uniform(0.1, 0.9, (len(lo) + 6, 3))
    return BoxRoomScene(room_lo, room_hi, lo, hi, albedo, n_plates)


# largest pitch of the room's random training poses (held-out views use 15 as well);
# a wider range trades horizontal coverage for floor / ceiling coverage
TRAIN_PITCH_DEG = 15.0


def sample_free_poses(scene, rng, n, margin=0.3, height=(1.0, 2.0), pitch_deg=15.0, clearance=0.3):
    """Random in-room camera poses, rejected when closer than ``clearance`` to solid space."""
    poses = []
    while len(poses) < n:
        p = np.array([rng.uniform(scene.room_lo[0] + margin, scene.room_hi[0] - margin),
                      rng.uniform(scene.room_lo[1] + margin, scene.room_hi[1] - margin),
                      rng.uniform(scene.room_lo[2] + height[0], scene.room_lo[2] + height[1])])
        yaw = rng.uniform(0.0, 2.0 * np.pi)
        pitch = np.deg2rad(rng.uniform(-pitch_deg, pitch_deg))
        if scene.sdf(p[None])[0] < clearance:
            continue
        poses.append(yaw_pitch_pose(p, yaw, pitch))
    return np.array(poses)


# ----------------------------------------------------------------------------
# grid / parameter containers
# ----------------------------------------------------------------------------
@dataclass
class GridSpec:
    nx: int
    ny: int
    nz: int
    origin: tuple
    voxel_size: float
    trunc: float
    dtype: str = "f32"          # "f32" | "f16" storage of the TSDF values

    @property
    def shape_zyx(self):
        return (self.nz, self.ny, self.nx)

    @property
    def aabb(self):
        o = np.asarray(self.origin, np.float64)
        return o, o + self.voxel_size * np.array([self.nx, self.ny, self.nz], np.float64)


@dataclass
class BoundsParams:
    d_s: float          # surface criterion D_s in metres (Alg. 1)
    t_near: float
    t_far: float
    step: float         # sample spacing in metres for the adaptive count
    nb_radius: int = 2  # neighbourhood radius: 2 -> 5x5x5 (Sec. 4.2)
    m_confirm: int = 15  # M, consecutive inside voxels (Sec. 4.2)
    n_max: int = 32
    n_fallback: int = 96


@dataclass
class MLPSpec:
    arch: int
    sdf: list                  # [(W (out,in) f32, b (out,) f32), ...]
    rgb: list
    center: tuple = (0.0, 0.0, 0.0)
    scale: float = 1.0         # x_tilde = (x - center) / scale ; f = scale * net_0
    inv_s: float = 64.0
    beta: float = 100.0
    alpha_eps: float = 1e-5
    n_feat: int = 16
    pe_sdf: int = 0            # positional-encoding octaves of the SDF input
    pe_dir: int = 0            # positional-encoding octaves of the view direction
    skip_layer: int = -1       # SDF layer whose input is concat(h, gamma(x)) / sqrt(2)
    opacity: int = 0           # SDF-to-opacity transform: 0 NeuS, 1 VolSDF Laplace density (a = inv_s)

    def packed(self, which):
        layers = self.sdf if which == "sdf" else self.rgb
        return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in layers]).astype(np.float32)


def round_bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def _geometric_sdf_layers(rng, dims_in, dims_out, radius, pe_cols=0, skip_layer=-1, skip_pe_cols=0,
                          inside_out=False):
    """SAL/IDR geometric initialisation: the network starts near |x| - radius
    (near radius - |x| with ``inside_out``, for scenes seen from the inside)."""
    layers = []
    n = len(dims_out)
    for l in range(n):
        fin, fout = dims_in[l], dims_out[l]
        if l == n - 1:
            W = rng.normal(math.sqrt(math.pi) / math.sqrt(fin), 1e-4, (fout, fin))
            b = np.full(fout, -radius)
            if inside_out:
                W, b = -W, -b
        else:
            W = rng.normal(0.0, math.sqrt(2.0) / math.sqrt(fout), (fout, fin))
            b = np.zeros(fout)
            if l == 0 and pe_cols:
                W[:, 3:] = 0.0
            if l == skip_layer and skip_pe_cols:
                W[:, fin - skip_pe_cols:] = 0.0
        layers.append((W, b))
    return layers


def _plain_layers(rng, dims_in, dims_out):
    layers = []
    for fin, fout in zip(dims_in, dims_out):
        W = rng.normal(0.0, 1.0 / math.sqrt(fin), (fout, fin))
        b = rng.normal(0.0, 0.05, fout)
        layers.append((W, b))
    return layers


def _finish(layers):
    return [(round_bf16(W.astype(np.float32)), round_bf16(b.astype(np.float32))) for W, b in layers]


TINY_SDF_DIMS = ([3, 64, 64, 64], [64, 64, 64, 17])
TINY_RGB_DIMS = ([25, 64, 64], [64, 64, 3])
ROOM_SDF_DIMS = ([39, 256, 256, 256, 256, 256, 256, 256], [256, 256, 256, 217, 256, 256, 256, 257])
ROOM_RGB_DIMS = ([289, 256, 256, 256, 256], [256, 256, 256, 256, 3])


def tiny_mlp(seed=SEED_MLP, radius=0.5) -> MLPSpec:
    rng = np.random.default_rng(seed)
    sdf = _geometric_sdf_layers(rng, *TINY_SDF_DIMS, radius=radius)
    rgb = _plain_layers(rng, *TINY_RGB_DIMS)
    return MLPSpec(ARCH_TINY, _finish(sdf), _finish(rgb), n_feat=16)


def room_mlp(seed=SEED_MLP, center=(0.0, 0.0, 1.5), scale=4.16, radius=0.6) -> MLPSpec:
    """8x256 SDF MLP (PE L=6, skip at layer 4) and 4x256 colour MLP (direction PE L=4).

    Geometric initialisation; a fitted parameter set can be loaded over it with
    :func:`load_mlp`.
    """
    rng = np.random.default_rng(seed)
    sdf = _geometric_sdf_layers(rng, *ROOM_SDF_DIMS, radius=radius, pe_cols=36, skip_layer=4, skip_pe_cols=36,
                                inside_out=True)
    rgb = _plain_layers(rng, *ROOM_RGB_DIMS)
    return MLPSpec(ARCH_ROOM, _finish(sdf), _finish(rgb), center=tuple(center), scale=scale,
                   n_feat=256, pe_sdf=6, pe_dir=4, skip_layer=4)


def save_mlp(spec: MLPSpec, path):
    arrs = {}
    for i, (W, b) in enumerate(spec.sdf):
        arrs[f"sdf{i}_W"], arrs[f"sdf{i}_b"] = W, b
    for i, (W, b) in enumerate(spec.rgb):
        arrs[f"rgb{i}_W"], arrs[f"rgb{i}_b"] = W, b
    np.savez_compressed(path, **arrs)


def load_mlp(spec: MLPSpec, path) -> MLPSpec:
    z = np.load(path)
    spec.sdf = [(round_bf16(z[f"sdf{i}_W"]), round_bf16(z[f"sdf{i}_b"])) for i in range(len(spec.sdf))]
    spec.rgb = [(round_bf16(z[f"rgb{i}_W"]), round_bf16(z[f"rgb{i}_b"])) for i in range(len(spec.rgb))]
    return spec


# ----------------------------------------------------------------------------
# workload presets
# ----------------------------------------------------------------------------
@dataclass
class Views:
    K: np.ndarray       # (V, 4) fx, fy, cx, cy   float32
    c2w: np.ndarray     # (V, 12) row-major 3x4    float32
    depth: np.ndarray   # (V, H, W) range          float32
    width: int
    height: int


@dataclass
class Workload:
    name: str
    grid: GridSpec
    bounds: BoundsParams
    views: Views
    scene: object
    rays_o: np.ndarray = field(default=None)   # (N, 3) float32
    rays_d: np.ndarray = field(default=None)


def render_depth_maps(scene, c2ws, fx, fy, cx, cy, width, height, noise_std=0.0, seed=SEED_NOISE):
    rng = np.random.default_rng(seed)
    depth = np.empty((len(c2ws), height, width), np.float32)
    for i, c2w in enumerate(c2ws):
        o, d = pinhole_rays(c2w, fx, fy, cx, cy, width, height)
        t = scene.ray_range(o, d)
        if noise_std > 0:
            t = t + rng.normal(0.0, noise_std, t.shape)
        depth[i] = t.reshape(height, width).astype(np.float32)
    return depth


def _views(c2ws, fx, fy, cx, cy, width, height, depth):
    V = len(c2ws)
    K = np.tile(np.array([fx, fy, cx, cy], np.float32), (V, 1))
    return Views(K, np.asarray(c2ws, np.float32).reshape(V, 12), depth, width, height)


def tiny_workload() -> Workload:
    """Sphere r=0.5 in the unit cube; 64^3 grid, D_T = 3 voxels; 8 views 64x64."""
    scene = SphereScene()
    vs = 1.0 / 64
    grid = GridSpec(64, 64, 64, (-0.5, -0.5, -0.5), vs, 3 * vs)
    fx = fy = 64.0
    cx = cy = 32.0
    c2ws = [look_at((2 * math.cos(a), 2 * math.sin(a), 0.0), (0, 0, 0)) for a in np.arange(8) * (np.pi / 4)]
    depth = render_depth_maps(scene, c2ws, fx, fy, cx, cy, 64, 64)
    az, el = np.deg2rad(22.5), np.deg2rad(20.0)
    eye = 2.0 * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    o, d = pinhole_rays(look_at(eye, (0, 0, 0)), fx, fy, cx, cy, 64, 64)
    bounds = BoundsParams(d_s=vs, t_near=0.0, t_far=4.0, step=vs, n_max=32)
    return Workload("tiny", grid, bounds, _views(c2ws, fx, fy, cx, cy, 64, 64, depth), scene,
                    o.astype(np.float32), d.astype(np.float32))


def room_scene(seed=SEED_SCENE):
    return make_box_room(seed, (-4.0, -3.0, 0.0), (4.0, 3.0, 3.0), n_boxes=20, n_plates=4)


ROOM_GRID = GridSpec(256, 256, 256, (-4.16, -4.16, 1.5 - 4.16), 8.32 / 256, 4 * 8.32 / 256)


def room_grid(n=256) -> GridSpec:
    vs = 8.32 / n
    return GridSpec(n, n, n, (-4.16, -4.16, 1.5 - 4.16), vs, 4 * vs)


def room_workload(n_views=100, width=640, height=480, grid_n=256, noise_std=0.005, with_views=True) -> Workload:
    """8x6x3 m room, 20 boxes + 4 plates; grid_n^3 grid with D_T = 4 voxels."""
    scene = room_scene()
    grid = room_grid(grid_n)
    vs = grid.voxel_size
    fx = fy = 500.0 * width / 640.0
    cx, cy = width / 2.0, height / 2.0
    c2ws = sample_free_poses(scene, np.random.default_rng(SEED_POSES), n_views, pitch_deg=TRAIN_PITCH_DEG)
    depth = render_depth_maps(scene, c2ws, fx, fy, cx, cy, width, height, noise_std) if with_views else None
    bounds = BoundsParams(d_s=vs, t_near=0.05, t_far=12.0, step=2 * vs, n_max=64)
    views = _views(c2ws, fx, fy, cx, cy, width, height, depth) if with_views else None
    return Workload("room", grid, bounds, views, scene)


def room_heldout_rays(i=0, width=640, height=480):
    scene = room_scene()
    c2w = sample_free_poses(scene, np.random.default_rng(SEED_HELDOUT), i + 1)[i]
    fx = fy = 500.0 * width / 640.0
    o, d = pinhole_rays(c2w, fx, fy, width / 2.0, height / 2.0, width, height)
    return o.astype(np.float32), d.astype(np.float32)


def room_panorama_rays(width=1024, height=512, center=(0.3, -0.2, 1.5)):
    o, d = equirect_rays(center, width, height)
    return o.astype(np.float32), d.astype(np.float32)


def room_panorama_centres(n=4):
    """Seeded in-room panorama centres, clear of solids (the ragged-batching case)."""
    poses = sample_free_poses(room_scene(), np.random.default_rng(SEED_HELDOUT + 100), n)
    return poses.reshape(n, 3, 4)[:, :, 3].copy()


def random_rays_from_views(views: Views, n, seed=SEED_TRAIN_RAYS):
    """Random training rays (and their view / pixel ids) drawn from the fused views."""
    rng = np.random.default_rng(seed)
    vi = rng.integers(0, len(views.c2w), n)
    px = rng.integers(0, views.width, n)
    py = rng.integers(0, views.height, n)
    c2w = views.c2w.reshape(-1, 3, 4).astype(np.float64)[vi]
    K = views.K.astype(np.float64)[vi]
    dc = np.stack([(px + 0.5 - K[:, 2]) / K[:, 0], (py + 0.5 - K[:, 3]) / K[:, 1], np.ones(n)], 1)
    d = np.einsum("nij,nj->ni", c2w[:, :, :3], dc)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = c2w[:, :, 3]
    return o.astype(np.float32), d.astype(np.float32), vi, px, py


def sub_sample(n_total, n, seed=SEED_RAYS):
    """Seeded sorted subset of ray indices."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=min(n, n_total), replace=False))


QUALITY_SEED = 31


def quality_pixels(n_rays, n_views, total=4096, seed=QUALITY_SEED):
    """Seeded pixel subsets for scoring image quality: `total` pixels spread over
    `n_views` views (the first total % n_views views take one more), a sorted
    subset of each view's n_rays rays, seed + v for view v."""
    base, extra = divmod(int(total), int(n_views))
    return [sub_sample(n_rays, base + (1 if v < extra else 0), seed=seed + v) for v in range(n_views)]


def random_tsdf(shape_zyx, seed, frac_neg=0.3):
    """Random normalised TSDF values in [-1, 1] with a share of exact -1 (unseen) voxels."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, shape_zyx).astype(np.float32)
    v[rng.uniform(size=shape_zyx) < frac_neg * 0.3] = -1.0
    return v


def analytic_tsdf(scene, grid: GridSpec):
    """Normalised clamped SDF of the analytic scene at voxel centres (an input stand-in
    for a fused grid, used at sizes where fusing on the CPU takes too long)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    o = np.asarray(grid.origin)
    out = np.empty((nz, ny, nx), np.float32)
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    for k in range(nz):
        x = np.stack([o[0] + (ii + 0.5) * grid.voxel_size, o[1] + (jj + 0.5) * grid.voxel_size,
                      np.full(ii.shape, o[2] + (k + 0.5) * grid.voxel_size)], -1).reshape(-1, 3)
        s = np.clip(scene.sdf(x) / grid.trunc, -1.0, 1.0)
        out[k] = s.reshape(ny, nx)
    return out


def fitted_path(name):
    import os
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", f"{name}_mlp.npz")


def scene_mlp(name) -> MLPSpec:
    """The network of a scene: the seeded initialisation refined by
    ``fit_scene_mlp`` (a stand-in for a pre-trained model), if its file exists."""
    import os
    spec = tiny_mlp() if name == "tiny" else room_mlp()
    p = fitted_path(name)
    if os.path.exists(p):
        load_mlp(spec, p)
    return spec


# ----------------------------------------------------------------------------
# torch versions of the heavy fixture geometry (same definitions as above), so
# full-size depth maps and distance grids can be generated on the device
# ----------------------------------------------------------------------------
def _t_boxes_entry(o, d, lo, hi):
    import torch
    inv = 1.0 / d
    t1 = (lo[None] - o[:, None, :]) * inv[:, None, :]
    t2 = (hi[None] - o[:, None, :]) * inv[:, None, :]
    t1 = torch.nan_to_num(t1, nan=-float("inf"))
    t2 = torch.nan_to_num(t2, nan=float("inf"))
    tmin = torch.amax(torch.minimum(t1, t2), 2)
    tmax = torch.amin(torch.maximum(t1, t2), 2)
    hit = (tmax >= tmin) & (tmin > 0)
    return torch.where(hit, tmin, torch.full_like(tmin, float("inf")))


def _t_box_exit(o, d, lo, hi):
    import torch
    inv = 1.0 / d
    t1 = torch.nan_to_num((lo[None] - o) * inv, nan=-float("inf"))
    t2 = torch.nan_to_num((hi[None] - o) * inv, nan=float("inf"))
    return torch.amin(torch.maximum(t1, t2), 1)


def ray_range_torch(scene, o, d):
    """Range of unit rays (torch float64 tensors) in a fixture scene."""
    import torch
    if isinstance(scene, SphereScene):
        c = torch.tensor(scene.center, dtype=o.dtype, device=o.device)
        oc = o - c
        b = (oc * d).sum(1)
        cc = (oc * oc).sum(1) - scene.radius ** 2
        disc = b * b - cc
        ok = disc >= 0
        sq = torch.sqrt(torch.clamp(disc, min=0))
        t0, t1 = -b - sq, -b + sq
        inf = torch.full_like(b, float("inf"))
        return torch.where(ok & (t0 > 0), t0, torch.where(ok & (t1 > 0), t1, inf))
    lo = torch.tensor(scene.box_lo, dtype=o.dtype, device=o.device)
    hi = torch.tensor(scene.box_hi, dtype=o.dtype, device=o.device)
    t_wall = _t_box_exit(o, d, torch.tensor(scene.room_lo, dtype=o.dtype, device=o.device),
                         torch.tensor(scene.room_hi, dtype=o.dtype, device=o.device))
    if lo.shape[0] == 0:
        return t_wall
    t_box = torch.amin(_t_boxes_entry(o, d, lo, hi), 1)
    return torch.minimum(t_wall, t_box)


def render_depth_maps_torch(scene, c2ws, fx, fy, cx, cy, width, height, noise_std=0.0, seed=SEED_NOISE, device="cuda"):
    """render_depth_maps on a torch device; returns a float32 tensor (V, H, W)."""
    import torch
    rng = np.random.default_rng(seed)
    u, v = torch.meshgrid(torch.arange(width, dtype=torch.float64, device=device) + 0.5,
                          torch.arange(height, dtype=torch.float64, device=device) + 0.5, indexing="xy")
    dc = torch.stack([(u - cx) / fx, (v - cy) / fy, torch.ones_like(u)], -1).reshape(-1, 3)
    out = torch.empty((len(c2ws), height, width), dtype=torch.float32, device=device)
    for i, c2w in enumerate(c2ws):
        P = torch.tensor(np.asarray(c2w), dtype=torch.float64, device=device)
        d = dc @ P[:, :3].T
        d = d / torch.linalg.norm(d, dim=1, keepdim=True)
        o = P[:, 3].expand_as(d)
        t = ray_range_torch(scene, o, d)
        if noise_std > 0:
            t = t + torch.tensor(rng.normal(0.0, noise_std, t.shape[0]), dtype=torch.float64, device=device)
        out[i] = t.reshape(height, width).to(torch.float32)
    return out


def sdf_torch(scene, x):
    import torch
    if isinstance(scene, SphereScene):
        return torch.linalg.norm(x - torch.tensor(scene.center, dtype=x.dtype, device=x.device), dim=1) - scene.radius
    rlo = torch.tensor(scene.room_lo, dtype=x.dtype, device=x.device)
    rhi = torch.tensor(scene.room_hi, dtype=x.dtype, device=x.device)
    d_room = torch.amin(torch.cat([x - rlo, rhi - x], 1), 1)
    q = torch.clamp(torch.maximum(rlo - x, x - rhi), min=0)
    out = torch.linalg.norm(q, dim=1)
    d_room = torch.where(out > 0, -out, d_room)
    if len(scene.box_lo) == 0:
        return d_room
    lo = torch.tensor(scene.box_lo, dtype=x.dtype, device=x.device)
    hi = torch.tensor(scene.box_hi, dtype=x.dtype, device=x.device)
    c = 0.5 * (lo + hi)
    h = 0.5 * (hi - lo)
    qq = torch.abs(x[:, None, :] - c[None]) - h[None]
    sb = torch.linalg.norm(torch.clamp(qq, min=0), dim=2) + torch.clamp(torch.amax(qq, 2), max=0)
    return torch.minimum(d_room, torch.amin(sb, 1))


def analytic_tsdf_torch(scene, grid: GridSpec, device="cuda", dtype=None):
    """analytic_tsdf on a torch device (float32 tensor (nz, ny, nx)); ``dtype`` is the
    arithmetic type (float64 by default, float32 for the 512^3 grid)."""
    import torch
    dt = torch.float64 if dtype is None else dtype
    o = torch.tensor(grid.origin, dtype=dt, device=device)
    jj, ii = torch.meshgrid(torch.arange(grid.ny, device=device), torch.arange(grid.nx, device=device), indexing="ij")
    out = torch.empty((grid.nz, grid.ny, grid.nx), dtype=torch.float32, device=device)
    for k in range(grid.nz):
        x = torch.stack([o[0] + (ii + 0.5) * grid.voxel_size, o[1] + (jj + 0.5) * grid.voxel_size,
                         torch.full(ii.shape, float(o[2] + (k + 0.5) * grid.voxel_size), dtype=dt,
                                    device=device)], -1).reshape(-1, 3).to(dt)
        out[k] = torch.clamp(sdf_torch(scene, x) / grid.trunc, -1.0, 1.0).reshape(grid.ny, grid.nx).to(torch.float32)
    return out


def room_workload_torch(device="cuda", n_views=100, width=640, height=480, grid_n=256, noise_std=0.005):
    """room_workload with the depth maps rendered on a torch device."""
    wl = room_workload(n_views, width, height, grid_n, noise_std, with_views=False)
    fx = fy = 500.0 * width / 640.0
    c2ws = sample_free_poses(wl.scene, np.random.default_rng(SEED_POSES), n_views, pitch_deg=TRAIN_PITCH_DEG)
    depth = render_depth_maps_torch(wl.scene, c2ws, fx, fy, width / 2.0, height / 2.0, width, height, noise_std,
                                    device=device)
    V = len(c2ws)
    wl.views = Views(np.tile(np.array([fx, fy, width / 2.0, height / 2.0], np.float32), (V, 1)),
                     np.asarray(c2ws, np.float32).reshape(V, 12), depth, width, height)
    return wl


# ----------------------------------------------------------------------------
# large: 20 x 20 x 4 m multi-room floor, 512^3 fp16 grid, 300 views of 1280x960
# ----------------------------------------------------------------------------
def large_scene(seed=SEED_SCENE + 10):
    """20x20x4 m floor split into four rooms by two 10 cm walls with 2 m doorways,
    200 random boxes (0.2-1.5 m sides) and 40 thin (2 cm) partition plates."""
    walls = [((-0.05, -10.0, 0.0), (0.05, -1.0, 4.0)), ((-0.05, 1.0, 0.0), (0.05, 10.0, 4.0)),
             ((-10.0, -0.05, 0.0), (-1.0, 0.05, 4.0)), ((1.0, -0.05, 0.0), (10.0, 0.05, 4.0))]
    return make_box_room(seed, (-10.0, -10.0, 0.0), (10.0, 10.0, 4.0), n_boxes=200, n_plates=40, interior_walls=walls)


def large_grid(n=512) -> GridSpec:
    vs = 20.48 / n
    return GridSpec(n, n, n, (-10.24, -10.24, 2.0 - 10.24), vs, 4 * vs, dtype="f16")


def large_bounds(grid: GridSpec) -> BoundsParams:
    vs = grid.voxel_size
    return BoundsParams(d_s=vs, t_near=0.05, t_far=30.0, step=2 * vs, n_max=64)


def large_poses(n=300):
    return sample_free_poses(large_scene(), np.random.default_rng(SEED_POSES + 10), n, pitch_deg=TRAIN_PITCH_DEG)


def large_panorama_centres(n=8):
    poses = sample_free_poses(large_scene(), np.random.default_rng(SEED_HELDOUT + 110), n)
    return poses.reshape(n, 3, 4)[:, :, 3].copy()


def render_depth_maps_torch_f32(scene, c2ws, fx, fy, cx, cy, width, height, noise_std=0.0, seed=SEED_NOISE,
                                device="cuda", chunk=1 << 18):
    """Depth maps of a box scene computed in float32 on a torch device, in ray chunks
    (for view counts and sizes where the float64 path is too slow)."""
    import torch
    rng = np.random.default_rng(seed)
    u, v = torch.meshgrid(torch.arange(width, dtype=torch.float32, device=device) + 0.5,
                          torch.arange(height, dtype=torch.float32, device=device) + 0.5, indexing="xy")
    dc = torch.stack([(u - cx) / fx, (v - cy) / fy, torch.ones_like(u)], -1).reshape(-1, 3)
    out = torch.empty((len(c2ws), height, width), dtype=torch.float32, device=device)
    flat = out.view(len(c2ws), -1)
    for i, c2w in enumerate(c2ws):
        P = torch.tensor(np.asarray(c2w), dtype=torch.float32, device=device)
        d = dc @ P[:, :3].T
        d = d / torch.linalg.norm(d, dim=1, keepdim=True)
        o = P[:, 3].expand_as(d)
        for a in range(0, d.shape[0], chunk):
            flat[i, a:a + chunk] = ray_range_torch(scene, o[a:a + chunk], d[a:a + chunk]).to(torch.float32)
        if noise_std > 0:
            flat[i] += torch.tensor(rng.normal(0.0, noise_std, flat.shape[1]), dtype=torch.float32, device=device)
    return out


def large_workload_torch(device="cuda", n_views=300, width=1280, height=960, noise_std=0.005):
    """The large configuration with its depth maps rendered on a torch device."""
    scene = large_scene()
    grid = large_grid()
    c2ws = large_poses(n_views)
    fx = fy = 1000.0 * width / 1280.0
    depth = render_depth_maps_torch_f32(scene, c2ws, fx, fy, width / 2.0, height / 2.0, width, height, noise_std,
                                        device=device)
    views = _views(c2ws, fx, fy, width / 2.0, height / 2.0, width, height, depth)
    return Workload("large", grid, large_bounds(grid), views, scene)

