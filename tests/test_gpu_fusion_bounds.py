"""GPU parity of fusion (K1), the inside mask (K2), ray bounds (K3) and the
offsets scan (K4) against the oracle's fp32-exact mode: bit for bit.

Inputs are seeded and synthetic; grids fed to the bounds kernel come from the
oracle or from the analytic fixture, never from the CUDA path."""
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


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a.view(np.uint16)


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def fuse_gpu(spec, views):
    g = T.Grid(spec).init()
    depth = views.depth if isinstance(views.depth, torch.Tensor) else dev(views.depth)
    g.integrate(depth.cuda().contiguous(), dev(views.K), dev(views.c2w))
    torch.cuda.synchronize()
    return g


def check_status_clean():
    rc, b = T.tsdfs_sync_status()
    assert rc == T.TSDFS_OK and b == 0


# ---------------------------------------------------------------- fusion ----
def test_grid_init():
    spec = synth.GridSpec(37, 29, 23, (0, 0, 0), 0.1, 0.3)
    g = T.Grid(spec).init()
    torch.cuda.synchronize()
    assert torch.all(g.V == -1.0) and torch.all(g.W == 0)


def test_tiny_fusion_bit_exact():
    wl = synth.tiny_workload()
    g = fuse_gpu(wl.grid, wl.views)
    V, W = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    assert np.array_equal(g.W.cpu().numpy(), W)
    assert np.array_equal(bits(g.V.cpu().numpy()), bits(V))
    check_status_clean()


def test_ragged_grid_fusion_bit_exact():
    wl = synth.tiny_workload()
    spec = synth.GridSpec(37, 29, 23, (-0.55, -0.41, -0.33), 0.031, 0.09)
    g = fuse_gpu(spec, wl.views)
    V, W = cgrid.integrate_projective(spec, wl.views, "f32")
    assert np.array_equal(g.W.cpu().numpy(), W)
    assert np.array_equal(bits(g.V.cpu().numpy()), bits(V))


def test_fusion_in_two_calls_equals_one():
    wl = synth.tiny_workload()
    g = T.Grid(wl.grid).init()
    d = dev(wl.views.depth)
    K, P = dev(wl.views.K), dev(wl.views.c2w)
    g.integrate(d[:3].contiguous(), K[:3].contiguous(), P[:3].contiguous())
    g.integrate(d[3:].contiguous(), K[3:].contiguous(), P[3:].contiguous())
    V, W = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    assert np.array_equal(g.W.cpu().numpy(), W)
    assert np.array_equal(bits(g.V.cpu().numpy()), bits(V))


def test_tiny_fusion_f16_storage_bit_exact():
    wl = synth.tiny_workload()
    spec = synth.GridSpec(**{**wl.grid.__dict__, "dtype": "f16"})
    g = fuse_gpu(spec, wl.views)
    V, W = cgrid.integrate_projective(spec, wl.views, "f32")
    assert np.array_equal(g.W.cpu().numpy(), W)
    assert np.array_equal(g.V.cpu().numpy().view(np.uint16), V)


@pytest.fixture(scope="module")
def room():
    wl = synth.room_workload_torch(device="cuda")
    return wl


def test_room_fusion_full_size_sampled_bit_exact(room):
    """256^3 grid, 100 views of 640x480 (the room workload): every voxel on the
    GPU; the oracle recomputes a seeded sample of 30000 voxels."""
    g = fuse_gpu(room.grid, room.views)
    views_np = synth.Views(room.views.K, room.views.c2w, room.views.depth.cpu().numpy(), 640, 480)
    n = room.grid.nx * room.grid.ny * room.grid.nz
    vox = synth.sub_sample(n, 30000, seed=21)
    V, W = cgrid.integrate_projective(room.grid, views_np, "f32", vox=vox)
    Vg = g.V.reshape(-1)[torch.as_tensor(vox).cuda()].cpu().numpy()
    Wg = g.W.reshape(-1)[torch.as_tensor(vox).cuda()].cpu().numpy()
    assert np.array_equal(Wg, W)
    assert np.array_equal(bits(Vg), bits(V))
    assert (W > 0).mean() > 0.15  # the 8x6x3 m room fills 25% of the 8.32 m grid cube
    check_status_clean()


# ------------------------------------------------------------ inside mask ----
def unpack_mask(words, n):
    b = np.unpackbits(words.view(np.uint8), bitorder="little")
    return b[:n].astype(bool)


@pytest.mark.parametrize("radius", [1, 2, 3])
@pytest.mark.parametrize("shape", [(64, 64, 64), (23, 29, 37)])
def test_inside_mask_bit_exact(radius, shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(radius)
    V = -rng.uniform(0, 1, shape).astype(np.float32)
    V[rng.uniform(size=shape) < 0.002] = 0.4
    spec = synth.GridSpec(nx, ny, nz, (0, 0, 0), 0.1, 0.3)
    g = T.Grid(spec, V=dev(V), W=torch.zeros(shape, dtype=torch.uint8, device="cuda"))
    m = g.inside_mask(radius)
    torch.cuda.synchronize()
    ref = cgrid.inside_mask(spec, V, radius).reshape(-1).astype(bool)
    got = unpack_mask(m.cpu().numpy(), nx * ny * nz)
    assert np.array_equal(got, ref)
    assert ref.any() and not ref.all()


# ----------------------------------------------------------------- bounds ----
def run_bounds(spec, V, o, d, bp, use_mask):
    g = T.Grid(spec, V=dev(V), W=torch.zeros(V.shape, dtype=torch.uint8, device="cuda"))
    mask = g.inside_mask(bp.nb_radius) if use_mask else None
    b = T.Bounds(len(o)).compute(g, dev(o), dev(d), bp, mask)
    torch.cuda.synchronize()
    return {k: getattr(b, k).cpu().numpy() for k in ("t_n", "t_f", "n", "offsets", "t_zero", "status")}


def assert_bounds_equal(got, ref, idx=None):
    sel = slice(None) if idx is None else idx
    assert np.array_equal(got["status"][sel], ref["status"])
    assert np.array_equal(got["n"][sel], ref["n"])
    assert np.array_equal(bits(got["t_n"][sel]), bits(ref["t_n"]))
    assert np.array_equal(bits(got["t_f"][sel]), bits(ref["t_f"]))
    tz_g, tz_r = got["t_zero"][sel], ref["t_zero"]
    assert np.array_equal(np.isnan(tz_g), np.isnan(tz_r))
    ok = ~np.isnan(tz_r)
    assert np.array_equal(bits(tz_g[ok]), bits(tz_r[ok]))


@pytest.mark.parametrize("use_mask", [False, True])
def test_tiny_bounds_bit_exact(use_mask):
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    ref = cgrid.ray_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f32")
    got = run_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, use_mask)
    assert_bounds_equal(got, ref)
    assert np.array_equal(got["offsets"], np.concatenate([[0], np.cumsum(ref["n"])]).astype(np.int32))
    assert set(np.unique(ref["status"])) == {0, 1, 2}
    check_status_clean()


def test_tiny_bounds_f16_grid_bit_exact():
    wl = synth.tiny_workload()
    spec = synth.GridSpec(**{**wl.grid.__dict__, "dtype": "f16"})
    V16, _ = cgrid.integrate_projective(spec, wl.views, "f32")
    ref = cgrid.ray_bounds(spec, V16, wl.rays_o, wl.rays_d, wl.bounds, "f32")
    g = T.Grid(spec, V=torch.as_tensor(V16.view(np.float16)).cuda(),
               W=torch.zeros(V16.shape, dtype=torch.uint8, device="cuda"))
    b = T.Bounds(4096).compute(g, dev(wl.rays_o), dev(wl.rays_d), wl.bounds)
    torch.cuda.synchronize()
    got = {k: getattr(b, k).cpu().numpy() for k in ("t_n", "t_f", "n", "offsets", "t_zero", "status")}
    assert_bounds_equal(got, ref)


@pytest.fixture(scope="module")
def room_grid():
    wl = synth.room_workload(with_views=False)
    V = synth.analytic_tsdf_torch(wl.scene, wl.grid, device="cuda").cpu().numpy()
    return wl, V


@pytest.mark.parametrize("rays", ["pinhole", "panorama"])
def test_room_bounds_full_size_sampled_bit_exact(room_grid, rays):
    """307200 pinhole / 524288 equirect rays on the 256^3 grid; the oracle
    recomputes a seeded sample of 4096 rays; offsets are the exclusive scan."""
    wl, V = room_grid
    o, d = synth.room_heldout_rays(0) if rays == "pinhole" else synth.room_panorama_rays()
    got = run_bounds(wl.grid, V, o, d, wl.bounds, use_mask=True)
    idx = synth.sub_sample(len(o), 4096, seed=22)
    ref = cgrid.ray_bounds(wl.grid, V, o[idx], d[idx], wl.bounds, "f32")
    assert_bounds_equal(got, ref, idx)
    cs = np.concatenate([[0], np.cumsum(got["n"].astype(np.int64))])
    assert np.array_equal(got["offsets"].astype(np.int64), cs)
    st = got["status"]
    assert (st == 1).mean() > 0.9
    assert got["n"][st == 1].max() <= wl.bounds.n_max
    check_status_clean()


def test_room_bounds_mask_and_direct_agree(room_grid):
    wl, V = room_grid
    o, d = synth.room_heldout_rays(1)
    a = run_bounds(wl.grid, V, o, d, wl.bounds, use_mask=True)
    b = run_bounds(wl.grid, V, o, d, wl.bounds, use_mask=False)
    for k in ("t_n", "t_f", "n", "offsets", "status"):
        assert np.array_equal(a[k], b[k])


def test_bounds_zero_rays_and_all_miss():
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    g = T.Grid(wl.grid, V=dev(V), W=torch.zeros(V.shape, dtype=torch.uint8, device="cuda"))
    b = T.Bounds(0)
    e = torch.empty((0, 3), device="cuda")
    b.compute(g, e, e, wl.bounds)
    torch.cuda.synchronize()
    assert b.offsets.cpu().tolist() == [0]
    o = np.tile(np.array([[5.0, 5.0, 5.0]], np.float32), (10000, 1))
    d = np.tile(np.array([[0.0, 0.0, 1.0]], np.float32), (10000, 1))
    got = run_bounds(wl.grid, V, o, d, wl.bounds, False)
    assert np.all(got["status"] == 0) and np.all(got["n"] == 0) and got["offsets"][-1] == 0


def _degenerate_rays():
    """Rays the voxel walk treats specially: axis-aligned in both senses (zero
    direction components), exact diagonals, origins on voxel boundaries and grid
    faces, origins inside the sphere, rays grazing the grid box, rays that miss."""
    vs = 1.0 / 64
    o, d = [], []
    for a in range(3):
        for sgn in (1.0, -1.0):
            for off in (0.0, 0.5 * vs, vs, 0.123, -0.31):
                p = np.array([off, -off, 0.25 * off])
                p[a] = -sgn * 0.9
                v = np.zeros(3)
                v[a] = sgn
                o.append(p); d.append(v)
    for v in ([1, 1, 1], [1, -1, 1], [-1, -1, -1], [1, 1, 0], [0, 1, -1]):
        v = np.asarray(v, np.float64)
        v /= np.linalg.norm(v)
        for p in ([-0.8, -0.8, -0.8], [0.0, 0.0, 0.0], [0.1, -0.2, 0.05], [-0.5, -0.5, -0.5], [8 * vs, 4 * vs, 0.0]):
            o.append(np.asarray(p, np.float64) - 0.0 * v); d.append(v)
    # grazing the box edges and faces, and parallel to a face just outside it
    for p, v in (([-0.9, 0.5, 0.0], [1, 0, 0]), ([-0.9, 0.5 - 1e-7, 0.5 - 1e-7], [1, 0, 0]),
                 ([-0.9, 0.5000001, 0.0], [1, 0, 0]), ([0.5, -0.9, 0.5], [0, 1, 0]),
                 ([-0.9, -0.9, 0.0], [1, 1e-7, 0]), ([0.0, 0.0, 0.49], [0, 0, 1]), ([0.0, 0.0, 0.0], [0, 0, 1])):
        v = np.asarray(v, np.float64)
        o.append(np.asarray(p, np.float64)); d.append(v / np.linalg.norm(v))
    return np.asarray(o, np.float32), np.asarray(d, np.float32)


@pytest.mark.parametrize("use_mask", [False, True])
def test_degenerate_rays_bit_exact(use_mask):
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    o, d = _degenerate_rays()
    for bp in (wl.bounds, synth.BoundsParams(**{**wl.bounds.__dict__, "t_near": 0.3})):
        ref = cgrid.ray_bounds(wl.grid, V, o, d, bp, "f32")
        got = run_bounds(wl.grid, V, o, d, bp, use_mask)
        assert_bounds_equal(got, ref)
        assert np.array_equal(got["offsets"], np.concatenate([[0], np.cumsum(ref["n"])]).astype(np.int32))
    assert set(np.unique(ref["status"])) >= {0, 1}
    check_status_clean()


def test_every_march_launch_shape_bit_exact_and_autotune():
    """The march's outputs do not depend on its launch shape: every shape the
    autotuner may pick reproduces the oracle bit for bit on a ragged ray count
    (several blocks and a partial one for each shape); the autotuner picks one of
    them and leaves correct outputs behind."""
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    n = 3001
    o, d = wl.rays_o[:n], wl.rays_d[:n]
    ref = cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")
    try:
        for block in (64, 128, 256):
            for per_sm in (1, 4, 64):
                T.tsdfs_set_bounds_launch_shape(block, per_sm)
                assert T.tsdfs_bounds_launch_shape() == (block, per_sm)
                for use_mask in (False, True):
                    assert_bounds_equal(run_bounds(wl.grid, V, o, d, wl.bounds, use_mask), ref)
        g = T.Grid(wl.grid, V=dev(V), W=torch.zeros(V.shape, dtype=torch.uint8, device="cuda"))
        b = T.Bounds(n)
        block, per_sm, ms = b.autotune(g, dev(o), dev(d), wl.bounds, g.inside_mask(wl.bounds.nb_radius), reps=2)
        torch.cuda.synchronize()
        assert block in (64, 128, 256) and per_sm in (4, 8, 16, 32, 64) and ms > 0
        assert T.tsdfs_bounds_launch_shape() == (block, per_sm)
        assert_bounds_equal({k: getattr(b, k).cpu().numpy() for k in ("t_n", "t_f", "n", "t_zero", "status")}, ref)
    finally:
        T.tsdfs_set_bounds_launch_shape(0, 0)
    assert T.tsdfs_bounds_launch_shape() == (128, 64)
    check_status_clean()
