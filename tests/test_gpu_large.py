"""The large configuration at full size (20x20x4 m floor, 512^3 fp16 grid, 300
views of 1280x960, 2048x1024 panoramas), checked on sampled outputs that the
oracle computes one by one: fusion bit for bit on seeded voxels, bounds bit
for bit on seeded rays of a whole panorama, the fp16 tensor-core render of
those rays within the render tolerances.  Inputs are seeded fixtures (depth
maps and the exact distance grid come from torch, not from the library)."""
import numpy as np
import pytest
import torch

from oracle import cgrid
from oracle import render as orr
from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()


def _halfbits(t):
    return t.contiguous().view(torch.int16).cpu().numpy().view(np.uint16)


def test_large_fusion_fp16_sampled_voxels_bit_exact():
    wl = synth.large_workload_torch(device="cuda")
    g = T.Grid(wl.grid).init()
    g.integrate(wl.views.depth.contiguous(), torch.tensor(wl.views.K, device="cuda"),
                torch.tensor(wl.views.c2w, device="cuda"))
    torch.cuda.synchronize()
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    # seeded voxels inside the floor's box (most are observed), plus a few anywhere
    rng = np.random.default_rng(81)
    vs, org = wl.grid.voxel_size, np.asarray(wl.grid.origin)
    lo = np.floor((np.array([-10.0, -10.0, 0.0]) - org) / vs).astype(np.int64)
    hi = np.floor((np.array([10.0, 10.0, 4.0]) - org) / vs).astype(np.int64)
    ijk = np.concatenate([rng.integers(lo, hi, (3000, 3)), rng.integers(0, 512, (1000, 3))])
    vox = (ijk[:, 2] * 512 + ijk[:, 1]) * 512 + ijk[:, 0]
    views = synth.Views(wl.views.K, wl.views.c2w, wl.views.depth.cpu().numpy(), wl.views.width, wl.views.height)
    V_or, W_or = cgrid.integrate_projective(wl.grid, views, "f32", vox=vox)
    V_gpu = _halfbits(g.V).reshape(-1)[vox]
    W_gpu = g.W.cpu().numpy().reshape(-1)[vox]
    assert np.array_equal(W_gpu, W_or)
    assert np.array_equal(V_gpu, V_or)
    assert (W_or > 0).mean() > 0.3


def test_large_bounds_and_render_sampled_rays():
    scene, spec_g = synth.large_scene(), synth.large_grid()
    bp = synth.large_bounds(spec_g)
    V16 = synth.analytic_tsdf_torch(scene, spec_g, device="cuda", dtype=torch.float32).to(torch.float16)
    g = T.Grid(spec_g, V=V16, W=torch.ones(V16.shape, dtype=torch.uint8, device="cuda"))
    c = synth.large_panorama_centres(8)[0]
    o, d = synth.room_panorama_rays(2048, 1024, center=tuple(c))
    n = len(o)
    bounds = T.Bounds(n).compute(g, torch.tensor(o, device="cuda"), torch.tensor(d, device="cuda"), bp, None)
    torch.cuda.synchronize()
    idx = synth.sub_sample(n, 4096, seed=82)
    ob = cgrid.ray_bounds(spec_g, _halfbits(V16), o[idx], d[idx], bp, "f32")
    for k in ("t_n", "t_f", "t_zero"):
        assert np.array_equal(getattr(bounds, k).cpu().numpy()[idx].view(np.uint32), ob[k].view(np.uint32)), k
    assert np.array_equal(bounds.n.cpu().numpy()[idx], ob["n"])
    assert np.array_equal(bounds.status.cpu().numpy()[idx], ob["status"])
    total = int(bounds.offsets[-1].item())
    assert total == int(bounds.n.sum().item())
    # fp16 tensor-core render of the whole panorama; the oracle renders a sample of it
    spec = synth.scene_mlp("room")
    mlp = T.Mlp(spec, T.TSDFS_PREC_F16)
    rend = T.Renderer(mlp, n, max(total, 1))
    out = rend.render(torch.tensor(o, device="cuda"), torch.tensor(d, device="cuda"), bounds)
    torch.cuda.synchronize()
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    sel = idx[:256]
    ob2 = cgrid.ray_bounds(spec_g, _halfbits(V16), o[sel], d[sel], bp, "f32")
    with torch.no_grad():
        ref = orr.render_bounded(orr.Net(spec), o[sel], d[sel], ob2["t_n"].astype(np.float64),
                                 ob2["t_f"].astype(np.float64), ob2["n"])
    er = np.abs(out.rgb.cpu().numpy()[sel] - ref["rgb"].numpy()).max(1)
    ok = ref["wsum"].numpy() > 1e-3
    ed = np.abs(out.depth.cpu().numpy()[sel][ok] - ref["depth"].numpy()[ok]) / np.abs(ref["depth"].numpy()[ok])
    assert er.max() < 2e-3 and ed.max() < 2e-3
