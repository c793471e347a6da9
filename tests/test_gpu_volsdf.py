"""GPU parity of the VolSDF opacity (Laplace-CDF density, alpha = 1 - exp(-sigma
delta)) through the render, the hierarchical comparator, the sampler inside the
bound and the backward, against the oracle with the same network switched to
that opacity."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import cgrid
from oracle import render as orr
from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu

DEPTH_REL_F32 = 1e-4
RGB_ABS = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def tiny():
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    b = cgrid.ray_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f32")
    spec = dataclasses.replace(synth.scene_mlp("tiny"), opacity=T.TSDFS_OPACITY_VOLSDF)
    return wl, b, spec


def bounds_dev(b):
    bb = T.Bounds(len(b["t_n"]))
    bb.t_n.copy_(dev(b["t_n"].astype(np.float32)))
    bb.t_f.copy_(dev(b["t_f"].astype(np.float32)))
    bb.status.copy_(dev(b["status"]))
    bb.n.copy_(dev(b["n"].astype(np.int32)))
    bb.offsets.copy_(dev(np.concatenate([[0], np.cumsum(b["n"])]).astype(np.int32)))
    return bb


def compare(got, ref, live, rgb_abs=RGB_ABS, depth_rel=DEPTH_REL_F32):
    ref = {k: (v.detach().numpy() if isinstance(v, torch.Tensor) else v) for k, v in ref.items()}
    assert np.max(np.abs(got["rgb"][live] - ref["rgb"][live])) < rgb_abs
    assert np.max(np.abs(got["wsum"][live] - ref["wsum"][live])) < rgb_abs
    ok = live & (ref["wsum"] > 1e-3)
    rel = np.abs(got["depth"][ok] - ref["depth"][ok]) / np.maximum(np.abs(ref["depth"][ok]), 1e-6)
    assert rel.max() < depth_rel


def host(out):
    return {k: getattr(out, k).cpu().numpy() for k in ("rgb", "depth", "wsum", "normal")}


def test_volsdf_render_f32_matches_oracle(tiny):
    wl, b, spec = tiny
    mlp = T.Mlp(spec)
    bb = bounds_dev(b)
    r = T.Renderer(mlp, len(b["n"]), int(b["n"].sum()))
    got = host(r.render(dev(wl.rays_o), dev(wl.rays_d), bb))
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    with torch.no_grad():
        ref = orr.render_bounded(orr.Net(spec), wl.rays_o, wl.rays_d, b["t_n"].astype(np.float64),
                                 b["t_f"].astype(np.float64), b["n"])
    live = b["n"] > 0
    compare(got, ref, live)
    # the opacity is really the other one: NeuS on the same inputs differs
    neus = host(T.Renderer(T.Mlp(synth.scene_mlp("tiny")), len(b["n"]), int(b["n"].sum())).render(
        dev(wl.rays_o), dev(wl.rays_d), bb))
    assert np.max(np.abs(neus["wsum"] - got["wsum"])) > 1e-2


def test_volsdf_render_f16_tracks_oracle(tiny):
    wl, b, spec = tiny
    mlp = T.Mlp(spec, T.TSDFS_PREC_F16)
    got = host(T.Renderer(mlp, len(b["n"]), int(b["n"].sum())).render(dev(wl.rays_o), dev(wl.rays_d), bounds_dev(b)))
    with torch.no_grad():
        ref = orr.render_bounded(orr.Net(spec), wl.rays_o, wl.rays_d, b["t_n"].astype(np.float64),
                                 b["t_f"].astype(np.float64), b["n"])
    live = b["n"] > 0
    er = np.abs(got["rgb"] - ref["rgb"].numpy())[live].max(1)
    assert np.percentile(er, 99) <= 2 * RGB_ABS and er.max() <= 8 * RGB_ABS


@pytest.mark.parametrize("n_coarse,n_fine", [(64, 32), (16, 8)])
def test_volsdf_comparator_f32_matches_oracle(tiny, n_coarse, n_fine):
    wl, _, spec = tiny
    bp = wl.bounds
    t0, te, ok = cgrid.clip_rays(wl.grid, wl.rays_o, wl.rays_d, bp.t_near, bp.t_far, "f32")
    g = T.Grid(wl.grid, V=torch.zeros(wl.grid.shape_zyx, device="cuda"),
               W=torch.zeros(wl.grid.shape_zyx, dtype=torch.uint8, device="cuda"))
    h = T.HierRenderer(T.Mlp(spec), 4096, n_coarse=n_coarse, n_fine=n_fine)
    got = host(h.render(g, dev(wl.rays_o), dev(wl.rays_d), bp.t_near, bp.t_far))
    live = np.nonzero(ok)[0]
    with torch.no_grad():
        ro = orr.render_hier(orr.Net(spec), wl.rays_o[live], wl.rays_d[live], t0[live].astype(np.float64),
                             te[live].astype(np.float64), n_coarse=n_coarse, n_fine=n_fine)
    compare({k: v[live] for k, v in got.items()}, ro, np.ones(len(live), bool))


def test_volsdf_in_bound_sampler_f32_matches_oracle(tiny):
    wl, b, spec = tiny
    counts, _ = orr.adaptive_counts(b["t_n"], b["t_f"], b["status"], 6.0, 2, 64, 64)
    bb = bounds_dev({**b, "n": counts})
    h = T.HierBoundedRenderer(T.Mlp(spec), len(counts), 8, int(counts.sum()))
    got = host(h.render(dev(wl.rays_o), dev(wl.rays_d), bb))
    with torch.no_grad():
        ref = orr.render_hier_bounded(orr.Net(spec), wl.rays_o, wl.rays_d, b["t_n"].astype(np.float64),
                                      b["t_f"].astype(np.float64), counts, 8)
    compare(got, ref, counts > 0)


def test_volsdf_backward_matches_oracle_gradient(tiny):
    wl, b, spec = tiny
    live = np.nonzero(b["status"] != 0)[0]
    idx = np.random.default_rng(43).choice(live, 96, replace=False)
    o, d = wl.rays_o[idx], wl.rays_d[idx]
    bs = {k: v[idx] for k, v in b.items() if isinstance(v, np.ndarray) and len(v) == len(b["t_n"])}
    rng = np.random.default_rng(8)
    d_rgb = rng.normal(0, 1, (96, 3)).astype(np.float32)
    d_depth = rng.normal(0, 1, 96).astype(np.float32)
    d_eik = np.full(96, 0.1, np.float32)
    mlp = T.Mlp(spec)
    offsets = np.concatenate([[0], np.cumsum(bs["n"])]).astype(np.int32)
    total = int(offsets[-1])
    d_sdf = torch.zeros_like(mlp.sdf_w)
    d_rw = torch.zeros_like(mlp.rgb_w)
    ws = torch.empty(T.tsdfs_backward_workspace_size(mlp, 96, total), dtype=torch.uint8, device="cuda")
    T.render_rays_backward(mlp, dev(o), dev(d), dev(bs["t_n"].astype(np.float32)), dev(bs["t_f"].astype(np.float32)),
                           dev(offsets), dev(bs["status"]), total, dev(d_rgb), dev(d_depth), dev(d_eik), d_sdf, d_rw, ws)
    torch.cuda.synchronize()
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    from test_gpu_backward import oracle_grads
    ref_sdf, ref_rgb = oracle_grads(spec, o, d, bs, d_rgb, d_depth, d_eik)
    for got, ref in [(d_sdf.cpu().numpy(), ref_sdf), (d_rw.cpu().numpy(), ref_rgb)]:
        assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-3
