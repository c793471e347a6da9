"""The FP64 finite-difference harness on the GPU (tsdfs_loss_f64) and the gradient
of render_rays_backward against it: central differences, h = 1e-6, of the FP64
functional L = sum g_rgb . rgb + g_depth depth + g_eik eik of the bounded render of
64 rays, over parameters of every layer of both networks."""
import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu

H = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()


def _setup(scene, n_rays, seed):
    from test_gpu_backward import case, dev
    o, d, b = case(scene, n_rays, seed)
    spec = synth.scene_mlp(scene)
    rng = np.random.default_rng(seed + 1)
    g_rgb = rng.normal(0, 1, (n_rays, 3)).astype(np.float32)
    g_depth = rng.normal(0, 1, n_rays).astype(np.float32)
    g_eik = np.full(n_rays, 0.1, np.float32)
    offsets = np.concatenate([[0], np.cumsum(b["n"])]).astype(np.int32)
    total = int(offsets[-1])
    t = {"o": dev(o), "d": dev(d), "t_n": dev(b["t_n"].astype(np.float32)), "t_f": dev(b["t_f"].astype(np.float32)),
         "off": dev(offsets), "st": dev(b["status"]), "g_rgb": dev(g_rgb), "g_depth": dev(g_depth),
         "g_eik": dev(g_eik)}
    return spec, o, d, b, g_rgb, g_depth, g_eik, total, t


def _loss64(mlp, w_sdf, w_rgb, t, total, ws, out):
    T.tsdfs_loss_f64(mlp, w_sdf, w_rgb, t["o"], t["d"], t["t_n"], t["t_f"], t["off"], t["st"], total, t["g_rgb"],
                     t["g_depth"], t["g_eik"], out, ws)
    return float(out.item())


@pytest.mark.parametrize("scene,n_rays", [("tiny", 64), ("room", 64)])
def test_fp64_functional_matches_oracle(scene, n_rays):
    """The harness computes the oracle's FP64 functional (same inputs, FP64 on both
    sides; only the summation order differs)."""
    spec, o, d, b, g_rgb, g_depth, g_eik, total, t = _setup(scene, n_rays, 51)
    mlp = T.Mlp(spec)
    w_sdf, w_rgb = mlp.sdf_w.double(), mlp.rgb_w.double()
    ws = torch.empty(T.tsdfs_loss_f64_workspace_size(n_rays, total), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    got = _loss64(mlp, w_sdf, w_rgb, t, total, ws, out)
    # the descriptor carries the network's constants as float32 (scale 4.16 is 4.1599998...):
    # give the oracle the same values, so that both sides compute the same function
    import dataclasses
    spec32 = dataclasses.replace(spec, scale=float(np.float32(spec.scale)),
                                 center=tuple(float(np.float32(c)) for c in spec.center),
                                 alpha_eps=float(np.float32(spec.alpha_eps)))
    with torch.no_grad():
        r = orr.render_bounded(orr.Net(spec32), o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])
    counts = torch.as_tensor(b["n"].astype(np.int64))
    eik_ray = torch.zeros(len(counts), dtype=torch.float64).index_add(
        0, torch.repeat_interleave(torch.arange(len(counts)), counts), r["eik"]) * torch.as_tensor(b["status"] == 1)
    ref = float((r["rgb"] * torch.as_tensor(g_rgb, dtype=torch.float64)).sum()
                + (r["depth"] * torch.as_tensor(g_depth, dtype=torch.float64)).sum()
                + (eik_ray * torch.as_tensor(g_eik, dtype=torch.float64)).sum())
    print(f"{scene}: L gpu f64 {got:.15e} oracle {ref:.15e}")
    assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


@pytest.mark.parametrize("scene,n_rays", [("tiny", 64), ("room", 64)])
def test_backward_matches_fp64_central_differences(scene, n_rays):
    """render_rays_backward (FP32) against FP64 central differences (h = 1e-6) of the
    harness's functional, for the largest-gradient parameter of every layer of both
    networks (weights and biases) and for seeded random ones."""
    spec, o, d, b, g_rgb, g_depth, g_eik, total, t = _setup(scene, n_rays, 52)
    mlp = T.Mlp(spec)
    d_sdf = torch.zeros_like(mlp.sdf_w)
    d_rw = torch.zeros_like(mlp.rgb_w)
    wsb = torch.empty(T.tsdfs_backward_workspace_size(mlp, n_rays, total), dtype=torch.uint8, device="cuda")
    T.render_rays_backward(mlp, t["o"], t["d"], t["t_n"], t["t_f"], t["off"], t["st"], total, t["g_rgb"], t["g_depth"],
                           t["g_eik"], d_sdf, d_rw, wsb)
    torch.cuda.synchronize()
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ws = torch.empty(T.tsdfs_loss_f64_workspace_size(n_rays, total), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    nets = {"sdf": (spec.sdf, d_sdf.cpu().numpy().astype(np.float64)),
            "rgb": (spec.rgb, d_rw.cpu().numpy().astype(np.float64))}
    rng = np.random.default_rng(9)
    checked, worst = 0, 0.0
    for which, (layers, grad) in nets.items():
        scale = np.abs(grad).max()
        # parameter indices: per layer, the largest-gradient weight and bias, and two random weights
        idx, off = [], 0
        for W, bvec in layers:
            nw, nb = W.size, bvec.size
            gw, gb = grad[off:off + nw], grad[off + nw:off + nw + nb]
            idx += [off + int(np.argmax(np.abs(gw))), off + nw + int(np.argmax(np.abs(gb)))]
            idx += [off + int(i) for i in rng.integers(0, nw, 2)]
            off += nw + nb
        for i in idx:
            w_sdf, w_rgb = mlp.sdf_w.double(), mlp.rgb_w.double()
            tgt = w_sdf if which == "sdf" else w_rgb
            base = float(tgt[i].item())
            tgt[i] = base + H
            lp = _loss64(mlp, w_sdf, w_rgb, t, total, ws, out)
            tgt[i] = base - H
            lm = _loss64(mlp, w_sdf, w_rgb, t, total, ws, out)
            fd = (lp - lm) / (2 * H)
            err = abs(fd - grad[i]) / scale
            worst = max(worst, err)
            checked += 1
            assert err < 2e-3, (which, i, fd, grad[i], scale)
    print(f"{scene}: {checked} parameters, max |fd - grad| / max |grad| = {worst:.2e}")
