"""Fit the seeded SDF / colour networks to an analytic synthetic scene.

The paper renders with a pre-trained neural surface field (MonoSDF / NeRF,
Sec. 4.2) whose trained weights are not available here.  This script makes a
stand-in: starting from the seeded geometric initialisation of
:mod:`synth`, it regresses the SDF network to the scene's analytic signed
distance (L1 + eikonal) and the colour network to the albedo of the surface
points seen by the training views, with Adam, seeded and single-threaded so
the result is reproducible on one machine.  The fitted parameters are stored
as ``data/<scene>_mlp.npz`` (values rounded to bfloat16) and loaded by
:func:`synth.scene_mlp`.

It is an input generator: its network code is a compact autograd version of
the architecture and is not used by the render path or its checks.

    python -m paper_2311_17878_gb300.fit_scene_mlp tiny
    python -m paper_2311_17878_gb300.fit_scene_mlp room --steps 4000
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np
import torch

from . import synth

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


class _Fit(torch.nn.Module):
    def __init__(self, spec: synth.MLPSpec):
        super().__init__()
        self.spec = spec
        self.sdf = torch.nn.ParameterList()
        for W, b in spec.sdf:
            self.sdf.append(torch.nn.Parameter(torch.tensor(W, dtype=torch.float32)))
            self.sdf.append(torch.nn.Parameter(torch.tensor(b, dtype=torch.float32)))
        self.rgb = torch.nn.ParameterList()
        for W, b in spec.rgb:
            self.rgb.append(torch.nn.Parameter(torch.tensor(W, dtype=torch.float32)))
            self.rgb.append(torch.nn.Parameter(torch.tensor(b, dtype=torch.float32)))

    @staticmethod
    def _enc(x, L):
        out = [x]
        for k in range(L):
            out += [torch.sin((2.0 ** k) * x), torch.cos((2.0 ** k) * x)]
        return torch.cat(out, -1)

    def sdf_net(self, x):
        s = self.spec
        xt = (x - torch.tensor(s.center, dtype=x.dtype)) / s.scale
        g = self._enc(xt, s.pe_sdf)
        h = g
        n = len(self.sdf) // 2
        for l in range(n):
            if l == s.skip_layer:
                h = torch.cat([h, g], -1) / math.sqrt(2.0)
            h = h @ self.sdf[2 * l].T + self.sdf[2 * l + 1]
            if l < n - 1:
                h = torch.nn.functional.softplus(h, beta=s.beta, threshold=20.0)
        return s.scale * h[:, 0], h[:, 1:]

    def rgb_net(self, x, v, nrm, feat):
        s = self.spec
        xt = (x - torch.tensor(s.center, dtype=x.dtype)) / s.scale
        venc = self._enc(v, s.pe_dir) if s.pe_dir else v
        h = torch.cat([xt, venc, nrm, feat], -1)
        n = len(self.rgb) // 2
        for l in range(n):
            h = h @ self.rgb[2 * l].T + self.rgb[2 * l + 1]
            h = torch.relu(h) if l < n - 1 else torch.sigmoid(h)
        return h

    def export(self):
        sdf = [(self.sdf[2 * i].detach().numpy(), self.sdf[2 * i + 1].detach().numpy()) for i in range(len(self.sdf) // 2)]
        rgb = [(self.rgb[2 * i].detach().numpy(), self.rgb[2 * i + 1].detach().numpy()) for i in range(len(self.rgb) // 2)]
        return sdf, rgb


def _surface_batch(scene, c2ws, K, W, H, rng, n):
    vi = rng.integers(0, len(c2ws), n)
    px = rng.uniform(0, W, n)
    py = rng.uniform(0, H, n)
    c2w = c2ws[vi]
    dc = np.stack([(px - K[2]) / K[0], (py - K[3]) / K[1], np.ones(n)], 1)
    d = np.einsum("nij,nj->ni", c2w[:, :, :3], dc)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = c2w[:, :, 3]
    if hasattr(scene, "box_lo"):
        t, ids = scene.ray_range(o, d, return_id=True)
        alb = scene.albedo_at(ids)
    else:
        t = scene.ray_range(o, d)
        alb = np.tile(np.asarray(scene.albedo), (n, 1))
    ok = np.isfinite(t)
    return o[ok] + t[ok, None] * d[ok], d[ok], alb[ok]


def fit(name, steps, batch, lr, seed=7, log_every=200):
    torch.manual_seed(seed)
    torch.set_num_threads(int(os.environ.get("FIT_THREADS", "8")))
    rng = np.random.default_rng(seed)
    if name == "tiny":
        spec = synth.tiny_mlp()
        wl = synth.tiny_workload()
        scene = wl.scene
        lo, hi = wl.grid.aabb
        c2ws = wl.views.c2w.reshape(-1, 3, 4).astype(np.float64)
        K = wl.views.K[0].astype(np.float64)
        Wd, Hd = wl.views.width, wl.views.height
        near_sigma = 0.02
    else:
        spec = synth.room_mlp()
        wl = synth.room_workload(with_views=False)
        scene = wl.scene
        lo, hi = wl.grid.aabb
        c2ws = synth.sample_free_poses(scene, np.random.default_rng(synth.SEED_POSES), 100)
        K = np.array([500.0, 500.0, 320.0, 240.0])
        Wd, Hd = 640, 480
        near_sigma = 0.05
    model = _Fit(spec)
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps, eta_min=lr * 0.05)
    t_start = time.time()
    for it in range(steps):
        ps, vs, alb = _surface_batch(scene, c2ws, K, Wd, Hd, rng, batch // 2)
        near = ps + rng.normal(0.0, near_sigma, ps.shape) * rng.uniform(0, 1, (len(ps), 1))
        uni = rng.uniform(lo, hi, (batch // 4, 3))
        pts = np.concatenate([ps, near, uni])
        target = scene.sdf(pts)
        x = torch.tensor(pts, dtype=torch.float32, requires_grad=True)
        f, feat = model.sdf_net(x)
        (g,) = torch.autograd.grad(f.sum(), x, create_graph=True)
        tgt = torch.tensor(target, dtype=torch.float32)
        l_sdf = torch.abs(f - tgt).mean()
        l_eik = ((g.norm(dim=1) - 1.0) ** 2).mean()
        ns = len(ps)
        nrm = g[:ns] / g[:ns].norm(dim=1, keepdim=True).clamp_min(1e-6)
        col = model.rgb_net(x[:ns], torch.tensor(vs, dtype=torch.float32), nrm, feat[:ns])
        l_rgb = torch.abs(col - torch.tensor(alb, dtype=torch.float32)).mean()
        loss = l_sdf + 0.1 * l_eik + l_rgb
        opt.zero_grad()
        loss.backward()
        opt.step()
        sched.step()
        if it % log_every == 0 or it == steps - 1:
            print(f"[{name}] it {it} sdf {l_sdf.item():.5f} eik {l_eik.item():.4f} rgb {l_rgb.item():.4f} "
                  f"({time.time() - t_start:.0f}s)", flush=True)
    sdf, rgb = model.export()
    spec.sdf = [(synth.round_bf16(W), synth.round_bf16(b)) for W, b in sdf]
    spec.rgb = [(synth.round_bf16(W), synth.round_bf16(b)) for W, b in rgb]
    os.makedirs(DATA, exist_ok=True)
    out = os.path.join(DATA, f"{name}_mlp.npz")
    synth.save_mlp(spec, out)
    print("wrote", out)
    return spec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("scene", choices=["tiny", "room"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--lr", type=float, default=None)
    a = ap.parse_args()
    if a.scene == "tiny":
        fit("tiny", a.steps or 1500, a.batch or 4096, a.lr or 2e-3)
    else:
        fit("room", a.steps or 4000, a.batch or 8192, a.lr or 5e-4)


if __name__ == "__main__":
    main()
