"""Pins of the oracle's coarse + fine sampler inside the TSDF bound (Tab. 2
"Ours", the supplementary ray study) and of the counts relative to the mean
interval (Sec. 3.4):

* the coarse section weights on a plane (linear SDF) telescope to a closed form;
* counts on dyadic lengths, where every FP32 step is exact, equal the formula
  evaluated by hand, including the clamps and the FALLBACK / MISS rules;
  on random lengths they are monotone in the length and average n_mean + [0, 1);
* with no fine samples the sampler is the TSDF-bounded midpoint render, and with
  the whole [t0, t_end] as its bound and fixed counts it is the hierarchical
  comparator;
* merged samples are sorted, inside the bound, contain the coarse midpoints and
  their widths tile the bound; a single coarse sample takes n_fine midpoints;
* on the sphere scene it converges to the dense render of the same bound;
* the dense reference (no opacity guard) converges in the sample count."""
import dataclasses
import math

import numpy as np
import pytest
import torch

from oracle import cgrid
from oracle import render as orr
from paper_2311_17878_gb300 import synth

DT = torch.float64


def test_coarse_weights_on_a_plane_telescope():
    """f(z) = c (z - z*) with c < 0: every section's slope is c (the first's
    "previous" slope 0 loses the min), so the section ends are the coarse values
    themselves and, with eps = 0, w_j = (Phi(f_j) - Phi(f_{j+1})) / Phi(f_0)."""
    inv_s = 64.0
    phi = lambda v: 1.0 / (1.0 + math.exp(-inv_s * v))
    for n, (lo, hi), c, zs in [(6, (0.5, 1.5), -1.0, 1.07), (17, (0.0, 3.0), -0.4, 2.2), (2, (1.0, 1.2), -2.0, 1.1)]:
        z = torch.tensor([[lo + (j + 0.5) * (hi - lo) / n for j in range(n)]], dtype=DT)
        f = c * (z - zs)
        w = orr.hier_coarse_weights(f, z, inv_s, 0.0)[0].numpy()
        fz = [c * (z[0, j].item() - zs) for j in range(n)]
        expect = [(phi(fz[j]) - phi(fz[j + 1])) / phi(fz[0]) for j in range(n - 1)]
        assert np.max(np.abs(w - np.array(expect))) < 1e-13


def test_adaptive_counts_dyadic_closed_form():
    # BOUNDED lengths 0.5, 1.5, 1.0, 1.0 -> mean 1.0; n_mean 4 -> spacing 0.25 (all exact)
    t_n = np.array([1.0, 2.0, 0.0, 3.0, 5.0, 0.0, 7.0, 2.0], np.float32)
    t_f = np.array([1.5, 3.5, 1.0, 4.0, 9.0, 0.0, 7.0, 2.0], np.float32)
    st = np.array([1, 1, 1, 1, 2, 0, 1, 1], np.uint8)
    # the last two BOUNDED rays have length 0 -> clamped to n_min; they lower the mean
    # to (0.5 + 1.5 + 1 + 1 + 0 + 0) / 6 = 2/3, so use them in a second case
    n, mean = orr.adaptive_counts(t_n[:6], t_f[:6], st[:6], 4.0, 1, 64, 96)
    assert mean == np.float32(1.0)
    assert n.tolist() == [2, 6, 4, 4, 96, 0]
    # clamps: n_max 5 caps the 1.5 m ray, n_min 3 lifts the 0.5 m one
    n, _ = orr.adaptive_counts(t_n[:6], t_f[:6], st[:6], 4.0, 3, 5, 7)
    assert n.tolist() == [3, 5, 4, 4, 7, 0]
    # zero-length BOUNDED rays: mean 4/6 -> rounded to FP32, n = clamp(ceil(0 / dl), n_min) = n_min
    n, mean = orr.adaptive_counts(t_n, t_f, st, 4.0, 2, 64, 96)
    assert mean == np.float32(4.0 / 6.0)
    assert n[6] == 2 and n[7] == 2
    # no BOUNDED ray: mean 0, FALLBACK / MISS rules only
    n, mean = orr.adaptive_counts(t_n[4:6], t_f[4:6], st[4:6], 4.0, 1, 64, 96)
    assert mean == 0.0 and n.tolist() == [96, 0]


def test_adaptive_counts_monotone_and_mean():
    rng = np.random.default_rng(3)
    L = rng.gamma(2.0, 0.4, 20000).astype(np.float32)
    t_n = rng.uniform(0.1, 5.0, L.size).astype(np.float32)
    t_f = (t_n + L).astype(np.float32)
    st = np.ones(L.size, np.uint8)
    n, mean = orr.adaptive_counts(t_n, t_f, st, 6.0, 1, 4096, 96)
    Lf = t_f - t_n
    o = np.argsort(Lf, kind="stable")
    assert np.all(np.diff(n[o]) >= 0)
    assert abs(mean - Lf.astype(np.float64).mean()) <= 1e-6 * mean
    # ceil adds at most one sample to the proportional count L / (mean / 6)
    assert 6.0 <= n.mean() < 7.0


def _tiny_bounds(n=96):
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    sel = synth.sub_sample(len(wl.rays_o), n, seed=4)
    o, d = wl.rays_o[sel], wl.rays_d[sel]
    b = cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")
    return wl, o, d, b


def test_no_fine_samples_is_the_bounded_render():
    wl, o, d, b = _tiny_bounds()
    net = orr.Net(synth.tiny_mlp())
    with torch.no_grad():
        got = orr.render_hier_bounded(net, o, d, b["t_n"], b["t_f"], b["n"], 0)
        ref = orr.render_bounded(net, o, d, b["t_n"], b["t_f"], b["n"])
    live = b["n"] > 0
    for k in ("rgb", "depth", "wsum", "normal"):
        assert torch.allclose(got[k][live], ref[k][live], atol=1e-14, rtol=0)
        assert torch.all(got[k][~live] == 0)


def test_whole_interval_fixed_counts_is_the_comparator():
    wl, o, d, _ = _tiny_bounds()
    net = orr.Net(synth.tiny_mlp())
    t0, te, ok = cgrid.clip_rays(wl.grid, o, d, wl.bounds.t_near, wl.bounds.t_far, "f64")
    o, d, t0, te = o[ok], d[ok], t0[ok], te[ok]
    with torch.no_grad():
        got = orr.render_hier_bounded(net, o, d, t0, te, np.full(len(t0), 16), 8)
        ref = orr.render_hier(net, o, d, t0, te, n_coarse=16, n_fine=8)
    for k in ("rgb", "depth", "wsum", "normal"):
        assert torch.allclose(got[k], ref[k], atol=1e-12, rtol=0)


@pytest.mark.parametrize("n_fine", [1, 8, 32])
def test_merged_samples_structure(n_fine):
    wl, o, d, b = _tiny_bounds()
    net = orr.Net(synth.tiny_mlp())
    rng = np.random.default_rng(n_fine)
    counts = np.where(b["n"] > 0, rng.integers(1, 12, len(b["n"])), 0)
    with torch.no_grad():
        out = orr.render_hier_bounded(net, o, d, b["t_n"], b["t_f"], counts, n_fine)
    for r in range(len(counts)):
        if counts[r] == 0:
            assert out["t"][r] is None and out["wsum"][r] == 0
            continue
        t = out["t"][r].numpy()
        lo, hi = float(b["t_n"][r]), float(b["t_f"][r])
        c = int(counts[r])
        assert len(t) == c + n_fine and np.all(np.diff(t) >= 0)
        assert np.all(t > lo) and np.all(t < hi)
        zc = lo + (np.arange(c) + 0.5) * ((hi - lo) / c)
        assert np.isin(zc, t).all()
        if c == 1:
            zf = lo + (np.arange(n_fine) + 0.5) * ((hi - lo) / n_fine)
            assert np.allclose(np.sort(np.concatenate([zc, zf])), t, atol=0, rtol=0)
        w = orr.section_widths(torch.as_tensor(t[None]), torch.tensor([lo], dtype=DT), torch.tensor([hi], dtype=DT),
                               torch.ones((1, len(t)), dtype=torch.bool))
        assert abs(float(w.sum()) - (hi - lo)) < 1e-12 and torch.all(w >= 0)


def test_converges_to_the_dense_render_of_the_bound():
    """Tiny sphere scene, geometric-init network, no opacity guard: with growing
    coarse and fine counts the sampler converges to the dense midpoint render of
    the same [t_n, t_f] (4096 samples) on the rays that hit inside it."""
    wl, o, d, b = _tiny_bounds(256)
    net = orr.Net(dataclasses.replace(synth.tiny_mlp(), alpha_eps=0.0))
    bd = b["status"] == 1
    o, d = o[bd], d[bd]
    tn, tf = b["t_n"][bd].astype(np.float64), b["t_f"][bd].astype(np.float64)
    with torch.no_grad():
        dense = orr.render_uniform(net, o, d, tn, tf, 4096)
    hit = dense["wsum"].numpy() > 0.5
    assert hit.sum() >= 30
    errs = []
    for n_mean, n_fine in [(4, 4), (8, 16), (32, 32)]:
        n, _ = orr.adaptive_counts(b["t_n"][bd], b["t_f"][bd], b["status"][bd], float(n_mean), 2, 4096, 64)
        with torch.no_grad():
            got = orr.render_hier_bounded(net, o, d, tn, tf, n, n_fine)
        errs.append((np.abs(got["depth"].numpy() - dense["depth"].numpy())[hit].max(),
                     np.abs(got["rgb"].numpy() - dense["rgb"].numpy())[hit].max()))
    assert errs[0][0] > errs[1][0] > errs[2][0] and errs[0][1] > errs[1][1] > errs[2][1]
    assert errs[2][0] < 1.5e-3 and errs[2][1] < 1.5e-3


def test_dense_reference_converges_without_the_guard():
    """R25: the unguarded dense render of the sphere scene changes by < 1e-5 from
    1024 to 8192 samples; with the guard eps every free-space section adds about
    eps of opacity, so a ray that misses everything gathers about n * eps."""
    wl, o, d, b = _tiny_bounds(64)
    net = orr.Net(synth.tiny_mlp())
    t0, te, ok = cgrid.clip_rays(wl.grid, o, d, wl.bounds.t_near, wl.bounds.t_far, "f64")
    o, d, t0, te = o[ok], d[ok], t0[ok], te[ok]
    r1 = orr.dense_reference(net, o, d, t0, te, n=1024)
    r8 = orr.dense_reference(net, o, d, t0, te, n=8192)
    for k in ("rgb", "wsum"):
        assert np.abs(r1[k].numpy() - r8[k].numpy()).max() < 1e-5
    miss = r8["wsum"].numpy() < 1e-3
    assert miss.sum() >= 3
    eps = net.spec.alpha_eps
    with torch.no_grad():
        g = orr.render_uniform(net, o[miss], d[miss], t0[miss], te[miss], 8192)
    assert np.all(np.abs(g["wsum"].numpy() - 8192 * eps) < 0.25 * 8192 * eps)
