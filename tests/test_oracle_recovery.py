"""Pins of the oracle's recovery pass (Sec. 4.5): which rays are rendered again
and what replaces them, on the 64^3 sphere fixture with its fitted networks."""
import numpy as np
import torch

from oracle import cgrid
from oracle import render as orr
from paper_2311_17878_gb300 import synth


def _case(n_rays=192):
    wl = synth.tiny_workload()
    V = synth.analytic_tsdf(wl.scene, wl.grid)
    idx = synth.sub_sample(len(wl.rays_o), n_rays, seed=71)
    o, d = wl.rays_o[idx].astype(np.float64), wl.rays_d[idx].astype(np.float64)
    b = cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")
    t0, te, ok = cgrid.clip_rays(wl.grid, o, d, wl.bounds.t_near, wl.bounds.t_far, "f64")
    return wl, o, d, b, t0, te, ok, orr.Net(synth.scene_mlp("tiny"))


def _render(net, o, d, b, t0, te, tau, status=None):
    return orr.render_recovered(net, o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"],
                                b["status"] if status is None else status, t0, te, tau)


def test_tau_zero_changes_nothing():
    wl, o, d, b, t0, te, ok, net = _case()
    out, again = _render(net, o, d, b, t0, te, 0.0)
    with torch.no_grad():
        ref = orr.render_bounded(net, o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])
    assert not again.any()
    for k in ("rgb", "depth", "wsum", "normal"):
        assert torch.equal(out[k], ref[k])


def test_tau_above_one_rerenders_every_bounded_ray_over_its_clip():
    wl, o, d, b, t0, te, ok, net = _case()
    out, again = _render(net, o, d, b, t0, te, 2.0)
    bounded = b["status"] == 1
    assert bounded.sum() > 20 and np.array_equal(again, bounded)
    with torch.no_grad():
        uni = orr.render_uniform(net, o[bounded], d[bounded], t0[bounded], te[bounded], 96)
        first = orr.render_bounded(net, o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])
    for k in ("rgb", "depth", "wsum", "normal"):
        assert torch.allclose(out[k][torch.as_tensor(bounded)], uni[k], rtol=0, atol=1e-12)
        assert torch.equal(out[k][torch.as_tensor(~bounded)], first[k][torch.as_tensor(~bounded)])


def test_selection_is_the_strict_weight_threshold():
    wl, o, d, b, t0, te, ok, net = _case()
    with torch.no_grad():
        first = orr.render_bounded(net, o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])
    w = first["wsum"].numpy()
    bounded = b["status"] == 1
    tau = float(np.median(w[bounded]))
    _, again = _render(net, o, d, b, t0, te, tau)
    assert np.array_equal(again, bounded & (w < tau))
    assert 0 < again.sum() < bounded.sum()
    # MISS and FALLBACK rays are never selected, whatever their weight
    st = b["status"].copy()
    st[:] = 2
    _, again2 = _render(net, o, d, b, t0, te, 2.0, status=st)
    assert not again2.any()


def test_recovery_finds_the_sphere_behind_a_wrong_interval():
    """Bounds placed in the free space in front of the sphere (what an unseen
    region of the grid does to Alg. 1) leave the weight near 0; recovery
    re-renders over the whole clip and finds the analytic hit."""
    wl, o, d, b, t0, te, ok, net = _case(512)
    bounded = b["status"] == 1
    tn = b["t_n"].astype(np.float64).copy()
    tf = b["t_f"].astype(np.float64).copy()
    wrong = bounded & (tn - t0 > 0.2)
    assert wrong.sum() > 10
    tf[wrong] = tn[wrong] - 0.1           # an interval that ends 10 cm before the near bound
    tn[wrong] = t0[wrong]
    tf[wrong] = np.maximum(tf[wrong], tn[wrong] + 1e-3)
    with torch.no_grad():
        bad = orr.render_bounded(net, o, d, tn, tf, b["n"])
    assert np.all(bad["wsum"].numpy()[wrong] < 0.5)
    out, again = orr.render_recovered(net, o, d, tn, tf, b["n"], b["status"], t0, te, 0.95)
    assert np.all(again[wrong])
    # the sphere r = 0.5 at the origin: analytic entry distance along each unit ray,
    # on the rays that pass well inside its rim (closest approach below 0.45)
    bq = np.sum(o * d, 1)
    disc = bq * bq - (np.sum(o * o, 1) - 0.25)
    t_hit = -bq - np.sqrt(np.maximum(disc, 0.0))
    core = wrong & (disc > 0.25 - 0.45 ** 2)
    assert core.sum() > 10
    dep = out["depth"].numpy()[core]
    assert np.all(np.abs(dep - t_hit[core]) < 0.03)
    assert np.all(out["wsum"].numpy()[core] > 0.9)
