"""Pins of the oracle's render half: SDF / colour networks, NeuS opacity,
compositing (Eq. 1, Eq. 2, rendered normal), the hierarchical comparator
and the training-loss gradient.

Each pin compares with something independent: finite differences, the
composition of affine maps, numpy's sin/cos, the telescoping closed form of
NeuS weights on a plane, invariants of Eq. 1, a brute-force quantile table.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

from oracle import render as orr
from paper_2311_17878_gb300 import synth

DT = torch.float64


def specs():
    return {"tiny": synth.tiny_mlp(), "room": synth.room_mlp()}


@pytest.mark.parametrize("arch", ["tiny", "room"])
def test_forward_mode_gradient_matches_reverse_mode(arch):
    net = orr.Net(specs()[arch])
    x = torch.tensor(np.random.default_rng(1).uniform(-1, 1, (200, 3)) * (0.5 if arch == "tiny" else 3.0), dtype=DT)
    _, g, _ = orr.sdf_forward(net, x)
    gr = orr.sdf_grad_reverse(net, x)
    assert torch.max(torch.abs(g - gr)).item() < 1e-12


@pytest.mark.parametrize("arch", ["tiny", "room"])
def test_gradient_matches_central_differences(arch):
    net = orr.Net(specs()[arch])
    x = torch.tensor(np.random.default_rng(2).uniform(-1, 1, (50, 3)) * (0.4 if arch == "tiny" else 3.0), dtype=DT)
    _, g, _ = orr.sdf_forward(net, x)
    h = 1e-6
    fd = torch.zeros_like(x)
    for a in range(3):
        e = torch.zeros(3, dtype=DT)
        e[a] = h
        fp, _, _ = orr.sdf_forward(net, x + e, with_grad=False)
        fm, _, _ = orr.sdf_forward(net, x - e, with_grad=False)
        fd[:, a] = (fp - fm) / (2 * h)
    assert torch.max(torch.abs(g - fd)).item() < 1e-6 * max(1.0, g.abs().max().item())


def _affine_spec(arch, seed=0):
    """Weights with every hidden pre-activation above 20/beta (the linear branch
    of softplus), so the SDF network is exactly affine in its encoded input."""
    s = specs()[arch]
    rng = np.random.default_rng(seed)
    layers = []
    for i, (W, b) in enumerate(s.sdf):
        W2 = np.abs(rng.normal(0, 0.05, W.shape))
        b2 = np.full(b.shape, 1.0)
        layers.append((W2, b2))
    s.sdf = layers
    return s


@pytest.mark.parametrize("arch", ["tiny", "room"])
def test_linear_regime_equals_composed_affine_map(arch):
    s = _affine_spec(arch)
    net = orr.Net(s)
    rng = np.random.default_rng(4)
    x = rng.uniform(-0.4, 0.4, (30, 3)) if arch == "tiny" else rng.uniform(-3, 3, (30, 3)) + np.array([0, 0, 1.5])
    f, g, feat = orr.sdf_forward(net, torch.tensor(x, dtype=DT))
    # encoded input computed with numpy, in the documented order
    xt = (x - np.asarray(s.center)) / s.scale
    enc = [xt]
    for k in range(s.pe_sdf):
        enc += [np.sin(2.0 ** k * xt), np.cos(2.0 ** k * xt)]
    gam = np.concatenate(enc, 1)
    # compose the affine maps: out = A_h h + c, with the skip splitting the layer
    A = np.eye(gam.shape[1])
    c = np.zeros(gam.shape[1])
    for l, (W, b) in enumerate(s.sdf):
        if l == s.skip_layer:
            A = np.concatenate([A, np.eye(gam.shape[1])], 0) / math.sqrt(2.0)
            c = np.concatenate([c, np.zeros(gam.shape[1])]) / math.sqrt(2.0)
        A = W @ A
        c = W @ c + b
    out = gam @ A.T + c
    assert np.max(np.abs(f.numpy() - s.scale * out[:, 0])) < 1e-9 * max(1, np.abs(out).max())
    assert np.max(np.abs(feat.numpy() - out[:, 1:])) < 1e-9 * max(1, np.abs(out).max())


def test_colour_network_constant_output():
    s = synth.tiny_mlp()
    W, b = s.rgb[-1]
    s.rgb[-1] = (np.zeros_like(W), np.array([0.0, math.log(3.0), -math.log(3.0)]))
    net = orr.Net(s)
    x = torch.zeros((5, 3), dtype=DT)
    c = orr.rgb_forward(net, x, x, x, torch.zeros((5, 16), dtype=DT))
    assert torch.allclose(c, torch.tensor([0.5, 0.75, 0.25], dtype=DT).expand(5, 3), atol=1e-15)


def _colour_numpy(spec, x, v, n_hat, feat):
    """The colour network written out per sample with numpy: the input row assembled
    by hand as (x_tilde, v, sin 2^k v, cos 2^k v for k < L, unit normal, feature),
    ReLU hidden layers, sigmoid output."""
    out = np.zeros((len(x), 3))
    for i in range(len(x)):
        row = list((x[i] - np.asarray(spec.center)) / spec.scale)
        row += list(v[i])
        for k in range(spec.pe_dir):
            row += [math.sin(2.0 ** k * v[i][a]) for a in range(3)]
            row += [math.cos(2.0 ** k * v[i][a]) for a in range(3)]
        row += list(n_hat[i]) + list(feat[i])
        h = np.array(row)
        for l, (W, b) in enumerate(spec.rgb):
            z = np.asarray(W, np.float64).dot(h) + np.asarray(b, np.float64)
            h = np.maximum(z, 0.0) if l + 1 < len(spec.rgb) else 1.0 / (1.0 + np.exp(-z))
        out[i] = h
    return out


def _colour_inputs(spec, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-2.0, 2.0, (n, 3)) + np.asarray(spec.center)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    nh = rng.normal(size=(n, 3))
    nh /= np.linalg.norm(nh, axis=1, keepdims=True)
    feat = rng.normal(0.0, 0.5, (n, spec.n_feat))
    return x, v, nh, feat


def _random_colour_layers(spec, rng, mode):
    """Random colour layers: 'mixed' (about half of the hidden units active), 'active'
    (every hidden unit above zero: non-negative weights on non-negative inputs beyond the
    first layer, unit biases) or 'inactive' (every hidden unit below zero)."""
    layers = []
    for l, (W, b) in enumerate(spec.rgb):
        fan_in = W.shape[1]
        W2 = rng.normal(0.0, 1.0 / math.sqrt(fan_in), W.shape)
        b2 = rng.normal(0.0, 0.1, b.shape)
        hidden = l + 1 < len(spec.rgb)
        if mode == "active" and hidden:
            # first layer: small weights on the signed input and a unit bias; later layers:
            # non-negative weights of mean 1 / fan_in on non-negative inputs
            W2 = np.abs(W2) / (0.8 * math.sqrt(fan_in)) if l > 0 else W2 * 0.05
            b2 = np.full(b.shape, 1.0)
        if mode == "inactive" and hidden:
            b2 = np.full(b.shape, -1e3)
        layers.append((W2, b2))
    return layers


@pytest.mark.parametrize("arch", ["tiny", "room"])
@pytest.mark.parametrize("mode", ["mixed", "active", "inactive"])
def test_colour_network_matches_numpy_matvec(arch, mode):
    """rgb_forward against the per-sample numpy matvec of the documented input row, on
    random weights; with every hidden unit active the network is the sigmoid of the
    composed affine map, with every hidden unit inactive the sigmoid of the output bias."""
    s = specs()[arch]
    rng = np.random.default_rng({"mixed": 11, "active": 12, "inactive": 13}[mode])
    s.rgb = _random_colour_layers(s, rng, mode)
    net = orr.Net(s)
    x, v, nh, feat = _colour_inputs(s, 24, seed=14)
    got = orr.rgb_forward(net, torch.tensor(x, dtype=DT), torch.tensor(v, dtype=DT), torch.tensor(nh, dtype=DT),
                          torch.tensor(feat, dtype=DT)).numpy()
    want = _colour_numpy(s, x, v, nh, feat)
    assert np.max(np.abs(got - want)) < 1e-13
    if mode == "inactive":
        b_last = np.asarray(s.rgb[-1][1], np.float64)
        assert np.max(np.abs(got - 1.0 / (1.0 + np.exp(-b_last)))) < 1e-15
    if mode == "active":
        # composed affine map of the input row: no unit may be clipped
        rows = np.stack([np.concatenate([(x[i] - np.asarray(s.center)) / s.scale, v[i]] +
                                        [f(2.0 ** k * v[i]) for k in range(s.pe_dir) for f in (np.sin, np.cos)] +
                                        [nh[i], feat[i]]) for i in range(len(x))])
        A, c = np.eye(rows.shape[1]), np.zeros(rows.shape[1])
        for W, b in s.rgb:
            A, c = np.asarray(W) @ A, np.asarray(W) @ c + np.asarray(b)
        assert np.max(np.abs(got - 1.0 / (1.0 + np.exp(-(rows @ A.T + c))))) < 1e-12
    if mode == "mixed":
        # the hidden layers really are mixed: each first-layer unit is active on some
        # samples and inactive on others, so a wrong activation would show
        z0 = np.stack([np.asarray(s.rgb[0][0]) @ np.concatenate(
            [(x[i] - np.asarray(s.center)) / s.scale, v[i]] +
            [f(2.0 ** k * v[i]) for k in range(s.pe_dir) for f in (np.sin, np.cos)] + [nh[i], feat[i]])
            for i in range(len(x))]) + np.asarray(s.rgb[0][1])
        frac = float((z0 > 0).mean())
        assert 0.3 < frac < 0.7


@pytest.mark.parametrize("arch", ["tiny", "room"])
def test_colour_network_reads_each_input_part(arch):
    """Changing any one part of the input row (position, direction, normal, feature)
    changes the colour exactly as the numpy matvec says, so no part is dropped or
    exchanged with another (the direction is encoded, not the position)."""
    s = specs()[arch]
    s.rgb = _random_colour_layers(s, np.random.default_rng(15), "mixed")
    net = orr.Net(s)
    x, v, nh, feat = _colour_inputs(s, 8, seed=16)
    rng = np.random.default_rng(17)
    for part in range(4):
        args = [a.copy() for a in (x, v, nh, feat)]
        args[part] = args[part] + rng.normal(0.0, s.scale if part == 0 else 0.3, args[part].shape)
        got = orr.rgb_forward(net, *[torch.tensor(a, dtype=DT) for a in args]).numpy()
        want = _colour_numpy(s, *args)
        base = _colour_numpy(s, x, v, nh, feat)
        assert np.max(np.abs(got - want)) < 1e-13
        assert np.max(np.abs(want - base)) > 1e-4


def test_plane_weights_telescoping_closed_form():
    """For f(t) = f0 + c t (c < 0) the section ends are exact, and with eps = 0
    T_i = Phi(f(b_i)) / Phi(f(b_0)), so sum w = 1 - Phi(f(b_n)) / Phi(f(b_0))."""
    inv_s = 64.0
    for n, (lo, hi) in [(1, (0.9, 1.1)), (7, (0.5, 1.4)), (96, (0.0, 3.0))]:
        t = torch.tensor([[lo + (i + 0.5) * (hi - lo) / n for i in range(n)]], dtype=DT)
        delta = torch.full_like(t, (hi - lo) / n)
        c = -0.8
        t_star = 1.05
        f = c * (t - t_star)
        dd = torch.full_like(t, c)
        alpha = orr.neus_alpha(f, dd, delta, inv_s, 0.0)
        mask = torch.ones_like(t, dtype=torch.bool)
        out = orr.composite(alpha, t, torch.zeros(1, n, 3, dtype=DT), torch.zeros(1, n, 3, dtype=DT), mask)
        phi = lambda v: 1.0 / (1.0 + math.exp(-inv_s * v))
        expect = 1.0 - phi(c * (hi - t_star)) / phi(c * (lo - t_star))
        assert abs(out["wsum"].item() - expect) < 1e-12
        b = [lo + i * (hi - lo) / n for i in range(n + 1)]
        w_exp = [(phi(c * (b[i] - t_star)) - phi(c * (b[i + 1] - t_star))) / phi(c * (b[0] - t_star)) for i in range(n)]
        assert np.max(np.abs(out["w"][0].numpy() - np.array(w_exp))) < 1e-12


def test_plane_depth_converges_to_hit():
    """Dense sampling over a wide interval: the NeuS weight density is a
    logistic centred on the zero crossing, so the depth converges to t*."""
    n, lo, hi = 4096, 0.0, 3.0
    t = torch.tensor([[lo + (i + 0.5) * (hi - lo) / n for i in range(n)]], dtype=DT)
    delta = torch.full_like(t, (hi - lo) / n)
    for c, t_star in [(-1.0, 1.3), (-0.5, 1.7)]:
        f = c * (t - t_star)
        alpha = orr.neus_alpha(f, torch.full_like(t, c), delta, 64.0, 0.0)
        out = orr.composite(alpha, t, torch.zeros(1, n, 3, dtype=DT), torch.zeros(1, n, 3, dtype=DT),
                            torch.ones_like(t, dtype=torch.bool))
        assert abs(out["depth"].item() - t_star) < 1e-5
        assert abs(out["wsum"].item() - 1.0) < 1e-12


def test_composite_invariants_and_special_cases():
    rng = np.random.default_rng(7)
    R, S = 40, 33
    counts = rng.integers(1, S + 1, R)
    mask = torch.arange(S).unsqueeze(0) < torch.tensor(counts).unsqueeze(1)
    alpha = torch.tensor(rng.uniform(0, 1, (R, S)) ** 3, dtype=DT)
    t = torch.tensor(np.sort(rng.uniform(0, 5, (R, S)), 1), dtype=DT)
    col = torch.tensor(rng.uniform(0, 1, (R, S, 3)), dtype=DT)
    nh = torch.tensor(rng.normal(size=(R, S, 3)), dtype=DT)
    out = orr.composite(alpha, t, col, nh, mask)
    w = out["w"]
    assert torch.all(w >= 0) and torch.all(out["wsum"] <= 1 + 1e-15)
    assert torch.all(w[~mask] == 0)
    # transmittance non-increasing
    T = torch.where(alpha > 0, w / alpha, torch.ones_like(w))
    a = alpha.numpy()
    Tn = np.cumprod(np.concatenate([np.ones((R, 1)), 1 - np.where(mask.numpy(), np.minimum(a, 1 - 2 ** -24), 0)[:, :-1]], 1), 1)
    assert np.all(np.diff(Tn, axis=1) <= 1e-15)
    assert np.allclose(w.numpy(), Tn * np.where(mask.numpy(), a, 0), atol=1e-14)
    # constant colour k: rgb = k * sum w
    k = torch.tensor([0.2, 0.5, 0.9], dtype=DT)
    out2 = orr.composite(alpha, t, k.expand(R, S, 3), nh, mask)
    assert torch.allclose(out2["rgb"], out2["wsum"].unsqueeze(1) * k, atol=1e-14)
    # n = 1: w = alpha
    one = orr.composite(alpha[:, :1], t[:, :1], col[:, :1], nh[:, :1], torch.ones((R, 1), dtype=torch.bool))
    assert torch.allclose(one["w"][:, 0], alpha[:, 0], atol=0)


def test_inverse_cdf_matches_quantile_table():
    """The inverse of the piecewise-linear CDF, against (a) numpy's linear
    interpolation of the (cdf, z) knots and (b) a brute-force fine-grid
    integration of the piecewise-constant density."""
    rng = np.random.default_rng(9)
    R, B = 6, 63
    z = np.arange(B + 1) * 0.0625 + rng.uniform(0, 0.03, (R, B + 1))
    w = rng.uniform(0, 1, (R, B)) ** 4
    s = orr.inverse_cdf(torch.tensor(z, dtype=DT), torch.tensor(w, dtype=DT), 32).numpy()
    ww = w + 1e-5
    u = (np.arange(32) + 0.5) / 32
    for r in range(R):
        cdf = np.concatenate([[0], np.cumsum(ww[r] / ww[r].sum())])
        assert np.max(np.abs(np.interp(u, cdf, z[r]) - s[r])) < 1e-12
        grid = np.linspace(z[r, 0], z[r, -1], 400001)
        mid = 0.5 * (grid[1:] + grid[:-1])
        j = np.clip(np.searchsorted(z[r], mid, side="right") - 1, 0, B - 1)
        dens = ww[r, j] / (z[r, j + 1] - z[r, j]) / ww[r].sum()
        cg = np.concatenate([[0], np.cumsum(dens * np.diff(grid))])
        # the brute-force CDF at the returned samples equals the requested quantiles
        assert np.max(np.abs(np.interp(s[r], grid, cg) - u)) < 1e-4  # one grid cell of mass


@pytest.mark.parametrize("n_coarse,n_fine", [(64, 32), (16, 8), (2, 1)])
def test_hier_samples_sorted_in_range_and_complete(n_coarse, n_fine):
    wl = synth.tiny_workload()
    net = orr.Net(synth.tiny_mlp())
    o, d = wl.rays_o[1000:1040], wl.rays_d[1000:1040]
    t0 = np.full(40, 1.0)
    te = np.full(40, 3.0)
    out = orr.render_hier(net, o, d, t0, te, n_coarse=n_coarse, n_fine=n_fine)
    t = out["t"].numpy()
    assert t.shape == (40, n_coarse + n_fine)
    # the coarse midpoints are all among the samples
    zc = 1.0 + (np.arange(n_coarse) + 0.5) * (2.0 / n_coarse)
    assert all(np.isin(zc, t[r]).all() for r in range(40))
    assert np.all(np.diff(t, axis=1) >= 0) and np.all(t > 1.0) and np.all(t < 3.0)
    assert torch.all(out["w"] >= 0) and torch.all(out["wsum"] <= 1 + 1e-12)


def test_midpoint_section_widths_are_uniform():
    t, dl, mask = orr.midpoint_samples([1.0, 2.0], [2.0, 2.5], [4, 3])
    w = orr.section_widths(t, torch.tensor([1.0, 2.0], dtype=DT), torch.tensor([2.0, 2.5], dtype=DT), mask)
    assert torch.allclose(w[mask], dl[mask], atol=1e-15)
    assert torch.allclose(t[0], torch.tensor([1.125, 1.375, 1.625, 1.875], dtype=DT))


@pytest.mark.parametrize("opacity", [orr.OPACITY_NEUS, orr.OPACITY_VOLSDF])
def test_training_loss_gradient_matches_central_differences(opacity):
    """Reverse-mode gradient of L1 colour + 0.1 eikonal (through grad f in the
    opacity, the colour-network normal and the eikonal term) against FP64
    central differences, h = 1e-6, on 64 rays; NeuS and VolSDF opacity."""
    wl = synth.tiny_workload()
    spec = dataclasses.replace(synth.tiny_mlp(), opacity=opacity)
    rng = np.random.default_rng(12)
    idx = rng.choice(4096, 64, replace=False)
    o, d = wl.rays_o[idx], wl.rays_d[idx]
    t_n = np.full(64, 1.35)
    t_f = np.full(64, 1.9)
    counts = rng.integers(3, 12, 64)
    status = np.ones(64, np.uint8)
    target = rng.uniform(0, 1, (64, 3))
    net = orr.Net(spec, requires_grad=True)
    loss, _ = orr.train_loss(net, o, d, t_n, t_f, counts, status, target)
    gs = orr.grads(net, loss)
    h = 1e-6
    checked = 0
    for pi, (p, g) in enumerate(zip(net.params(), gs)):
        flat = p.detach().reshape(-1)
        for e in rng.choice(flat.numel(), min(4, flat.numel()), replace=False):
            with torch.no_grad():
                old = flat[e].item()
                p.view(-1)[e] = old + h
                lp, _ = orr.train_loss(net, o, d, t_n, t_f, counts, status, target)
                p.view(-1)[e] = old - h
                lm, _ = orr.train_loss(net, o, d, t_n, t_f, counts, status, target)
                p.view(-1)[e] = old
            fd = (lp.item() - lm.item()) / (2 * h)
            an = g.reshape(-1)[e].item()
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(an), (pi, e, fd, an)
            checked += 1
    assert checked >= 20
