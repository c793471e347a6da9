"""CPU oracle for the render half of TSDF-Sampling: sample placement, the SDF and
colour MLPs with the analytic SDF gradient, NeuS opacity and volume-rendering
compositing (Eq. 1, Eq. 2, the rendered normal of Sec. C.1), the 64+32
hierarchical comparator and the same sampler inside the TSDF bound, counts
relative to the mean interval, the dense reference render and the training loss.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain PyTorch CPU ops in float64.  The SDF gradient is carried by explicit
forward-mode tangents (one tangent per input axis); reverse-mode autograd
of the same network is kept as a cross-check (:func:`sdf_grad_reverse`).
Parameter gradients of the training loss come from autograd through the
explicit forward computation.

Readings taken here (numbered as in the design notes):
  R12 midpoint placement t_i = t_n + (i + 1/2) (t_f - t_n) / n, no jitter;
  R13 softplus_beta(z) = log(1 + exp(beta z)) / beta, and z itself when
      beta z > 20 (derivative 1 there);
  R14 positional encoding (x, sin(2^k x), cos(2^k x)), k = 0..L-1, of
      x_tilde = (x - center) / scale; the SDF in world units is scale * net_0;
  R15 the skip layer's input is concat(h, gamma(x_tilde)) / sqrt(2);
  R16 NeuS opacity with section ends f -/+ (1/2) Delta min(v . grad f, 0),
      alpha = clamp((Phi(f-) - Phi(f+) + eps) / (Phi(f-) + eps), 0, 1),
      Phi(x) = sigmoid(inv_s x);
  R17 black background; R18 depth and normal are 0 when sum w < 1e-8;
  R19 hierarchical comparator as in :func:`render_hier`;
  R21 section widths: boundaries at the interval ends and halfway between
      neighbouring samples (equal to (t_f - t_n)/n for midpoint placement);
  R23 coarse + fine inside the TSDF bound as in :func:`render_hier_bounded`;
  R24 counts relative to the mean interval as in :func:`adaptive_counts`;
  R25 the dense reference image is rendered without the opacity guard;
  R26 VolSDF opacity: alpha = 1 - exp(-sigma delta) with sigma(f) = a Psi(-f),
      Psi the Laplace CDF of scale 1/a (a = inv_s); the comparator's section
      opacity uses the density at the section's mid value.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64
OPACITY_NEUS, OPACITY_VOLSDF = 0, 1   # the network's SDF-to-opacity transform (R16 / R26)
LOG_T_CLAMP = 1.0 - 2.0 ** -24
WSUM_MIN = 1e-8


# ----------------------------------------------------------------------------
# network parameters
# ----------------------------------------------------------------------------
class Net:
    """The SDF and colour networks of an :class:`MLPSpec`, as float64 tensors."""

    def __init__(self, spec, requires_grad=False):
        self.spec = spec
        self.sdf = [(torch.tensor(np.asarray(W), dtype=DT, requires_grad=requires_grad),
                     torch.tensor(np.asarray(b), dtype=DT, requires_grad=requires_grad)) for W, b in spec.sdf]
        self.rgb = [(torch.tensor(np.asarray(W), dtype=DT, requires_grad=requires_grad),
                     torch.tensor(np.asarray(b), dtype=DT, requires_grad=requires_grad)) for W, b in spec.rgb]

    def params(self):
        return [p for W, b in self.sdf + self.rgb for p in (W, b)]


def softplus(z, beta):
    """R13: log(1 + exp(beta z)) / beta, linear for beta z > 20."""
    bz = beta * z
    return torch.where(bz > 20.0, z, torch.log1p(torch.exp(torch.clamp(bz, max=20.0))) / beta)


def softplus_slope(z, beta):
    """d softplus_beta / dz = sigmoid(beta z), and 1 on the linear branch."""
    bz = beta * z
    return torch.where(bz > 20.0, torch.ones_like(z), torch.sigmoid(bz))


def encode(x, octaves):
    """gamma(x) = (x, sin(2^0 x), cos(2^0 x), ..., sin(2^{L-1} x), cos(2^{L-1} x))
    and its Jacobian as tangents (N, 3, E): entry [n, a, e] = d gamma_e / d x_a."""
    N = x.shape[0]
    parts = [x]
    eye = torch.eye(3, dtype=x.dtype).expand(N, 3, 3)
    jac = [eye]
    for k in range(octaves):
        f = 2.0 ** k
        s, c = torch.sin(f * x), torch.cos(f * x)
        parts += [s, c]
        jac += [torch.diag_embed(f * c), torch.diag_embed(-f * s)]
    return torch.cat(parts, 1), torch.cat(jac, 2)


def normalise_points(spec, x):
    return (x - torch.tensor(spec.center, dtype=x.dtype)) / spec.scale


def sdf_forward(net, x, with_grad=True):
    """SDF network at world points x (N, 3).

    Returns f (N,) in world units, grad_x f (N, 3) (forward-mode tangents) and
    the feature vector (N, F).  Hidden layers use softplus_beta; the output
    layer is linear; row 0 of the output is the SDF, the rest the feature.
    """
    spec = net.spec
    xt = normalise_points(spec, x)
    g, jg = encode(xt, spec.pe_sdf)
    h, dh = g, jg
    last = len(net.sdf) - 1
    for l, (W, b) in enumerate(net.sdf):
        if l == spec.skip_layer:
            h = torch.cat([h, g], 1) / math.sqrt(2.0)
            dh = torch.cat([dh, jg], 2) / math.sqrt(2.0)
        z = h @ W.T + b
        dz = dh @ W.T if with_grad else None
        if l < last:
            h = softplus(z, spec.beta)
            if with_grad:
                dh = softplus_slope(z, spec.beta).unsqueeze(1) * dz
        else:
            h, dh = z, dz
    f = spec.scale * h[:, 0]
    grad = dh[:, :, 0] if with_grad else None      # d(scale net_0)/dx = d net_0 / d x_tilde
    return f, grad, h[:, 1:]


def sdf_grad_reverse(net, x):
    """Cross-check of the forward-mode gradient: reverse-mode autograd of f."""
    x = x.detach().clone().requires_grad_(True)
    f, _, _ = sdf_forward(net, x, with_grad=False)
    (g,) = torch.autograd.grad(f.sum(), x)
    return g


def rgb_forward(net, x, v, n_hat, feat):
    """Colour network: input (x_tilde, dir encoding, unit normal, feature),
    ReLU hidden layers, sigmoid output."""
    spec = net.spec
    xt = normalise_points(spec, x)
    venc = encode(v, spec.pe_dir)[0] if spec.pe_dir > 0 else v
    h = torch.cat([xt, venc, n_hat, feat], 1)
    last = len(net.rgb) - 1
    for l, (W, b) in enumerate(net.rgb):
        z = h @ W.T + b
        h = torch.relu(z) if l < last else torch.sigmoid(z)
    return h


def eval_samples(net, x, v):
    """All per-sample quantities: f, grad f, v.grad f, unit normal, colour."""
    f, g, feat = sdf_forward(net, x)
    gn = torch.linalg.norm(g, dim=1, keepdim=True)
    n_hat = g / gn
    rgb = rgb_forward(net, x, v, n_hat, feat)
    return dict(f=f, grad=g, dd=(g * v).sum(1), n_hat=n_hat, rgb=rgb, gnorm=gn[:, 0])


# ----------------------------------------------------------------------------
# NeuS opacity + compositing (Eq. 1, Eq. 2, rendered normal)
# ----------------------------------------------------------------------------
def neus_alpha(f, dd, delta, inv_s, eps):
    """R16: discrete NeuS opacity of a section of width delta around the sample."""
    c = torch.clamp(dd, max=0.0)
    f_lo = f - 0.5 * delta * c
    f_hi = f + 0.5 * delta * c
    p_lo = torch.sigmoid(inv_s * f_lo)
    p_hi = torch.sigmoid(inv_s * f_hi)
    if eps == 0.0:  # no guard: a section whose near end underflows to Phi = 0 lies deep inside, opaque
        ratio = torch.where(p_lo > 0, (p_lo - p_hi) / torch.where(p_lo > 0, p_lo, 1.0), torch.ones_like(p_lo))
        return torch.clamp(ratio, 0.0, 1.0)
    return torch.clamp((p_lo - p_hi + eps) / (p_lo + eps), 0.0, 1.0)


def volsdf_density(f, a):
    """R26: VolSDF / MonoSDF density sigma(f) = a Psi(-f), Psi the CDF of the zero-mean
    Laplace law of scale 1/a."""
    return a * torch.where(f >= 0, 0.5 * torch.exp(-a * f), 1.0 - 0.5 * torch.exp(a * f))


def volsdf_alpha(f, delta, a):
    """Eq. 1 as printed: alpha = 1 - exp(-sigma delta)."""
    return -torch.expm1(-volsdf_density(f, a) * delta)


def section_alpha(spec, f, dd, delta, eps=None):
    """Opacity of the section of width delta around a sample, by the network's transform."""
    if getattr(spec, "opacity", OPACITY_NEUS) == OPACITY_VOLSDF:
        return volsdf_alpha(f, delta, spec.inv_s)
    return neus_alpha(f, dd, delta, spec.inv_s, spec.alpha_eps if eps is None else eps)


def composite(alpha, t, rgb, n_hat, mask):
    """Eq. 1/2 on padded (R, S) arrays; mask marks real samples.

    log T_0 = 0, log T_{i+1} = log T_i + log1p(-min(alpha_i, 1 - 2^-24)),
    w_i = exp(log T_i) alpha_i; colour = sum w c; depth = sum w t / sum w;
    normal = sum w n / sum w (0 when sum w < 1e-8).
    """
    alpha = torch.where(mask, alpha, torch.zeros_like(alpha))
    lt = torch.log1p(-torch.clamp(alpha, max=LOG_T_CLAMP))
    logT = torch.cat([torch.zeros_like(lt[:, :1]), torch.cumsum(lt[:, :-1], 1)], 1)
    w = torch.exp(logT) * alpha
    wsum = w.sum(1)
    ok = wsum >= WSUM_MIN
    safe = torch.where(ok, wsum, torch.ones_like(wsum))
    color = (w.unsqueeze(2) * rgb).sum(1)
    depth = torch.where(ok, (w * t).sum(1) / safe, torch.zeros_like(wsum))
    normal = torch.where(ok.unsqueeze(1), (w.unsqueeze(2) * n_hat).sum(1) / safe.unsqueeze(1), torch.zeros_like(color))
    return dict(rgb=color, depth=depth, wsum=wsum, normal=normal, w=w)


def section_widths(t, lo, hi, mask):
    """R21: boundaries b_0 = lo, b_i = (t_{i-1} + t_i)/2, b_n = hi; widths b_{i+1} - b_i."""
    R, S = t.shape
    counts = mask.sum(1)
    prev = torch.cat([lo.unsqueeze(1), t[:, :-1]], 1)
    b_lo = torch.where(torch.arange(S).unsqueeze(0) == 0, lo.unsqueeze(1), 0.5 * (prev + t))
    nxt = torch.cat([t[:, 1:], hi.unsqueeze(1)], 1)
    is_last = torch.arange(S).unsqueeze(0) == (counts - 1).unsqueeze(1)
    b_hi = torch.where(is_last, hi.unsqueeze(1), 0.5 * (t + nxt))
    return torch.where(mask, b_hi - b_lo, torch.zeros_like(t))


def _padded(counts):
    counts = torch.as_tensor(np.asarray(counts), dtype=torch.int64)
    S = int(counts.max()) if len(counts) else 0
    S = max(S, 1)
    mask = torch.arange(S).unsqueeze(0) < counts.unsqueeze(1)
    return counts, S, mask


def render_samples(net, o, d, t, delta, mask, eps=None):
    """Evaluate and composite padded samples t (R, S) with widths delta (opacity
    guard eps: the network's own unless given)."""
    R, S = t.shape
    x = o.unsqueeze(1) + t.unsqueeze(2) * d.unsqueeze(1)
    sel = mask.reshape(-1)
    xs = x.reshape(-1, 3)[sel]
    vs = d.unsqueeze(1).expand(R, S, 3).reshape(-1, 3)[sel]
    ev = eval_samples(net, xs, vs)
    spec = net.spec

    def scatter(val, fill=0.0):
        shape = (R * S,) + tuple(val.shape[1:])
        out = torch.full(shape, fill, dtype=val.dtype)
        out = out.index_put((torch.nonzero(sel)[:, 0],), val)
        return out.reshape((R, S) + tuple(val.shape[1:]))

    f = scatter(ev["f"], 1.0)
    dd = scatter(ev["dd"])
    rgb = scatter(ev["rgb"])
    nh = scatter(ev["n_hat"])
    alpha = section_alpha(spec, f, dd, delta, eps)
    out = composite(alpha, t, rgb, nh, mask)
    out["alpha"] = alpha
    out["eik"] = (ev["gnorm"] - 1.0) ** 2
    out["sample_mask"] = sel
    return out


def midpoint_samples(t_n, t_f, counts):
    """R12: t_i = t_n + (i + 1/2) * (t_f - t_n) / n (Sec. 3.4: equal spacing)."""
    counts, S, mask = _padded(counts)
    t_n = torch.as_tensor(np.asarray(t_n), dtype=DT)
    t_f = torch.as_tensor(np.asarray(t_f), dtype=DT)
    n = torch.clamp(counts, min=1).to(DT)
    delta = (t_f - t_n) / n
    i = torch.arange(S, dtype=DT).unsqueeze(0)
    t = t_n.unsqueeze(1) + (i + 0.5) * delta.unsqueeze(1)
    t = torch.where(mask, t, torch.zeros_like(t))
    dl = torch.where(mask, delta.unsqueeze(1).expand_as(t), torch.zeros_like(t))
    return t, dl, mask


def render_bounded(net, rays_o, rays_d, t_n, t_f, counts, eps=None):
    """The TSDF-bounded render: n_r midpoint samples in [t_n, t_f] per ray
    (Sec. 3.3-3.4), evaluated and composited (Eq. 1, Eq. 2, normal)."""
    o = torch.as_tensor(np.asarray(rays_o), dtype=DT)
    d = torch.as_tensor(np.asarray(rays_d), dtype=DT)
    t, dl, mask = midpoint_samples(t_n, t_f, counts)
    return render_samples(net, o, d, t, dl, mask, eps)


STATUS_BOUNDED = 1   # ray status written by the bounds pass: 0 MISS, 1 BOUNDED, 2 FALLBACK
STATUS_FALLBACK = 2


def render_recovered(net, rays_o, rays_d, t_n, t_f, counts, status, t0, t_end, tau, n_fallback=96):
    """Sec. 4.5 (threshold tau of Tab. 5): render the TSDF-bounded samples; every
    BOUNDED ray whose accumulated weight stays below tau is rendered again with
    n_fallback midpoints over its whole [t0, t_end], and that render replaces the
    first.  Returns (merged outputs, boolean mask of the re-rendered rays)."""
    with torch.no_grad():
        first = render_bounded(net, rays_o, rays_d, t_n, t_f, counts)
    status = np.asarray(status)
    again = (status == STATUS_BOUNDED) & (first["wsum"].numpy() < tau)
    out = {k: first[k].clone() for k in ("rgb", "depth", "wsum", "normal")}
    if again.any():
        with torch.no_grad():
            second = render_uniform(net, np.asarray(rays_o)[again], np.asarray(rays_d)[again],
                                    np.asarray(t0)[again], np.asarray(t_end)[again], n_fallback)
        idx = torch.as_tensor(np.nonzero(again)[0])
        for k in out:
            out[k][idx] = second[k]
    return out, again


def render_uniform(net, rays_o, rays_d, t0, t_end, n, eps=None):
    """n midpoint samples over [t0, t_end] (the fallback and the dense reference)."""
    return render_bounded(net, rays_o, rays_d, t0, t_end, np.full(len(np.asarray(t0)), n, np.int64), eps)


def dense_reference(net, rays_o, rays_d, t0, t_end, n=2048, chunk=64):
    """The reference image: n midpoint samples over the whole [t0, t_end], without
    the opacity guard (R25): the guard gives every free-space section an opacity
    of about eps, which over n samples adds up to n * eps (1 % at n = 1024), so
    only the unguarded sum converges to the continuous render as n grows."""
    outs = []
    N = len(np.asarray(t0))
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        with torch.no_grad():
            r = render_uniform(net, np.asarray(rays_o)[s:e], np.asarray(rays_d)[s:e],
                               np.asarray(t0)[s:e], np.asarray(t_end)[s:e], n, eps=0.0)
        outs.append({k: r[k] for k in ("rgb", "depth", "wsum", "normal")})
    return {k: torch.cat([o[k] for o in outs]) for k in outs[0]}


# ----------------------------------------------------------------------------
# 64 + 32 hierarchical comparator (R19)
# ----------------------------------------------------------------------------
def hier_coarse_weights(f, z, inv_s, eps, opacity=0):
    """Weights of the sections between consecutive coarse samples, from SDF
    values only: mid value, slope (f_{j+1} - f_j)/(z_{j+1} - z_j), slope taken as
    min(own, previous) (previous of the first = 0), clipped to [-1e3, 0];
    opacity as R16 with the section's ends (NeuS), or the density at the mid
    value over the section (VolSDF, R26); w = alpha * prod (1 - alpha)."""
    mid = 0.5 * (f[:, 1:] + f[:, :-1])
    dz = z[:, 1:] - z[:, :-1]
    if opacity == OPACITY_VOLSDF:
        alpha = volsdf_alpha(mid, dz, inv_s)
        T = torch.cumprod(torch.cat([torch.ones_like(alpha[:, :1]), 1.0 - alpha[:, :-1]], 1), 1)
        return alpha * T
    slope = (f[:, 1:] - f[:, :-1]) / dz
    prev = torch.cat([torch.zeros_like(slope[:, :1]), slope[:, :-1]], 1)
    c = torch.clamp(torch.minimum(slope, prev), -1e3, 0.0)
    f_lo = mid - 0.5 * c * dz
    f_hi = mid + 0.5 * c * dz
    p_lo, p_hi = torch.sigmoid(inv_s * f_lo), torch.sigmoid(inv_s * f_hi)
    alpha = torch.clamp((p_lo - p_hi + eps) / (p_lo + eps), 0.0, 1.0)
    T = torch.cumprod(torch.cat([torch.ones_like(alpha[:, :1]), 1.0 - alpha[:, :-1]], 1), 1)
    return alpha * T


def inverse_cdf(z, w, n_fine, pdf_floor=1e-5):
    """Deterministic inverse-transform samples u_k = (k + 1/2)/n_fine over the
    bins [z_j, z_{j+1}] with pdf proportional to w_j + pdf_floor, linear within a bin."""
    pdf = w + pdf_floor
    pdf = pdf / pdf.sum(1, keepdim=True)
    cdf = torch.cat([torch.zeros_like(pdf[:, :1]), torch.cumsum(pdf, 1)], 1)
    u = (torch.arange(n_fine, dtype=z.dtype) + 0.5) / n_fine
    u = u.unsqueeze(0).expand(z.shape[0], n_fine).contiguous()
    j = torch.searchsorted(cdf, u, right=True) - 1
    j = torch.clamp(j, 0, pdf.shape[1] - 1)
    c0 = torch.gather(cdf, 1, j)
    p = torch.gather(pdf, 1, j)
    z0 = torch.gather(z, 1, j)
    z1 = torch.gather(z, 1, j + 1)
    return z0 + (u - c0) / p * (z1 - z0)


def render_hier(net, rays_o, rays_d, t0, t_end, n_coarse=64, n_fine=32):
    """Hierarchical render over [t0, t_end]: n_coarse midpoints, n_fine inverse-CDF samples
    (64 + 32 is the comparator of Tab. 2)."""
    spec = net.spec
    o = torch.as_tensor(np.asarray(rays_o), dtype=DT)
    d = torch.as_tensor(np.asarray(rays_d), dtype=DT)
    t0 = torch.as_tensor(np.asarray(t0), dtype=DT)
    te = torch.as_tensor(np.asarray(t_end), dtype=DT)
    R = o.shape[0]
    i = torch.arange(n_coarse, dtype=DT).unsqueeze(0)
    zc = t0.unsqueeze(1) + (i + 0.5) * ((te - t0) / n_coarse).unsqueeze(1)
    xc = (o.unsqueeze(1) + zc.unsqueeze(2) * d.unsqueeze(1)).reshape(-1, 3)
    fc, _, _ = sdf_forward(net, xc, with_grad=False)
    w = hier_coarse_weights(fc.reshape(R, n_coarse), zc, spec.inv_s, spec.alpha_eps, spec.opacity)
    zf = inverse_cdf(zc, w, n_fine)
    t, _ = torch.sort(torch.cat([zc, zf], 1), 1)
    mask = torch.ones_like(t, dtype=torch.bool)
    dl = section_widths(t, t0, te, mask)
    out = render_samples(net, o, d, t, dl, mask)
    out["t"] = t
    return out


# ----------------------------------------------------------------------------
# coarse + fine inside the TSDF bound (R23) and counts relative to the mean (R24)
# ----------------------------------------------------------------------------
def adaptive_counts(t_n, t_f, status, n_mean, n_min, n_max, n_fallback):
    """R24 (Sec. 3.4: equal spacing, so a count proportional to the interval's
    length; the supplementary ray study scales it against the average bound).
    In FP32 as the library states it: L = t_f - t_n, mean = the FP64 mean of L
    over the BOUNDED rays rounded to FP32 (0 with none), dl = mean / n_mean,
    n = clamp(ceil(L / dl), n_min, n_max) (n_min when dl = 0 or L / dl is NaN);
    FALLBACK rays n_fallback, MISS rays 0.  Returns (counts int32, mean float32)."""
    t_n = np.asarray(t_n, np.float32)
    t_f = np.asarray(t_f, np.float32)
    status = np.asarray(status)
    L = np.subtract(t_f, t_n, dtype=np.float32)
    bnd = status == STATUS_BOUNDED
    mean = np.float32(np.mean(L[bnd].astype(np.float64))) if bnd.any() else np.float32(0.0)
    dl = np.float32(mean / np.float32(n_mean))
    n = np.zeros(len(L), np.int32)
    if dl > 0:
        with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
            q = np.ceil(np.divide(L, dl, dtype=np.float32))
        q = np.where(np.isnan(q), n_min, np.clip(q, n_min, n_max))
    else:
        q = np.full(len(L), n_min, np.float32)
    n[bnd] = q[bnd].astype(np.int32)
    n[status == STATUS_FALLBACK] = n_fallback
    return n, mean


def render_hier_bounded(net, rays_o, rays_d, t_n, t_f, counts, n_fine):
    """R23 (Tab. 2 "Ours", the supplementary ray study): the hierarchical sampler
    inside each ray's [t_n, t_f].  counts[r] coarse midpoints of [t_n, t_f],
    SDF values only; section weights as :func:`hier_coarse_weights`; n_fine
    inverse-CDF samples (:func:`inverse_cdf`); with a single coarse sample (no
    section) the fine samples are the midpoints of n_fine equal parts of the
    interval; coarse and fine merged in order, section widths as R21 with the
    outer boundaries at t_n and t_f; rays with no coarse sample render to zero."""
    spec = net.spec
    o = torch.as_tensor(np.asarray(rays_o), dtype=DT)
    d = torch.as_tensor(np.asarray(rays_d), dtype=DT)
    lo_all = torch.as_tensor(np.asarray(t_n), dtype=DT)
    hi_all = torch.as_tensor(np.asarray(t_f), dtype=DT)
    counts = np.asarray(counts, np.int64)
    R = len(counts)
    out = {"rgb": torch.zeros((R, 3), dtype=DT), "depth": torch.zeros(R, dtype=DT),
           "wsum": torch.zeros(R, dtype=DT), "normal": torch.zeros((R, 3), dtype=DT)}
    t_all = [None] * R
    for c in np.unique(counts[counts > 0]):
        idx = np.nonzero(counts == c)[0]
        it = torch.as_tensor(idx)
        lo, hi = lo_all[it], hi_all[it]
        i = torch.arange(int(c), dtype=DT).unsqueeze(0)
        zc = lo.unsqueeze(1) + (i + 0.5) * ((hi - lo) / int(c)).unsqueeze(1)
        if n_fine == 0:
            zf = zc[:, :0]
        elif c >= 2:
            xc = (o[it].unsqueeze(1) + zc.unsqueeze(2) * d[it].unsqueeze(1)).reshape(-1, 3)
            fc, _, _ = sdf_forward(net, xc, with_grad=False)
            w = hier_coarse_weights(fc.reshape(len(idx), int(c)), zc, spec.inv_s, spec.alpha_eps, spec.opacity)
            zf = inverse_cdf(zc, w, n_fine)
        else:
            k = torch.arange(n_fine, dtype=DT).unsqueeze(0)
            zf = lo.unsqueeze(1) + (k + 0.5) * ((hi - lo) / n_fine).unsqueeze(1)
        t, _ = torch.sort(torch.cat([zc, zf], 1), 1)
        mask = torch.ones_like(t, dtype=torch.bool)
        dl = section_widths(t, lo, hi, mask)
        r = render_samples(net, o[it], d[it], t, dl, mask)
        for key in out:
            out[key][it] = r[key]
        for j, rr in enumerate(idx):
            t_all[rr] = t[j]
    out["t"] = t_all
    return out


# ----------------------------------------------------------------------------
# training loss (L1 colour + 0.1 eikonal on the bounded samples)
# ----------------------------------------------------------------------------
def train_loss(net, rays_o, rays_d, t_n, t_f, counts, status, target_rgb, eik_weight=0.1):
    """mean_{rays, channels} |C - C*| + eik_weight * mean_{samples of BOUNDED rays} (|grad f| - 1)^2."""
    out = render_bounded(net, rays_o, rays_d, t_n, t_f, counts)
    tgt = torch.as_tensor(np.asarray(target_rgb), dtype=DT)
    l1 = torch.abs(out["rgb"] - tgt).mean()
    counts_t = torch.as_tensor(np.asarray(counts), dtype=torch.int64)
    bounded = torch.as_tensor(np.asarray(status) == 1)
    per_sample_bounded = torch.repeat_interleave(bounded, counts_t)
    eik = out["eik"]
    nb = int(per_sample_bounded.sum())
    eik_term = (eik * per_sample_bounded).sum() / max(nb, 1)
    return l1 + eik_weight * eik_term, out


def grads(net, loss):
    ps = net.params()
    gs = torch.autograd.grad(loss, ps)
    return gs


def to_numpy(out):
    return {k: (v.detach().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}


def psnr(a, b, peak=1.0):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)
