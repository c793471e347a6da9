"""Pins of the oracle's VolSDF opacity (the Laplace-CDF density of VolSDF /
MonoSDF in Eq. 1 as printed, alpha = 1 - exp(-sigma delta)):

* the density equals a times scipy's Laplace CDF of -f with scale 1/a;
* on a plane hit head-on the weights telescope: sum w = 1 - exp(-sum sigma delta)
  exactly, and the midpoint sum of sigma delta is the closed-form optical depth
  within the midpoint rule's error bound;
* the comparator's section weights use the density at the mid value;
* the training-loss gradient through the VolSDF opacity matches central
  differences (in tests/test_oracle_render.py, parametrised on the opacity)."""
import math

import numpy as np
import pytest
import torch

from oracle import render as orr

DT = torch.float64


def test_density_is_the_laplace_cdf():
    stats = pytest.importorskip("scipy.stats")
    for a in (8.0, 64.0, 100.0):
        f = np.linspace(-0.3, 0.3, 2001)
        got = orr.volsdf_density(torch.tensor(f, dtype=DT), a).numpy()
        ref = a * stats.laplace.cdf(-f, loc=0.0, scale=1.0 / a)
        assert np.max(np.abs(got - ref)) < 1e-12 * a


def _tau(u, a):
    """Optical depth of sigma(-(t - t*)) from -inf to t* + u: a * integral of the
    Laplace CDF, (1/2) e^{a u} for u <= 0 and a u + (1/2) e^{-a u} for u > 0."""
    return 0.5 * math.exp(a * u) if u <= 0 else a * u + 0.5 * math.exp(-a * u)


@pytest.mark.parametrize("a", [16.0, 64.0])
def test_plane_weights_and_optical_depth(a):
    t_star = 1.3
    for n, (lo, hi) in [(7, (1.0, 1.6)), (96, (0.5, 2.0)), (4096, (0.0, 3.0))]:
        t = torch.tensor([[lo + (i + 0.5) * (hi - lo) / n for i in range(n)]], dtype=DT)
        delta = torch.full_like(t, (hi - lo) / n)
        f = -(t - t_star)
        alpha = orr.volsdf_alpha(f, delta, a)
        out = orr.composite(alpha, t, torch.zeros(1, n, 3, dtype=DT), torch.zeros(1, n, 3, dtype=DT),
                            torch.ones_like(t, dtype=torch.bool))
        x = float((orr.volsdf_density(f, a) * delta).sum())
        assert abs(out["wsum"].item() - (1.0 - math.exp(-x))) < 1e-12
        # midpoint rule: |error| <= (hi - lo) h^2 / 24 * max |sigma''|, sigma'' <= a^3 / 2
        h = (hi - lo) / n
        exact = _tau(hi - t_star, a) - _tau(lo - t_star, a)
        assert abs(x - exact) <= (hi - lo) * h * h / 24 * a ** 3 / 2 + 1e-12


def test_comparator_sections_use_the_mid_density():
    a = 64.0
    z = torch.tensor([[0.9, 1.1, 1.25, 1.3, 1.6]], dtype=DT)
    f = torch.tensor([[0.3, 0.1, 0.02, -0.01, -0.3]], dtype=DT)
    w = orr.hier_coarse_weights(f, z, a, 1e-5, orr.OPACITY_VOLSDF)[0].numpy()
    T, ref = 1.0, []
    for j in range(4):
        mid = 0.5 * (f[0, j].item() + f[0, j + 1].item())
        sig = a * (0.5 * math.exp(-a * mid) if mid >= 0 else 1.0 - 0.5 * math.exp(a * mid))
        al = 1.0 - math.exp(-sig * (z[0, j + 1].item() - z[0, j].item()))
        ref.append(al * T)
        T *= 1.0 - al
    assert np.max(np.abs(w - np.array(ref))) < 1e-14
