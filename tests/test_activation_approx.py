"""The tensor-core kernel evaluates softplus_beta and its slope from one tanh:
t = tanh(beta z / 2), slope = (1 + t)/2, softplus = max(z, 0) + (ln 2 - log(1 + |t|))/beta,
with log(1 + u) on [0, 1] as a fitted polynomial.  Pin the identity and the
polynomial's error bound against numpy."""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def coefficients():
    src = open(os.path.join(ROOT, "paper_2311_17878_gb300", "csrc", "tc_common.cuh")).read()
    body = src[src.index("float log1p_unit(float u)"):]
    body = body[:body.index("return p * u;")]
    return [float(v) for v in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]


def poly(u, c):
    p = np.full_like(u, c[0])
    for ci in c[1:]:
        p = p * u + ci
    return p * u


def test_log1p_polynomial_error_bound():
    c = coefficients()
    assert len(c) == 4
    u = np.linspace(0.0, 1.0, 200001)
    assert np.max(np.abs(poly(u, c) - np.log1p(u))) < 8e-5
    # exact at both ends: softplus -> 0 as z -> -inf (u -> 1), and the value at z = 0
    assert poly(np.array([0.0]), c)[0] == 0.0
    assert abs(poly(np.array([1.0]), c)[0] - math.log(2)) < 1e-7


def test_tanh_form_of_softplus_and_slope():
    beta = 100.0
    z = np.concatenate([np.linspace(-0.5, 0.5, 20001), [0.0, 1e-6, -1e-6, 3.0, -3.0]])
    t = np.tanh(beta * z / 2)
    slope = 0.5 * (1 + t)
    sp = np.maximum(z, 0) + (math.log(2) - np.log1p(np.abs(t))) / beta
    ref_sp = np.logaddexp(0.0, beta * z) / beta
    ref_slope = 1.0 / (1.0 + np.exp(-beta * z))
    assert np.max(np.abs(sp - ref_sp)) < 1e-12
    assert np.max(np.abs(slope - ref_slope)) < 1e-12
    # with the fitted polynomial the softplus error stays below 8e-5 / beta, under half an
    # FP16 ulp of softplus(0) = ln 2 / beta, the smallest activation that is not tiny
    sp_poly = np.maximum(z, 0) + (math.log(2) - poly(np.abs(t), coefficients())) / beta
    assert np.max(np.abs(sp_poly - ref_sp)) < 8e-5 / beta + 1e-12
    assert 8e-5 / beta < 0.5 * np.spacing(np.float16(math.log(2) / beta))
