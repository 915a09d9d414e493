"""Pins of the oracle's user-integrand family (a host function called from its
own sampling loop) against facts outside that path: the same function
written as a built-in family, and closed-form integrals."""
import math

import numpy as np
import pytest

import closed_forms as CF
import oracle as O
import user_sources as U
from paper_2010_09341_gb300 import workloads as W


def test_user_genz_gauss_equals_builtin_family():
    """The user source of the Genz Gaussian through the callback gives the
    built-in family's sums (the same FP64 formula, term for term)."""
    d, N, n = 5, 30, 20_000
    p = W.genz_params("genz_gauss", d, seed=3)
    O.set_user(U.host_function(U.GENZ_GAUSS))
    e = O.uniform_edges(d, N)
    e = O.refine(d, N, O.iterate(d, N, e, "genz_gauss", p, 0, 0, 0, n)["hist"], e)
    a = O.iterate(d, N, e, "genz_gauss", p, 1, 2, 1, n)
    b = O.iterate(d, N, e, "user", p, 1, 2, 1, n)
    assert b["S1"] == pytest.approx(a["S1"], rel=1e-14)
    assert b["S2"] == pytest.approx(a["S2"], rel=1e-14)
    assert np.allclose(b["hist"], a["hist"], rtol=1e-13, atol=0)


def test_user_sine_product_integrates_to_one():
    d = 4
    O.set_user(U.host_function(U.SINE))
    r = O.integrate(d, 40, "user", [], 50_000, 6, threads=4)
    assert abs(r["I"] - 1.0) < 4 * r["sigma"]


def test_user_mixed_closed_form():
    """g/((x0-m)^2+g^2) prod_j h(x_j), h = 1 + a x below 1/2 and 2 x^1.5 above:
    (atan((1-m)/g) + atan(m/g)) (1/2 + a/8 + 0.8 (1 - 2^-2.5))^(d-1)."""
    d, m, g, a = 3, 0.35, 0.05, 0.7
    O.set_user(U.host_function(U.MIXED))
    exact = (math.atan((1 - m) / g) + math.atan(m / g)) * (0.5 + a / 8 + 0.8 * (1 - 0.5 ** 2.5)) ** (d - 1)
    r = O.integrate(d, 50, "user", [m, g, a], 100_000, 6, threads=4)
    assert abs(r["I"] - exact) < 4 * r["sigma"], (r["I"], exact, r["sigma"])
