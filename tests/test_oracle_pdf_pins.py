"""Pins of the oracle's tabulated parton density (bicubic Hermite in
(ln x, ln Q^2) with finite-difference tangents) and of the LO toy built on it,
against facts outside that code: the knot values themselves, polynomials the
scheme reproduces exactly, the analytic density the table samples, and the
LO toy with its analytic density."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2010_09341_gb300 import workloads as W


def test_knot_values_are_reproduced():
    xg, u0, u1, v0, v1 = W.pdf_grid(24, 12)
    O.set_pdf_grid(xg, u0, u1, v0, v1)
    u = np.linspace(u0, u1, 24)
    v = np.linspace(v0, v1, 12)
    for i in (0, 1, 7, 22, 23):
        for j in (0, 3, 11):
            assert O.pdf_xg(math.exp(u[i]), math.exp(v[j])) == pytest.approx(xg[i, j], rel=1e-12, abs=1e-300)


def test_tensor_quadratics_are_exact_inside():
    """Central-difference tangents are exact for quadratics, and a cubic
    Hermite piece with exact values and tangents reproduces a quadratic, so
    q(u) r(v) is reproduced in every cell whose four knots are inside."""
    nx, nq = 11, 9
    u0, u1, v0, v1 = -5.0, 0.0, 2.0, 9.0
    u = np.linspace(u0, u1, nx)
    v = np.linspace(v0, v1, nq)
    q = lambda a: 0.3 + 0.7 * a - 0.2 * a * a
    r = lambda b: 1.1 - 0.4 * b + 0.05 * b * b
    O.set_pdf_grid(np.outer(q(u), r(v)), u0, u1, v0, v1)
    rng = np.random.default_rng(1)
    hu, hv = (u1 - u0) / (nx - 1), (v1 - v0) / (nq - 1)
    for _ in range(200):
        a = rng.uniform(u0 + hu, u1 - hu)
        b = rng.uniform(v0 + hv, v1 - hv)
        assert O.pdf_xg(math.exp(a), math.exp(b)) == pytest.approx(q(a) * r(b), rel=1e-12)


def test_interpolation_converges_to_the_sampled_density():
    """Against x g = N x^1/2 (1-x)^b(Q^2) itself: the error falls at least 6x
    when the knot spacing halves (third order inside).  Uniform knots in ln x
    are coarsest where (1-x)^b is steepest (x -> 1): the largest error of the
    79 x 39 grid is there, below 1% up to x = 0.8."""
    from scipy.special import beta
    rng = np.random.default_rng(2)
    xs = np.exp(rng.uniform(math.log(1e-5), math.log(0.8), 300))
    qs = np.exp(rng.uniform(math.log(20.0), math.log(900.0), 300))
    errs = []
    for nx, nq in ((40, 20), (79, 39)):
        xg, u0, u1, v0, v1 = W.pdf_grid(nx, nq)
        O.set_pdf_grid(xg, u0, u1, v0, v1)
        e = 0.0
        for x, q in zip(xs, qs):
            b = 3.0 + 0.5 * (math.log(q * q) - v0) / (v1 - v0)
            exact = math.sqrt(x) * (1 - x) ** b / beta(0.5, b + 1)
            e = max(e, abs(O.pdf_xg(x, q * q) - exact) / exact)
        errs.append(e)
    assert errs[1] < errs[0] / 6.0, errs
    assert errs[1] < 1e-2


def test_lo_on_the_grid_approaches_the_analytic_lo_toy():
    """With the LO toy's own density tabulated (no scale dependence), the
    gridded LO integrand equals the analytic one to the interpolation error,
    sample for sample and in the iteration sums."""
    xg, u0, u1, v0, v1 = W.pdf_grid(160, 8, b1=0.0)
    O.set_pdf_grid(xg, u0, u1, v0, v1)
    p = W.lo_params()
    N = 100
    e = O.uniform_edges(3, N)
    a = O.iterate(3, N, e, "lo", p, 0, 0, 0, 200_000, threads=4)
    b = O.iterate(3, N, e, "lo_pdf", p, 0, 0, 0, 200_000, threads=4)
    assert b["S1"] == pytest.approx(a["S1"], rel=2e-4)
    assert b["S2"] == pytest.approx(a["S2"], rel=4e-4)
