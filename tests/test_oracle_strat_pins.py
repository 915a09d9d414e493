"""Pins of the oracle's stratified + importance hybrid (Lepage 1980's combined
mode) against facts that do not come from the oracle itself:

  * with one hypercube (B = 0) it is plain importance sampling, sample for
    sample (the plain oracle is pinned separately);
  * every sample lies in its hypercube, whose strata are the mixed-radix
    digits of the hypercube index, computed here by integer division;
  * for a linear integrand on the uniform grid the variance of the estimate
    has the closed form sum_j 1/(12 M_j^2) / n (independent uniforms inside
    strata of width 1/M_j);
  * estimates of integrals with closed forms lie within a few sigma, and
    stratification lowers sigma on a smooth integrand.
"""
import math

import numpy as np
import pytest

import closed_forms as CF
import oracle as O
from paper_2010_09341_gb300 import workloads as W


def _digits(h, bits):
    """Mixed-radix digits of h with radices 2^bits[j], lowest first (plain
    integer division and remainder)."""
    out = []
    for b in bits:
        M = 2 ** int(b)
        out.append(h % M)
        h //= M
    return out


def test_strata_bits_spread_evenly():
    for d in range(1, 9):
        for B in range(0, 3 * d + 2):
            bits = O.strata_bits(d, B)
            assert bits.sum() == B
            assert bits.max() - bits.min() <= 1
            assert list(bits) == sorted(bits, reverse=True)


@pytest.mark.parametrize("family,params", [("sum", []), ("gauss_sym", [0.2])])
def test_one_hypercube_is_plain_sampling(family, params):
    """B = 0: one hypercube of P = n samples; the stratified word is the Philox
    word itself, so every sample and every sum equals plain sampling's."""
    d, N, n = 3, 20, 3000
    e = O.uniform_edges(d, N)
    # a non-uniform grid as well
    e2 = O.refine(d, N, O.iterate(d, N, e, "gauss_sym", [0.1], 0, 0, 0, 2000)["hist"], e)
    for edges in (e, e2):
        for s in (0, 1, 17, 2999):
            a = O.sample(d, N, edges, family, params, 4, 2, 1, s)
            b = O.sample_strat(d, N, edges, family, params, 4, 2, 1, 0, n, s)
            assert np.array_equal(a[0], b[0])
            assert np.array_equal(a[1], b[1])
            assert a[2] == b[2] and a[3] == b[3]
        p = O.iterate(d, N, edges, family, params, 4, 2, 1, n)
        q = O.iterate_strat(d, N, edges, family, params, 4, 2, 1, 0, n)
        assert p["S1"] == q["S1"] and p["S2"] == q["S2"]
        assert np.array_equal(p["hist"], q["hist"])
        I_p, var_p = O.iteration_result(p["S1"], p["S2"], n)
        I_q, var_q = O.strat_result(q["S1"], q["Q"], 1, n)
        assert I_q == pytest.approx(I_p, rel=1e-15)
        assert var_q == pytest.approx(var_p, rel=1e-9)


@pytest.mark.parametrize("d,B,P", [(1, 5, 3), (2, 6, 2), (3, 7, 2), (5, 12, 2)])
def test_samples_lie_in_their_hypercube(d, B, P):
    """On the uniform grid x = y.  Sample s of hypercube h = s // P has
    floor(x_j M_j) = k_j (digit j of h) and its offset inside the stratum is the
    Philox uniform r_j 2^-32, to the 2^-32 lattice."""
    N = 16
    e = O.uniform_edges(d, N)
    bits = O.strata_bits(d, B)
    M = [2 ** int(b) for b in bits]
    H = 2 ** B
    hs = range(H) if H <= 512 else list(range(256)) + list(range(H - 256, H))
    counts = [np.zeros(m, dtype=np.int64) for m in M]
    for h in hs:
        k = _digits(h, bits)
        for p in range(P):
            s = h * P + p
            bins, x, J, f = O.sample_strat(d, N, e, "sum", [], 9, 1, 2, B, P, s)
            assert J == pytest.approx(1.0, abs=1e-12)
            for j in range(d):
                u = O.draw(s, 2, j, 9, 1) / 2.0 ** 32
                assert math.floor(x[j] * M[j]) == k[j]
                assert abs(x[j] * M[j] - k[j] - u) <= M[j] * 2.0 ** -32 + 1e-12
                assert bins[j] == math.floor(x[j] * N) or abs(x[j] * N - round(x[j] * N)) < 1e-9
                counts[j][k[j]] += 1
    if H <= 512:
        for j in range(d):
            assert np.all(counts[j] == P * H // M[j])


@pytest.mark.parametrize("d,B", [(3, 14), (2, 13), (6, 15)])
def test_linear_integrand_variance_closed_form(d, B):
    """f = sum x on the uniform grid: inside a hypercube the x_j are independent
    uniforms on intervals of width 1/M_j, so Var(v | h) = sum_j 1/(12 M_j^2) for
    every h and Var(I) = sum_j 1/(12 M_j^2) / n with n = H P.  With P = 2 the
    estimate's relative spread is sqrt(2 / H) (< 1.3% here)."""
    P = 2
    N = 8
    e = O.uniform_edges(d, N)
    H = 2 ** B
    acc = O.iterate_strat(d, N, e, "sum", [], 3, 0, 0, B, P, threads=4)
    I, var = O.strat_result(acc["S1"], acc["Q"], H, P)
    M = [2.0 ** b for b in O.strata_bits(d, B)]
    want = sum(1.0 / (12.0 * m * m) for m in M) / (H * P)
    assert var == pytest.approx(want, rel=6 * math.sqrt(2.0 / H))
    assert abs(I - d / 2.0) < 5 * math.sqrt(want)


def test_stratification_lowers_sigma_on_smooth_integrand():
    """Genz Gaussian, d = 2, uniform grid, n = 2^15: stratification with 2^14
    hypercubes must cut sigma well below plain sampling's (the within-stratum
    variance of a smooth f falls like 1/M^2)."""
    d, N = 2, 16
    params = W.genz_params("genz_gauss", d, seed=5, c_lo=0.5, c_hi=2.0)
    e = O.uniform_edges(d, N)
    n = 2 ** 15
    p = O.iterate(d, N, e, "genz_gauss", params, 0, 0, 0, n)
    _, var_p = O.iteration_result(p["S1"], p["S2"], n)
    q = O.iterate_strat(d, N, e, "genz_gauss", params, 0, 0, 0, 14, 2)
    I_q, var_q = O.strat_result(q["S1"], q["Q"], 2 ** 14, 2)
    assert math.sqrt(var_q) < 0.05 * math.sqrt(var_p)
    exact = CF.genz_gauss(params, d)
    assert abs(I_q - exact) < 5 * math.sqrt(var_q)


@pytest.mark.parametrize("family,d,B,P,n_iter", [("gauss_sym", 4, 14, 3, 6),
                                                 ("genz_prod", 3, 12, 4, 5),
                                                 ("genz_osc", 5, 13, 2, 4)])
def test_stratified_runs_agree_with_closed_forms(family, d, B, P, n_iter):
    """Full stratified runs with grid refinement: the combined estimate lies
    within 4 sigma of the closed form and chi^2/dof is moderate."""
    N = 32
    if family == "gauss_sym":
        params = [0.1]
        exact = math.erf(5.0) ** d
    elif family == "genz_prod":
        params = W.genz_params("genz_prod", d, seed=2)
        exact = CF.genz_prod(params, d)
    else:
        params = W.genz_osc_params(d, seed=1)
        exact = CF.genz_osc(params)
    r = O.integrate_strat(d, N, family, params, B, P, n_iter, threads=4)
    assert abs(r["I"] - exact) < 4 * r["sigma"], (r["I"], exact, r["sigma"])
    assert r["chi2_dof"] < 5.0
