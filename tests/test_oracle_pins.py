"""Pins of the FP64 oracle against facts that do not come from the oracle.

Sources of truth used here:
  * cuRAND's host Philox4x32-10 generator (an independent implementation),
  * closed-form integrals and adaptive quadrature (calculus),
  * tensor Gauss-Legendre quadrature for d <= 2,
  * textbook special cases (uniform grid = plain Monte Carlo, f = 1),
  * grid invariants and hand-derived rebinning examples.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import closed_forms as CF
import oracle as O
from paper_2010_09341_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


# ------------------------------------------------------------------ Philox
def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    pytest.skip("libcurand not available")


@pytest.mark.parametrize("seed", [0, 1, 0x9E3779B97F4A7C15, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4x32-10 generator with offset 0 emits block b as
    Philox(ctr = (0, 0, b, 0), key = (seed_lo, seed_hi)).  The oracle's block
    function, written from Salmon et al., must reproduce every word."""
    lib = _curand()
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        nblk = 4096
        ref = np.zeros(4 * nblk, dtype=np.uint32)
        assert lib.curandGenerate(gen, ref.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(ref.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    mine = np.concatenate([O.philox4x32_10([0, 0, b, 0], key) for b in range(nblk)])
    assert np.array_equal(mine, ref)


def test_draw_counter_layout():
    """r_j of sample s, iteration t is word j%4 of Philox((s_lo, s_hi, t, j/4), (seed, id))."""
    s = (5 << 32) | 77
    for j in range(9):
        blk = O.philox4x32_10([77, 5, 3, j // 4], [11, 42])
        assert O.draw(s, 3, j, 11, 42) == int(blk[j % 4])


def test_uniform_words_are_uniform():
    """Bit balance of 4e4 words: every bit set with frequency 1/2 within 5 sigma."""
    words = np.array([O.draw(s, 0, j, 0, 0) for s in range(10000) for j in range(4)],
                     dtype=np.uint64)
    bits = np.array([(words >> b) & 1 for b in range(32)], dtype=np.float64)
    freq = bits.mean(axis=1)
    assert np.all(np.abs(freq - 0.5) < 5 * 0.5 / math.sqrt(words.size))


# ----------------------------------------------------------- single sample
def test_uniform_grid_maps_identity():
    """On the uniform grid x_j = r_j / 2^32 (to rounding) and J = 1 (to rounding)."""
    d, N = 5, 50
    e = O.uniform_edges(d, N)
    for s in range(200):
        bins, x, J, f = O.sample(d, N, e, "sum", [], 7, 3, 2, s)
        r = np.array([O.draw(s, 2, j, 7, 3) for j in range(d)], dtype=np.float64)
        y = r / 2.0 ** 32
        assert np.allclose(x, y, rtol=0, atol=4e-16)
        assert np.array_equal(bins, np.floor(y * N).astype(np.int32))
        # N * (e[i+1] - e[i]) with e[k] = k/N carries up to ~1 ulp(1)/Delta per dim
        assert abs(J - 1.0) < d * N * 4 * np.spacing(1.0)
        assert abs(f - x.sum()) < 1e-14


def test_bin_index_and_fraction_on_nonuniform_grid():
    """x lies inside its bin; the bin index depends only on r and N."""
    d, N = 3, 7
    rng = np.random.default_rng(5)
    inner = np.sort(rng.uniform(0, 1, size=(d, N - 1)), axis=1)
    e = np.concatenate([np.zeros((d, 1)), inner, np.ones((d, 1))], axis=1)
    for s in range(300):
        bins, x, J, _ = O.sample(d, N, e, "const", [], 1, 0, 0, s)
        ub, _, _, _ = O.sample(d, N, O.uniform_edges(d, N), "const", [], 1, 0, 0, s)
        assert np.array_equal(bins, ub)
        for j in range(d):
            assert e[j, bins[j]] <= x[j] <= e[j, bins[j] + 1]
        widths = e[np.arange(d), bins + 1] - e[np.arange(d), bins]
        assert abs(J - np.prod(N * widths)) <= 1e-12 * J


def test_bin_counts_uniform_in_y():
    """Samples are uniform in y, so each bin receives n/N samples (chi^2 test)."""
    d, N, n = 3, 50, 200000
    acc = O.iterate(d, N, O.uniform_edges(d, N), "const", [], 0, 0, 0, n, counts=True)
    c = acc["counts"]
    assert np.all(c.sum(axis=1) == n)
    exp = n / N
    chi2 = ((c - exp) ** 2 / exp).sum(axis=1)
    # chi^2 with 49 dof: mean 49, sd ~9.9; 49 + 6 sd is far in the tail
    assert np.all(chi2 < 49 + 6 * 9.9)


# ---------------------------------------------------- iteration statistics
def test_iteration_result_textbook():
    """v in {0, 2} (n = 2): mean 1, unbiased sample variance 2, variance of the
    mean 1; a constant gives zero variance."""
    I, var = O.iteration_result(2.0, 4.0, 2)
    assert I == 1.0 and var == 1.0
    I, var = O.iteration_result(5.0 * 10, 25.0 * 10, 10)
    assert I == 5.0 and var == 0.0


def test_uniform_grid_first_iteration_is_plain_mc():
    """Iteration 0 on the uniform grid is the plain MC mean of f at x = r/2^32."""
    d, N, n = 3, 50, 4000
    params = W.genz_params("genz_gauss", d, seed=4)
    acc = O.iterate(d, N, O.uniform_edges(d, N), "genz_gauss", params, 9, 1, 0, n)
    vals = []
    for s in range(n):
        y = np.array([O.draw(s, 0, j, 9, 1) for j in range(d)], dtype=np.float64) / 2.0 ** 32
        vals.append(O.integrand("genz_gauss", d, params, y))
    vals = np.array(vals)
    assert abs(acc["S1"] / n - vals.mean()) < 1e-13
    assert abs(acc["S2"] - (vals ** 2).sum()) < 1e-12 * acc["S2"]


def test_histogram_rows_sum_to_S2():
    """Every sample adds v^2 once per dimension, so each histogram row sums to S2."""
    d, N = 6, 20
    rng = np.random.default_rng(1)
    inner = np.sort(rng.uniform(0, 1, size=(d, N - 1)), axis=1)
    e = np.concatenate([np.zeros((d, 1)), inner, np.ones((d, 1))], axis=1)
    acc = O.iterate(d, N, e, "genz_prod", W.genz_params("genz_prod", d, 3), 0, 0, 1, 20000)
    assert np.allclose(acc["hist"].sum(axis=1), acc["S2"], rtol=1e-12, atol=0)


def test_const_on_uniform_grid_exact():
    r = O.integrate(4, 50, "const", [], 1000, 1)
    assert abs(r["iters"][0][0] - 1.0) < 1e-14
    assert r["iters"][0][1] < 1e-9


def test_jacobian_has_unit_mean_on_any_grid():
    """E_y[J] = prod_j sum_i Delta_j[i] = 1 on any grid: f = 1 integrates to 1."""
    d, N, n = 4, 10, 200000
    rng = np.random.default_rng(2)
    inner = np.sort(rng.uniform(0, 1, size=(d, N - 1)), axis=1)
    e = np.concatenate([np.zeros((d, 1)), inner, np.ones((d, 1))], axis=1)
    acc = O.iterate(d, N, e, "const", [], 0, 0, 0, n)
    I, var = O.iteration_result(acc["S1"], acc["S2"], n)
    assert abs(I - 1.0) < 4 * math.sqrt(var)


# ------------------------------------------------------------- refinement
def _random_grid(rng, d, N):
    inner = np.sort(rng.uniform(0, 1, size=(d, N - 1)), axis=1)
    return np.concatenate([np.zeros((d, 1)), inner, np.ones((d, 1))], axis=1)


def test_refine_invariants():
    rng = np.random.default_rng(0)
    for N in (2, 3, 50, 100, 1024):
        d = 4
        e = _random_grid(rng, d, N)
        h = rng.exponential(1.0, size=(d, N)) * rng.uniform(0, 1, size=(d, 1))
        h[0, : N // 2] = 0.0  # dimension with empty bins
        out = O.refine(d, N, h, e, 1.5)
        assert np.all(out[:, 0] == 0.0) and np.all(out[:, -1] == 1.0)
        assert np.all(np.diff(out, axis=1) >= 0.0)
        assert np.all(np.abs(np.diff(out, axis=1).sum(axis=1) - 1.0) < 1e-14)


def test_refine_uniform_fixed_point():
    """Equal weights on the uniform grid leave it unchanged, up to the rounding
    of the running weight sum (which grows with the number of bins summed)."""
    for N in (10, 50, 100, 1024):
        e = O.uniform_edges(3, N)
        out = O.refine(3, N, np.full((3, N), 2.5), e, 1.5)
        assert np.all(np.abs(out - e) <= (2 + N / 8) * np.spacing(1.0))


def test_refine_alpha_zero_is_identity():
    """alpha = 0 makes every positive weight 1: the grid must not move."""
    rng = np.random.default_rng(3)
    e = _random_grid(rng, 3, 40)
    h = rng.uniform(0.1, 5.0, size=(3, 40))
    out = O.refine(3, 40, h, e, 0.0)
    assert np.allclose(out, e, rtol=0, atol=1e-15)


def test_refine_worked_example_empty_region():
    """Hand-derived: N = 10 uniform grid, weight only in bins 3..6.  Smoothing
    spreads it to bins 2..7 (6 bins); alpha = 0 gives each weight 1, so the
    10 new bins split [0.2, 0.8] evenly: e'_k = 0.2 + 0.06 k, k = 1..9."""
    N = 10
    h = np.zeros((1, N))
    h[0, 3:7] = [1.0, 4.0, 2.0, 3.0]
    out = O.refine(1, N, h, O.uniform_edges(1, N), 0.0)
    exp = np.concatenate([[0.0], 0.2 + 0.06 * np.arange(1, N), [1.0]])
    assert np.allclose(out[0], exp, rtol=0, atol=1e-15)


def test_refine_worked_example_two_bins():
    """Hand-derived from Lepage's compression with N = 2, no smoothing,
    weights (1, 4) so d = (0.2, 0.8), alpha = 1:
      rho_0 = 0.8/ln 5, rho_1 = 0.2/ln 1.25, delta = (rho_0 + rho_1)/2;
      rho_0 < delta, so the edge sits in bin 1 at 0.5 + 0.5 (delta - rho_0)/rho_1."""
    r0 = 0.8 / math.log(5.0)
    r1 = 0.2 / math.log(1.25)
    dl = (r0 + r1) / 2
    exp = 0.5 + 0.5 * (dl - r0) / r1
    out = O.refine(1, 2, np.array([[1.0, 4.0]]), O.uniform_edges(1, 2), 1.0, smooth=False)
    assert abs(out[0, 1] - exp) < 1e-15
    assert 0.61 < out[0, 1] < 0.62


def test_refine_narrows_bins_where_weight_is_high():
    N = 20
    h = np.arange(1, N + 1, dtype=np.float64)[None, :] ** 2
    out = O.refine(1, N, h, O.uniform_edges(1, N), 1.5)
    w = np.diff(out[0])
    assert np.all(np.diff(w) < 0)


def test_refine_zero_histogram_keeps_grid():
    rng = np.random.default_rng(4)
    e = _random_grid(rng, 2, 30)
    out = O.refine(2, 30, np.zeros((2, 30)), e, 1.5)
    assert np.array_equal(out, e)


def test_adaptation_reduces_variance():
    """A peaked integrand: the adapted grid cuts the per-iteration sigma by a
    large factor (a broken compression or rebin would not)."""
    r = O.integrate(4, 50, "gauss_sym", [0.1], 50000, 6)
    s = [b for _, b in r["iters"]]
    assert s[0] / s[-1] > 20


# ------------------------------------------------------------- combination
def test_combine_closed_forms():
    Ib, sb, c2 = O.combine([1.0, 1.0, 1.0, 1.0], [2.0, 2.0, 2.0, 2.0])
    assert Ib == 1.0 and abs(sb - 1.0) < 1e-15 and c2 == 0.0
    Ib, sb, c2 = O.combine([1.0, 3.0], [1.0, 1.0])
    assert Ib == 2.0 and abs(sb - 1 / math.sqrt(2)) < 1e-15 and c2 == 2.0
    Ib, sb, c2 = O.combine([1.0, 4.0], [1.0, 2.0])  # weights 1, 1/4
    assert abs(Ib - (1.0 + 1.0) / 1.25) < 1e-15
    Ib, sb, c2 = O.combine([2.0, 5.0], [0.0, 1.0])
    assert Ib == 2.0 and sb == 0.0


# ----------------------------------------------------------- closed forms
def _check(r, exact, k=3.0):
    assert abs(r["I"] - exact) < k * r["sigma"], (r["I"], exact, r["sigma"])
    assert r["chi2_dof"] < 5.0


def test_closed_form_gauss_sym_d4():
    r = O.integrate(4, 50, "gauss_sym", [0.1], 100000, 5, alpha=1.5, seed=0)
    _check(r, CF.gauss_sym(4, 0.1))
    assert r["sigma"] < 2e-3


def test_closed_form_gauss_sym_d8():
    r = O.integrate(8, 50, "gauss_sym", [0.1], 200000, 8, alpha=1.5, seed=0)
    _check(r, CF.gauss_sym(8, 0.1))


def test_closed_form_genz_osc_d8():
    p = W.genz_osc_params(8, seed=1)
    r = O.integrate(8, 50, "genz_osc", p, 100000, 5, seed=1)
    _check(r, CF.genz_osc(p))
    assert r["sigma"] < 1e-3 * abs(CF.genz_osc(p)) + 1e-3


@pytest.mark.parametrize("d", [2, 5, 9])
def test_closed_form_genz_gauss(d):
    p = W.genz_params("genz_gauss", d, seed=10 + d)
    r = O.integrate(d, 50, "genz_gauss", p, 100000, 5)
    _check(r, CF.genz_gauss(p, d))


@pytest.mark.parametrize("d", [2, 5, 9])
def test_closed_form_genz_prod(d):
    p = W.genz_params("genz_prod", d, seed=20 + d)
    r = O.integrate(d, 50, "genz_prod", p, 100000, 5)
    _check(r, CF.genz_prod(p, d))


@pytest.mark.parametrize("d", [2, 4, 6])
def test_closed_form_genz_corner(d):
    p = W.genz_params("genz_corner", d, seed=30 + d)
    exact = CF.genz_corner_incl_excl(p)
    assert abs(exact - CF.genz_corner_laplace(p)) < 1e-10 * exact
    r = O.integrate(d, 50, "genz_corner", p, 100000, 5)
    _check(r, exact)


def test_corner_laplace_form_d16():
    """At d = 16 the inclusion-exclusion sum cancels; the 1-D form must still be
    positive and below the integrand's maximum 1."""
    p = W.genz_params("genz_corner", 16, seed=5)
    v = CF.genz_corner_laplace(p)
    assert 0 < v < 1


def test_closed_form_sum_toy():
    r = O.integrate(10, 50, "sum", [], 50000, 4)
    _check(r, 5.0)


def test_lo_against_quadrature():
    p = W.lo_params()
    exact = CF.lo_value(p)
    r = O.integrate(3, 100, "lo", p, 200000, 8, threads=4)
    _check(r, exact)
    assert r["sigma"] < 2e-2 * exact


# ------------------------------------------------------ brute force, d <= 2
def _gauss_legendre_2d(fn, n=400):
    xg, wg = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (xg + 1)
    w = 0.5 * wg
    tot = 0.0
    for i in range(n):
        for k in range(n):
            tot += w[i] * w[k] * fn(np.array([x[i], x[k]]))
    return tot


@pytest.mark.parametrize("family", ["genz_gauss", "genz_prod", "genz_corner"])
def test_brute_force_d2(family):
    p = W.genz_params(family, 2, seed=40)
    q = _gauss_legendre_2d(lambda x: O.integrand(family, 2, p, x), n=200)
    exact = {"genz_gauss": lambda: CF.genz_gauss(p, 2), "genz_prod": lambda: CF.genz_prod(p, 2),
             "genz_corner": lambda: CF.genz_corner_incl_excl(p)}[family]()
    assert abs(q - exact) < 1e-9 * abs(exact)
    r = O.integrate(2, 50, family, p, 50000, 5)
    _check(r, q)


def test_oracle_reproduces_golden_fixture_bitwise():
    """tests/golden/config1_oracle.json was written by tests/golden/make_golden.py
    (oracle only); the oracle must reproduce it exactly on this machine."""
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config1_oracle.json")
    g = json.load(open(path))
    r = O.integrate(4, 50, "gauss_sym", [0.1], 100_000, 5, alpha=1.5, seed=0)
    assert [[float(I).hex(), float(s).hex()] for I, s in r["iters"]] == g["iters"]
    assert float(r["I"]).hex() == g["I"] and float(r["sigma"]).hex() == g["sigma"]
    assert hashlib.sha256(r["edges"].astype("<f8").tobytes()).hexdigest() == g["edges_sha256"]


def test_oracle_reproduces_path_fixtures_bitwise():
    """tests/golden/paths_oracle.json (tests/golden/make_golden.py, oracle only):
    the stratified run, the LO toy on a density grid and an observable
    histogram reproduce exactly on this machine, so that any change of the
    oracle's arithmetic on those paths shows."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    try:
        import make_golden as MG
    finally:
        sys.path.remove(here)
    g = json.load(open(os.path.join(here, "paths_oracle.json")))
    r = MG.paths()
    for key in ("strat", "lo_pdf", "histogram"):
        assert r[key] == g[key], key


def test_trace_is_sample_by_sample_and_sums_to_iterate():
    """oracle.trace runs oracle_sample per sample (host threads): the same
    bins, points and weights, and its weights add up to the iteration sums."""
    d, N = 5, 30
    p = W.genz_params("genz_gauss", d, seed=4)
    rng = np.random.default_rng(5)
    inner = np.sort(rng.uniform(0, 1, size=(d, N - 1)), axis=1)
    e = np.concatenate([np.zeros((d, 1)), inner, np.ones((d, 1))], axis=1)
    s0, cnt = (1 << 32) - 300, 2000
    bins, x, v = O.trace(d, N, e, "genz_gauss", p, 3, 7, 2, s0, cnt, threads=3)
    for k in (0, 1, 299, 300, 1999):
        ob, ox, J, f = O.sample(d, N, e, "genz_gauss", p, 3, 7, 2, s0 + k)
        assert np.array_equal(bins[k], ob) and np.array_equal(x[k], ox) and v[k] == J * f
    acc = O.iterate(d, N, e, "genz_gauss", p, 3, 7, 2, cnt, s_begin=s0, s_end=s0 + cnt)
    assert abs(v.sum() - acc["S1"]) <= 1e-13 * abs(acc["S1"])
    assert abs((v * v).sum() - acc["S2"]) <= 1e-13 * acc["S2"]
