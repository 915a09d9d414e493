"""Observable histograms of an iteration's weights (vegas_histogram) against
the FP64 oracle's.

Tolerances: FP64 per bin 1e-12 relative (plus 1e-15 of the total for bins
that cancel); FP32: the points carry FP32 rounding, so a sample within ~1e-7
of a bin edge may fall in the neighbouring bin: per bin 2e-4 of the total
weight, totals 1e-5 (the iteration's own tolerance).
"""
import numpy as np
import pytest

import oracle as O
import user_sources as U
from gpu_helpers import PRECS, native
from paper_2010_09341_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(V, family, d, N, n, prec, params, strata=0):
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=1.5, seed=3, integral_id=8, precision=prec)
    ctx = V.vegas_create(cfg, family, params)
    if strata:
        V.vegas_set_strata(ctx, strata)
    return ctx


def _compare(prec, g1, g2, o1, o2):
    tot = np.sum(np.abs(o1))
    if prec == "fp64":
        assert np.all(np.abs(g1 - o1) <= 1e-12 * np.abs(o1) + 1e-15 * tot)
        assert np.all(np.abs(g2 - o2) <= 1e-12 * np.abs(o2) + 1e-15 * np.sum(o2))
    else:
        assert abs(g1.sum() - o1.sum()) <= 1e-5 * tot
        assert np.max(np.abs(g1 - o1)) <= 2e-4 * tot


@pytest.mark.parametrize("strata", [0, -1])
@pytest.mark.parametrize("prec", PRECS)
def test_coordinate_histogram_matches_oracle(prec, strata):
    V = native()
    d, N, n = 4, 40, 300_000
    p = W.genz_params("genz_gauss", d, seed=3)
    ctx = _ctx(V, "genz_gauss", d, N, n, prec, p, strata)
    V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    g1, g2 = V.vegas_histogram(ctx, 1, 2, 17, 0.1, 0.9)
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    B, P, used = V.vegas_get_strata(ctx)
    o1, o2 = O.histogram(d, N, e, "genz_gauss", p, 3, 8, 1, used, 2, 17, 0.1, 0.9, B=B, P=P, threads=8)
    assert g1[0] > 0 and g1[-1] > 0
    _compare(prec, g1, g2, o1, o2)


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_bins_add_up_to_the_iteration(prec):
    """The histogram of iteration t on the grid iteration t samples with adds up
    to that iteration's S1 and S2."""
    V = native()
    d, N, n = 5, 50, 200_003
    p = W.genz_params("genz_prod", d, seed=4)
    ctx = _ctx(V, "genz_prod", d, N, n, prec, p)
    V.vegas_step(ctx)
    g1, g2 = V.vegas_histogram(ctx, 1, 0, 64, 0.0, 1.0)
    V.vegas_iterate(ctx)
    S1, S2, _ = V.vegas_get_sums(ctx)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(g1.sum().item() - S1) <= tol * abs(S1)
    assert abs(g2.sum().item() - S2) <= tol * abs(S2)


@pytest.mark.parametrize("obs,lo,hi", [(-1, 60.0, 120.0 + 1e-9), (-2, -0.95, 0.95)])
@pytest.mark.parametrize("prec", ["fp64", "fp32_acc64"])
def test_lo_observables(prec, obs, lo, hi):
    V = native()
    N, n = 100, 400_000
    p = W.lo_params()
    ctx = _ctx(V, "lo", 3, N, n, prec, p)
    for _ in range(2):
        V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    g1, g2 = V.vegas_histogram(ctx, 2, obs, 30, lo, hi)
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    o1, o2 = O.histogram(3, N, e, "lo", p, 3, 8, 2, n, obs, 30, lo, hi, threads=8)
    assert g1[0] == 0 and g1[-1] == 0   # the cuts
    _compare(prec, g1, g2, o1, o2)


def test_user_integrand_histogram():
    V = native()
    d, N, n = 3, 30, 100_000
    params = np.array([0.35, 0.05, 0.7])
    O.set_user(U.host_function(U.MIXED))
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=1.5, seed=3, integral_id=8, precision="fp64")
    ctx = V.vegas_create(cfg, "user", params, source=U.MIXED)
    V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    g1, g2 = V.vegas_histogram(ctx, 1, 0, 25, 0.0, 1.0)
    o1, o2 = O.histogram(d, N, e, "user", params, 3, 8, 1, n, 0, 25, 0.0, 1.0, threads=8)
    _compare("fp64", g1.cpu().numpy(), g2.cpu().numpy(), o1, o2)


def test_histogram_validation():
    V = native()
    from paper_2010_09341_gb300 import _native as nat
    ctx = _ctx(V, "sum", 3, 10, 1000, "fp64", [])
    for args in [(0, 3, 10, 0.0, 1.0), (0, -1, 10, 0.0, 1.0), (0, 0, 0, 0.0, 1.0), (0, 0, 1025, 0.0, 1.0),
                 (0, 0, 10, 1.0, 1.0), (-1, 0, 10, 0.0, 1.0)]:
        with pytest.raises(nat.VegasError):
            V.vegas_histogram(ctx, *args)


def test_full_size_histogram_sums():
    """1e7 samples of the d = 8 Gaussian in FP32: the histogram of x_0 adds up
    to the iteration's S1, and its peak is at the centre."""
    V = native()
    d, N, n = 8, 50, 10_000_000
    ctx = _ctx(V, "gauss_sym", d, N, n, "fp32_acc64", W.gauss_sym_params(0.1))
    V.vegas_step(ctx)
    g1, _ = V.vegas_histogram(ctx, 1, 0, 100, 0.0, 1.0)
    V.vegas_iterate(ctx)
    S1, _, _ = V.vegas_get_sums(ctx)
    g1 = g1.cpu().numpy()
    assert abs(g1.sum() - S1) <= 1e-5 * abs(S1)
    assert abs(np.argmax(g1[1:-1]) - 49.5) <= 1.5
