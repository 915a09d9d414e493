"""User integrands compiled at run time (vegas_create_user) against the FP64
oracle evaluating the same source compiled for the host.

Tolerances as for the built-in families: bins bit-exact; I_t, S2 and the
histograms relative 1e-12 (FP64) and 1e-5 (FP32) on the same input grid;
sigma_t 1e-9 (FP64).  Per-sample FP32 values: the FP32 path's math functions
(sin, pow, exp in float) carry a few ulps, 2e-5 of the integrand's scale.
"""
import math
import time

import numpy as np
import pytest

import oracle as O
import user_sources as U
from gpu_helpers import BIN_TOL, PRECS, TOL, assert_hist_close, native, random_grid
from paper_2010_09341_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _make(V, source, params, d, N, n, prec, seed=0, iid=0, strata=0):
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=1.5, seed=seed, integral_id=iid,
                   precision=prec)
    ctx = V.vegas_create(cfg, "user", params, source=source)
    if strata:
        V.vegas_set_strata(ctx, strata)
    return ctx


CASES = [("genz_gauss", U.GENZ_GAUSS, 5, 50, 100_003), ("sine", U.SINE, 4, 40, 65_536),
         ("mixed", U.MIXED, 3, 50, 77_777), ("sine12", U.SINE, 12, 20, 50_001)]


def _params(name, d):
    if name == "genz_gauss":
        return W.genz_params("genz_gauss", d, seed=3)
    if name == "mixed":
        return np.array([0.35, 0.05, 0.7])
    return np.zeros(0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,src,d,N,n", CASES)
def test_user_iteration_parity_on_shared_grid(name, src, d, N, n, prec):
    V = native()
    p = _params(name, d)
    O.set_user(U.host_function(src))
    ctx = _make(V, src, p, d, N, n, prec)
    V.vegas_step(ctx)                      # a refined, non-uniform grid
    e = V.vegas_get_grid(ctx)
    I, sigma, n_ok, n_nf = V.vegas_iterate(ctx)
    S1, S2, h = V.vegas_get_sums(ctx)
    acc = O.iterate(d, N, e, "user", p, 0, 0, 1, n, threads=8)
    Io, var = O.iteration_result(acc["S1"], acc["S2"], n - acc["n_nonfinite"])
    tol = TOL[prec]
    assert n_nf == acc["n_nonfinite"] == 0
    assert abs(I - Io) <= tol * abs(Io), (I, Io)
    assert abs(S2 - acc["S2"]) <= tol * abs(acc["S2"])
    assert_hist_close(h, acc["hist"], tol, BIN_TOL[prec])
    if prec == "fp64":
        assert abs(sigma - math.sqrt(var)) <= 1e-9 * math.sqrt(var)


@pytest.mark.parametrize("prec", PRECS)
def test_user_trace_bins_bit_exact(prec):
    V = native()
    d, N = 5, 30
    p = _params("mixed", d)
    O.set_user(U.host_function(U.MIXED))
    ctx = _make(V, U.MIXED, p, d, N, 1000, prec, seed=4, iid=6)
    e = random_grid(d, N, seed=2)
    V.vegas_set_grid(ctx, e)
    bins, x, w = V.vegas_trace(ctx, 2, (1 << 32) - 500, 1000)
    bins, x, w = bins.cpu().numpy(), x.cpu().numpy(), w.cpu().numpy()
    vs = []
    for k in range(0, 1000, 3):
        ob, ox, J, f = O.sample(d, N, e, "user", p, 4, 6, 2, (1 << 32) - 500 + k)
        assert np.array_equal(bins[k], ob)
        assert np.allclose(x[k], ox, rtol=0, atol=4e-16 if prec == "fp64" else 3e-7)
        vs.append(J * f)
    vs = np.array(vs)
    ws = w[::3]
    if prec == "fp64":
        assert np.all(np.abs(ws - vs) <= 1e-13 * np.abs(vs) + 1e-300)
    else:
        assert np.all(np.abs(ws - vs) <= 2e-5 * np.abs(vs) + 2e-5 * np.mean(np.abs(vs)))


@pytest.mark.parametrize("prec", PRECS)
def test_user_source_equals_builtin_family(prec):
    """The Genz Gaussian as user source and as the built-in family: the same
    sums on the same grid (FP64: 1e-12; FP32: the built-in family forms the
    exponential with the hardware ex2, the user source calls expf, 1e-5)."""
    V = native()
    d, N, n = 6, 50, 200_000
    p = W.genz_params("genz_gauss", d, seed=3)
    a = _make(V, U.GENZ_GAUSS, p, d, N, n, prec)
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=1.5, seed=0, integral_id=0, precision=prec)
    b = V.vegas_create(cfg, "genz_gauss", p)
    V.vegas_step(b)
    V.vegas_set_grid(a, V.vegas_get_grid(b))
    V.vegas_set_iteration(a, 1)
    ra = V.vegas_iterate(a)
    rb = V.vegas_iterate(b)
    assert abs(ra[0] - rb[0]) <= TOL[prec] * abs(rb[0])


def test_user_stratified_matches_oracle():
    V = native()
    d, N, n = 4, 40, 100_000
    O.set_user(U.host_function(U.SINE))
    ctx = _make(V, U.SINE, [], d, N, n, "fp64", strata=-1)
    Bt, P, used = V.vegas_get_strata(ctx)
    e = O.uniform_edges(d, N)
    I, sigma, _, _ = V.vegas_iterate(ctx)
    acc = O.iterate_strat(d, N, e, "user", [], 0, 0, 0, Bt, P, threads=8)
    Io, var = O.strat_result(acc["S1"], acc["Q"], 2 ** Bt, P)
    assert abs(I - Io) <= 1e-12 * abs(Io)
    assert abs(sigma - math.sqrt(var)) <= 1e-9 * math.sqrt(var)


def test_user_full_run_closed_form():
    V = native()
    it = V.Integrator(n_dim=6, n_events=1_000_000, precision="fp32_acc64")
    it.compile(U.SINE)
    res = it.run_integration(8)
    assert abs(res["I"] - 1.0) < 4 * res["sigma"], res


def test_user_compile_error_is_reported():
    V = native()
    from paper_2010_09341_gb300 import _native as nat
    with pytest.raises(nat.VegasError) as ei:
        _make(V, U.BROKEN, [], 3, 10, 1000, "fp32_kahan")
    assert ei.value.status == nat.VEGAS_EJIT
    assert "this_is_not_defined" in str(ei.value)


def test_user_kernels_are_cached():
    """A second context with the same source, precision and dimension reuses the
    compiled module (no second run-time compilation)."""
    V = native()
    src = U.SINE + "\n// cache probe\n"
    t0 = time.perf_counter()
    _make(V, src, [], 7, 20, 1000, "fp32_kahan")
    first = time.perf_counter() - t0
    t0 = time.perf_counter()
    _make(V, src, [], 7, 20, 1000, "fp32_kahan")
    second = time.perf_counter() - t0
    assert second < 0.25 * first, (first, second)


def test_user_params_limit():
    V = native()
    from paper_2010_09341_gb300 import _native as nat
    with pytest.raises(nat.VegasError):
        _make(V, U.SINE, np.zeros(73), 2, 10, 1000, "fp64")
