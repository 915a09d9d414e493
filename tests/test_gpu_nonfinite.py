"""Integrand values that are not finite (NaN, +Inf, -Inf).

The estimator takes the finite values only: in plain sampling a non-finite
value is counted (n_nonfinite) and left out of the sums and of n; in the
stratified hybrid it counts as 0 and every hypercube keeps its P samples.
The GPU must count and exclude exactly the samples the FP64 oracle does
(the same user source compiled for the host), and its sums must agree at
the parity tolerances.  An iteration without any finite value has no
estimate: it returns VEGAS_ENONFINITE, leaves the combination of the other
iterations as it was, and its refinement keeps the grid.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
import user_sources as U
from gpu_helpers import BIN_TOL, PRECS, TOL, assert_hist_close, native, random_grid

pytestmark = pytest.mark.gpu


def _make(V, source, d, N, n, prec, strata=0):
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=1.5, seed=0, integral_id=0, precision=prec)
    ctx = V.vegas_create(cfg, "user", np.zeros(0), source=source)
    if strata:
        V.vegas_set_strata(ctx, strata)
    return ctx


@pytest.mark.parametrize("strata", [0, -1])
@pytest.mark.parametrize("warm", [False, True])
@pytest.mark.parametrize("prec", PRECS)
def test_nonfinite_counted_and_excluded_like_the_oracle(prec, warm, strata):
    V = native()
    d, N, n = 4, 40, 100_003
    O.set_user(U.host_function(U.NONFINITE))
    ctx = _make(V, U.NONFINITE, d, N, n, prec, strata)
    t = 0
    if warm:  # the FP32 modes then use fixed-point histogram cells
        V.vegas_step(ctx)
        t = 1
    e = random_grid(d, N, seed=4, spread=0.5)
    V.vegas_set_grid(ctx, e)
    I, sigma, n_ok, n_nf = V.vegas_iterate(ctx)
    S1, S2, h = V.vegas_get_sums(ctx)
    if strata:
        Bt, P, used = V.vegas_get_strata(ctx)
        acc = O.iterate_strat(d, N, e, "user", [], 0, 0, t, Bt, P, threads=8)
        Io, var = O.strat_result(acc["S1"], acc["Q"], 2 ** Bt, P)
        n_expect = used
    else:
        acc = O.iterate(d, N, e, "user", [], 0, 0, t, n, threads=8)
        Io, var = O.iteration_result(acc["S1"], acc["S2"], n - acc["n_nonfinite"])
        n_expect = n - acc["n_nonfinite"]
    tol = TOL[prec]
    assert acc["n_nonfinite"] > 1000          # a few per cent of the samples
    assert n_nf == acc["n_nonfinite"]         # the same samples, exactly
    assert n_ok == n_expect
    assert abs(I - Io) <= tol * abs(Io), (I, Io)
    assert abs(S2 - acc["S2"]) <= tol * abs(acc["S2"])
    assert_hist_close(h, acc["hist"], tol, BIN_TOL[prec])
    if prec == "fp64" and not strata:
        assert abs(sigma - math.sqrt(var)) <= 1e-9 * math.sqrt(var)


@pytest.mark.parametrize("prec", PRECS)
def test_fp32_square_overflow_counts_as_nonfinite(prec):
    """A finite J f whose square exceeds the FP32 range (1e20 where x_0 > 31/32,
    first iteration, uniform grid: J = 1, no rescale yet): the FP32 modes, whose
    sums take (J f)^2, count those samples in n_nonfinite and leave them out;
    the FP64 path keeps them and equals the oracle, which counts none."""
    V = native()
    d, N, n = 3, 32, 60_001
    O.set_user(U.host_function(U.HUGE))
    ctx = _make(V, U.HUGE, d, N, n, prec)
    e = O.uniform_edges(d, N)
    I, sigma, n_ok, n_nf = V.vegas_iterate(ctx)
    acc = O.iterate(d, N, e, "user", [], 0, 0, 0, n, threads=8)
    assert acc["n_nonfinite"] == 0
    if prec == "fp64":
        Io, _ = O.iteration_result(acc["S1"], acc["S2"], n)
        assert n_nf == 0 and n_ok == n
        assert abs(I - Io) <= TOL[prec] * abs(Io), (I, Io)
    else:
        _, x, _ = O.trace(d, N, e, "user", [], 0, 0, 0, 0, n, threads=8)
        huge = int(np.count_nonzero(x[:, 0] > 0.96875))
        assert 1000 < huge < 3000            # about 1/32 of the samples
        assert n_nf == huge and n_ok == n - huge
        # the rest: 1 + x_1 over the samples with x_0 <= 31/32, each weighted by 1
        keep = x[:, 0] <= 0.96875
        Io = float(np.sum(1.0 + x[keep, 1])) / (n - huge)
        assert abs(I - Io) <= TOL[prec] * abs(Io), (I, Io)


@pytest.mark.parametrize("strata", [0, -1])
@pytest.mark.parametrize("prec", PRECS)
def test_all_nonfinite_iteration_is_left_out(prec, strata):
    """Two finite iterations of a user integrand, then (through a checkpoint
    moved into a context whose integrand is NaN everywhere) one without any
    finite value: VEGAS_ENONFINITE, the combined result unchanged, and the
    grid unchanged by its refinement."""
    V = native()
    from paper_2010_09341_gb300 import _native as nat
    d, N, n = 3, 30, 50_000
    good = _make(V, U.SINE, d, N, n, prec, strata)
    V.vegas_step(good)
    V.vegas_step(good)
    before = V.vegas_result(good)
    e1 = V.vegas_get_grid(good)
    blob = V.vegas_export_state(good)
    bad = _make(V, U.ALL_NAN, d, N, n, prec)
    V.vegas_import_state(bad, blob)
    r = nat.VegasIterResult()
    st = nat.load().vegas_step(bad.handle, ctypes.byref(r))
    assert st == nat.VEGAS_ENONFINITE
    if strata:
        _, _, used = V.vegas_get_strata(bad)
        assert r.n_nonfinite == used and r.n == used
    else:
        assert r.n_nonfinite == n and r.n == 0
    after = V.vegas_result(bad)
    assert after["I"] == before["I"] and after["sigma"] == before["sigma"]
    assert after["chi2_dof"] == before["chi2_dof"]
    assert after["n_iter"] == before["n_iter"] + 1
    assert np.array_equal(V.vegas_get_grid(bad), e1)
