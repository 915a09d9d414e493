"""Stratified + importance hybrid (vegas_set_strata) on the GPU against the
FP64 oracle's stratified iteration.

Tolerances:
  * bin indices: bit-exact (integer work: the stratum word and the split);
  * iteration estimate I_t: relative 1e-12 (FP64 path), 1e-5 (FP32 paths) on
    the same input grid; S2 and the histograms likewise;
  * sigma_t: relative 1e-9 in FP64.  In the FP32 paths sigma_t comes from the
    spread of the values about their hypercube's mean, and each FP32 value
    carries an error of about 1e-7 of v (the 23-bit in-bin fraction, FP32
    rounding), so its relative error is about 1e-7 |v| / spread: 2e-3 is
    asserted, with smooth integrands whose spread inside a hypercube is
    1e-2 to 1e-1 of v.
"""
import math

import numpy as np
import pytest

import oracle as O
from gpu_helpers import BIN_TOL, PRECS, TOL, assert_hist_close, native, params_for, random_grid

pytestmark = pytest.mark.gpu

SIGMA_TOL = {"fp64": 1e-9, "fp32_acc64": 2e-3, "fp32_kahan": 2e-3}


def _make(V, family, d, N, n, prec, B, seed=0, iid=0, limit=0):
    p = params_for(family, d)
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, events_limit=limit, alpha=1.5, seed=seed,
                   integral_id=iid, precision=prec)
    ctx = V.vegas_create(cfg, family, p)
    V.vegas_set_strata(ctx, B)
    return ctx, p


def _expected_strata(B_req, d, n):
    """The stated rule, restated: B = the request (or the most) that keeps
    P = floor(n / 2^B) >= 2, at most 16 d and 31."""
    bmax = 0
    while n // 2 ** (bmax + 1) >= 2:
        bmax += 1
    B = bmax if B_req < 0 else min(B_req, bmax)
    B = min(B, 16 * d, 31)
    return B, n // 2 ** B


@pytest.mark.parametrize("B_req,d,n", [(-1, 8, 10_000_000), (-1, 1, 10 ** 9), (-1, 3, 2),
                                       (-1, 2, 3), (5, 4, 100_000), (40 // 2, 2, 1000),
                                       (-1, 20, 1 << 16), (31, 32, 10 ** 12)])
def test_strata_geometry_follows_the_rule(B_req, d, n):
    V = native()
    ctx, _ = _make(V, "sum", d, 8, n, "fp64", B_req)
    B, P, used = V.vegas_get_strata(ctx)
    eB, eP = _expected_strata(B_req, d, n)
    assert (B, P, used) == (eB, eP, eP * 2 ** eB)
    V.vegas_set_strata(ctx, 0)
    assert V.vegas_get_strata(ctx) == (0, 0, n)


def test_strata_rejects_bad_requests():
    V = native()
    from paper_2010_09341_gb300 import _native as nat
    ctx, _ = _make(V, "sum", 4, 8, 1000, "fp32_acc64", -1)
    for B in (-2, 32):
        with pytest.raises(nat.VegasError):
            V.vegas_set_strata(ctx, B)
    # stratified iterations are not sharded
    with pytest.raises(nat.VegasError):
        V.vegas_sample_shard(ctx, 0, 500)
    # FP32 modes: one hypercube's samples must fit one block's fixed-point cells
    ctx2, _ = _make(V, "sum", 1, 2, 10 ** 9, "fp32_acc64", 0)
    with pytest.raises(nat.VegasError):
        V.vegas_set_strata(ctx2, 1)


TRACE_CASES = [("gauss_sym", 4, 50, 100_000, -1), ("genz_osc", 8, 50, 200_003, -1),
               ("genz_prod", 9, 30, 77_777, 10), ("sum", 20, 10, 1 << 16, -1),
               ("genz_corner", 2, 64, 5_000, 3), ("lo", 3, 100, 300_000, -1)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("family,d,N,n,B", TRACE_CASES)
def test_strat_trace_bins_bit_exact(family, d, N, n, B, prec):
    V = native()
    ctx, p = _make(V, family, d, N, n, prec, B, seed=5, iid=9)
    e = random_grid(d, N, seed=d * N + 1)
    V.vegas_set_grid(ctx, e)
    Bt, P, used = V.vegas_get_strata(ctx)
    t = 2
    for s0, cnt in [(0, min(used, 1200)), (used - 900, 900)]:
        bins, x, w = V.vegas_trace(ctx, t, s0, cnt)
        bins, x, w = bins.cpu().numpy(), x.cpu().numpy(), w.cpu().numpy()
        ks = list(range(0, cnt, 5 if d > 8 else 3))
        vs, js = [], []
        for k in ks:
            ob, ox, J, f = O.sample_strat(d, N, e, family, p, 5, 9, t, Bt, P, s0 + k)
            assert np.array_equal(bins[k], ob), (k, bins[k], ob)
            atol = 4e-16 if prec == "fp64" else 3e-7
            assert np.allclose(x[k], ox, rtol=0, atol=atol)
            v = J * f
            vs.append(v if math.isfinite(v) else 0.0)
            js.append(abs(J))
        vs, js, ws = np.array(vs), np.array(js), w[ks]
        if prec == "fp64":
            # the cosine's argument differs by ~1e-16 (fused vs separate
            # multiply-add), an absolute error in f near its zeros
            atol = 1e-14 * js if family == "genz_osc" else 1e-300
            assert np.all(np.abs(ws - vs) <= 1e-13 * np.abs(vs) + atol)
        else:
            scale = np.mean(np.abs(vs))
            rel = 2e-4 if family == "lo" else 2e-5
            atol = 2e-6 * scale + (4e-6 * js if family == "genz_osc" else 0.0)
            ok = np.abs(ws - vs) <= rel * np.abs(vs) + atol
            if family == "lo":
                ok |= (vs == 0.0) != (ws == 0.0)
            assert np.all(ok)


ITER_CASES = [("gauss_sym", 4, 50, 100_000, -1), ("genz_osc", 8, 50, 200_003, -1),
              ("genz_gauss", 5, 50, 50_033, 12), ("genz_prod", 9, 30, 77_777, -1),
              ("sum", 10, 50, 65_536, -1), ("genz_gauss", 32, 20, 20_011, -1),
              ("gauss_sym", 1, 1024, 4099, -1), ("genz_corner", 3, 40, 300_000, 9)]


@pytest.mark.parametrize("warm", [False, True])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("family,d,N,n,B", ITER_CASES)
def test_strat_iteration_parity_on_shared_grid(family, d, N, n, B, prec, warm):
    V = native()
    ctx, p = _make(V, family, d, N, n, prec, B)
    if warm:
        V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    t = 1 if warm else 0
    Bt, P, used = V.vegas_get_strata(ctx)
    I, sigma, n_ok, n_nf = V.vegas_iterate(ctx)
    S1, S2, h = V.vegas_get_sums(ctx)
    acc = O.iterate_strat(d, N, e, family, p, 0, 0, t, Bt, P, threads=8)
    Io, var = O.strat_result(acc["S1"], acc["Q"], 2 ** Bt, P)
    tol = TOL[prec]
    assert n_ok == used
    assert n_nf == acc["n_nonfinite"]
    assert abs(I - Io) <= tol * abs(Io) + 1e-300, (I, Io)
    assert abs(S2 - acc["S2"]) <= tol * abs(acc["S2"]) + 1e-300
    assert_hist_close(h, acc["hist"], tol, BIN_TOL[prec])
    assert abs(sigma - math.sqrt(var)) <= SIGMA_TOL[prec] * math.sqrt(var), (sigma, math.sqrt(var))


def test_strat_full_run_fp64_matches_oracle_every_iteration():
    """Five stratified iterations with refinement, FP64: every iteration's
    estimate, sigma and refined grid, and the combination, against the oracle."""
    V = native()
    d, N, n, iters = 4, 50, 100_000, 5
    ctx, p = _make(V, "gauss_sym", d, N, n, "fp64", -1)
    Bt, P, used = V.vegas_get_strata(ctx)
    e = O.uniform_edges(d, N)
    its = []
    for t in range(iters):
        I, sigma, _, _ = V.vegas_iterate(ctx)
        acc = O.iterate_strat(d, N, e, "gauss_sym", p, 0, 0, t, Bt, P, threads=8)
        Io, var = O.strat_result(acc["S1"], acc["Q"], 2 ** Bt, P)
        assert abs(I - Io) <= 1e-12 * abs(Io)
        assert abs(sigma - math.sqrt(var)) <= 1e-9 * math.sqrt(var)
        its.append((Io, math.sqrt(var)))
        V.vegas_refine(ctx)
        e = O.refine(d, N, acc["hist"], e, 1.5)
        assert np.max(np.abs(V.vegas_get_grid(ctx) - e)) < 1e-12
    res = V.vegas_result(ctx)
    Ib, sb, c2 = O.combine([a for a, _ in its], [b for _, b in its])
    assert abs(res["I"] - Ib) <= 1e-12 * abs(Ib)
    assert abs(res["sigma"] - sb) <= 1e-9 * sb
    assert abs(res["I"] - math.erf(5.0) ** d) < 4 * res["sigma"]


@pytest.mark.parametrize("prec", PRECS)
def test_strat_events_limit_splits_launches_only(prec):
    V = native()
    d, N, n = 6, 50, 300_000
    a, _ = _make(V, "genz_gauss", d, N, n, prec, -1)
    b, _ = _make(V, "genz_gauss", d, N, n, prec, -1, limit=10_007)
    for _ in range(3):
        ra = V.vegas_step(a)
        rb = V.vegas_step(b)
        tol = TOL[prec]
        assert abs(ra[0] - rb[0]) <= tol * abs(ra[0])
        assert abs(ra[1] - rb[1]) <= SIGMA_TOL[prec] * ra[1]


def test_strat_full_size_d8_iteration():
    """The bench's d = 8 Gaussian at 1e7 samples, FP32 sampling with FP64 sums,
    stratified (2^22 hypercubes of 2 samples): the second iteration on the
    GPU's grid against the oracle (16 host threads)."""
    V = native()
    d, N, n = 8, 50, 10_000_000
    ctx, p = _make(V, "gauss_sym", d, N, n, "fp32_acc64", -1)
    V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    Bt, P, used = V.vegas_get_strata(ctx)
    assert (Bt, P) == (22, 2)
    I, sigma, n_ok, _ = V.vegas_iterate(ctx)
    acc = O.iterate_strat(d, N, e, "gauss_sym", p, 0, 0, 1, Bt, P, threads=16)
    Io, var = O.strat_result(acc["S1"], acc["Q"], 2 ** Bt, P)
    assert abs(I - Io) <= 1e-5 * abs(Io)
    assert abs(sigma - math.sqrt(var)) <= SIGMA_TOL["fp32_acc64"] * math.sqrt(var)
    assert abs(I - math.erf(5.0) ** d) < 5 * sigma


def test_strat_checkpoint_keeps_the_setting():
    V = native()
    d, N, n = 3, 30, 40_000
    a, _ = _make(V, "genz_prod", d, N, n, "fp64", 7)
    V.vegas_step(a)
    blob = V.vegas_export_state(a)
    b, _ = _make(V, "genz_prod", d, N, n, "fp64", 0)
    V.vegas_import_state(b, blob)
    assert V.vegas_get_strata(b) == V.vegas_get_strata(a)
    ra = V.vegas_iterate(a)
    rb = V.vegas_iterate(b)
    assert ra[0] == rb[0] and ra[1] == rb[1]


def test_strat_largest_hypercube_count():
    """The most hypercubes allowed, 2^31 of 2 samples (n = 2^32 + 12345 requested,
    2^32 used): sample indices pass 2^32 inside the iteration.  Bins of the
    first and last samples bit-exact against the oracle, the estimate within
    5 sigma of the closed form."""
    V = native()
    d, N, n = 4, 50, (1 << 32) + 12345
    ctx, p = _make(V, "gauss_sym", d, N, n, "fp32_acc64", -1)
    Bt, P, used = V.vegas_get_strata(ctx)
    assert (Bt, P, used) == (31, 2, 1 << 32)
    e = O.uniform_edges(d, N)
    for s0 in (0, used - 600):
        bins, x, w = V.vegas_trace(ctx, 0, s0, 600)
        bins = bins.cpu().numpy()
        for k in range(0, 600, 7):
            ob, _, _, _ = O.sample_strat(d, N, e, "gauss_sym", p, 0, 0, 0, Bt, P, s0 + k)
            assert np.array_equal(bins[k], ob)
    I, sigma, n_ok, _ = V.vegas_iterate(ctx)
    assert n_ok == used
    assert abs(I - math.erf(5.0) ** d) < 5 * sigma
