"""GPU path (C ABI, sm_103a kernels) against the FP64 oracle.

Tolerances (stated per quantity):
  * bin indices and Philox words: bit-exact (integer work);
  * iteration estimate I_t: relative 1e-12 for the FP64 path, 1e-5 for the
    FP32 paths, on the same input grid;
  * S2: same tolerances; histograms row by row: every bin within the same
    tolerance of its row's sum, bins holding >= 1e-3 of their row within
    1e-12 (FP64) / 1e-4 (FP32 fixed-point cells) of their own value;
  * refined edges from identical histograms: absolute 1e-13.
"""
import ctypes
import math

import numpy as np
import pytest

import closed_forms as CF
import oracle as O
from gpu_helpers import BIN_TOL, PRECS, TOL, assert_hist_close, curand_ref_lib, native, params_for, random_grid

pytestmark = pytest.mark.gpu


def _make(V, family, d, N, n, prec, seed=0, iid=0, limit=0, alpha=1.5, params=None):
    p = params_for(family, d) if params is None else params
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, events_limit=limit, alpha=alpha, seed=seed,
                   integral_id=iid, precision=prec)
    return V.vegas_create(cfg, family, p), p


# ------------------------------------------------------------------ Philox
def test_device_philox_matches_oracle_and_curand():
    V = native()
    import torch
    rng = np.random.default_rng(11)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = 0
    key[:16] = 0
    ctr[16:32] = 0xFFFFFFFF
    key[16:32] = 0xFFFFFFFF
    tc = torch.from_numpy(ctr.view(np.int32)).cuda()
    tk = torch.from_numpy(key.view(np.int32)).cuda()
    mine = V.vegas_philox(tc, tk).cpu().numpy().view(np.uint32)
    torch.cuda.synchronize()
    ref = O.philox_many(ctr, key)
    assert np.array_equal(mine, ref)
    lib = curand_ref_lib()
    out = torch.empty_like(tc)
    assert lib.curand_ref_philox(ctypes.c_void_p(tc.data_ptr()), ctypes.c_void_p(tk.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), n) == 0
    assert np.array_equal(mine, out.cpu().numpy().view(np.uint32))


# ---------------------------------------------------------- per-sample trace
TRACE_CASES = [("gauss_sym", 4, 50), ("genz_osc", 8, 50), ("genz_gauss", 5, 17),
               ("genz_prod", 9, 64), ("genz_corner", 16, 50), ("sum", 20, 10),
               ("lo", 3, 100), ("const", 32, 2)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("family,d,N", TRACE_CASES)
def test_trace_bins_bit_exact(family, d, N, prec):
    V = native()
    ctx, p = _make(V, family, d, N, 1000, prec, seed=5, iid=9)
    e = random_grid(d, N, seed=d * N)
    V.vegas_set_grid(ctx, e)
    t = 3
    starts = [(0, 1500), ((1 << 32) - 700, 1400)]  # crosses the s_hi word
    for s0, cnt in starts:
        bins, x, w = V.vegas_trace(ctx, t, s0, cnt)
        bins, x, w = bins.cpu().numpy(), x.cpu().numpy(), w.cpu().numpy()
        ks = list(range(0, cnt, 7 if d > 8 else 3))
        vs = []
        js = []
        for k in ks:
            ob, ox, J, f = O.sample(d, N, e, family, p, 5, 9, t, s0 + k)
            assert np.array_equal(bins[k], ob), (k, bins[k], ob)
            if prec == "fp64":
                assert np.allclose(x[k], ox, rtol=0, atol=4e-16)
            else:
                assert np.allclose(x[k], ox, rtol=0, atol=3e-7)
            vs.append(J * f)
            js.append(abs(J))
        vs = np.array(vs)
        js = np.array(js)
        ws = w[ks]
        if prec == "fp64":
            assert np.all(np.abs(ws - vs) <= 1e-13 * np.abs(vs) + 1e-300)
        else:
            # FP32 per-sample error is relative to the integrand's scale: where
            # f is tiny (tails, zeros of cos, (1-x)^3 near x = 1) cancellation
            # makes its own relative error large.
            # The LO toy's Breit-Wigner has d ln f / d ln shat ~ 37 on its
            # shoulders, and FP32 shat = X1 X2 s0 carries up to ~5e-7 of
            # rounding (each coordinate ~2e-7, two products): up to 2e-5 in f,
            # so its per-sample bound is 5e-5.
            scale = np.mean(np.abs(vs))
            # The oscillatory family's FP32 cosine has an absolute error (its
            # argument carries ~1e-6 of FP32 rounding), which J multiplies.
            rel = 5e-5 if family == "lo" else 2e-5
            atol = 2e-6 * scale + (4e-6 * js if family == "genz_osc" else 0.0)
            ok = np.abs(ws - vs) <= rel * np.abs(vs) + atol
            assert np.all(ok), np.max(np.abs(ws - vs) / (np.abs(vs) + scale))
            if family == "lo":  # the cuts classify every traced point as the oracle does
                assert np.array_equal(vs == 0.0, ws == 0.0)


# --------------------------------------------------------------- iteration
ITER_CASES = [("gauss_sym", 4, 50, 100_000), ("genz_osc", 8, 50, 200_003),
              ("genz_gauss", 5, 50, 50_033), ("genz_prod", 9, 30, 77_777),
              ("genz_corner", 6, 50, 100_000), ("sum", 10, 50, 65_536),
              ("lo", 3, 100, 300_000), ("const", 3, 2, 2), ("gauss_sym", 1, 1024, 4099),
              ("genz_gauss", 32, 20, 20_011)]


def _compare_iteration(V, ctx, p, family, d, N, n, prec, e, t, seed=0, iid=0):
    I, sigma, n_ok, n_nf = V.vegas_iterate(ctx)
    S1, S2, h = V.vegas_get_sums(ctx)
    acc = O.iterate(d, N, e, family, p, seed, iid, t, n, threads=8)
    Io, var = O.iteration_result(acc["S1"], acc["S2"], n - acc["n_nonfinite"])
    tol = TOL[prec]
    assert n_nf == acc["n_nonfinite"] == 0
    assert abs(I - Io) <= tol * abs(Io) + 1e-300, (I, Io)
    assert abs(S2 - acc["S2"]) <= tol * abs(acc["S2"]) + 1e-300
    assert_hist_close(h, acc["hist"], tol, BIN_TOL[prec])
    if var > 0 and prec == "fp64":
        assert abs(sigma - math.sqrt(var)) <= 1e-9 * math.sqrt(var)
    return acc


@pytest.mark.parametrize("warm", [False, True])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("family,d,N,n", ITER_CASES)
def test_iteration_parity_on_shared_grid(family, d, N, n, prec, warm):
    """warm: one iteration runs first, so the FP32 modes accumulate this one
    in fixed-point histogram cells scaled from it (the first iteration of a
    context uses FP32 cells)."""
    V = native()
    ctx, p = _make(V, family, d, N, n, prec)
    t = 0
    if warm:
        V.vegas_iterate(ctx)
        t = 1
    e = random_grid(d, N, seed=1, spread=0.5)
    V.vegas_set_grid(ctx, e)
    _compare_iteration(V, ctx, p, family, d, N, n, prec, e, t)


def _lo_grids(V, d, N):
    """The LO toy's grids for the cut-flip census: uniform, a random one, and
    the grid six FP64 iterations of 1e6 samples adapt to."""
    ctx, _ = _make(V, "lo", d, N, 1_000_000, "fp64")
    for _ in range(6):
        V.vegas_step(ctx)
    return {"uniform": O.uniform_edges(d, N), "random": random_grid(d, N, seed=1, spread=0.5),
            "adapted": V.vegas_get_grid(ctx)}


@pytest.mark.parametrize("prec", ["fp32_acc64", "fp32_kahan"])
def test_lo_fp32_cut_flips(prec):
    """The LO toy's hard cuts (the mass window and |cos theta| < 0.95) in FP32:
    every one of 3e5 samples is traced on three grids and classified (inside
    or outside the cuts) by the GPU and by the oracle.  The samples classified
    differently (flips) are counted and their weight bounded; the rest of the
    iteration, and the whole of it, agree with the oracle to 1e-5."""
    V = native()
    d, N, n = 3, 100, 300_000
    p = params_for("lo", d)
    for name, e in _lo_grids(V, d, N).items():
        ctx, _ = _make(V, "lo", d, N, n, prec, params=p)
        V.vegas_set_grid(ctx, e)
        I, _, _, n_nf = V.vegas_iterate(ctx)
        S1, S2, h = V.vegas_get_sums(ctx)
        bins, _, w = V.vegas_trace(ctx, 0, 0, n)
        bins, w = bins.cpu().numpy(), w.cpu().numpy()
        ob, _, v = O.trace(d, N, e, "lo", p, 0, 0, 0, 0, n, threads=16)
        assert np.array_equal(bins, ob), name
        flip = (w == 0.0) != (v == 0.0)
        So = v.sum()
        # measured: no flips on these grids (FP32 X carries ~2e-7 relative)
        assert flip.sum() <= 2, (name, int(flip.sum()))
        assert np.abs(v[flip]).sum() + np.abs(w[flip]).sum() <= 1e-6 * abs(So), name
        keep = ~flip
        assert abs(w[keep].sum() - v[keep].sum()) <= 1e-5 * abs(v[keep].sum()), name
        acc = O.iterate(d, N, e, "lo", p, 0, 0, 0, n, threads=16)
        assert n_nf == acc["n_nonfinite"] == 0
        assert abs(I - acc["S1"] / n) <= 1e-5 * abs(acc["S1"] / n), (name, I, acc["S1"] / n)
        assert abs(S2 - acc["S2"]) <= 1e-5 * acc["S2"], name
        assert_hist_close(h, acc["hist"], 1e-5, BIN_TOL[prec])


def test_refine_parity_from_identical_histograms():
    V = native()
    for prec in PRECS:
        d, N, n = 6, 50, 200_000
        ctx, p = _make(V, "genz_gauss", d, N, n, prec)
        e = random_grid(d, N, seed=3, spread=0.3)
        V.vegas_set_grid(ctx, e)
        V.vegas_iterate(ctx)
        _, _, h = V.vegas_get_sums(ctx)
        V.vegas_refine(ctx)
        eg = V.vegas_get_grid(ctx)
        eo = O.refine(d, N, h, e, 1.5)
        assert np.max(np.abs(eg - eo)) < 1e-13
        assert np.all(eg[:, 0] == 0.0) and np.all(eg[:, -1] == 1.0)
        assert np.all(np.diff(eg, axis=1) >= 0)


def test_full_run_fp64_matches_oracle_every_iteration():
    """Configuration: d = 4 symmetric Gaussian a = 0.1, 50 bins, 1e5 samples,
    5 iterations, alpha = 1.5, seed 0, FP64 throughout.  Every iteration,
    the refined grids and the combination agree with the oracle to 1e-12; the
    result is within 3 sigma of erf(5)^4."""
    V = native()
    d, N, n, m = 4, 50, 100_000, 5
    ctx, p = _make(V, "gauss_sym", d, N, n, "fp64")
    res = V.vegas_run(ctx, m)
    ref = O.integrate(d, N, "gauss_sym", p, n, m, alpha=1.5, seed=0)
    for (I, s, _, _), (Io, so) in zip(res["iters"], ref["iters"]):
        assert abs(I - Io) <= 1e-12 * abs(Io)
        assert abs(s - so) <= 1e-9 * so
    assert abs(res["I"] - ref["I"]) <= 1e-12 * abs(ref["I"])
    assert abs(res["sigma"] - ref["sigma"]) <= 1e-9 * ref["sigma"]
    assert abs(res["chi2_dof"] - ref["chi2_dof"]) <= 1e-6 * max(1.0, ref["chi2_dof"])
    assert abs(res["I"] - CF.gauss_sym(4, 0.1)) < 3 * res["sigma"]


@pytest.mark.parametrize("prec", ["fp32_acc64", "fp32_kahan"])
def test_fp32_run_per_iteration_on_gpu_grid(prec):
    """FP32 runs diverge from FP64 ones through the grid; per iteration, with
    the oracle fed the GPU's own grid, the estimates agree to 1e-5, and the
    combined result is within 3 sigma of the closed form."""
    V = native()
    d, N, n, m = 8, 50, 200_000, 6
    ctx, p = _make(V, "gauss_sym", d, N, n, prec)
    for t in range(m):
        e = V.vegas_get_grid(ctx)
        _compare_iteration(V, ctx, p, "gauss_sym", d, N, n, prec, e, t)
        V.vegas_refine(ctx)
    r = V.vegas_result(ctx)
    assert r["n_iter"] == m
    assert abs(r["I"] - CF.gauss_sym(8, 0.1)) < 3 * r["sigma"]


def test_events_limit_split_matches_single_launch():
    V = native()
    d, N, n = 5, 50, 123_457
    a, p = _make(V, "genz_prod", d, N, n, "fp64")
    b, _ = _make(V, "genz_prod", d, N, n, "fp64", limit=10_000)
    ra = V.vegas_run(a, 3)
    rb = V.vegas_run(b, 3)
    for x, y in zip(ra["iters"], rb["iters"]):
        assert abs(x[0] - y[0]) <= 1e-13 * abs(x[0])
    assert np.max(np.abs(V.vegas_get_grid(a) - V.vegas_get_grid(b))) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_checkpoint_resume(prec):
    """Export after 3 iterations, continue 2 more; a fresh context that imports
    the blob and runs 2 iterations gives the same results.  Shared-memory
    atomics add in a run-dependent order, so equality holds to the path's
    rounding (FP64 1e-12, FP32 1e-6), not bit for bit."""
    V = native()
    d, N, n = 6, 40, 60_000
    a, p = _make(V, "genz_gauss", d, N, n, prec)
    V.vegas_run(a, 3)
    V.vegas_refine(a)
    blob = V.vegas_export_state(a)
    ra = V.vegas_run(a, 2)
    b, _ = _make(V, "genz_gauss", d, N, n, prec)
    V.vegas_import_state(b, blob)
    assert V.vegas_get_iteration(b) == 3
    rb = V.vegas_run(b, 2)
    tol = 1e-12 if prec == "fp64" else 1e-6
    for x, y in zip(ra["iters"], rb["iters"]):
        assert abs(x[0] - y[0]) <= tol * abs(x[0]) and x[2:] == y[2:]
    assert np.max(np.abs(V.vegas_get_grid(a) - V.vegas_get_grid(b))) < (1e-13 if prec == "fp64" else 1e-6)
    assert rb["n_iter"] == 5 and abs(ra["I"] - rb["I"]) <= tol * abs(ra["I"])


def test_integrator_paper_usage_sum_toy():
    """The usage of Sec. 3.1: n_dim = 10, n_events = 1e6, events_limit = 1e5,
    f = sum x_i, 5 iterations; the exact value is 5."""
    V = native()
    it = V.Integrator(n_dim=10, n_events=10 ** 6, events_limit=10 ** 5, precision="fp32_kahan")
    it.compile("sum")
    r = it.run_integration(n_iter=5)
    assert abs(r["I"] - 5.0) < 3 * r["sigma"]
    assert r["sigma"] < 1e-3


def test_invalid_arguments_rejected():
    V = native()
    from paper_2010_09341_gb300 import _native as nat
    with pytest.raises(nat.VegasError):
        V.vegas_create(V.Config(n_dim=3, n_events=1000), "genz_gauss", [1.0, 2.0])
    with pytest.raises(nat.VegasError):
        V.vegas_create(V.Config(n_dim=4, n_events=1000), "lo", params_for("lo", 3))
    ctx, _ = _make(V, "gauss_sym", 2, 10, 1000, "fp64")
    bad = O.uniform_edges(2, 10)
    bad[0, 3] = 0.9
    with pytest.raises(nat.VegasError):
        V.vegas_set_grid(ctx, bad)


# -------------------------------------------------------- full-size checks
@pytest.mark.parametrize("family", ["gauss_sym", "genz_osc"])
@pytest.mark.parametrize("prec", ["fp32_acc64", "fp32_kahan", "fp64"])
def test_full_size_d8_iteration(family, prec):
    """d = 8, 50 bins, 1e7 samples, the launch configuration the benchmark
    times (after a first iteration, as in the benchmark's steady state): the
    whole iteration against the oracle run on all host cores."""
    V = native()
    d, N, n = 8, 50, 10_000_000
    p = params_for(family, d, seed=1) if family == "genz_osc" else params_for(family, d)
    ctx, _ = _make(V, family, d, N, n, prec, params=p)
    V.vegas_iterate(ctx)
    V.vegas_refine(ctx)
    e = V.vegas_get_grid(ctx)
    _compare_iteration(V, ctx, p, family, d, N, n, prec, e, 1)


def test_full_size_lo_iteration():
    """d = 3 LO toy, 100 bins, 1e8 samples, FP32 with Kahan sums, after one
    iteration (fixed-point histogram cells): estimate and S2 within 1e-5,
    histograms row by row as in the iteration parity tests."""
    V = native()
    d, N, n = 3, 100, 100_000_000
    ctx, p = _make(V, "lo", d, N, n, "fp32_kahan")
    V.vegas_iterate(ctx)
    V.vegas_refine(ctx)
    e = V.vegas_get_grid(ctx)
    I, _, _, _ = V.vegas_iterate(ctx)
    _, S2, h = V.vegas_get_sums(ctx)
    acc = O.iterate(d, N, e, "lo", p, 0, 0, 1, n, threads=16)
    Io = acc["S1"] / n
    assert abs(I - Io) <= 1e-5 * abs(Io)
    assert abs(S2 - acc["S2"]) <= 1e-5 * acc["S2"]
    assert_hist_close(h, acc["hist"], 1e-5, BIN_TOL["fp32_kahan"])


@pytest.mark.parametrize("prec", ["fp32_acc64", "fp32_kahan"])
def test_fp32_tiny_integral_corner_d16(prec):
    """Genz corner peak in d = 16 has an integral near 1e-20 while f reaches 1:
    the FP32 paths rescale v by powers of two each iteration so that v^2 stays
    in FP32's normal range.  The result must agree with the closed form."""
    V = native()
    d, N, n = 16, 50, 1_000_000
    p = params_for("genz_corner", d, seed=5)
    ctx, _ = _make(V, "genz_corner", d, N, n, prec, params=p)
    r = V.vegas_run(ctx, 8)
    exact = CF.genz_corner_laplace(p)
    assert abs(r["I"] - exact) < 4 * r["sigma"], (r["I"], exact, r["sigma"])
    assert r["sigma"] < 0.05 * exact


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_two_shards_equal_one_context(prec):
    """Two contexts on one GPU take the two halves of every iteration; their
    accumulators are summed (as an all-reduce would) and both finalize and
    refine: the results equal a single context's, and the shards' grids stay
    identical."""
    V = native()
    import torch
    d, N, n = 6, 40, 300_001
    p = params_for("genz_prod", d)
    ref, _ = _make(V, "genz_prod", d, N, n, prec, params=p)
    sh = [_make(V, "genz_prod", d, N, n, prec, params=p)[0] for _ in range(2)]
    tol = TOL[prec]
    for t in range(3):
        Ir = V.vegas_iterate(ref)[0]
        half = n // 2
        V.vegas_sample_shard(sh[0], 0, half)
        V.vegas_sample_shard(sh[1], half, n - half)
        (a, na), (b, nb) = V.vegas_accumulators(sh[0]), V.vegas_accumulators(sh[1])
        tot, ntot = a + b, na + nb
        for s_, n_ in ((a, na), (b, nb)):
            s_.copy_(tot)
            n_.copy_(ntot)
        I0 = V.vegas_finalize(sh[0])[0]
        I1 = V.vegas_finalize(sh[1])[0]
        assert I0 == I1
        assert abs(I0 - Ir) <= tol * abs(Ir)
        for c in (ref, sh[0], sh[1]):
            V.vegas_refine(c)
        assert np.array_equal(V.vegas_get_grid(sh[0]), V.vegas_get_grid(sh[1]))


@pytest.mark.parametrize("prec", PRECS)
def test_step_equals_iterate_then_refine(prec):
    """vegas_step (finalize and refinement in one launch) gives the same
    iterations and grids as vegas_iterate followed by vegas_refine."""
    V = native()
    d, N, n = 7, 50, 200_000
    p = params_for("genz_gauss", d)
    a, _ = _make(V, "genz_gauss", d, N, n, prec, params=p)
    b, _ = _make(V, "genz_gauss", d, N, n, prec, params=p)
    tol = TOL[prec]
    for _ in range(4):
        Ia = V.vegas_step(a)[0]
        Ib = V.vegas_iterate(b)[0]
        V.vegas_refine(b)
        assert abs(Ia - Ib) <= tol * abs(Ib)
        ea, eb = V.vegas_get_grid(a), V.vegas_get_grid(b)
        assert np.max(np.abs(ea - eb)) <= (1e-13 if prec == "fp64" else 1e-5)
    ra, rb = V.vegas_result(a), V.vegas_result(b)
    assert abs(ra["I"] - rb["I"]) <= tol * abs(rb["I"]) and ra["n_iter"] == rb["n_iter"] == 4


def _tight_combination_params():
    # Genz Gaussian with c = 1e-3: f = exp(-1e-6 sum (x - w)^2), so one
    # iteration of 1e5 samples has sigma / I ~ 1e-9 and (I / sigma)^2 ~ 1e18:
    # a one-pass chi^2 (sum w I^2 - Ibar sum w I) would keep no digit of it.
    return np.array([1e-3, 1e-3, 0.3, 0.6])


def test_combination_chi2_without_cancellation():
    """The running combination against the oracle's two-pass one on the same
    iteration records (FP64, five iterations of an integrand whose iterations
    agree to nine digits): Ibar to 1e-15, sigma to 1e-12, chi^2/dof to 1e-6."""
    V = native()
    d, N, n, m = 2, 20, 100_000, 5
    p = _tight_combination_params()
    # alpha = 0 keeps the uniform grid (a refined grid would carry the bin
    # counts' sampling noise into J, and sigma / I would rise to ~1e-5)
    ctx, _ = _make(V, "genz_gauss", d, N, n, "fp64", params=p, alpha=0.0)
    r = V.vegas_run(ctx, m)
    I = np.array([x[0] for x in r["iters"]])
    s = np.array([x[1] for x in r["iters"]])
    assert np.max(s / I) < 1e-8
    Io, so, co = O.combine(I, s)
    assert abs(r["I"] - Io) <= 1e-15 * abs(Io)
    assert abs(r["sigma"] - so) <= 1e-12 * so
    assert co > 0.05 and abs(r["chi2_dof"] - co) <= 1e-6 * co, (r["chi2_dof"], co)
    # the batched form keeps the same running sums.  It runs in the FP32
    # modes only, whose sums cannot resolve a relative variance per sample of
    # 1e-12; with c = 0.1 (relative variance ~1e-6) and 1e7 samples per
    # iteration sigma / I ~ 3e-7, so (I / sigma)^2 ~ 1e13, where a one-pass
    # chi^2 would keep about two digits.
    n = 10_000_000
    p = np.array([0.1, 0.1, 0.3, 0.6])
    b = V.Batch(max_slots=2, pool_bytes=4 << 20, precision="fp32_acc64")
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=0.0, seed=0, integral_id=0, precision="fp32_acc64")
    slot = b.add(cfg, "genz_gauss", p)
    its = []
    for _ in range(m):
        b.step()
        its.append(b.wait()[slot])
    Ib = np.array([x["I_t"] for x in its])
    sb = np.array([x["sigma_t"] for x in its])
    assert np.max(sb / Ib) < 1e-6
    Io, so, co = O.combine(Ib, sb)
    last = its[-1]
    assert abs(last["I"] - Io) <= 1e-15 * abs(Io)
    assert abs(last["sigma"] - so) <= 1e-12 * so
    assert co > 0.05 and abs(last["chi2_dof"] - co) <= 1e-6 * co, (last["chi2_dof"], co)
    b.close()


@pytest.mark.parametrize("prec", PRECS)
def test_histogram_rows_sum_to_s2(prec):
    """Every sample adds its (J f)^2 once to one bin of every dimension, so each
    row of an iteration's histograms sums to S2: a lost or doubled shared-memory
    update in any dimension would break it.  Three iterations (the FP32 modes'
    first in FP32 cells, then fixed-point cells), 1e6 + 3 samples, d = 8: rows
    to 1e-12 (FP64) and 1e-6 (FP32: each v^2 is rounded to 2^-19 of the mean
    in a fixed-point cell)."""
    V = native()
    d, N, n = 8, 50, 1_000_003
    ctx, _ = _make(V, "genz_gauss", d, N, n, prec)
    tol = 1e-12 if prec == "fp64" else 1e-6
    for _ in range(3):
        V.vegas_iterate(ctx)
        _, S2, h = V.vegas_get_sums(ctx)
        rows = np.asarray(h).reshape(d, N).sum(axis=1)
        assert np.all(np.abs(rows - S2) <= tol * S2), (rows / S2 - 1.0)
        V.vegas_refine(ctx)
