"""The LO toy on a tabulated density grid (VEGAS_F_LO_PDF, vegas_set_pdf_grid)
against the FP64 oracle's grid interpolation.

Tolerances: bins bit-exact; FP64 per-sample values 1e-13 relative and
iteration results 1e-12; FP32 per iteration 1e-5 as for every family, per
sample 2e-4 (the interpolation's cell index comes from an FP32 log2, which
moves the point by ~1e-6 of a cell inside a C1 interpolant, on top of the LO
toy's Breit-Wigner slope).
"""
import math

import numpy as np
import pytest

import oracle as O
from gpu_helpers import PRECS, native
from paper_2010_09341_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_IT = {"fp64": 1e-12, "fp32_acc64": 1e-5, "fp32_kahan": 1e-5}


def _grid(nx=96, nq=48, b1=0.5):
    import torch
    xg, u0, u1, v0, v1 = W.pdf_grid(nx, nq, b1=b1)
    O.set_pdf_grid(xg, u0, u1, v0, v1)
    return torch.from_numpy(xg).cuda(), (u0, u1, v0, v1)


def _make(V, N, n, prec, grid, seed=0, iid=0, strata=0, limit=0):
    cfg = V.Config(n_dim=3, n_events=n, n_bins=N, events_limit=limit, alpha=1.5, seed=seed,
                   integral_id=iid, precision=prec)
    ctx = V.vegas_create(cfg, "lo_pdf", W.lo_params())
    if strata:
        V.vegas_set_strata(ctx, strata)
    V.vegas_set_pdf_grid(ctx, grid[0], *grid[1])
    return ctx


def _adapted_edges(V, grid, N):
    """A grid adapted to the integrand by three FP64 iterations (most points of a
    uniform or random grid fall outside the invariant-mass window)."""
    a = _make(V, N, 200_000, "fp64", grid, seed=7)
    for _ in range(3):
        V.vegas_step(a)
    return V.vegas_get_grid(a)


@pytest.mark.parametrize("prec", PRECS)
def test_pdf_trace_bins_bit_exact(prec):
    V = native()
    grid = _grid()
    N = 100
    ctx = _make(V, N, 1000, prec, grid, seed=3, iid=5)
    e = _adapted_edges(V, grid, N)
    V.vegas_set_grid(ctx, e)
    p = W.lo_params()
    s0, cnt = (1 << 32) - 1000, 2000
    bins, x, w = V.vegas_trace(ctx, 1, s0, cnt)
    bins, x, w = bins.cpu().numpy(), x.cpu().numpy(), w.cpu().numpy()
    vs = []
    for k in range(0, cnt, 2):
        ob, ox, J, f = O.sample(3, N, e, "lo_pdf", p, 3, 5, 1, s0 + k)
        assert np.array_equal(bins[k], ob)
        vs.append(J * f)
    vs = np.array(vs)
    ws = w[::2]
    assert np.count_nonzero(vs) > 50
    if prec == "fp64":
        assert np.all(np.abs(ws - vs) <= 1e-13 * np.abs(vs) + 1e-300)
    else:
        ok = np.abs(ws - vs) <= 2e-4 * np.abs(vs) + 2e-6 * np.mean(np.abs(vs))
        ok |= (vs == 0.0) != (ws == 0.0)   # cut edges within FP32 rounding of a point
        assert np.all(ok)
        assert np.count_nonzero((vs == 0.0) != (ws == 0.0)) <= 2


@pytest.mark.parametrize("strata", [0, -1])
@pytest.mark.parametrize("prec", PRECS)
def test_pdf_iteration_parity_on_shared_grid(prec, strata):
    V = native()
    grid = _grid()
    N, n = 100, 400_000
    ctx = _make(V, N, n, prec, grid, strata=strata)
    V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    I, sigma, n_ok, _ = V.vegas_iterate(ctx)
    p = W.lo_params()
    if strata:
        Bt, P, used = V.vegas_get_strata(ctx)
        acc = O.iterate_strat(3, N, e, "lo_pdf", p, 0, 0, 1, Bt, P, threads=8)
        Io, var = O.strat_result(acc["S1"], acc["Q"], 2 ** Bt, P)
    else:
        acc = O.iterate(3, N, e, "lo_pdf", p, 0, 0, 1, n, threads=8)
        Io, var = O.iteration_result(acc["S1"], acc["S2"], n)
    tol = TOL_IT[prec]
    assert abs(I - Io) <= tol * abs(Io), (I, Io)
    if prec == "fp64":
        assert abs(sigma - math.sqrt(var)) <= 1e-9 * math.sqrt(var)


@pytest.mark.parametrize("strata", [0, -1])
@pytest.mark.parametrize("prec", PRECS)
def test_pdf_odd_cell_count_and_small_odd_grid(prec, strata):
    """d N = 99 cells (the FP32 cells end 4 bytes past an 8-byte boundary: the
    density grid after them starts at the next 16-byte boundary) and a 15 x 9
    knot grid (odd in both directions; the FP32 path's pairs reach the last
    padded column): the iteration after one refinement equals the oracle's."""
    V = native()
    grid = _grid(nx=15, nq=9)
    N, n = 33, 150_001
    ctx = _make(V, N, n, prec, grid, strata=strata)
    V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    I, sigma, n_ok, _ = V.vegas_iterate(ctx)
    p = W.lo_params()
    if strata:
        Bt, P, used = V.vegas_get_strata(ctx)
        acc = O.iterate_strat(3, N, e, "lo_pdf", p, 0, 0, 1, Bt, P, threads=8)
        Io, var = O.strat_result(acc["S1"], acc["Q"], 2 ** Bt, P)
    else:
        acc = O.iterate(3, N, e, "lo_pdf", p, 0, 0, 1, n, threads=8)
        Io, var = O.iteration_result(acc["S1"], acc["S2"], n)
    tol = TOL_IT[prec]
    assert Io != 0.0
    assert abs(I - Io) <= tol * abs(Io), (I, Io)


def test_pdf_full_run_fp64_matches_oracle_every_iteration():
    V = native()
    grid = _grid()
    N, n = 100, 200_000
    ctx = _make(V, N, n, "fp64", grid)
    p = W.lo_params()
    e = O.uniform_edges(3, N)
    for t in range(4):
        I, sigma, _, _ = V.vegas_iterate(ctx)
        acc = O.iterate(3, N, e, "lo_pdf", p, 0, 0, t, n, threads=8)
        Io, var = O.iteration_result(acc["S1"], acc["S2"], n)
        assert abs(I - Io) <= 1e-12 * abs(Io)
        V.vegas_refine(ctx)
        e = O.refine(3, N, acc["hist"], e, 1.5)
        assert np.max(np.abs(V.vegas_get_grid(ctx) - e)) < 1e-12


def test_pdf_grid_of_the_lo_density_reproduces_the_lo_toy():
    """A grid of the LO toy's own density (no scale dependence, 160 knots in
    ln x): on the first iteration (the same uniform grid, so the same samples)
    the gridded integrand's estimate equals the analytic family's to the
    interpolation error; after refinement the two runs sample different
    points and agree within their errors."""
    V = native()
    grid = _grid(160, 8, b1=0.0)
    N, n = 100, 2_000_000
    a = _make(V, N, n, "fp64", grid)
    cfg = V.Config(n_dim=3, n_events=n, n_bins=N, alpha=1.5, seed=0, integral_id=0, precision="fp64")
    b = V.vegas_create(cfg, "lo", W.lo_params())
    ra = V.vegas_step(a)
    rb = V.vegas_step(b)
    assert abs(ra[0] - rb[0]) <= 3e-4 * abs(rb[0])
    for _ in range(4):
        V.vegas_step(a)
        V.vegas_step(b)
    ca, cb = V.vegas_result(a), V.vegas_result(b)
    assert abs(ca["I"] - cb["I"]) <= 4 * math.hypot(ca["sigma"], cb["sigma"]) + 3e-4 * abs(cb["I"])


def test_pdf_grid_required_and_validated():
    V = native()
    from paper_2010_09341_gb300 import _native as nat
    import torch
    cfg = V.Config(n_dim=3, n_events=1000, n_bins=20, precision="fp32_kahan")
    ctx = V.vegas_create(cfg, "lo_pdf", W.lo_params())
    with pytest.raises(nat.VegasError):
        V.vegas_iterate(ctx)          # no grid yet
    big = torch.zeros((100, 62), dtype=torch.float64, device="cuda")   # 6200 > 6144 values
    with pytest.raises(nat.VegasError):
        V.vegas_set_pdf_grid(ctx, big, -10.0, 0.0, 1.0, 10.0)
    with pytest.raises(nat.VegasError):
        V.vegas_set_pdf_grid(ctx, torch.zeros((4, 4), dtype=torch.float64, device="cuda"), 0.0, -1.0, 1.0, 2.0)
    other = V.vegas_create(cfg, "lo", W.lo_params())
    with pytest.raises(nat.VegasError):
        V.vegas_set_pdf_grid(other, torch.zeros((4, 4), dtype=torch.float64, device="cuda"), -1.0, 0.0, 1.0, 2.0)
    # the batched form does not take the family
    b = V.Batch(max_slots=4, pool_bytes=1 << 20, precision="fp32_kahan")
    with pytest.raises(nat.VegasError):
        b.add(cfg, "lo_pdf", W.lo_params())
    b.close()


def test_pdf_full_size_iteration_fp32_kahan():
    """1e7 samples per iteration, FP32 with Kahan sums: the third iteration on
    the GPU's grid against the oracle (16 host threads)."""
    V = native()
    grid = _grid()
    N, n = 100, 10_000_000
    ctx = _make(V, N, n, "fp32_kahan", grid)
    V.vegas_step(ctx)
    V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    I, sigma, _, _ = V.vegas_iterate(ctx)
    acc = O.iterate(3, N, e, "lo_pdf", W.lo_params(), 0, 0, 2, n, threads=16)
    Io, var = O.iteration_result(acc["S1"], acc["S2"], n)
    assert abs(I - Io) <= 1e-5 * abs(Io)
