"""vegas_step_many: one iteration of several integrals, their iteration
results and refinements in one launch, against vegas_step on twin contexts
and against the FP64 oracle.

Tolerances: the twins run the same kernels on the same inputs; only the order
of the FP64 atomic additions of the block sums differs.  The first iteration
(the same uniform grid) agrees to 1e-13.  Later iterations sample refined
grids whose FP64 edges differ at the rounding level, and in the FP32 modes
an edge that moves across a float rounding boundary moves the samples of its
bin by one float ulp (6e-8 relative; I by about 1e-9 per such entry): FP32
1e-6 on I and sigma and 1e-7 on the edges, FP64 1e-10; chi^2/dof to that
times its cancelled terms, (I/sigma)^2/(m - 1).  The first iteration
against the oracle: as the plain parity tests (FP64 1e-12).
"""
import math

import numpy as np
import pytest

import oracle as O
from gpu_helpers import native, params_for

pytestmark = pytest.mark.gpu

MIX = [("gauss_sym", 8, 50, 300_000, "fp32_acc64", 0),
       ("genz_osc", 5, 40, 200_000, "fp64", 0),
       ("genz_corner", 3, 30, 150_000, "fp32_kahan", -1),
       ("genz_prod", 12, 20, 100_003, "fp32_kahan", 0)]


def _make(V, fam, d, N, n, prec, strata, iid, stream=None):
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=1.5, seed=5, integral_id=iid, precision=prec)
    ctx = V.vegas_create(cfg, fam, params_for(fam, d), stream=stream)
    if strata:
        V.vegas_set_strata(ctx, strata)
    return ctx


def _close(a, b, tol):
    return abs(a - b) <= tol * max(abs(a), abs(b)) + 1e-300


def _tols(prec):
    return (1e-10, 1e-10) if prec == "fp64" else (1e-6, 1e-7)


def test_step_many_equals_step_on_twins():
    V = native()
    many = [_make(V, *m, iid=k) for k, m in enumerate(MIX)]
    twins = [_make(V, *m, iid=k) for k, m in enumerate(MIX)]
    V.vegas_step_many(many)
    for c in twins:
        V.vegas_step(c, sync=False)
    for a, b in zip(many, twins):
        ra, rb = V.vegas_result(a), V.vegas_result(b)
        assert _close(ra["I"], rb["I"], 1e-13) and _close(ra["sigma"], rb["sigma"], 1e-13), (ra, rb)
    for _ in range(3):
        V.vegas_step_many(many)
        for c in twins:
            V.vegas_step(c, sync=False)
    for a, b, m in zip(many, twins, MIX):
        tr, tg = _tols(m[4])
        ra, rb = V.vegas_result(a), V.vegas_result(b)
        assert ra["n_iter"] == rb["n_iter"] == 4
        for key in ("I", "sigma"):
            assert _close(ra[key], rb[key], tr), (key, ra, rb)
        # chi^2/dof = (sum w I^2 - I sum w I)/(m - 1) cancels terms of size
        # sum w I^2 ~ (I/sigma)^2: a change of the I_t by tr moves it by ~tr of that
        scale = (rb["I"] / rb["sigma"]) ** 2 / 3
        assert abs(ra["chi2_dof"] - rb["chi2_dof"]) <= 10 * tr * (1 + scale), (ra, rb)
        assert np.max(np.abs(V.vegas_get_grid(a) - V.vegas_get_grid(b))) <= tg
        assert V.vegas_get_iteration(a) == V.vegas_get_iteration(b) == 4


def test_step_many_on_a_user_stream():
    """Contexts on a caller's (non-default) stream: back-to-back steps with no
    host synchronisation, and a read on that stream right after them, see the
    same results as vegas_step on twins on the default stream (the twin
    tolerances above)."""
    V = native()
    import torch
    s = torch.cuda.Stream()
    mix = MIX[:3]
    many = [_make(V, *m, iid=k, stream=s) for k, m in enumerate(mix)]
    twins = [_make(V, *m, iid=k) for k, m in enumerate(mix)]
    for _ in range(4):
        V.vegas_step_many(many)
    for _ in range(4):
        for c in twins:
            V.vegas_step(c, sync=False)
    for a, b, m in zip(many, twins, mix):
        tr, tg = _tols(m[4])
        ra, rb = V.vegas_result(a), V.vegas_result(b)
        assert ra["n_iter"] == rb["n_iter"] == 4
        assert _close(ra["I"], rb["I"], tr) and _close(ra["sigma"], rb["sigma"], tr), (ra, rb)
        assert np.max(np.abs(V.vegas_get_grid(a) - V.vegas_get_grid(b))) <= tg


def test_step_many_first_iteration_matches_oracle():
    V = native()
    fam, d, N, n = "genz_gauss", 6, 40, 200_000
    a = _make(V, fam, d, N, n, "fp64", 0, iid=3)
    b = _make(V, "sum", 2, 10, 50_000, "fp32_kahan", 0, iid=4)
    V.vegas_step_many([a, b])
    p = params_for(fam, d)
    acc = O.iterate(d, N, O.uniform_edges(d, N), fam, p, 5, 3, 0, n, threads=8)
    Io, var = O.iteration_result(acc["S1"], acc["S2"], n)
    r = V.vegas_result(a)
    assert _close(r["I"], Io, 1e-12)
    assert _close(r["sigma"], math.sqrt(var), 1e-9)
    e = O.refine(d, N, acc["hist"], O.uniform_edges(d, N), 1.5)
    assert np.max(np.abs(V.vegas_get_grid(a) - e)) < 1e-12
    # the sum toy: I = d/2 exactly in expectation, within its error
    rb = V.vegas_result(b)
    assert abs(rb["I"] - 1.0) < 5 * rb["sigma"]


def test_step_many_eight_contexts_up_to_32_dimensions():
    V = native()
    dims = [1, 2, 4, 8, 9, 16, 17, 32]
    many = [_make(V, "genz_gauss", d, 16, 20_000, "fp32_kahan", 0, iid=k) for k, d in enumerate(dims)]
    twins = [_make(V, "genz_gauss", d, 16, 20_000, "fp32_kahan", 0, iid=k) for k, d in enumerate(dims)]
    for _ in range(2):
        V.vegas_step_many(many)
        for c in twins:
            V.vegas_step(c, sync=False)
    tr, tg = _tols("fp32_kahan")
    for a, b in zip(many, twins):
        assert _close(V.vegas_result(a)["I"], V.vegas_result(b)["I"], tr)
        assert np.max(np.abs(V.vegas_get_grid(a) - V.vegas_get_grid(b))) <= tg


def test_step_many_validation():
    V = native()
    import torch
    from paper_2010_09341_gb300 import _native as nat
    from paper_2010_09341_gb300 import workloads as W
    a = _make(V, "sum", 2, 10, 1000, "fp64", 0, iid=0)
    b = _make(V, "sum", 2, 10, 1000, "fp64", 0, iid=1)
    other = _make(V, "sum", 2, 10, 1000, "fp64", 0, iid=2, stream=torch.cuda.Stream())
    nine = [_make(V, "sum", 2, 10, 1000, "fp64", 0, iid=10 + k) for k in range(9)]
    cfg = V.Config(n_dim=3, n_events=1000, n_bins=20, precision="fp32_kahan")
    nogrid = V.vegas_create(cfg, "lo_pdf", W.lo_params())
    for bad in ([], [a, a], [a, other], nine, [a, nogrid]):
        with pytest.raises(nat.VegasError):
            V.vegas_step_many(bad)
    # nothing ran for the rejected calls
    assert V.vegas_get_iteration(a) == 0
    V.vegas_step_many([a, b])
    assert V.vegas_get_iteration(a) == V.vegas_get_iteration(b) == 1
