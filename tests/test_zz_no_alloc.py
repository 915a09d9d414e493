"""The no-allocation entry point against the workspace-based one.

vegas_iterate_noalloc serves callers that cannot allocate device memory at
call time (a runtime that owns the device's memory through its own pool, a
plugin that must not grow the memory footprint): its scratch is a fixed
array inside the library.  Here it must give the same sums as vegas_iterate
on a context (same configuration, grid and iteration), within the tolerances
the parity tests use, on two calls in a row (the second call must not see
the first call's leftovers in the shared array).

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import BIN_TOL, TOL, assert_hist_close, native, params_for, random_grid

pytestmark = pytest.mark.gpu


# events_limit below n_events splits one call into several launches that add
# into the same scratch array (the last case: four launches, the last ragged)
@pytest.mark.parametrize("prec,family,d,N,n,limit", [("fp32_acc64", "gauss_sym", 8, 50, 1_000_000, 0),
                                                      ("fp32_kahan", "genz_osc", 6, 64, 500_001, 0),
                                                      ("fp64", "genz_gauss", 5, 40, 200_003, 0),
                                                      ("fp32_kahan", "genz_corner", 4, 30, 300_007, 80_000)])
def test_noalloc_matches_workspace_path(prec, family, d, N, n, limit):
    V = native()
    import torch
    p = params_for(family, d)
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, events_limit=limit, alpha=1.5, seed=3, integral_id=11,
                   precision=prec)
    sums = torch.empty(3 + d * N, dtype=torch.float64, device="cuda")
    tol = TOL[prec]
    for call, t in enumerate((0, 5)):
        e = random_grid(d, N, seed=100 + call, spread=0.5)
        # reference: the workspace-based entry point on a fresh context
        ctx = V.vegas_create(cfg, family, p)
        V.vegas_set_grid(ctx, e)
        V.vegas_set_iteration(ctx, t)
        V.vegas_iterate(ctx)
        S1, S2, h = V.vegas_get_sums(ctx)
        V.vegas_destroy(ctx)
        # the no-allocation entry point through the C ABI
        edges = torch.from_numpy(np.ascontiguousarray(e)).cuda()
        sums.fill_(np.nan)
        V.vegas_iterate_noalloc(cfg, family, p, t, edges, sums)
        torch.cuda.synchronize()
        out = sums.cpu().numpy()
        assert abs(out[0] - S1) <= tol * abs(S1)
        assert abs(out[1] - S2) <= tol * abs(S2)
        assert_hist_close(out[2:2 + d * N].reshape(d, N), h, tol, BIN_TOL[prec])
        assert out[2 + d * N] == 0.0   # no non-finite values in these families


def test_noalloc_rejects_oversized_grid():
    V = native()
    import torch
    from paper_2010_09341_gb300 import _native as nat
    d, N = 8, 600  # 4800 cells > 4096
    cfg = V.Config(n_dim=d, n_events=1000, n_bins=N, precision="fp32_acc64")
    edges = torch.zeros((d, N + 1), dtype=torch.float64, device="cuda")
    sums = torch.zeros(3 + d * N, dtype=torch.float64, device="cuda")
    with pytest.raises(nat.VegasError):
        V.vegas_iterate_noalloc(cfg, "gauss_sym", params_for("gauss_sym", d), 0, edges, sums)
    assert b"static scratch limit" in nat.load().vegas_last_error_string()
