"""Sample indices on both sides of 2^32 in the sampling kernel.

After the first iteration the FP32 modes take a loop whose sample index is
the block's high word plus a 32-bit low word when the block's samples stay
below a multiple of 2^32, and the general 64-bit loop otherwise.  An
iteration of more than 2^32 samples, sampled here in two shards (the first
samples, and a range that straddles 2^32, so that one block crosses it while
the others lie wholly below or wholly above), must accumulate exactly the
samples the oracle does: S1, S2 at the FP32 tolerance, the histograms as in
the parity tests, no non-finite values.  Two iterations of 2e5 samples come
first, so that the fixed-point histogram scale is set (a settled iteration)."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import BIN_TOL, TOL, assert_hist_close, native, params_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32_acc64", "fp32_kahan"])
@pytest.mark.parametrize("family", ["gauss_sym", "genz_gauss"])
def test_sums_across_two_to_the_32(family, prec):
    V = native()
    d, N = 4, 50
    p = params_for(family, d)
    cfg = V.Config(n_dim=d, n_events=200_000, n_bins=N, alpha=1.5, seed=3, integral_id=1, precision=prec)
    ctx = V.vegas_create(cfg, family, p)
    V.vegas_step(ctx)
    V.vegas_step(ctx)
    e = V.vegas_get_grid(ctx)
    n = (1 << 32) + 50_000
    V.vegas_set_events(ctx, n)
    ranges = [(0, 60_000), ((1 << 32) - 37_001, 74_003)]
    for s0, cnt in ranges:
        V.vegas_sample_shard(ctx, s0, cnt)
    _, _, n_ok, n_nf = V.vegas_finalize(ctx)
    S1, S2, h = V.vegas_get_sums(ctx)
    accs = [O.iterate(d, N, e, family, p, 3, 1, 2, n, s_begin=s0, s_end=s0 + cnt, threads=8) for s0, cnt in ranges]
    So1 = sum(a["S1"] for a in accs)
    So2 = sum(a["S2"] for a in accs)
    ho = sum(a["hist"] for a in accs)
    tol = TOL[prec]
    assert n_nf == 0 and sum(a["n_nonfinite"] for a in accs) == 0
    assert abs(S1 - So1) <= tol * abs(So1), (S1, So1)
    assert abs(S2 - So2) <= tol * abs(So2), (S2, So2)
    assert_hist_close(h, ho, tol, BIN_TOL[prec])
    assert np.all(h >= 0)
