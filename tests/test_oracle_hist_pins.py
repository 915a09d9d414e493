"""Pins of the oracle's observable histograms against facts outside that
code: the iteration sums the bins must add up to, a histogram of the Philox
uniforms themselves, and the cuts of the LO toy."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2010_09341_gb300 import workloads as W


@pytest.mark.parametrize("B,P", [(0, 0), (10, 3)])
def test_bins_add_up_to_the_iteration_sums(B, P):
    d, N = 4, 30
    p = W.genz_params("genz_gauss", d, seed=3)
    e = O.uniform_edges(d, N)
    e = O.refine(d, N, O.iterate(d, N, e, "genz_gauss", p, 0, 0, 0, 20000)["hist"], e)
    n = 3 * 2 ** 10 if P else 20_000
    S1b, S2b = O.histogram(d, N, e, "genz_gauss", p, 1, 2, 1, n, obs=2, nb=17, lo=0.1, hi=0.9, B=B, P=P)
    if P:
        acc = O.iterate_strat(d, N, e, "genz_gauss", p, 1, 2, 1, B, P)
    else:
        acc = O.iterate(d, N, e, "genz_gauss", p, 1, 2, 1, n)
    assert S1b.sum() == pytest.approx(acc["S1"], rel=1e-12)
    assert S2b.sum() == pytest.approx(acc["S2"], rel=1e-12)
    assert S1b[0] > 0 and S1b[-1] > 0      # under- and overflow bins are used


def test_constant_on_the_uniform_grid_is_a_histogram_of_the_uniforms():
    """f = 1 on the uniform grid: v = 1 and x_k = r_k / 2^32, so bin b holds the
    number of Philox words of dimension k in it (counted here directly)."""
    d, N, n, k, t = 3, 10, 5000, 1, 2
    e = O.uniform_edges(d, N)
    S1b, _ = O.histogram(d, N, e, "const", [], 7, 4, t, n, obs=k, nb=20, lo=0.0, hi=1.0)
    u = np.array([O.draw(s, t, k, 7, 4) for s in range(n)], dtype=np.float64) / 2.0 ** 32
    counts, _ = np.histogram(u, bins=np.linspace(0.0, 1.0, 21))
    assert S1b[0] == 0 and S1b[-1] == 0
    assert np.allclose(S1b[1:-1], counts, rtol=0, atol=1e-9)


def test_lo_cuts_leave_nothing_outside_the_window():
    """The LO toy keeps 60 <= sqrt(shat) <= 120 GeV and |cos theta| < 0.95:
    no weight falls outside those ranges (up to the closed upper edge)."""
    N = 100
    p = W.lo_params()
    e = O.uniform_edges(3, N)
    for _ in range(2):
        acc = O.iterate(3, N, e, "lo", p, 0, 0, 0, 50_000)
        e = O.refine(3, N, acc["hist"], e)
    m1, _ = O.histogram(3, N, e, "lo", p, 0, 0, 5, 100_000, obs=-1, nb=30, lo=60.0, hi=120.0 + 1e-9)
    c1, _ = O.histogram(3, N, e, "lo", p, 0, 0, 5, 100_000, obs=-2, nb=19, lo=-0.95, hi=0.95)
    assert m1.sum() > 0
    assert m1[0] == 0 and m1[-1] == 0
    assert c1[0] == 0 and c1[-1] == 0
    # the Breit-Wigner peak: the bin holding M = 91.19 GeV carries the most weight
    centre = 60.0 + (np.argmax(m1[1:-1]) + 0.5) * (60.0 + 1e-9) / 30
    assert abs(centre - 91.19) < 2.0
