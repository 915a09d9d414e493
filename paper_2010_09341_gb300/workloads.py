"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module draws the integrand parameters, batch mixes and request streams
that stand in for the paper's physics workload (the single-top LO example of
Sec. 3.1 is not available).  It holds none of the method's arithmetic: no
sampling, no grid, no integrand evaluation, only numpy random draws with fixed
seeds.  Both sides receive its output as plain parameter arrays.

Parameter layouts (one float64 array per integral):
  const, sum      : []
  gauss_sym       : [a]
  genz_osc        : [u, c_1..c_d]
  genz_gauss      : [c_1..c_d, w_1..w_d]
  genz_prod       : [c_1..c_d, w_1..w_d]
  genz_corner     : [c_1..c_d]
  lo              : [sqrtS, M, Gamma, cos_cut, mll_lo, mll_hi, norm]
"""
from __future__ import annotations

from dataclasses import dataclass, field

import math

import numpy as np

# LO-style 2->2 toy: 13 TeV collider, Z-like Breit-Wigner, |cos theta| < 0.95,
# invariant-mass window 60..120 GeV, GeV^-2 -> pb conversion.
LO_PARAMS = (13000.0, 91.19, 2.49, 0.95, 60.0, 120.0, 0.3894e9)


def gauss_sym_params(a: float = 0.1) -> np.ndarray:
    return np.array([a], dtype=np.float64)


def genz_osc_params(d: int, seed: int = 1, u: float = 0.3) -> np.ndarray:
    """Oscillatory Genz family: u fixed, c_i ~ U(0, 1) from ``seed``."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, size=d)
    return np.concatenate([[u], c]).astype(np.float64)


def genz_params(family: str, d: int, seed: int, c_lo: float = 0.5, c_hi: float = 5.0):
    """Genz Gaussian / product-peak / corner-peak: c_i ~ U(c_lo, c_hi), w_i ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(c_lo, c_hi, size=d)
    w = rng.uniform(0.0, 1.0, size=d)
    if family in ("genz_gauss", "genz_prod"):
        return np.concatenate([c, w]).astype(np.float64)
    if family == "genz_corner":
        return c.astype(np.float64)
    raise ValueError(family)


def lo_params() -> np.ndarray:
    return np.array(LO_PARAMS, dtype=np.float64)


# Grid of a synthetic parton density (no PDF sets are available here): the
# LO toy's x^-1/2 (1-x)^b shape with a mild scale dependence of b, normalised
# to unit integral at every scale, tabulated as x g(x, Q^2) on uniform knots
# in ln x and ln Q^2 (the layout of the density grids the paper's companion
# tool interpolates).
PDF_X_MIN, PDF_Q_MIN, PDF_Q_MAX = 1e-6, 10.0, 1000.0


def pdf_grid(nx: int = 96, nq: int = 48, b0: float = 3.0, b1: float = 0.5):
    """(xg[nx, nq], u0, u1, v0, v1): x g(x, Q^2) = N(Q^2) x^(1/2) (1-x)^b(Q^2)
    with b = b0 + b1 ln(Q^2/Qmin^2)/ln(Qmax^2/Qmin^2) and N = 1/B(1/2, b+1);
    u = ln x from ln(1e-6) to 0, v = ln Q^2 from ln(10^2) to ln(1000^2).
    b1 = 0 gives the LO toy's own density at every scale."""
    from scipy.special import beta
    u0, u1 = math.log(PDF_X_MIN), 0.0
    v0, v1 = math.log(PDF_Q_MIN ** 2), math.log(PDF_Q_MAX ** 2)
    u = np.linspace(u0, u1, nx)
    v = np.linspace(v0, v1, nq)
    x = np.exp(u)[:, None]
    b = b0 + b1 * (v - v0) / (v1 - v0)
    N = 1.0 / beta(0.5, b + 1.0)
    xg = N[None, :] * np.sqrt(x) * (1.0 - np.minimum(x, 1.0)) ** b[None, :]
    xg[-1, :] = 0.0  # x = 1
    return np.ascontiguousarray(xg), u0, u1, v0, v1


@dataclass
class Integral:
    """One integration problem: family, dimension, parameters, samples/iteration."""
    family: str
    d: int
    params: np.ndarray
    n_events: int
    n_bins: int = 50
    n_iter: int = 10
    alpha: float = 1.5
    seed: int = 0
    integral_id: int = 0
    target_rel: float = 0.0
    budget: int = 0
    arrival: float = 0.0
    extra: dict = field(default_factory=dict)


def batch_mix(n_integrals: int = 512, seed: int = 2, d_lo: int = 2, d_hi: int = 16,
              n_lo: float = 1e4, n_hi: float = 1e7, n_bins: int = 50):
    """Uneven batch: d ~ U{d_lo..d_hi}, family ~ U{genz_gauss, genz_prod,
    genz_corner}, c ~ U(0.5, 5), w ~ U(0, 1), samples per iteration
    log-uniform in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    fams = ("genz_gauss", "genz_prod", "genz_corner")
    out = []
    for k in range(n_integrals):
        d = int(rng.integers(d_lo, d_hi + 1))
        fam = fams[int(rng.integers(0, 3))]
        n = int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))))
        pseed = int(rng.integers(0, 2**31 - 1))
        out.append(Integral(fam, d, genz_params(fam, d, pseed), n, n_bins=n_bins,
                            seed=0, integral_id=k))
    return out


def request_stream(rate: float, n_requests: int, seed: int = 3, d_lo: int = 1,
                   d_hi: int = 20, t_lo: float = 1e-5, t_hi: float = 1e-3,
                   max_budget: int = 10**9, n_bins: int = 50):
    """Poisson arrivals at ``rate`` per second of mixed integration requests.

    Each request: d ~ U{d_lo..d_hi}; family uniform over genz_gauss,
    genz_prod, genz_corner, genz_osc and lo (lo only where d == 3);
    per-request parameter seed = request id; relative-error target
    log-uniform in [t_lo, t_hi]; total sample budget ``max_budget``.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for k in range(n_requests):
        d = int(rng.integers(d_lo, d_hi + 1))
        fams = ["genz_gauss", "genz_prod", "genz_corner", "genz_osc"]
        if d == 3:
            fams.append("lo")
        fam = fams[int(rng.integers(0, len(fams)))]
        target = float(np.exp(rng.uniform(np.log(t_lo), np.log(t_hi))))
        if fam == "genz_osc":
            p = genz_osc_params(d, seed=k)
        elif fam == "lo":
            p = lo_params()
        else:
            p = genz_params(fam, d, seed=k)
        out.append(Integral(fam, d, p, 0, n_bins=n_bins, seed=0, integral_id=k,
                            target_rel=target, budget=max_budget, arrival=float(t[k])))
    return out
