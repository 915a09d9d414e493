"""Closed-form and quadrature values of the test integrals.

Each function states the integral over [0,1]^d exactly from calculus, written
independently of the oracle (which only evaluates integrands pointwise).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import integrate as si
from scipy.special import erf


def gauss_sym(d, a=0.1):
    """int (a sqrt(pi))^-d exp(-sum (x-1/2)^2/a^2) = erf(1/(2a))^d."""
    return erf(0.5 / a) ** d


def genz_osc(params):
    """int cos(2 pi u + c.x) = Re[e^{i 2 pi u} prod (e^{i c} - 1)/(i c)]."""
    u, c = params[0], np.asarray(params[1:])
    return math.cos(2 * math.pi * u + c.sum() / 2) * float(np.prod(2 * np.sin(c / 2) / c))


def genz_gauss(params, d):
    c, w = np.asarray(params[:d]), np.asarray(params[d:])
    return float(np.prod(math.sqrt(math.pi) / (2 * c) * (erf(c * (1 - w)) + erf(c * w))))


def genz_prod(params, d):
    c, w = np.asarray(params[:d]), np.asarray(params[d:])
    return float(np.prod(c * (np.arctan(c * (1 - w)) + np.arctan(c * w))))


def genz_corner_incl_excl(c):
    """(1/(d! prod c)) sum_S (-1)^|S| / (1 + sum_{i in S} c_i); fine for small d."""
    c = list(c)
    d = len(c)
    tot = 0.0
    for k in range(d + 1):
        for S in itertools.combinations(range(d), k):
            tot += (-1) ** k / (1.0 + sum(c[i] for i in S))
    return tot / (math.factorial(d) * float(np.prod(c)))


def genz_corner_laplace(c):
    """(1/d!) int_0^inf t^d e^-t prod (1 - e^{-c_i t})/(c_i t) dt, from
    1/a^{d+1} = (1/d!) int t^d e^{-a t} dt with a = 1 + c.x."""
    c = np.asarray(c, dtype=np.float64)
    d = len(c)

    def g(t):
        if t == 0.0:
            return 0.0
        return t ** d * math.exp(-t) * float(np.prod(-np.expm1(-c * t) / (c * t)))

    val, _ = si.quad(g, 0.0, np.inf, epsabs=0, epsrel=1e-13, limit=500)
    return val / math.factorial(d)


def lo_value(params):
    """LO toy: c-integral (1+c^2) over |c| < cut in closed form, times the
    (x1, x2) integral done through tau = x1 x2:
      int dtau BW(tau S)/(tau S) L(tau),  L(tau) = int_{ln tau}^0 g(e^t) g(tau e^-t) dt.
    """
    sqrtS, M, G, cut, mlo, mhi, norm = params
    S = sqrtS * sqrtS
    cfac = 2 * cut + 2 * cut ** 3 / 3.0

    def g(x):
        return (35.0 / 32.0) * (1 - x) ** 3 / math.sqrt(x)

    def lum(tau):
        val, _ = si.quad(lambda t: g(math.exp(t)) * g(tau * math.exp(-t)), math.log(tau), 0.0,
                         epsabs=0, epsrel=1e-12, limit=200)
        return val

    def outer(tau):
        sh = tau * S
        bw = 1.0 / ((sh - M * M) ** 2 + M * M * G * G)
        return bw / sh * lum(tau)

    tlo, thi, t0 = (mlo / sqrtS) ** 2, (mhi / sqrtS) ** 2, (M / sqrtS) ** 2
    w = M * G / S
    pts = sorted(p for p in (t0 - 3 * w, t0, t0 + 3 * w) if tlo < p < thi)
    val, _ = si.quad(outer, tlo, thi, points=pts, epsabs=0, epsrel=1e-10, limit=400)
    return cfac * val * norm
