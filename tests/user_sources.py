"""User integrand sources for the run-time compiled family, and their host
build for the oracle.

Each source defines ``template <class T> __device__ T user_integrand(const T *x,
int d, const T *p)``, the signature vegas_create_user takes.  For the oracle
the same text is compiled by g++ as host C++ (``__device__`` defined away, the
math functions of <cmath> in scope) and its double instance exported; the
oracle then calls it through its own sampling loop.  The source is the input
(the integrand), not the method's arithmetic.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")

# Genz Gaussian written by a user: f = exp(-sum (c_j (x_j - w_j))^2), p = [c..., w...]
GENZ_GAUSS = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    T q = T(0);
    for (int j = 0; j < d; ++j) {
        const T t = p[j] * (x[j] - p[d + j]);
        q += t * t;
    }
    return exp(-q);
}
"""

# prod_j (pi/2) sin(pi x_j): integral 1 over [0,1]^d
SINE = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    const T hp = T(1.5707963267948966);
    T f = T(1);
    for (int j = 0; j < d; ++j) f *= hp * sin(T(3.141592653589793) * x[j]);
    return f;
}
"""

# a product of a Lorentzian peak and a polynomial, parameters [m, g, a]:
# f = g / ((x0 - m)^2 + g^2) * (1 + a x1) * ... (uses pow and a branch)
MIXED = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    const T m = p[0], g = p[1], a = p[2];
    T f = g / ((x[0] - m) * (x[0] - m) + g * g);
    for (int j = 1; j < d; ++j) f *= (x[j] < T(0.5)) ? T(1) + a * x[j] : pow(x[j], T(1.5)) * T(2);
    return f;
}
"""

# NaN where x_0 < 2^-6, +Inf where x_1 > 1 - 2^-6, -Inf where
# 1/2 <= x_2 < 1/2 + 2^-11 (d >= 3), else 1 + sum x_j^2.  The thresholds are
# exact in FP32 and FP64, so both precisions see the same regions; the
# non-finite values are formed at run time from x.
NONFINITE = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    const T z = x[0] - x[0];
    if (x[0] < T(0.015625)) return z / z;
    if (x[1] > T(0.984375)) return T(1) / z;
    if (x[2] >= T(0.5) && x[2] < T(0.50048828125)) return T(-1) / z;
    T f = T(1);
    for (int j = 0; j < d; ++j) f += x[j] * x[j];
    return f;
}
"""

# finite everywhere, but (J f)^2 exceeds the FP32 range where x_0 > 31/32
HUGE = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    if (x[0] > T(0.96875)) return T(1e20);
    return T(1) + x[1];
}
"""

# NaN everywhere
ALL_NAN = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    const T z = x[0] - x[0];
    return z / z;
}
"""

BROKEN = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    return this_is_not_defined(x[0]);
}
"""

_PRELUDE = """#include <cmath>
using std::exp; using std::sin; using std::cos; using std::pow; using std::log; using std::sqrt;
#define __device__
"""


def host_function(source: str) -> int:
    """Compile ``source`` for the host and return the address of its double
    instance, double f(const double *x, int d, const double *p)."""
    os.makedirs(BUILD, exist_ok=True)
    key = hashlib.sha256(source.encode()).hexdigest()[:16]
    so = os.path.join(BUILD, "user_%s.so" % key)
    if not os.path.exists(so):
        src = os.path.join(BUILD, "user_%s.cpp" % key)
        with open(src, "w") as f:
            f.write(_PRELUDE + source + '\nextern "C" double user_f64(const double *x, int d, const double *p) '
                    '{ return user_integrand<double>(x, d, p); }\n')
        tmp = so + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, src])
        os.replace(tmp, so)
    lib = ctypes.CDLL(so)
    _keep.append(lib)
    return ctypes.cast(lib.user_f64, ctypes.c_void_p).value


_keep = []
