"""FP64 CPU oracle for one VEGAS iteration (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and the two share no code: this package wraps
``vegas_oracle.c`` through ctypes, compiled with gcc by :func:`build`.

The method is VEGAS (Lepage 1978/1980), which the paper names as the
algorithm VegasFlow implements (Sec. 1) and whose iterate -> refine loop it
distributes (Sec. 3.1, 3.2).  See ``vegas_oracle.c`` for the restated steps
and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vegas_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

FAMILIES = {
    "const": 0,
    "sum": 1,
    "gauss_sym": 2,
    "genz_osc": 3,
    "genz_gauss": 4,
    "genz_prod": 5,
    "genz_corner": 6,
    "lo": 7,
    "user": 8,
    "lo_pdf": 9,
}

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``vegas_oracle.c`` into ``liboracle.so`` with gcc.

    ``-ffp-contract=off`` keeps every multiply and add separately rounded, so
    the oracle gives the same FP64 bits on x86-64 and aarch64 hosts.
    """
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u32, i32, i64, u64 = ctypes.c_uint32, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        dp, ip, lp, up = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint32))
        lib.oracle_philox4x32_10.argtypes = [up, up, up]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_philox_many.argtypes = [i64, up, up, up]
        lib.oracle_philox_many.restype = None
        lib.oracle_draw.argtypes = [u64, u32, i32, u32, u32]
        lib.oracle_draw.restype = u32
        lib.oracle_integrand.argtypes = [i32, i32, dp, i32, dp]
        lib.oracle_integrand.restype = ctypes.c_double
        lib.oracle_n_params.argtypes = [i32, i32]
        lib.oracle_n_params.restype = i32
        lib.oracle_sample.argtypes = [i32, i32, dp, i32, dp, i32, u32, u32, u32, u64,
                                      ip, dp, dp, dp]
        lib.oracle_sample.restype = None
        lib.oracle_trace.argtypes = [i32, i32, dp, i32, dp, i32, u32, u32, u32, u64, i64, ip, dp, dp]
        lib.oracle_trace.restype = None
        lib.oracle_iterate.argtypes = [i32, i32, dp, i32, dp, i32, u32, u32, u32, i64, i64,
                                       dp, dp, dp, lp, lp]
        lib.oracle_iterate.restype = None
        lib.oracle_iteration_result.argtypes = [ctypes.c_double, ctypes.c_double, i64, dp, dp]
        lib.oracle_iteration_result.restype = None
        lib.oracle_refine.argtypes = [i32, i32, dp, dp, ctypes.c_double, i32, dp]
        lib.oracle_refine.restype = None
        lib.oracle_combine.argtypes = [i32, dp, dp, dp, dp, dp]
        lib.oracle_combine.restype = None
        lib.oracle_histogram.argtypes = [i32, i32, dp, i32, dp, i32, u32, u32, u32, i32, i64, i64, i64,
                                         i32, i32, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_histogram.restype = None
        lib.oracle_set_pdf_grid.argtypes = [i32, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, dp]
        lib.oracle_set_pdf_grid.restype = None
        lib.oracle_pdf_xg.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.oracle_pdf_xg.restype = ctypes.c_double
        lib.oracle_set_user.argtypes = [ctypes.c_void_p]
        lib.oracle_set_user.restype = None
        lib.oracle_strata_bits.argtypes = [i32, i32, ip]
        lib.oracle_strata_bits.restype = None
        lib.oracle_sample_strat.argtypes = [i32, i32, dp, i32, dp, i32, u32, u32, u32, i32, i64,
                                            u64, ip, dp, dp, dp]
        lib.oracle_sample_strat.restype = None
        lib.oracle_iterate_strat.argtypes = [i32, i32, dp, i32, dp, i32, u32, u32, u32, i32, i64,
                                             i64, i64, dp, dp, dp, dp, dp, lp]
        lib.oracle_iterate_strat.restype = None
        lib.oracle_strat_result.argtypes = [ctypes.c_double, ctypes.c_double, i64, i64, dp, dp]
        lib.oracle_strat_result.restype = None
        _lib = lib
        return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one 128-bit counter under one 64-bit key."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_philox4x32_10(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def philox_many(ctr, key):
    """Philox4x32-10 of n counters (n x 4 u32) under n keys (n x 2 u32)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    assert c.shape[0] == k.shape[0]
    out = np.zeros_like(c)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_philox_many(c.shape[0], c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def draw(s: int, t: int, j: int, seed: int, integral_id: int) -> int:
    """Uniform u32 word r_j of sample s in iteration t."""
    return int(_load().oracle_draw(s, t, j, seed, integral_id))


def n_params(family: str, d: int) -> int:
    return int(_load().oracle_n_params(FAMILIES[family], d))


def integrand(family: str, d: int, params, x) -> float:
    p = _f64(params if len(params) else [0.0])
    xx = _f64(x)
    return float(_load().oracle_integrand(FAMILIES[family], d, _dptr(p), len(params), _dptr(xx)))


def uniform_edges(d: int, N: int) -> np.ndarray:
    """Initial grid: e_j[k] = k/N for every dimension (d rows of N+1)."""
    return np.tile(np.arange(N + 1, dtype=np.float64) / N, (d, 1))


def sample(d, N, edges, family, params, seed, integral_id, t, s):
    """One sample: (bins[d], x[d], J, f)."""
    lib = _load()
    e = _f64(edges).reshape(d, N + 1)
    p = _f64(params if len(params) else [0.0])
    bins = np.zeros(d, dtype=np.int32)
    x = np.zeros(d, dtype=np.float64)
    J = ctypes.c_double()
    f = ctypes.c_double()
    lib.oracle_sample(d, N, _dptr(e), FAMILIES[family], _dptr(p), len(params), seed,
                      integral_id, t, s, bins.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      _dptr(x), ctypes.byref(J), ctypes.byref(f))
    return bins, x, J.value, f.value


def trace(d, N, edges, family, params, seed, integral_id, t, s_begin, count, threads=1):
    """Samples s_begin .. s_begin + count - 1: (bins[count, d] int32, x[count, d], v[count])
    with v = J f; ``threads`` > 1 splits the range over host threads."""
    lib = _load()
    e = _f64(edges).reshape(d, N + 1)
    p = _f64(params if len(params) else [0.0])
    bins = np.zeros((count, d), dtype=np.int32)
    x = np.zeros((count, d), dtype=np.float64)
    v = np.zeros(count, dtype=np.float64)
    threads = max(1, min(int(threads), max(1, count)))
    bounds = np.linspace(0, count, threads + 1).astype(np.int64)

    def run(a, b):
        if b <= a:
            return
        lib.oracle_trace(d, N, _dptr(e), FAMILIES[family], _dptr(p), len(params), seed, integral_id, t,
                         int(s_begin + a), int(b - a),
                         bins[a:b].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(x[a:b]),
                         _dptr(v[a:b]))

    ths = [threading.Thread(target=run, args=(int(bounds[i]), int(bounds[i + 1]))) for i in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    return bins, x, v


def iterate(d, N, edges, family, params, seed, integral_id, t, n, s_begin=0, s_end=None,
            threads=1, counts=False):
    """Accumulate samples [s_begin, s_end) of iteration t (default: all n).

    Returns a dict with S1, S2, hist (d x N), n_nonfinite and, if ``counts``,
    the per-bin sample counts.  ``threads`` > 1 splits the range into
    contiguous pieces run on host threads (the C call releases the GIL) and
    adds the pieces in thread order.
    """
    lib = _load()
    if s_end is None:
        s_end = s_begin + n
    e = _f64(edges).reshape(d, N + 1)
    p = _f64(params if len(params) else [0.0])
    fam = FAMILIES[family]
    threads = max(1, min(int(threads), max(1, s_end - s_begin)))
    bounds = np.linspace(s_begin, s_end, threads + 1).astype(np.int64)
    parts = []

    def run(a, b, slot):
        S1 = ctypes.c_double(0.0)
        S2 = ctypes.c_double(0.0)
        nn = ctypes.c_int64(0)
        h = np.zeros((d, N), dtype=np.float64)
        c = np.zeros((d, N), dtype=np.int64) if counts else None
        lib.oracle_iterate(d, N, _dptr(e), fam, _dptr(p), len(params), seed, integral_id, t,
                           int(a), int(b), ctypes.byref(S1), ctypes.byref(S2), _dptr(h),
                           c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if counts else None,
                           ctypes.byref(nn))
        slot.append((S1.value, S2.value, h, c, nn.value))

    slots = [[] for _ in range(threads)]
    if threads == 1:
        run(bounds[0], bounds[1], slots[0])
    else:
        ths = [threading.Thread(target=run, args=(bounds[i], bounds[i + 1], slots[i]))
               for i in range(threads)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    S1 = 0.0
    S2 = 0.0
    nn = 0
    h = np.zeros((d, N), dtype=np.float64)
    c = np.zeros((d, N), dtype=np.int64) if counts else None
    for sl in slots:
        a1, a2, hh, cc, n0 = sl[0]
        S1 += a1
        S2 += a2
        h += hh
        nn += n0
        if counts:
            c += cc
        parts.append(sl[0])
    out = {"S1": S1, "S2": S2, "hist": h, "n_nonfinite": nn}
    if counts:
        out["counts"] = c
    return out


def iteration_result(S1, S2, n):
    lib = _load()
    I = ctypes.c_double()
    var = ctypes.c_double()
    lib.oracle_iteration_result(S1, S2, n, ctypes.byref(I), ctypes.byref(var))
    return I.value, var.value


def refine(d, N, hist, edges, alpha=1.5, smooth=True):
    lib = _load()
    h = _f64(hist).reshape(d, N)
    e = _f64(edges).reshape(d, N + 1)
    out = np.zeros((d, N + 1), dtype=np.float64)
    lib.oracle_refine(d, N, _dptr(h), _dptr(e), alpha, 1 if smooth else 0, _dptr(out))
    return out


def combine(I, sigma):
    lib = _load()
    a = _f64(I)
    s = _f64(sigma)
    Ib = ctypes.c_double()
    sb = ctypes.c_double()
    c2 = ctypes.c_double()
    lib.oracle_combine(len(a), _dptr(a), _dptr(s), ctypes.byref(Ib), ctypes.byref(sb),
                       ctypes.byref(c2))
    return Ib.value, sb.value, c2.value


def integrate(d, N, family, params, n, n_iter, alpha=1.5, seed=0, integral_id=0,
              threads=1, edges=None, smooth=True):
    """Full run: n_iter iterations, refining the grid after each one.

    Returns dict(I, sigma, chi2_dof, iters=[(I_t, sigma_t)], edges).
    """
    e = uniform_edges(d, N) if edges is None else _f64(edges).reshape(d, N + 1)
    its = []
    for t in range(n_iter):
        acc = iterate(d, N, e, family, params, seed, integral_id, t, n, threads=threads)
        n_eff = n - acc["n_nonfinite"]
        I, var = iteration_result(acc["S1"], acc["S2"], n_eff)
        its.append((I, float(np.sqrt(var))))
        e = refine(d, N, acc["hist"], e, alpha, smooth)
    Ib, sb, c2 = combine([a for a, _ in its], [b for _, b in its])
    return {"I": Ib, "sigma": sb, "chi2_dof": c2, "iters": its, "edges": e}


# ------------------------------------------- stratified + importance hybrid
def strata_bits(d: int, B: int) -> np.ndarray:
    """Halvings of each dimension for 2^B hypercubes (Lepage 1980's combined
    mode, with the strata counts read as powers of two)."""
    out = np.zeros(d, dtype=np.int32)
    _load().oracle_strata_bits(d, B, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


def sample_strat(d, N, edges, family, params, seed, integral_id, t, B, P, s):
    """One sample s of a stratified iteration: (bins[d], x[d], J, f)."""
    lib = _load()
    e = _f64(edges).reshape(d, N + 1)
    p = _f64(params if len(params) else [0.0])
    bins = np.zeros(d, dtype=np.int32)
    x = np.zeros(d, dtype=np.float64)
    J = ctypes.c_double()
    f = ctypes.c_double()
    lib.oracle_sample_strat(d, N, _dptr(e), FAMILIES[family], _dptr(p), len(params), seed,
                            integral_id, t, B, P, s,
                            bins.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(x),
                            ctypes.byref(J), ctypes.byref(f))
    return bins, x, J.value, f.value


def iterate_strat(d, N, edges, family, params, seed, integral_id, t, B, P, h_begin=0,
                  h_end=None, threads=1):
    """Hypercubes [h_begin, h_end) (default all 2^B) of a stratified iteration
    with P samples each.  Returns dict(S1, S2, Q, hist, n_nonfinite); pieces run
    on host threads are added in thread order."""
    lib = _load()
    if h_end is None:
        h_end = 1 << B
    e = _f64(edges).reshape(d, N + 1)
    p = _f64(params if len(params) else [0.0])
    fam = FAMILIES[family]
    threads = max(1, min(int(threads), max(1, h_end - h_begin)))
    bounds = np.linspace(h_begin, h_end, threads + 1).astype(np.int64)
    slots = [[] for _ in range(threads)]

    def run(a, b, slot):
        S1, S2, Q = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        nn = ctypes.c_int64(0)
        h = np.zeros((d, N), dtype=np.float64)
        vbuf = np.zeros(max(1, P), dtype=np.float64)
        lib.oracle_iterate_strat(d, N, _dptr(e), fam, _dptr(p), len(params), seed, integral_id, t,
                                 B, P, int(a), int(b), _dptr(vbuf), ctypes.byref(S1),
                                 ctypes.byref(S2), ctypes.byref(Q), _dptr(h), ctypes.byref(nn))
        slot.append((S1.value, S2.value, Q.value, h, nn.value))

    if threads == 1:
        run(bounds[0], bounds[1], slots[0])
    else:
        ths = [threading.Thread(target=run, args=(bounds[i], bounds[i + 1], slots[i]))
               for i in range(threads)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    out = {"S1": 0.0, "S2": 0.0, "Q": 0.0, "hist": np.zeros((d, N)), "n_nonfinite": 0}
    for sl in slots:
        a1, a2, q, hh, n0 = sl[0]
        out["S1"] += a1
        out["S2"] += a2
        out["Q"] += q
        out["hist"] += hh
        out["n_nonfinite"] += n0
    return out


def strat_result(S1, Q, H, P):
    """(I, var) of a stratified iteration over H hypercubes of P samples."""
    lib = _load()
    I = ctypes.c_double()
    var = ctypes.c_double()
    lib.oracle_strat_result(S1, Q, H, P, ctypes.byref(I), ctypes.byref(var))
    return I.value, var.value


def integrate_strat(d, N, family, params, B, P, n_iter, alpha=1.5, seed=0, integral_id=0,
                    threads=1, edges=None, smooth=True):
    """Full stratified run (2^B hypercubes of P samples per iteration), refining
    after each iteration.  Returns dict(I, sigma, chi2_dof, iters, edges)."""
    e = uniform_edges(d, N) if edges is None else _f64(edges).reshape(d, N + 1)
    its = []
    for t in range(n_iter):
        acc = iterate_strat(d, N, e, family, params, seed, integral_id, t, B, P, threads=threads)
        I, var = strat_result(acc["S1"], acc["Q"], 1 << B, P)
        its.append((I, float(np.sqrt(var))))
        e = refine(d, N, acc["hist"], e, alpha, smooth)
    Ib, sb, c2 = combine([a for a, _ in its], [b for _, b in its])
    return {"I": Ib, "sigma": sb, "chi2_dof": c2, "iters": its, "edges": e}


# ------------------------------------------------------- user integrands
def set_user(fn_address: int) -> None:
    """Family "user" evaluates the host function at fn_address,
    double f(const double *x, int d, const double *p) (the test compiles the
    user's source for the host)."""
    _load().oracle_set_user(ctypes.c_void_p(fn_address))


# ------------------------------------------------------ parton-density grid
_pdf_keep = []


def set_pdf_grid(xg, u0, u1, v0, v1) -> None:
    """Family "lo_pdf" takes x g(x, Q^2) from xg (nx x nq) on uniform knots in
    ln x from u0 to u1 and ln Q^2 from v0 to v1."""
    t = _f64(xg)
    nx, nq = t.shape
    _pdf_keep[:] = [t]
    _load().oracle_set_pdf_grid(nx, nq, u0, u1, v0, v1, _dptr(t))


def pdf_xg(x: float, q2: float) -> float:
    return float(_load().oracle_pdf_xg(x, q2))


# --------------------------------------------------- observable histograms
def histogram(d, N, edges, family, params, seed, integral_id, t, n, obs, nb, lo, hi, B=0, P=0,
              threads=1):
    """Observable histogram of the n samples of iteration t (stratified when P
    > 0): (S1[nb + 2], S2[nb + 2]) with bin 0 below lo and bin nb + 1 at or
    above hi.  Pieces run on host threads are added in thread order."""
    lib = _load()
    e = _f64(edges).reshape(d, N + 1)
    p = _f64(params if len(params) else [0.0])
    threads = max(1, min(int(threads), max(1, n)))
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    outs = [np.zeros(2 * (nb + 2)) for _ in range(threads)]

    def run(i):
        lib.oracle_histogram(d, N, _dptr(e), FAMILIES[family], _dptr(p), len(params), seed,
                             integral_id, t, B, P, int(bounds[i]), int(bounds[i + 1]), obs, nb, lo, hi,
                             _dptr(outs[i]))

    ths = [threading.Thread(target=run, args=(i,)) for i in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    tot = np.zeros(2 * (nb + 2))
    for o in outs:
        tot += o
    return tot[:nb + 2], tot[nb + 2:]
