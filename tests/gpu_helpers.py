"""Helpers shared by the GPU tests: library build, contexts, oracle runs."""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2010_09341_gb300 import workloads as W

TOL = {"fp64": 1e-12, "fp32_acc64": 1e-5, "fp32_kahan": 1e-5}
PRECS = ["fp64", "fp32_acc64", "fp32_kahan"]
# Histogram bins that hold at least BIG_FRAC of their row, relative to their own
# value.  FP32: the fixed-point cells round each v^2 to 2^-19 of the previous
# iteration's mean v^2 (half a quantum of 2^-18), so a bin holding a fraction
# phi of a row of N bins, filled by about n/N samples, carries a rounding error
# of about 2^-19 / (phi sqrt(N n)) relative, 2^-19 / (phi N) if every rounding
# went one way: at phi = 1e-3, N >= 20, at most 1e-4.
BIG_FRAC = 1e-3
BIN_TOL = {"fp64": 1e-12, "fp32_acc64": 1e-4, "fp32_kahan": 1e-4}


def assert_hist_close(h, ho, tol, bin_tol, big_frac=BIG_FRAC):
    """Histograms (d, N) against the oracle's, row by row: every bin within
    tol of its row's sum, and bins holding at least big_frac of their row
    within bin_tol of their own value."""
    h = np.asarray(h, dtype=np.float64).reshape(ho.shape)
    rows = ho.sum(axis=1, keepdims=True)
    err = np.abs(h - ho)
    bad = err > tol * rows
    assert not bad.any(), ("row", np.max(err / np.maximum(rows, 1e-300)))
    big = ho >= big_frac * rows
    if big.any():
        rel = err[big] / ho[big]
        assert np.all(rel <= bin_tol), ("bin", float(rel.max()))

_built = False


def native():
    """Build (if needed) and return the vegas Python binding; skip without a GPU."""
    global _built
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not _built:
        from paper_2010_09341_gb300 import build as B
        B.build()
        _built = True
    from paper_2010_09341_gb300 import vegas as V
    return V


def params_for(family, d, seed=7):
    if family in ("const", "sum"):
        return np.zeros(0)
    if family == "gauss_sym":
        return W.gauss_sym_params(0.1)
    if family == "genz_osc":
        return W.genz_osc_params(d, seed=seed)
    if family == "lo":
        return W.lo_params()
    return W.genz_params(family, d, seed=seed)


def random_grid(d, N, seed=0, spread=1.0):
    """A valid non-uniform grid: sorted uniforms mixed with the uniform grid."""
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(0, 1, size=(d, N - 1)), axis=1)
    uni = np.tile(np.arange(1, N) / N, (d, 1))
    inner = np.sort(spread * inner + (1 - spread) * uni, axis=1)
    return np.concatenate([np.zeros((d, 1)), inner, np.ones((d, 1))], axis=1)


def curand_ref_lib():
    """Compile tests/cuda/curand_philox_ref.cu with nvcc (cached) and load it."""
    import ctypes
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "cuda", "curand_philox_ref.cu")
    out_dir = os.path.join(here, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcurandref.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        from paper_2010_09341_gb300.build import nvcc
        subprocess.check_call([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                               "-shared", "-Xcompiler", "-fPIC", "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.curand_ref_philox.restype = ctypes.c_int
    lib.curand_ref_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_longlong]
    return lib
