"""The FP64 path's 2^x (vegas::fexp2, the table-driven method of Tang, ACM
TOMS 1989) against CUDA's exp2 on the same GPU: within 2 ulp over normal
results, the same subnormal results to one unit of the last place, and the
same 0, infinity and NaN outside the normal range."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from gpu_helpers import native

pytestmark = pytest.mark.gpu


def _lib():
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "cuda", "exp2_check.cu")
    dev = os.path.join(here, "..", "paper_2010_09341_gb300", "csrc", "vegas_device.cuh")
    out = os.path.join(here, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "libexp2check.so")
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(src), os.path.getmtime(dev)):
        from paper_2010_09341_gb300.build import nvcc
        subprocess.check_call([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                               "-shared", "-Xcompiler", "-fPIC", "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.exp2_check.restype = ctypes.c_int
    lib.exp2_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]
    return lib


def test_fp64_exp2_matches_cuda():
    native()
    import torch
    rng = np.random.default_rng(17)
    x = np.concatenate([
        rng.uniform(-1100.0, 1030.0, 400_000),
        rng.uniform(-300.0, 0.0, 400_000),          # the Gaussian families' range
        rng.uniform(-1.0 / 64, 1.0 / 64, 100_000),
        np.arange(-64 * 1100, 64 * 1030) / 64.0,    # every table point k/64
        np.array([0.0, -0.0, 1.0, -1.0, 0.5 / 64, -0.5 / 64, -1021.0, np.nextafter(-1021.0, -2000.0),
                  -1022.0, -1022.5, -1074.0, -1074.5, -1075.0, -1080.0, -1080.5, -1e300, 1023.0,
                  np.nextafter(1023.0, 2000.0), 1023.9, 1024.0, 1e300, 1e-300, -np.inf, np.inf, np.nan]),
    ])
    xt = torch.from_numpy(x).cuda()
    mine = torch.empty_like(xt)
    ref = torch.empty_like(xt)
    assert _lib().exp2_check(xt.data_ptr(), mine.data_ptr(), ref.data_ptr(), x.size) == 0
    m, r = mine.cpu().numpy(), ref.cpu().numpy()
    assert np.array_equal(np.isnan(m), np.isnan(r))
    ok = ~np.isnan(r)
    m, r, xs = m[ok], r[ok], x[ok]
    assert np.array_equal(np.isinf(m), np.isinf(r))
    tiny = np.finfo(np.float64).tiny
    normal = (r >= tiny) & np.isfinite(r)
    ulp = np.spacing(r[normal])
    err = np.abs(m[normal] - r[normal]) / ulp
    assert err.max() <= 2.0, (err.max(), xs[normal][np.argmax(err)])
    sub = (r < tiny) & ~np.isinf(r)
    # below the normal range both round to multiples of 2^-1074
    assert np.all(np.abs(m[sub] - r[sub]) <= 2.0 ** -1074), np.max(np.abs(m[sub] - r[sub]))
    assert np.all(m[xs < -1076.0] == 0.0)
