"""ctypes binding of ``libvegas.so`` (the C ABI in ``include/vegas.h``).

Argument marshalling only: every step of an iteration runs in the library's
CUDA kernels.  PyTorch supplies device memory (the workspace) and streams.
There is no CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvegas.so")

(VEGAS_OK, VEGAS_EINVAL, VEGAS_ENOMEM, VEGAS_ECUDA, VEGAS_ETIMEOUT, VEGAS_EBUSY, VEGAS_ENONFINITE,
 VEGAS_EJIT) = range(8)
VEGAS_FP64, VEGAS_FP32_ACC64, VEGAS_FP32_KAHAN = 0, 1, 2
PRECISIONS = {"fp64": VEGAS_FP64, "fp32_acc64": VEGAS_FP32_ACC64, "fp32_kahan": VEGAS_FP32_KAHAN}
FAMILIES = {"const": 0, "sum": 1, "gauss_sym": 2, "genz_osc": 3, "genz_gauss": 4,
            "genz_prod": 5, "genz_corner": 6, "lo": 7, "user": 8, "lo_pdf": 9}
MAX_USER_PARAMS = 72
MAX_DIM, MAX_BINS, MAX_ITERS = 32, 1024, 4096


class VegasConfig(ctypes.Structure):
    _fields_ = [("n_dim", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("n_events", ctypes.c_int64), ("events_limit", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("seed", ctypes.c_uint32),
                ("integral_id", ctypes.c_uint32), ("precision", ctypes.c_int32),
                ("smooth", ctypes.c_int32)]


class VegasIntegrand(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("n_dim", ctypes.c_int32),
                ("params", ctypes.POINTER(ctypes.c_double)), ("n_params", ctypes.c_int32)]


class VegasIterResult(ctypes.Structure):
    _fields_ = [("I", ctypes.c_double), ("sigma", ctypes.c_double), ("n", ctypes.c_int64),
                ("n_nonfinite", ctypes.c_int64)]


class VegasResult(ctypes.Structure):
    _fields_ = [("I", ctypes.c_double), ("sigma", ctypes.c_double),
                ("chi2_dof", ctypes.c_double), ("n_iter", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class VegasBatchShape(ctypes.Structure):
    _fields_ = [("tile_samples", ctypes.c_int32), ("threads", ctypes.c_int32), ("layout", ctypes.c_int32)]


class VegasBatchResult(ctypes.Structure):
    _fields_ = [("slot", ctypes.c_int32), ("t", ctypes.c_int32), ("it", VegasIterResult),
                ("comb", VegasResult)]


class VegasError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        lib = load()
        msg = lib.vegas_strerror(status).decode()
        extra = lib.vegas_last_error_string().decode() if status == VEGAS_ECUDA else ""
        if status == VEGAS_EJIT:
            extra = lib.vegas_jit_log().decode(errors="replace").strip()
        super().__init__("%s: %s%s" % (what, msg, (" (" + extra + ")") if extra else ""))


_lib = None

# Every symbol include/vegas.h declares, with its ctypes signature.
_P = ctypes.c_void_p
_SIGS = {
    "vegas_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(VegasConfig)]),
    "vegas_create": (ctypes.c_int, [ctypes.POINTER(VegasConfig), ctypes.POINTER(VegasIntegrand),
                                    _P, _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "vegas_iterate": (ctypes.c_int, [_P, ctypes.POINTER(VegasIterResult)]),
    "vegas_sample_shard": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64]),
    "vegas_accumulators": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(_P)]),
    "vegas_finalize": (ctypes.c_int, [_P, ctypes.POINTER(VegasIterResult)]),
    "vegas_step": (ctypes.c_int, [_P, ctypes.POINTER(VegasIterResult)]),
    "vegas_step_many": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32]),
    "vegas_refine": (ctypes.c_int, [_P]),
    "vegas_result": (ctypes.c_int, [_P, ctypes.POINTER(VegasResult)]),
    "vegas_run": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(VegasIterResult),
                                 ctypes.POINTER(VegasResult)]),
    "vegas_get_grid": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "vegas_set_grid": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "vegas_get_sums": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "vegas_set_events": (ctypes.c_int, [_P, ctypes.c_int64]),
    "vegas_get_iteration": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "vegas_set_iteration": (ctypes.c_int, [_P, ctypes.c_int32]),
    "vegas_trace": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P, _P, _P]),
    "vegas_set_strata": (ctypes.c_int, [_P, ctypes.c_int32]),
    "vegas_create_user": (ctypes.c_int, [ctypes.POINTER(VegasConfig), ctypes.c_char_p,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int32, _P, _P,
                                         ctypes.c_size_t, ctypes.POINTER(_P)]),
    "vegas_jit_log": (ctypes.c_char_p, []),
    "vegas_histogram": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, _P]),
    "vegas_set_pdf_grid": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "vegas_get_strata": (ctypes.c_int, [_P, _P, _P, _P]),
    "vegas_export_state": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "vegas_import_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "vegas_philox": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
    "vegas_iterate_noalloc": (ctypes.c_int, [ctypes.POINTER(VegasConfig),
                                             ctypes.POINTER(VegasIntegrand), ctypes.c_int32,
                                             _P, _P, _P]),
    "vegas_profile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "vegas_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]),
    "vegas_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_size_t]),
    "vegas_batch_slot_bytes": (ctypes.c_size_t, [ctypes.POINTER(VegasConfig)]),
    "vegas_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_size_t,
                                          ctypes.POINTER(_P)]),
    "vegas_batch_add": (ctypes.c_int, [_P, ctypes.POINTER(VegasConfig), ctypes.POINTER(VegasIntegrand),
                                       ctypes.POINTER(ctypes.c_int32)]),
    "vegas_batch_remove": (ctypes.c_int, [_P, ctypes.c_int32]),
    "vegas_batch_step": (ctypes.c_int, [_P]),
    "vegas_batch_wait": (ctypes.c_int, [_P, ctypes.POINTER(VegasBatchResult), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "vegas_batch_get_grid": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "vegas_batch_set_events": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64]),
    "vegas_batch_set_tile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "vegas_batch_set_shape": (ctypes.c_int, [_P, ctypes.POINTER(VegasBatchShape)]),
    "vegas_batch_get_shape": (ctypes.c_int, [_P, ctypes.POINTER(VegasBatchShape)]),
    "vegas_batch_autotune_shapes": (ctypes.c_int, [_P, ctypes.POINTER(VegasBatchShape), ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                                   ctypes.POINTER(ctypes.c_int32)]),
    "vegas_batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                            ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "vegas_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t),
                                        ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int32)]),
    "vegas_batch_destroy": (None, [_P]),
    "vegas_batch_last_error": (ctypes.c_char_p, []),
    "vegas_destroy": (None, [_P]),
    "vegas_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vegas_last_error_string": (ctypes.c_char_p, []),
}


def declared_symbols():
    return list(_SIGS)


def load():
    """Load libvegas.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libvegas.so is not built (%s); run paper_2010_09341_gb300.build.build()"
                          % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, what=""):
    if status != VEGAS_OK:
        raise VegasError(status, what)
    return status
