"""Python face of the C ABI: the same call names as ``include/vegas.h``.

Marshalling only.  Device memory (the workspace, trace outputs) comes from
PyTorch; the stream is PyTorch's current CUDA stream unless one is given.
:class:`Integrator` mirrors the paper's usage (Sec. 3.1): construct with
``n_dim``, ``n_events`` and ``events_limit``, ``compile`` an integrand,
``run_integration(n_iter)``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as nat
from ._native import check


@dataclass
class Config:
    n_dim: int
    n_events: int
    n_bins: int = 50
    events_limit: int = 0
    alpha: float = 1.5
    seed: int = 0
    integral_id: int = 0
    precision: str = "fp32_kahan"
    smooth: bool = True

    def to_c(self) -> nat.VegasConfig:
        return nat.VegasConfig(int(self.n_dim), int(self.n_bins), int(self.n_events),
                               int(self.events_limit), float(self.alpha), int(self.seed),
                               int(self.integral_id), nat.PRECISIONS[self.precision],
                               1 if self.smooth else 0)


class Context:
    """A live vegas_ctx plus the PyTorch workspace it points into."""

    def __init__(self, handle, cfg: Config, family: str, params, workspace, stream):
        self.handle = handle
        self.cfg = cfg
        self.family = family
        self.params = np.asarray(params, dtype=np.float64)
        self.workspace = workspace
        self.stream = stream

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                nat.load().vegas_destroy(h)
            except Exception:
                pass
            self.handle = None


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream, ctypes.c_void_p(stream.cuda_stream)


def vegas_workspace_bytes(cfg: Config) -> int:
    c = cfg.to_c()
    return int(nat.load().vegas_workspace_bytes(ctypes.byref(c)))


def vegas_create(cfg: Config, family: str, params=(), stream=None, workspace=None,
                 source: str = None) -> Context:
    """A context for a built-in family, or, with family "user", for the CUDA C++
    ``source`` defining ``template <class T> __device__ T user_integrand(const
    T *x, int d, const T *p)`` (compiled at run time by the library)."""
    lib = nat.load()
    c = cfg.to_c()
    nbytes = lib.vegas_workspace_bytes(ctypes.byref(c))
    if nbytes == 0:
        raise nat.VegasError(nat.VEGAS_EINVAL, "vegas_workspace_bytes")
    if workspace is None:
        workspace = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    pp = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if p.size else None
    stream, sp = _stream_ptr(stream)
    h = ctypes.c_void_p()
    if family == "user":
        if source is None:
            raise ValueError("family 'user' needs the integrand's source")
        check(lib.vegas_create_user(ctypes.byref(c), source.encode(), pp, int(p.size), sp,
                                    ctypes.c_void_p(workspace.data_ptr()),
                                    ctypes.c_size_t(workspace.numel()), ctypes.byref(h)),
              "vegas_create_user")
    else:
        itg = nat.VegasIntegrand(nat.FAMILIES[family], int(cfg.n_dim), pp, int(p.size))
        check(lib.vegas_create(ctypes.byref(c), ctypes.byref(itg), sp,
                               ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
                               ctypes.byref(h)), "vegas_create")
    return Context(h, cfg, family, p, workspace, stream)


def vegas_iterate(ctx: Context, sync: bool = True):
    """One iteration; with sync returns (I, sigma, n, n_nonfinite)."""
    lib = nat.load()
    if not sync:
        check(lib.vegas_iterate(ctx.handle, None), "vegas_iterate")
        return None
    r = nat.VegasIterResult()
    st = lib.vegas_iterate(ctx.handle, ctypes.byref(r))
    if st not in (nat.VEGAS_OK, nat.VEGAS_ENONFINITE):
        check(st, "vegas_iterate")
    return r.I, r.sigma, r.n, r.n_nonfinite


def vegas_step(ctx: Context, sync: bool = True):
    """vegas_iterate + vegas_refine in fewer launches; with sync returns the iteration."""
    lib = nat.load()
    if not sync:
        check(lib.vegas_step(ctx.handle, None), "vegas_step")
        return None
    r = nat.VegasIterResult()
    st = lib.vegas_step(ctx.handle, ctypes.byref(r))
    if st not in (nat.VEGAS_OK, nat.VEGAS_ENONFINITE):
        check(st, "vegas_step")
    return r.I, r.sigma, r.n, r.n_nonfinite


MAX_STEP_MANY = 8


def vegas_step_many(ctxs) -> None:
    """One vegas_step of each context (distinct, on one stream), with all their
    iteration results and refinements in one launch (asynchronous)."""
    arr = (nat._P * len(ctxs))(*[c.handle for c in ctxs])
    check(nat.load().vegas_step_many(arr, len(ctxs)), "vegas_step_many")


def vegas_sample_shard(ctx: Context, s_begin: int, count: int) -> None:
    check(nat.load().vegas_sample_shard(ctx.handle, int(s_begin), int(count)), "vegas_sample_shard")


def vegas_accumulators(ctx: Context):
    """(sums, nonfinite): CUDA tensor views of the context's FP64 accumulators
    (2 + d*N values) and its int64 non-finite count, inside the workspace."""
    sp = ctypes.c_void_p()
    cnt = ctypes.c_int64()
    nfp = ctypes.c_void_p()
    check(nat.load().vegas_accumulators(ctx.handle, ctypes.byref(sp), ctypes.byref(cnt),
                                        ctypes.byref(nfp)), "vegas_accumulators")
    base = ctx.workspace.data_ptr()
    off = sp.value - base
    sums = ctx.workspace[off: off + 8 * cnt.value].view(torch.float64)
    off2 = nfp.value - base
    nonfinite = ctx.workspace[off2: off2 + 8].view(torch.int64)
    return sums, nonfinite


def vegas_finalize(ctx: Context, sync: bool = True):
    lib = nat.load()
    if not sync:
        check(lib.vegas_finalize(ctx.handle, None), "vegas_finalize")
        return None
    r = nat.VegasIterResult()
    st = lib.vegas_finalize(ctx.handle, ctypes.byref(r))
    if st not in (nat.VEGAS_OK, nat.VEGAS_ENONFINITE):
        check(st, "vegas_finalize")
    return r.I, r.sigma, r.n, r.n_nonfinite


def vegas_refine(ctx: Context):
    check(nat.load().vegas_refine(ctx.handle), "vegas_refine")


def vegas_result(ctx: Context):
    r = nat.VegasResult()
    check(nat.load().vegas_result(ctx.handle, ctypes.byref(r)), "vegas_result")
    return {"I": r.I, "sigma": r.sigma, "chi2_dof": r.chi2_dof, "n_iter": r.n_iter}


def vegas_run(ctx: Context, n_iter: int):
    its = (nat.VegasIterResult * n_iter)()
    r = nat.VegasResult()
    check(nat.load().vegas_run(ctx.handle, int(n_iter), its, ctypes.byref(r)), "vegas_run")
    return {"I": r.I, "sigma": r.sigma, "chi2_dof": r.chi2_dof, "n_iter": r.n_iter,
            "iters": [(x.I, x.sigma, x.n, x.n_nonfinite) for x in its]}


def vegas_get_grid(ctx: Context, out=None) -> np.ndarray:
    """The grid edges (d, N+1) FP64; into ``out`` (C-contiguous float64, e.g. a
    pinned buffer's numpy view) when given."""
    d, N = ctx.cfg.n_dim, ctx.cfg.n_bins
    if out is None:
        e = np.zeros((d, N + 1), dtype=np.float64)
    else:
        e = out
        if e.dtype != np.float64 or not e.flags["C_CONTIGUOUS"] or e.size != d * (N + 1):
            raise ValueError("out must be a C-contiguous float64 array of d*(N+1) values")
    check(nat.load().vegas_get_grid(ctx.handle, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
          "vegas_get_grid")
    return e


def vegas_set_grid(ctx: Context, edges) -> None:
    d, N = ctx.cfg.n_dim, ctx.cfg.n_bins
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.float64).reshape(d, N + 1))
    check(nat.load().vegas_set_grid(ctx.handle, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
          "vegas_set_grid")


def vegas_get_sums(ctx: Context):
    """(S1, S2, hist[d, N]) of the last iteration, FP64."""
    d, N = ctx.cfg.n_dim, ctx.cfg.n_bins
    s = np.zeros(2 + d * N, dtype=np.float64)
    check(nat.load().vegas_get_sums(ctx.handle, s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
          "vegas_get_sums")
    return s[0], s[1], s[2:].reshape(d, N)


def vegas_set_events(ctx: Context, n_events: int) -> None:
    check(nat.load().vegas_set_events(ctx.handle, int(n_events)), "vegas_set_events")
    ctx.cfg.n_events = int(n_events)


def vegas_get_iteration(ctx: Context) -> int:
    t = ctypes.c_int32()
    check(nat.load().vegas_get_iteration(ctx.handle, ctypes.byref(t)), "vegas_get_iteration")
    return int(t.value)


def vegas_set_iteration(ctx: Context, t: int) -> None:
    check(nat.load().vegas_set_iteration(ctx.handle, int(t)), "vegas_set_iteration")


def vegas_trace(ctx: Context, t: int, s_begin: int, count: int):
    """Per-sample (bins[count, d] int32, x[count, d] f64, w[count] f64) as CUDA tensors."""
    d = ctx.cfg.n_dim
    bins = torch.empty((count, d), dtype=torch.int32, device="cuda")
    x = torch.empty((count, d), dtype=torch.float64, device="cuda")
    w = torch.empty((count,), dtype=torch.float64, device="cuda")
    check(nat.load().vegas_trace(ctx.handle, int(t), int(s_begin), int(count),
                                 ctypes.c_void_p(bins.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(w.data_ptr())), "vegas_trace")
    return bins, x, w


def vegas_set_strata(ctx: Context, B: int) -> None:
    """Stratified + importance hybrid from the next iteration: 2^B hypercubes
    (0: plain sampling, -1: as many as leave 2 samples per hypercube)."""
    check(nat.load().vegas_set_strata(ctx.handle, int(B)), "vegas_set_strata")


def vegas_histogram(ctx: Context, t: int, observable: int, nbins: int, lo: float, hi: float):
    """Observable histogram of iteration t's weights: (sum v, sum v^2) per bin as
    float64 CUDA tensors of nbins + 2 (bin 0 below lo, the last at or above hi).
    observable: a coordinate index, or -1 (sqrt(shat)) / -2 (cos theta) for the
    LO families."""
    out = torch.empty(2 * (nbins + 2), dtype=torch.float64, device="cuda")
    check(nat.load().vegas_histogram(ctx.handle, int(t), int(observable), int(nbins), float(lo), float(hi),
                                     ctypes.c_void_p(out.data_ptr())), "vegas_histogram")
    return out[:nbins + 2], out[nbins + 2:]


def vegas_set_pdf_grid(ctx: Context, xg: torch.Tensor, u0: float, u1: float, v0: float,
                       v1: float) -> None:
    """Density grid of an "lo_pdf" context: xg (nx, nq) float64 CUDA tensor of
    x g(x, Q^2) on uniform knots in ln x (u0..u1) and ln Q^2 (v0..v1).  The
    context keeps a reference to the tensor."""
    assert xg.is_cuda and xg.dtype == torch.float64 and xg.dim() == 2
    xg = xg.contiguous()
    check(nat.load().vegas_set_pdf_grid(ctx.handle, ctypes.c_void_p(xg.data_ptr()), int(xg.shape[0]),
                                        int(xg.shape[1]), float(u0), float(u1), float(v0), float(v1)),
          "vegas_set_pdf_grid")
    ctx.pdf_grid = xg


def vegas_get_strata(ctx: Context):
    """(B, P, n_used) of the next iteration (B = P = 0 when plain)."""
    B = ctypes.c_int32()
    P = ctypes.c_int64()
    n = ctypes.c_int64()
    check(nat.load().vegas_get_strata(ctx.handle, ctypes.byref(B), ctypes.byref(P), ctypes.byref(n)),
          "vegas_get_strata")
    return B.value, P.value, n.value


def vegas_export_state(ctx: Context) -> bytes:
    lib = nat.load()
    size = ctypes.c_size_t(0)
    check(lib.vegas_export_state(ctx.handle, None, ctypes.byref(size)), "vegas_export_state")
    buf = ctypes.create_string_buffer(size.value)
    check(lib.vegas_export_state(ctx.handle, buf, ctypes.byref(size)), "vegas_export_state")
    return buf.raw[: size.value]


def vegas_import_state(ctx: Context, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    check(nat.load().vegas_import_state(ctx.handle, buf, ctypes.c_size_t(len(blob))),
          "vegas_import_state")


def vegas_philox(ctr: torch.Tensor, key: torch.Tensor, stream=None) -> torch.Tensor:
    """Device Philox4x32-10: ctr (n, 4) and key (n, 2) int32/uint32 CUDA tensors."""
    assert ctr.is_cuda and key.is_cuda and ctr.shape[-1] == 4 and key.shape[-1] == 2
    ctr = ctr.contiguous()
    key = key.contiguous()
    out = torch.empty_like(ctr)
    _, sp = _stream_ptr(stream)
    check(nat.load().vegas_philox(ctypes.c_void_p(ctr.data_ptr()), ctypes.c_void_p(key.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), int(ctr.shape[0]), sp),
          "vegas_philox")
    return out


def vegas_iterate_noalloc(cfg: Config, family: str, params, t: int, edges: torch.Tensor,
                          sums: torch.Tensor, stream=None) -> None:
    """One iteration's sums without any device allocation by the library.

    For callers that cannot allocate device memory at call time (a runtime
    that owns the device's memory through its own pool, a plugin that must not
    grow the footprint).  ``edges`` (d x (N+1) float64) and ``sums``
    (3 + d*N float64: S1, S2, the histograms, the non-finite count) are the
    caller's CUDA tensors; scratch lives in a fixed array inside the library
    (n_dim * n_bins <= 4096).  Calls that overlap on the GPU race on that array.
    """
    assert edges.is_cuda and sums.is_cuda
    assert edges.dtype == torch.float64 and sums.dtype == torch.float64
    assert edges.is_contiguous() and sums.is_contiguous()
    assert edges.numel() == cfg.n_dim * (cfg.n_bins + 1) and sums.numel() >= 3 + cfg.n_dim * cfg.n_bins
    c = cfg.to_c()
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    itg = nat.VegasIntegrand(nat.FAMILIES[family], int(cfg.n_dim),
                             p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if p.size else None,
                             int(p.size))
    _, sp = _stream_ptr(stream)
    check(nat.load().vegas_iterate_noalloc(ctypes.byref(c), ctypes.byref(itg), int(t),
                                           ctypes.c_void_p(edges.data_ptr()),
                                           ctypes.c_void_p(sums.data_ptr()), sp),
          "vegas_iterate_noalloc")


def vegas_profile(ctx: Context, enable: bool = True) -> None:
    check(nat.load().vegas_profile(ctx.handle, 1 if enable else 0), "vegas_profile")


def vegas_profile_read(ctx: Context, cap: int = 1 << 16):
    """Sampling-kernel durations (ms) of the iterations since the last read."""
    buf = (ctypes.c_float * cap)()
    cnt = ctypes.c_int32()
    check(nat.load().vegas_profile_read(ctx.handle, buf, int(cap), ctypes.byref(cnt)),
          "vegas_profile_read")
    return [buf[i] for i in range(cnt.value)]


def vegas_destroy(ctx: Context) -> None:
    if ctx.handle:
        nat.load().vegas_destroy(ctx.handle)
        ctx.handle = None


class Integrator:
    """The paper's usage pattern (Sec. 3.1) over the C ABI.

    >>> it = Integrator(n_dim=10, n_events=10**6, events_limit=10**5)
    >>> it.compile("sum")
    >>> res = it.run_integration(n_iter=5)
    """

    def __init__(self, n_dim, n_events, events_limit=0, n_bins=50, alpha=1.5, seed=0,
                 integral_id=0, precision="fp32_kahan", smooth=True, stream=None, strata=0):
        self.cfg = Config(n_dim, n_events, n_bins, events_limit, alpha, seed, integral_id,
                          precision, smooth)
        self.stream = stream
        self.strata = strata   # vegas_set_strata's B: 0 plain, -1 automatic
        self.ctx = None

    def compile(self, integrand: str, params=()):
        """A built-in family's name, or CUDA C++ source defining user_integrand
        (the paper's compile(integrand); compiled at run time)."""
        if integrand in nat.FAMILIES:
            self.ctx = vegas_create(self.cfg, integrand, params, stream=self.stream)
        else:
            self.ctx = vegas_create(self.cfg, "user", params, stream=self.stream, source=integrand)
        if self.strata:
            vegas_set_strata(self.ctx, self.strata)
        return self

    def run_integration(self, n_iter: int):
        if self.ctx is None:
            raise RuntimeError("compile() an integrand first")
        return vegas_run(self.ctx, n_iter)


class Batch:
    """The batched form of the C ABI (vegas_batch_*): many integrals, one
    iteration of each per step, replayed as one CUDA graph.

    ``pool_bytes`` of device memory hold the added integrals' grids and
    accumulators (``vegas_batch_slot_bytes`` each); ``max_slots`` bounds their
    number.  Workspace from PyTorch.
    """

    def __init__(self, max_slots: int, pool_bytes: int, precision: str = "fp32_kahan",
                 stream=None, workspace=None):
        lib = nat.load()
        nbytes = lib.vegas_batch_workspace_bytes(int(max_slots), ctypes.c_size_t(int(pool_bytes)))
        if nbytes == 0:
            raise nat.VegasError(nat.VEGAS_EINVAL, "vegas_batch_workspace_bytes")
        if workspace is None:
            workspace = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self.precision = precision
        # default: the library's own stream (graphs cannot use the legacy stream)
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        torch.cuda.synchronize()  # the workspace allocation is complete
        h = ctypes.c_void_p()
        check(lib.vegas_batch_create(int(max_slots), nat.PRECISIONS[precision], sp,
                                     ctypes.c_void_p(workspace.data_ptr()),
                                     ctypes.c_size_t(workspace.numel()), ctypes.byref(h)),
              "vegas_batch_create")
        self.handle = h
        self.max_slots = int(max_slots)
        self._buf = (nat.VegasBatchResult * self.max_slots)()
        self.cfgs = {}
        self.families = {}

    @staticmethod
    def slot_bytes(cfg: Config) -> int:
        c = cfg.to_c()
        return int(nat.load().vegas_batch_slot_bytes(ctypes.byref(c)))

    def add(self, cfg: Config, family: str, params=()) -> int:
        """Admit an integral; raises VegasError with status EBUSY / ENOMEM when full."""
        c = cfg.to_c()
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        itg = nat.VegasIntegrand(nat.FAMILIES[family], int(cfg.n_dim),
                                 p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if p.size else None,
                                 int(p.size))
        slot = ctypes.c_int32()
        check(nat.load().vegas_batch_add(self.handle, ctypes.byref(c), ctypes.byref(itg),
                                         ctypes.byref(slot)), "vegas_batch_add")
        self.cfgs[int(slot.value)] = cfg
        self.families[int(slot.value)] = family
        return int(slot.value)

    def remove(self, slot: int) -> None:
        check(nat.load().vegas_batch_remove(self.handle, int(slot)), "vegas_batch_remove")
        self.cfgs.pop(int(slot), None)
        self.families.pop(int(slot), None)

    def step(self) -> None:
        check(nat.load().vegas_batch_step(self.handle), "vegas_batch_step")

    def wait(self):
        """Results of the last step: {slot: dict(t, I_t, sigma_t, n, n_nonfinite, I, sigma, chi2_dof, n_iter)}."""
        cnt = ctypes.c_int32()
        check(nat.load().vegas_batch_wait(self.handle, self._buf, self.max_slots, ctypes.byref(cnt)),
              "vegas_batch_wait")
        out = {}
        for k in range(cnt.value):
            r = self._buf[k]
            out[int(r.slot)] = {"t": r.t, "I_t": r.it.I, "sigma_t": r.it.sigma, "n": r.it.n,
                                "n_nonfinite": r.it.n_nonfinite, "I": r.comb.I,
                                "sigma": r.comb.sigma, "chi2_dof": r.comb.chi2_dof,
                                "n_iter": r.comb.n_iter}
        return out

    # the layout of vegas_batch_result as a numpy record
    RESULT_DTYPE = np.dtype([("slot", "<i4"), ("t", "<i4"), ("I_t", "<f8"), ("sigma_t", "<f8"),
                             ("n", "<i8"), ("n_nonfinite", "<i8"), ("I", "<f8"), ("sigma", "<f8"),
                             ("chi2_dof", "<f8"), ("n_iter", "<i4"), ("reserved", "<i4")])

    def wait_array(self) -> np.ndarray:
        """Results of the last step as a numpy record array (one entry per
        integral stepped; fields as vegas_batch_result), a copy."""
        cnt = ctypes.c_int32()
        check(nat.load().vegas_batch_wait(self.handle, self._buf, self.max_slots, ctypes.byref(cnt)),
              "vegas_batch_wait")
        return np.frombuffer(self._buf, dtype=self.RESULT_DTYPE, count=cnt.value).copy()

    def grid(self, slot: int) -> np.ndarray:
        cfg = self.cfgs[int(slot)]
        e = np.zeros((cfg.n_dim, cfg.n_bins + 1), dtype=np.float64)
        check(nat.load().vegas_batch_get_grid(self.handle, int(slot),
                                              e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
              "vegas_batch_get_grid")
        return e

    def set_events(self, slot: int, n_events: int) -> None:
        check(nat.load().vegas_batch_set_events(self.handle, int(slot), int(n_events)),
              "vegas_batch_set_events")
        self.cfgs[int(slot)].n_events = int(n_events)

    def set_tile(self, tile_samples: int) -> None:
        check(nat.load().vegas_batch_set_tile(self.handle, int(tile_samples)), "vegas_batch_set_tile")

    def autotune(self, candidates, reps: int = 3):
        """Time the sampling kernel per candidate tile size; keep the fastest."""
        cand = (ctypes.c_int32 * len(candidates))(*[int(c) for c in candidates])
        ms = (ctypes.c_float * len(candidates))()
        best = ctypes.c_int32()
        check(nat.load().vegas_batch_autotune(self.handle, cand, len(candidates), int(reps), ms,
                                              ctypes.byref(best)), "vegas_batch_autotune")
        return int(best.value), [float(x) for x in ms]

    def shape(self) -> dict:
        """The sampling kernel's launch shape: tile_samples, threads, layout."""
        sh = nat.VegasBatchShape()
        check(nat.load().vegas_batch_get_shape(self.handle, ctypes.byref(sh)), "vegas_batch_get_shape")
        return {"tile_samples": sh.tile_samples, "threads": sh.threads, "layout": sh.layout}

    def set_shape(self, tile_samples: int, threads: int, layout: int = -1) -> None:
        sh = nat.VegasBatchShape(int(tile_samples), int(threads), int(layout))
        check(nat.load().vegas_batch_set_shape(self.handle, ctypes.byref(sh)), "vegas_batch_set_shape")

    def tune_key(self) -> str:
        """Key of the autotuner's cache: precision, then the active slots'
        largest bin count and dimension and their families."""
        cfgs = list(self.cfgs.values())
        fams = sorted(set(self.families.values()))
        n_max = max((c.n_bins for c in cfgs), default=0)
        d_max = max((c.n_dim for c in cfgs), default=0)
        return "%s|N%d|d%d|%s" % (self.precision, n_max, d_max, ",".join(fams))

    def autotune_shapes(self, candidates, reps: int = 3, cache: str = None):
        """Pick the sampling kernel's launch shape (tile samples, threads per
        block, shared-memory layout) for the current slots.  ``candidates``:
        (tile_samples, threads, layout) triples.  With ``cache`` (a JSON file
        path) a shape stored under this batch's tune_key() is applied without
        measuring, and a measured one is stored.  Returns (shape dict, times
        in ms per candidate or None when taken from the cache)."""
        import json
        import os
        key = self.tune_key()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            hit = table.get(key)
            if hit is not None:
                try:
                    self.set_shape(hit["tile_samples"], hit["threads"], hit["layout"])
                    return self.shape(), None
                except nat.VegasError:
                    pass  # no longer fits: measure again
        arr = (nat.VegasBatchShape * len(candidates))(
            *[nat.VegasBatchShape(int(t), int(th), int(lay)) for t, th, lay in candidates])
        ms = (ctypes.c_float * len(candidates))()
        best = ctypes.c_int32()
        check(nat.load().vegas_batch_autotune_shapes(self.handle, arr, len(candidates), int(reps), ms,
                                                     ctypes.byref(best)), "vegas_batch_autotune_shapes")
        shape = self.shape()
        times = [float(x) for x in ms]
        if cache:
            table[key] = dict(shape, ms=times[best.value])
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            tmp = cache + ".tmp%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return shape, times

    def info(self):
        n = ctypes.c_int32()
        free = ctypes.c_size_t()
        largest = ctypes.c_size_t()
        tile = ctypes.c_int32()
        check(nat.load().vegas_batch_info(self.handle, ctypes.byref(n), ctypes.byref(free),
                                          ctypes.byref(largest), ctypes.byref(tile)),
              "vegas_batch_info")
        return {"n_active": n.value, "pool_free": free.value, "pool_largest": largest.value,
                "tile_samples": tile.value}

    def close(self) -> None:
        if getattr(self, "handle", None):
            nat.load().vegas_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
