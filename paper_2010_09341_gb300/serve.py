"""Continuous-batching server of VEGAS integrations over the batched C ABI.

Requests (integrand family, dimension, parameters, relative-error target,
sample budget) arrive over time.  Every loop turn the server

  1. admits arrived requests while a slot and pool memory are free
     (``vegas_batch_add`` refuses with EBUSY / ENOMEM otherwise; refused
     requests wait in arrival order),
  2. runs one batched step -- one VEGAS iteration of every admitted
     integral in one graph launch -- so new work overlaps the old on the GPU,
  3. retires every integral whose combined estimate reached its target
     (sigma / |I| <= target after at least ``min_iters`` iterations) or whose
     budget is spent, and records its latency (arrival to retirement).

A request may be cancelled between steps (``Server.cancel``): it leaves the
queue or frees its slot at once and is reported as cancelled, not completed.
The summary adds the admission refusals (slot or pool full), the longest
queue and the fraction of the wall time spent waiting for batched steps.

Samples per iteration: ``n_first`` for the first ``warm_iters`` iterations
(grid adaptation), then what the target needs from the current estimate,
n = total_needed / remaining_iterations, rounded up to a power of two and
kept within [n_first, n_cap] and the budget, where n_cap = max(n_max,
step_samples / active integrals): when few integrals are active their
iterations grow so that a step still fills the GPU.

Give-up rule: from ``give_up_after`` iterations on, an integral whose
projected total, used * (rel / target)^2, exceeds ``give_up`` times its
budget is retired unconverged at once instead of spending the rest of the
budget (the projection assumes the per-sample variance stays as it is; grid
adaptation only lowers it, hence the factor).

The paper's own distribution of one integration over devices (Sec. 3.1,
3.2) is not a server; this module is the serving form of the method.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import vegas as V
from ._native import VEGAS_EBUSY, VEGAS_ENOMEM, VegasError


@dataclass
class Request:
    family: str
    d: int
    params: np.ndarray
    target_rel: float
    budget: int = 10 ** 9
    arrival: float = 0.0
    seed: int = 0
    integral_id: int = 0
    n_bins: int = 50
    alpha: float = 1.5
    # filled by the server
    admitted: float = -1.0
    done: float = -1.0
    result: dict = field(default_factory=dict)
    converged: bool = False
    gave_up: bool = False
    cancelled: bool = False


def _pow2_ceil(x: float) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1.0, x)))))


@dataclass
class SamplePolicy:
    """Samples per iteration and the give-up rule (module docstring)."""
    n_first: int = 1 << 17
    n_max: int = 1 << 24
    warm_iters: int = 2
    iters_to_target: int = 4
    adaptive: bool = True
    step_samples: int = 1 << 28
    give_up: float = 4.0
    give_up_after: int = 6

    def first_n(self, r: Request) -> int:
        return min(self.n_first, max(2, r.budget))

    def next_n(self, r: Request, used: int, res: dict, n_active: int = 1) -> int:
        """Samples for the next iteration of one integral."""
        m = res["n_iter"]
        left = r.budget - used
        if not self.adaptive or m < self.warm_iters or res["sigma"] <= 0 or res["I"] == 0:
            return max(2, min(self.n_first, left))
        rel = res["sigma"] / abs(res["I"])
        need_total = used * (rel / r.target_rel) ** 2
        more = max(0.0, need_total - used)
        n = _pow2_ceil(more / self.iters_to_target)
        n_cap = max(self.n_max, _pow2_ceil(self.step_samples / max(1, n_active)) // 2)
        return int(max(2, min(max(self.n_first, n), n_cap, left)))

    def hopeless(self, r: Request, used: int, res: dict) -> bool:
        """The projected total exceeds give_up x budget."""
        if self.give_up <= 0 or res["n_iter"] < self.give_up_after or res["sigma"] <= 0 or res["I"] == 0:
            return False
        rel = res["sigma"] / abs(res["I"])
        return used * (rel / r.target_rel) ** 2 > self.give_up * r.budget

    # -- the same rules over arrays (one entry per active integral) --------
    @staticmethod
    def _pow2_ceil_array(x):
        # exponents above 62 would overflow int64; every cap applied afterwards is smaller
        e = np.minimum(62.0, np.maximum(0.0, np.ceil(np.log2(np.maximum(1.0, x)))))
        return np.left_shift(np.int64(1), e.astype(np.int64))

    def next_n_array(self, budget, target, used, n_iter, I, sigma, n_active: int):
        """next_n for every entry: int64 array."""
        left = budget - used
        warm = (n_iter < self.warm_iters) | (sigma <= 0) | (I == 0)
        if not self.adaptive:
            warm = np.ones_like(warm)
        # entries that take the first-iterations rule (warm) may divide by zero
        # here; their value is not used
        with np.errstate(divide="ignore", invalid="ignore"):
            rel = np.where(I != 0, sigma / np.abs(I), 0.0)
            need_total = used * (rel / target) ** 2
        more = np.maximum(0.0, need_total - used)
        n = self._pow2_ceil_array(more / self.iters_to_target)
        n_cap = max(self.n_max, _pow2_ceil(self.step_samples / max(1, n_active)) // 2)
        adapt = np.maximum(2, np.minimum(np.minimum(np.maximum(self.n_first, n), n_cap), left))
        first = np.maximum(2, np.minimum(self.n_first, left))
        return np.where(warm, first, adapt).astype(np.int64)

    def hopeless_array(self, budget, target, used, n_iter, I, sigma):
        """hopeless for every entry: bool array."""
        if self.give_up <= 0:
            return np.zeros(len(used), dtype=bool)
        ok = (n_iter >= self.give_up_after) & (sigma > 0) & (I != 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            rel = np.where(I != 0, sigma / np.abs(I), 0.0)
            return ok & (used * (rel / target) ** 2 > self.give_up * budget)


class Server:
    """Tiles of 2^17 samples by default: at saturation (1e4 requests/s) the
    served mix ran 576 integrals/s with the batch's default 8192-sample tiles,
    652 with 32768, 666 with 131072 and 658 with 262144 (one GB300)."""

    def __init__(self, max_slots: int = 1024, pool_bytes: int = 512 << 20,
                 precision: str = "fp32_kahan", n_first: int = 1 << 17, n_max: int = 1 << 24,
                 warm_iters: int = 2, min_iters: int = 3, iters_to_target: int = 4,
                 adaptive: bool = True, tile_samples: int | None = 1 << 17,
                 step_samples: int = 1 << 28, give_up: float = 4.0, give_up_after: int = 6):
        self.batch = V.Batch(max_slots=max_slots, pool_bytes=pool_bytes, precision=precision)
        if tile_samples:
            self.batch.set_tile(tile_samples)
        self.precision = precision
        self.policy = SamplePolicy(int(n_first), int(n_max), warm_iters, iters_to_target, adaptive,
                                   int(step_samples), float(give_up), int(give_up_after))
        self.min_iters = min_iters
        self.active = {}      # slot -> [Request, samples used, n per iteration]
        self.queue = []       # arrived, not yet admitted (arrival order)
        self.steps = 0
        self.samples = 0
        self.refusals = 0     # admissions refused because the slots or the pool were full
        self.max_queue = 0
        self.busy_s = 0.0     # wall time inside the batched steps (launch to results)
        self.cancelled = []
        # per-slot state as arrays, for the vectorised step
        self.used = np.zeros(max_slots, dtype=np.int64)
        self.n_cur = np.zeros(max_slots, dtype=np.int64)
        self.budget = np.zeros(max_slots, dtype=np.float64)
        self.target = np.zeros(max_slots, dtype=np.float64)

    def _admit(self, now: float) -> None:
        while self.queue:
            r = self.queue[0]
            n0 = self.policy.first_n(r)
            cfg = V.Config(n_dim=r.d, n_events=n0, n_bins=r.n_bins, alpha=r.alpha, seed=r.seed,
                           integral_id=r.integral_id, precision=self.precision)
            try:
                slot = self.batch.add(cfg, r.family, r.params)
            except VegasError as e:
                if e.status in (VEGAS_EBUSY, VEGAS_ENOMEM):
                    self.refusals += 1
                    return  # full: wait for retirements
                raise
            r.admitted = now
            self.active[slot] = [r, 0, n0]
            self.used[slot] = 0
            self.n_cur[slot] = n0
            self.budget[slot] = r.budget
            self.target[slot] = r.target_rel
            self.queue.pop(0)

    def step(self, now_fn) -> list:
        """One batched iteration of all active integrals; returns retired requests.

        The rules run over arrays of all active integrals at once (the
        SamplePolicy array forms); only integrals that retire or change their
        samples per iteration are touched one by one."""
        if not self.active:
            return []
        t0 = time.perf_counter()
        self.batch.step()
        a = self.batch.wait_array()
        self.busy_s += time.perf_counter() - t0
        self.steps += 1
        now = now_fn()
        slots = a["slot"].astype(np.int64)
        used = self.used[slots] + a["n"] + a["n_nonfinite"]
        self.used[slots] = used
        self.samples += int(self.n_cur[slots].sum())
        I, sigma, m = a["I"], a["sigma"], a["n_iter"]
        budget, target = self.budget[slots], self.target[slots]
        conv = (m >= self.min_iters) & (sigma <= target * np.abs(I)) & (I != 0)
        hopeless = ~conv & (used < budget) & self.policy.hopeless_array(budget, target, used, m, I, sigma)
        done = conv | (used >= budget) | hopeless
        retired = []
        for k in np.flatnonzero(done):
            slot = int(slots[k])
            r = self.active.pop(slot)[0]
            r.done = now
            r.converged = bool(conv[k])
            r.gave_up = bool(hopeless[k])
            r.result = {"t": int(a["t"][k]), "I_t": float(a["I_t"][k]), "sigma_t": float(a["sigma_t"][k]),
                        "n": int(a["n"][k]), "n_nonfinite": int(a["n_nonfinite"][k]), "I": float(I[k]),
                        "sigma": float(sigma[k]), "chi2_dof": float(a["chi2_dof"][k]), "n_iter": int(m[k]),
                        "samples": int(used[k])}
            self.batch.remove(slot)
            retired.append(r)
        keep = ~done
        if keep.any():
            nn = self.policy.next_n_array(budget[keep], target[keep], used[keep], m[keep], I[keep], sigma[keep],
                                          len(self.active))
            ks = slots[keep]
            for slot, n_new in zip(ks[nn != self.n_cur[ks]], nn[nn != self.n_cur[ks]]):
                self.batch.set_events(int(slot), int(n_new))
            self.n_cur[ks] = nn
            for slot, n_new in zip(ks, nn):
                rec = self.active[int(slot)]
                rec[1] = int(self.used[slot])
                rec[2] = int(n_new)
        return retired

    def cancel(self, r: Request, now: float) -> bool:
        """Withdraw a queued or active request between steps; False if it is
        neither (not yet arrived, or already retired)."""
        k = next((k for k, q in enumerate(self.queue) if q is r), None)
        if k is not None:
            self.queue.pop(k)
        else:
            slot = next((s for s, rec in self.active.items() if rec[0] is r), None)
            if slot is None:
                return False
            self.active.pop(slot)
            self.batch.remove(slot)
        r.cancelled = True
        r.done = now
        self.cancelled.append(r)
        return True

    def run(self, requests, time_limit: float = 60.0, realtime: bool = True, on_step=None):
        """Serve ``requests`` (sorted by arrival time, seconds from start).

        With ``realtime`` the arrivals follow the wall clock; otherwise every
        request is queued at start.  ``on_step(server, now)`` runs after every
        step (it may cancel requests).  Returns summary statistics.
        """
        pending = sorted(requests, key=lambda q: q.arrival)
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0)
        done = []
        i = 0
        while True:
            now = clock()
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                self.queue.append(pending[i])
                i += 1
            self.max_queue = max(self.max_queue, len(self.queue))
            self._admit(now)
            if not self.active:
                if i >= len(pending) and not self.queue:
                    break
                if realtime and i < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[i].arrival - clock())))
                continue
            done.extend(self.step(clock))
            if on_step is not None:
                on_step(self, clock())
            if clock() > time_limit:
                break
        wall = clock()
        out = summarize(done, wall, self.steps, self.samples, len(requests))
        out.update({"cancelled": len(self.cancelled), "admit_refusals": self.refusals,
                    "max_queue": self.max_queue, "busy_frac": self.busy_s / wall if wall > 0 else 0.0})
        return out


def summarize(done, wall: float, steps: int, samples: int, n_requests: int) -> dict:
    lat = np.array([r.done - r.arrival for r in done]) if done else np.zeros(0)
    conv = sum(1 for r in done if r.converged)
    return {
        "requests": n_requests, "completed": len(done), "converged": conv,
        "gave_up": sum(1 for r in done if r.gave_up),
        "wall_s": wall, "integrals_per_s": len(done) / wall if wall > 0 else 0.0,
        "converged_per_s": conv / wall if wall > 0 else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
        "steps": steps, "samples": samples,
        "samples_per_s": samples / wall if wall > 0 else 0.0,
    }


def serve_single_fp64(requests, n_first: int = 1 << 17, n_max: int = 1 << 24, warm_iters: int = 2,
                      min_iters: int = 3, iters_to_target: int = 4, time_limit: float = 60.0,
                      step_samples: int = 1 << 28, give_up: float = 4.0, give_up_after: int = 6):
    """The plain FP64 single-integral form: one context per request, one at a
    time, the same sample schedule, stopping and give-up rules as the server
    (one integral active, so its iterations may grow to step_samples / 2)."""
    t0 = time.perf_counter()
    done = []
    samples = 0
    steps = 0
    policy = SamplePolicy(n_first, n_max, warm_iters, iters_to_target, True, int(step_samples),
                          float(give_up), int(give_up_after))
    for r in sorted(requests, key=lambda q: q.arrival):
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        n = policy.first_n(r)
        cfg = V.Config(n_dim=r.d, n_events=n, n_bins=r.n_bins, alpha=r.alpha, seed=r.seed,
                       integral_id=r.integral_id, precision="fp64")
        ctx = V.vegas_create(cfg, r.family, r.params)
        used = 0
        while True:
            V.vegas_step(ctx, sync=True)  # iterate + refine (a refine after the last is unused)
            steps += 1
            samples += n
            used += n
            res = V.vegas_result(ctx)
            conv = res["n_iter"] >= min_iters and res["sigma"] <= r.target_rel * abs(res["I"]) and res["I"] != 0
            hopeless = not conv and used < r.budget and policy.hopeless(r, used, res)
            if conv or used >= r.budget or hopeless:
                r.converged = bool(conv)
                r.gave_up = bool(hopeless)
                r.result = dict(res)
                r.result["samples"] = used
                break
            nn = policy.next_n(r, used, res)
            if nn != n:
                V.vegas_set_events(ctx, nn)
                n = nn
        V.vegas_destroy(ctx)
        r.done = time.perf_counter() - t0
        done.append(r)
        if r.done > time_limit:
            break
    return summarize(done, time.perf_counter() - t0, steps, samples, len(requests))


def requests_from(integrals, budget: int | None = None, target: float | None = None):
    """Requests from workload ``Integral`` records (see workloads.request_stream)."""
    out = []
    for it in integrals:
        out.append(Request(family=it.family, d=it.d, params=np.asarray(it.params, dtype=np.float64),
                           target_rel=target if target is not None else it.target_rel,
                           budget=budget if budget is not None else (it.budget or 10 ** 9),
                           arrival=it.arrival, seed=it.seed, integral_id=it.integral_id,
                           n_bins=it.n_bins, alpha=it.alpha))
    return out
