"""Several devices or processes for one integral, over torch.distributed.

One VEGAS integral shards naturally: sample s of iteration t draws the same
Philox words on every device, so rank r takes the contiguous sample range
[r n / R, (r+1) n / R) of each iteration, the ranks sum their accumulators
(S1, S2, histograms, non-finite count) with one all-reduce, and every rank
then finalizes and refines identically -- the paper's multi-device use of one
integration, where each iteration's partial results are combined before the
grid is refined (Sec. 3.1, Sec. 3.2).  The union of the shards is exactly the
single-device iteration.

The orchestration here works on any object with the shard interface
(``sample_shard``, ``accumulators``, ``finalize``, ``refine``, and optionally
``exchange_begin`` / ``exchange_end``, called around the collective);
:class:`GpuShard` adapts a C-ABI context.  Independent integrals need no
exchange: they run as replicas (one set per rank).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class ShardLost(RuntimeError):
    """The exchange of an iteration failed: a rank of the group left, died or
    did not answer within the process group's timeout.  The iteration's sums
    are incomplete, so it is not finalized; the caller decides whether to
    rebuild the group or give up."""


def shard_range(n: int, rank: int, world: int):
    """(first sample, count) of rank's share of n samples."""
    s0 = (rank * n) // world
    s1 = ((rank + 1) * n) // world
    return s0, s1 - s0


class GpuShard:
    """Shard interface over a C-ABI context (paper_2010_09341_gb300.vegas)."""

    def __init__(self, ctx):
        from . import vegas as V
        self.V = V
        self.ctx = ctx

    @property
    def n_events(self) -> int:
        return self.ctx.cfg.n_events

    def sample_shard(self, s0: int, count: int) -> None:
        self.V.vegas_sample_shard(self.ctx, s0, count)

    def accumulators(self):
        return self.V.vegas_accumulators(self.ctx)

    def exchange_begin(self) -> None:
        # The accumulators are written on the context's stream, which need not
        # be the stream the collective orders itself after.
        self.ctx.stream.synchronize()

    def exchange_end(self) -> None:
        # The collective wrote the summed accumulators in the order of the
        # current stream; finalize reads them on the context's stream.
        self.ctx.stream.wait_stream(torch.cuda.current_stream(self.ctx.stream.device))

    def finalize(self):
        return self.V.vegas_finalize(self.ctx, sync=True)

    def refine(self) -> None:
        self.V.vegas_refine(self.ctx)


def sharded_iterate(shard, group=None):
    """One iteration of one integral over all ranks of ``group``; returns the
    iteration result (I, sigma, n, n_nonfinite), the same on every rank."""
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    s0, count = shard_range(shard.n_events, rank, world)
    shard.sample_shard(s0, count)
    sums, nonfinite = shard.accumulators()
    begin = getattr(shard, "exchange_begin", None)
    if begin is not None:
        begin()
    try:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(nonfinite, op=dist.ReduceOp.SUM, group=group)
    except RuntimeError as e:  # a lost peer or a timeout (the backends raise RuntimeError subclasses)
        raise ShardLost("rank %d of %d: the iteration's exchange failed: %s" % (rank, world, e)) from e
    end = getattr(shard, "exchange_end", None)
    if end is not None:
        end()
    return shard.finalize()


def sharded_run(shard, n_iter: int, group=None):
    """run_integration over the ranks: n_iter rounds of sharded iterate and
    refine (no refine after the last).  Returns the per-iteration results."""
    out = []
    for k in range(n_iter):
        out.append(sharded_iterate(shard, group))
        if k + 1 < n_iter:
            shard.refine()
    return out


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Largest value of x over the ranks (timings are taken as the slowest rank)."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def replica_integral_ids(rank: int, per_rank: int):
    """Distinct Philox integral ids for a rank's replicas (weak scaling)."""
    return [rank * per_rank + k for k in range(per_rank)]
