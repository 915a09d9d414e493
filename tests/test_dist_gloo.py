"""Multi-rank orchestration on CPU ranks (gloo, world size 2).

The shard interface is backed by the FP64 oracle here (a test double of the
C-ABI context), so the sharding, the all-reduce of the accumulators and the
identical finalize/refine on every rank run without a GPU.  Parity: the
sharded run equals the single-rank oracle run to 1e-12.
"""
import datetime
import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2010_09341_gb300 import dist as D
from paper_2010_09341_gb300 import workloads as W


class OracleShard:
    """Shard interface over the oracle: accumulators in a CPU float64 tensor."""

    def __init__(self, family, d, N, n, params, seed=0, iid=0, alpha=1.5):
        self.family, self.d, self.N, self.n_events = family, d, N, n
        self.params, self.seed, self.iid, self.alpha = params, seed, iid, alpha
        self.edges = O.uniform_edges(d, N)
        self.t = 0
        self.sums = torch.zeros(2 + d * N, dtype=torch.float64)
        self.nonfinite = torch.zeros(1, dtype=torch.int64)
        self.log = []

    def sample_shard(self, s0, count):
        self.log.append("sample")
        acc = O.iterate(self.d, self.N, self.edges, self.family, self.params, self.seed, self.iid,
                        self.t, self.n_events, s_begin=s0, s_end=s0 + count)
        self.sums.zero_()
        self.sums[0] = acc["S1"]
        self.sums[1] = acc["S2"]
        self.sums[2:] = torch.from_numpy(acc["hist"].reshape(-1))
        self.nonfinite[0] = acc["n_nonfinite"]

    def accumulators(self):
        return self.sums, self.nonfinite

    def exchange_begin(self):
        self.log.append("begin")
        self.pre = float(self.sums[0])

    def exchange_end(self):
        # the collective has summed the accumulators by now
        self.log.append("end" if float(self.sums[0]) != self.pre else "end-unsummed")

    def finalize(self):
        self.log.append("finalize")
        ne = self.n_events - int(self.nonfinite[0])
        I, var = O.iteration_result(float(self.sums[0]), float(self.sums[1]), ne)
        self.t += 1
        return I, float(np.sqrt(var)), ne, int(self.nonfinite[0])

    def refine(self):
        h = self.sums[2:].numpy().reshape(self.d, self.N)
        self.edges = O.refine(self.d, self.N, h, self.edges, self.alpha)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, N, n = 4, 20, 20_003
        p = W.genz_params("genz_gauss", d, seed=9)
        sh = OracleShard("genz_gauss", d, N, n, p, seed=3, iid=5)
        its = D.sharded_run(sh, 3)
        slow = D.max_over_ranks(1.0 + rank)
        q.put((rank, its, sh.edges, slow, sh.log))
    finally:
        dist.destroy_process_group()


def test_sharded_run_equals_single_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda x: x[0])
    d, N, n = 4, 20, 20_003
    p = W.genz_params("genz_gauss", d, seed=9)
    ref = O.integrate(d, N, "genz_gauss", p, n, 3, seed=3, integral_id=5)
    for rank, its, edges, slow, log in out:
        assert slow == 2.0  # the slowest rank's value on every rank
        # the exchange hooks bracket the collective of every iteration
        assert log == ["sample", "begin", "end", "finalize"] * 3
        for (I, s, ne, nf), (Io, so) in zip(its, ref["iters"]):
            assert abs(I - Io) <= 1e-12 * abs(Io)
            assert abs(s - so) <= 1e-9 * so
    # every rank refined to the same grid
    assert np.array_equal(out[0][2], out[1][2])


def test_shard_ranges_partition_the_samples():
    for n in (1, 2, 7, 1000, 10 ** 7 + 3):
        for world in (1, 2, 3, 8):
            got = [D.shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0
            assert sum(c for _, c in got) == n
            for (a, ca), (b, _) in zip(got, got[1:]):
                assert a + ca == b


def test_replica_ids_distinct():
    ids = [i for r in range(4) for i in D.replica_integral_ids(r, 2)]
    assert len(set(ids)) == len(ids) == 8


def _leaving_worker(rank, world, port, q):
    """Rank 1 takes part in one iteration and then leaves without a word;
    rank 0 goes on to a second iteration, whose exchange must fail."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    d, N, n = 3, 20, 10_001
    p = W.genz_params("genz_gauss", d, seed=9)
    sh = OracleShard("genz_gauss", d, N, n, p, seed=3, iid=5)
    first = D.sharded_iterate(sh)
    if rank == 1:
        time.sleep(1.0)          # the peer's first exchange is complete by now
        q.put((rank, "left", first, ""))
        q.close()
        q.join_thread()
        os._exit(0)              # no goodbye: the process group is not destroyed
    sh.refine()
    t0 = time.time()
    try:
        D.sharded_iterate(sh)
        q.put((rank, "no error", first, ""))
    except D.ShardLost as e:
        q.put((rank, "lost after %.1f s" % (time.time() - t0), first, str(e)))
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_rank_that_leaves_is_detected():
    """Failure detection on the host, no GPU involved: when a rank dies
    between iterations, the survivor's next exchange raises ShardLost (the
    dropped connection, or at worst the group's 20 s timeout) instead of
    hanging, and the iteration before it is still the single-rank result."""
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_leaving_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out = dict((r[0], r[1:]) for r in out)
    assert out[1][0] == "left"
    status, first, msg = out[0]
    assert status.startswith("lost"), status
    assert "exchange failed" in msg
    d, N, n = 3, 20, 10_001
    p = W.genz_params("genz_gauss", d, seed=9)
    ref = O.integrate(d, N, "genz_gauss", p, n, 1, seed=3, integral_id=5)
    Io, so = ref["iters"][0]
    assert abs(first[0] - Io) <= 1e-12 * abs(Io) and out[1][1][0] == first[0]
