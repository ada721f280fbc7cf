"""Multi-process paths on CPU (gloo, world_size 2): request sharding across ranks and the
whole-job statistics, and the benchmark's max-over-ranks timing."""
import os
import socket
import time

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_01855_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2509_01855_gb300.serve import (SlotPool, combine_stats, run_schedule,
                                                  shard_requests)
        import bench
        reqs = synth.serving_requests(40, rate=400.0, kmin=8, kmax=10)
        mine = shard_requests(reqs, rank, world)

        class S:
            def __init__(self, N):
                self.N, self.nbytes = N, 1

        pool = SlotPool(10 ** 9, 3, lambda N: S(N), lambda s: None, lambda N: 1)

        def solve(slot, req):
            time.sleep(0.002 * (1 + rank))
            return {"status": "ok"}

        t0 = time.perf_counter()
        res = run_schedule(mine, pool, solve, n_workers=3, realtime=True)
        st = combine_stats(res, time.perf_counter() - t0, dist)
        mx = bench.max_over_ranks(float(rank + 1), dist)
        q.put((rank, [r["id"] for r in res], st, mx))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_combine():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    ids0, ids1 = set(out[0][1]), set(out[1][1])
    assert not (ids0 & ids1) and len(ids0 | ids1) == 40      # every request exactly once
    for _, _, st, mx in out:
        assert st["requests"] == 40 and st["solved"] == 40 and st["ranks"] == 2
        assert mx == 2.0                                        # max over ranks
    assert out[0][2]["p99_ms"] == out[1][2]["p99_ms"]           # same whole-job statistics
