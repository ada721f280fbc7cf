"""Host logic of the serving loop (no GPU): admission by slot count and memory, continuous
batching, failure isolation."""
import threading
import time

import pytest

from paper_2509_01855_gb300.serve import SlotPool, run_schedule, summarize


class FakeSlot:
    def __init__(self, N, nbytes):
        self.N = N
        self.nbytes = nbytes


def _pool(budget, max_slots, log):
    def make(N):
        log.append(("make", N))
        return FakeSlot(N, N)          # bytes = N

    def free(s):
        log.append(("free", s.N))
    return SlotPool(budget, max_slots, make, free, lambda N: N)


def test_admission_reuses_and_evicts():
    log = []
    pool = _pool(budget=1100, max_slots=3, log=log)
    a = pool.try_acquire(256)
    b = pool.try_acquire(512)
    assert pool.try_acquire(512) is None          # 256 + 512 + 512 > 1100, nothing idle
    pool.release(a)
    c = pool.try_acquire(256)                      # reuses the idle 256 slot
    assert c is a and log.count(("make", 256)) == 1
    pool.release(c)
    d = pool.try_acquire(512)                      # evicts the idle 256 slot to fit
    assert d is not None and d.N == 512 and ("free", 256) in log
    assert pool.used == 1024 and pool.evicted == 1
    with pytest.raises(MemoryError):
        pool.try_acquire(4096)                     # one slot larger than the whole budget


def test_slot_count_limit():
    log = []
    pool = _pool(budget=10 ** 9, max_slots=2, log=log)
    s1 = pool.try_acquire(8)
    s2 = pool.try_acquire(8)
    assert pool.try_acquire(8) is None
    pool.release(s1)
    assert pool.try_acquire(8) is s1
    del s2


def test_continuous_batching_overlaps_and_isolates_failures():
    log = []
    pool = _pool(budget=10 ** 9, max_slots=4, log=log)
    active = {"now": 0, "peak": 0}
    lock = threading.Lock()

    def solve(slot, req):
        with lock:
            active["now"] += 1
            active["peak"] = max(active["peak"], active["now"])
        time.sleep(0.02)
        with lock:
            active["now"] -= 1
        if req["id"] == 3:
            raise RuntimeError("injected failure")
        return {"status": "ok", "value": req["id"] * 2}

    reqs = [dict(id=i, arrival=0.002 * i, N=256 << (i % 3)) for i in range(16)]
    res = run_schedule(reqs, pool, solve, n_workers=4, realtime=True)
    assert [r["id"] for r in res] == list(range(16))
    assert active["peak"] >= 2                     # requests overlapped
    assert res[3]["status"] == "error" and "injected" in res[3]["error"]
    assert all(r["status"] == "ok" and r["value"] == 2 * r["id"] for r in res if r["id"] != 3)
    assert all(r["latency"] >= r["service"] - 1e-9 for r in res)
    st = summarize(res, 1.0)
    assert st["solved"] == 15 and st["failed"] == 1
    # later requests were admitted while earlier ones were still running
    assert min(r["t_admit"] for r in res if r["id"] >= 4) < max(r["t_done"] for r in res if r["id"] < 4)
