"""Serving: continuous batching of Newton-Krylov trajectory solves on one GPU.

Requests (orbit raising with grid size N, target radius r_f, final time t_f) arrive over time.
A request is admitted as soon as a solver slot for its N is free or device memory allows a new
one; admitted requests run concurrently, each slot on its own CUDA stream driven by its own
host thread (the C calls release the GIL), so their kernels overlap on the device. A slot owns
a bk_problem of its grid size, a Newton workspace and pinned host buffers, and is reused by
later requests of the same N (bk_problem_set_params); idle slots of other sizes are evicted
when memory or the slot cache is full. Each request's result does not depend on what else runs: every slot has
its own buffers and every reduction has a fixed order.

Latency = time the solution reaches host memory - arrival time.
"""
import collections
import threading
import time

import numpy as np

A_NOMINAL = 0.01


class SlotPool:
    """Admission by slot count and device-memory budget (host logic, no GPU).

    make_slot(N) -> slot object with attributes N and nbytes; free_slot(slot) releases it.
    """

    def __init__(self, budget_bytes, max_slots, make_slot, free_slot, slot_bytes):
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.make_slot = make_slot
        self.free_slot = free_slot
        self.slot_bytes = slot_bytes          # N -> bytes estimate before creation
        self.idle = collections.OrderedDict()  # id(slot) -> slot, least recently used first
        self.busy = {}
        self.used = 0
        self.created = 0
        self.evicted = 0

    def _count(self):
        return len(self.idle) + len(self.busy)

    def try_acquire(self, N):
        for k, s in self.idle.items():
            if s.N == N:
                del self.idle[k]
                self.busy[k] = s
                return s
        need = self.slot_bytes(N)
        if need > self.budget:
            raise MemoryError("one slot of N=%d needs %d bytes, more than the budget %d"
                              % (N, need, self.budget))
        # evict idle slots of other sizes (least recently used first) until the new one fits
        while (self.used + need > self.budget or self._count() >= self.max_slots) and self.idle:
            k, s = next(iter(self.idle.items()))
            del self.idle[k]
            self.used -= s.nbytes
            self.free_slot(s)
            self.evicted += 1
        if self.used + need > self.budget or self._count() >= self.max_slots:
            return None
        s = self.make_slot(N)
        self.used += s.nbytes
        self.created += 1
        self.busy[id(s)] = s
        return s

    def release(self, slot):
        del self.busy[id(slot)]
        self.idle[id(slot)] = slot

    def close(self):
        for s in list(self.idle.values()) + list(self.busy.values()):
            self.free_slot(s)
        self.idle.clear()
        self.busy.clear()
        self.used = 0


def run_schedule(requests, pool, solve, n_workers, realtime=True, clock=time.perf_counter):
    """Continuous batching driver (host logic). requests: dicts with id, arrival (s), N.
    solve(slot, req) -> dict. Returns the list of per-request results (dicts with latency)."""
    cv = threading.Condition()
    pending = []
    results = []
    state = {"done_arrivals": False, "error": None}
    t_start = clock()

    def worker():
        while True:
            with cv:
                while True:
                    if state["error"] is not None:
                        return
                    pick = None
                    for i, req in enumerate(pending):
                        try:
                            slot = pool.try_acquire(req["N"])
                        except MemoryError as e:
                            pick = (i, None, req, str(e))
                            break
                        if slot is not None:
                            pick = (i, slot, req, None)
                            break
                    if pick is not None:
                        del pending[pick[0]]
                        break
                    if state["done_arrivals"] and not pending:
                        return
                    cv.wait(timeout=0.005)
            i, slot, req, err = pick
            t0 = clock()
            if slot is None:
                res = {"status": "rejected", "error": err}
            else:
                try:
                    res = solve(slot, req)
                except Exception as e:  # a failed request must not stop the server
                    res = {"status": "error", "error": repr(e)}
            t1 = clock()
            arrival_abs = t_start + req["arrival"] if realtime else t0
            res.update(id=req["id"], N=req["N"], t_admit=t0 - t_start, t_done=t1 - t_start,
                       latency=t1 - arrival_abs, service=t1 - t0)
            with cv:
                if slot is not None:
                    pool.release(slot)
                results.append(res)
                cv.notify_all()

    threads = [threading.Thread(target=worker, daemon=True) for _ in range(n_workers)]
    for th in threads:
        th.start()
    for req in sorted(requests, key=lambda r: r["arrival"]):
        if realtime:
            delay = t_start + req["arrival"] - clock()
            if delay > 0:
                time.sleep(delay)
        with cv:
            pending.append(req)
            cv.notify_all()
    with cv:
        state["done_arrivals"] = True
        cv.notify_all()
    for th in threads:
        th.join()
    return sorted(results, key=lambda r: r["id"])


def summarize(results, wall):
    ok = [r for r in results if r.get("status") == "ok"]
    lat = np.array([r["latency"] for r in ok]) if ok else np.array([np.nan])
    return {"requests": len(results), "solved": len(ok),
            "failed": len(results) - len(ok),
            "solves_per_s": len(ok) / wall if wall > 0 else float("nan"),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(np.mean(lat) * 1e3), "wall_s": wall}


class Server:
    """GPU server for orbit-raising requests (one bk_problem per slot, one stream per slot)."""

    def __init__(self, dtype=None, max_slots=16, budget_bytes=None, newton_opts=None, restart=30, cache_slots=None):
        """max_slots: concurrent solves (worker threads, streams). cache_slots: solver slots kept
        (busy + idle; default 4 x max_slots) within the memory budget, so that idle slots of
        every size stay for later requests instead of being evicted and rebuilt (a slot's
        problem, plans and workspace take milliseconds to build, and their frees synchronise
        the device)."""
        import torch
        from . import _lib, api
        self.torch, self.api, self.lib = torch, api, _lib
        self.dtype = dtype or torch.float64
        self.max_slots = max_slots
        self.newton_opts = dict(newton_opts or {})
        self.restart = restart
        free, total = torch.cuda.mem_get_info()
        self.budget = int(budget_bytes if budget_bytes is not None else 0.5 * free)
        self._tau = {}
        self._bytes = {}
        self._lock = threading.Lock()
        self.cache_slots = int(cache_slots if cache_slots is not None else 4 * max_slots)
        self.pool = SlotPool(self.budget, max(self.cache_slots, max_slots), self._make_slot, self._free_slot,
                             self._slot_bytes)

    def _nodes(self, N):
        if N not in self._tau:
            t, _ = self.api.Plan(N, t0=-1.0, tf=1.0).grid()
            self._tau[N] = t.numpy()
        return self._tau[N]

    def _slot_bytes(self, N):
        # measured on the first slot of this size; before that a generous estimate
        return self._bytes.get(N, 600 * (N + 1) * (8 if self.dtype == self.torch.float64 else 6) + (64 << 20))

    def _make_slot(self, N):
        torch, api = self.torch, self.api

        class Slot:
            pass
        s = Slot()
        s.N = N
        s.stream = torch.cuda.Stream()
        with torch.cuda.stream(s.stream):
            s.prob = api.Problem(self.lib.BK_ORBIT, N, self.dtype, 0.0, 1.0, (A_NOMINAL, 1.5),
                                 stream=s.stream)
            s.ws = api.newton_workspace(s.prob, self.restart)
            s.z = torch.zeros(s.prob.kkt_len, dtype=torch.float64, device="cuda")
        s.h_in = torch.zeros(s.prob.kkt_len, dtype=torch.float64).pin_memory()
        s.h_out = torch.zeros(s.prob.kkt_len, dtype=torch.float64).pin_memory()
        s.tau = self._nodes(N)
        s.nbytes = s.prob.device_bytes() + s.ws.numel() * 8 + s.z.numel() * 8
        self._bytes[N] = s.nbytes
        s.stream.synchronize()   # this slot only: other slots keep running
        return s

    def _free_slot(self, s):
        s.stream.synchronize()
        s.prob.close()
        del s.ws, s.z

    def guess(self, slot, rf, tf):
        from .synth import orbit_guess
        t = tf * 0.5 * (slot.tau + 1.0)
        X, U = orbit_guess(t, rf, tf)
        prob = slot.prob
        P = prob.pitch
        h = slot.h_in.numpy()
        h[:] = 0.0
        for m in range(4):
            h[m * P:m * P + prob.L] = X[m]
        for q in range(2):
            h[(4 + q) * P:(4 + q) * P + prob.L] = U[q]

    def solve(self, slot, req):
        torch, api = self.torch, self.api
        rf, tf = req["rf"], req["tf"]
        slot.prob.set_params(0.0, tf, (A_NOMINAL, rf))
        self.guess(slot, rf, tf)
        with torch.cuda.stream(slot.stream):
            slot.z.copy_(slot.h_in, non_blocking=True)
            info = api.newton_solve(slot.prob, slot.z, workspace=slot.ws, restart=self.restart,
                                    stream=slot.stream, raise_on_fail=False, **self.newton_opts)
            slot.h_out.copy_(slot.z, non_blocking=True)
        slot.stream.synchronize()
        st = "ok" if info["status"] == 0 else self.lib.STATUS.get(info["status"], "error")
        return {"status": st, "newton_iterations": info["iterations"],
                "krylov_iterations": info["krylov_iterations"], "residual": info["residual"],
                "solution": slot.h_out.numpy().copy() if req.get("keep") else None,
                "theta_f": float(slot.h_out[1 * slot.prob.pitch + slot.prob.L - 1])}

    def run(self, requests, realtime=True):
        t0 = time.perf_counter()
        res = run_schedule(requests, self.pool, self.solve, self.max_slots, realtime=realtime)
        wall = time.perf_counter() - t0
        return res, summarize(res, wall)

    def close(self):
        self.pool.close()


def shard_requests(requests, rank, world):
    """Requests of one rank when `world` GPUs serve one stream: request i goes to rank
    i mod world (independent solves need no exchange between ranks)."""
    return [r for i, r in enumerate(sorted(requests, key=lambda r: r["arrival"])) if i % world == rank]


def combine_stats(local_results, wall, dist=None):
    """Whole-job statistics over ranks: total solved / max wall time, latency percentiles over
    every rank's requests (all-gathered). Without a process group it is summarize()."""
    if dist is None:
        return summarize(local_results, wall)
    import torch
    world = dist.get_world_size()
    lat = torch.tensor([r["latency"] for r in local_results if r.get("status") == "ok"], dtype=torch.float64)
    n = torch.tensor([lat.numel(), len(local_results)], dtype=torch.int64)
    counts = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, n)
    maxn = int(max(c[0] for c in counts))
    padded = torch.full((max(maxn, 1),), float("nan"), dtype=torch.float64)
    padded[:lat.numel()] = lat
    gathered = [torch.zeros_like(padded) for _ in range(world)]
    dist.all_gather(gathered, padded)
    allv = torch.cat(gathered)
    allv = allv[~torch.isnan(allv)].numpy()
    w = torch.tensor([wall], dtype=torch.float64)
    dist.all_reduce(w, op=dist.ReduceOp.MAX)
    solved = int(sum(c[0] for c in counts))
    total = int(sum(c[1] for c in counts))
    return {"requests": total, "solved": solved, "failed": total - solved,
            "solves_per_s": solved / float(w.item()),
            "p50_ms": float(np.percentile(allv, 50) * 1e3) if allv.size else float("nan"),
            "p99_ms": float(np.percentile(allv, 99) * 1e3) if allv.size else float("nan"),
            "mean_ms": float(np.mean(allv) * 1e3) if allv.size else float("nan"),
            "wall_s": float(w.item()), "ranks": world}
