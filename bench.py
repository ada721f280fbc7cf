"""Benchmark of the Birkhoff hot path on GB300.

Default workload: one Newton-Krylov solve of the planar orbit-raising problem on the CGL grid
with N = 2^20 (L = 1,048,577 nodes), FP64, from the tangential-thrust spiral initial guess.
A step is the whole path: residual (Birkhoff products of f), linearisation (B^T lambda,
per-node preconditioner factors, terminal Schur data), preconditioned GMRES on the KKT system
(KKT products = B and B^T on every state component, preconditioner sweeps), line search.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload newton_f64|newton_f32ir|newton_bounded|apply_f64|apply_f32] [--N 20]

--workload newton_bounded solves the same transfer with its thrust components bounded (FP64,
barrier stages; see bounded_table).

With the default --sweep 1 the line also carries the product sweep (N = 2^10..2^24), the FFT vs
dense tensor-core crossover, the minimum-time orbit table (Eq. ot, free final time,
N = 2^10..2^20: Newton and KKT-solve counts per N, the measure of Table tab:m), and the bounded
orbit table (the same transfer with its thrust components bounded, barrier stages, N = 2^10..2^20).

Prints one JSON line on rank 0. With N > 1 (torchrun) every rank solves its own instance
(replicas; the path has no data-path collective) and the time is the max over ranks.
--impl reference times the matrix-free FP64 CPU oracle (test infrastructure) on a bounded sample:
one solve of the same problem at N = 2^12 per step, labelled with the N it ran.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

RF, TF, A_NOM = 1.5, 20.0, 0.01
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 FMA rate of GB300: 152 SMs x 2 FP64 FMA / clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s
# (nominal 1.25 TFLOP/s); the transforms of the FP64 path are bound by it, not by HBM.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5 TFLOP/s nominal FFMA


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="newton_f64",
                    choices=["newton_f64", "newton_f32ir", "newton_bounded", "apply_f64", "apply_f32", "serve",
                             "peaks"])
    ap.add_argument("--serve-requests", type=int, default=0,
                    help="serving requests (default 4096, offered at 0.8 of the closed-loop rate, plus "
                         "1024 each at 0.5 and 0.95; -1 skips serving in the default line)")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--N", type=int, default=20, help="log2 of the grid size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", type=int, default=1, help="1 (default): add the apply sweep N=2^10..2^24")
    ap.add_argument("--profile", action="store_true",
                    help="apply and newton workloads: after timing, run one more product or solve (L2 "
                         "flushed first) between cudaProfilerStart and cudaProfilerStop, for ncu "
                         "--profile-from-start off")
    return ap.parse_args()


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        return rank, world, dist
    if torch.cuda.is_available():
        torch.cuda.set_device(0)
    return 0, 1, None


def barrier(dist):
    import torch
    if dist is not None:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(x, dist):
    import torch
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def read_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smmax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        load = [r for r in rows if r["power"] > 200.0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["smmax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "samples_under_load": len(load)}


def l2_flush_buffer():
    import torch
    return torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > 2 x L2


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def make_orbit(N, dtype):
    import torch
    from paper_2509_01855_gb300 import _lib, api, synth
    prob = api.Problem(_lib.BK_ORBIT, N, dtype, 0.0, TF, (A_NOM, RF))
    t, _ = api.Plan(N, t0=0.0, tf=TF).grid()
    X, U = synth.orbit_guess(t.numpy(), RF, TF)
    z0 = prob.pack(X, U)
    return prob, z0


def run_newton(args, rank, world, dist):
    import torch
    from paper_2509_01855_gb300 import _lib, api
    N = 1 << args.N
    dtype = torch.float32 if args.workload == "newton_f32ir" else torch.float64
    prob, z0 = make_orbit(N, dtype)
    if args.workload == "newton_bounded":
        lo, hi = orbit_bounds()
        prob.set_control_bounds(lo, hi)
        prob.set_barrier(BOUNDED_MU[0], BOUNDED_MU[1])
    ws = api.newton_workspace(prob)
    z = torch.empty_like(z0)
    flush = l2_flush_buffer()
    infos = []

    def step():
        z.copy_(z0)
        return api.newton_solve(prob, z, workspace=ws)

    for _ in range(args.warmup):
        infos.append(step())
    lib = _lib.lib()
    barrier(dist)
    launches0 = lib.bk_launch_count()
    times = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            infos.append(step())
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier(dist)
    launches = lib.bk_launch_count() - launches0
    ms = sum(times) / len(times)
    ms_max = max_over_ranks(ms, dist)
    if args.profile:
        # one more solve (L2 flushed first) between cudaProfilerStart and cudaProfilerStop
        flush.zero_()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()

    # end to end through the public API: pinned host initial guess in, solution out
    zh = z0.cpu().pin_memory()
    outh = torch.empty_like(zh).pin_memory()
    zd = torch.empty_like(z0)
    e2e_times = []
    for i in range(max(2, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        zd.copy_(zh, non_blocking=True)
        api.newton_solve(prob, zd, workspace=ws)
        outh.copy_(zd, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(sum(e2e_times) / len(e2e_times), dist)
    nbytes = z0.numel() * z0.element_size()
    last = infos[-1]
    err = None
    if dtype == torch.float32:
        # trajectory difference between the FP32-inner solve and an FP64 solve of the same problem
        # (untimed; tests/test_gpu_fullsize.py compares both with the oracle at this N)
        p64, _ = make_orbit(N, torch.float64)
        z64 = z0.clone()
        api.newton_solve(p64, z64, workspace=api.newton_workspace(p64))
        X32, U32, _, _ = prob.split(z)
        X64, U64, _, _ = p64.split(z64)
        err = {"state_max_abs": float((X32 - X64).abs().max()), "control_max_abs": float((U32 - U64).abs().max()),
               "state_scale": float(X64.abs().max())}
        p64.close()
    res = dict(ms=ms_max, launches=launches, clocks=clk.summary(),
               e2e={"value": world * 1000.0 / e2e_ms, "unit": "solves/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
               solve=dict(newton_iterations=last["iterations"], krylov_iterations=last["krylov_iterations"],
                          kkt_solves=last["kkt_solves"], backtracks=last["backtracks"], residual=last["residual"],
                          error_vs_f64_gpu_solve=err))
    return res


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
TRANSFORM_SOURCES = ("bk_birkhoff.cu", "bk_fft.cuh", "bk_plan.cuh", "bk_common.cuh")


def transform_source_hash():
    """First 16 hex digits of the SHA-256 of the transform sources (in TRANSFORM_SOURCES order)."""
    csrc = os.path.join(ROOT, "paper_2509_01855_gb300", "csrc")
    sha = hashlib.sha256()
    for f in TRANSFORM_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            sha.update(fh.read())
    return sha.hexdigest()[:16]


def recorded_traffic(dtype_name, N):
    """DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one 4-component product
    at N from profiles/traffic.json, or None when no capture exists for (dtype, N) or the
    transform sources changed since it was taken (source hash check)."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    e = rec.get("%s_2p%d" % (dtype_name, int(math.log2(N))))
    if not e or e.get("source_sha256_16") != transform_source_hash():
        return None
    return int(e["traffic_bytes_per_product"])


def measure_apply(N, dtype, reps=20, trans=False, dense=None, profile=False):
    """Birkhoff apply B v (or B^T v) on 4 components, cold L2 between repetitions (CUDA events).
    dense: None keeps the plan's default path; True / False force the tensor-core dense product
    or the FFT chain (FP32, N <= 1024)."""
    import torch
    from paper_2509_01855_gb300 import api
    plan = api.Plan(N, n_comp=4, max_batch=1, dtype=dtype, t0=0.0, tf=TF)
    if dense is not None:
        plan.set_dense(dense)
    g = torch.Generator(device="cuda")
    g.manual_seed(2509_01855)
    v = plan.empty(1)
    v[:, :, :N + 1] = torch.randn(1, 4, N + 1, dtype=dtype, device="cuda", generator=g)
    out = plan.empty(1)
    flush = l2_flush_buffer()
    fn = api.birkhoff_apply_T if trans else api.birkhoff_apply
    for _ in range(3):
        fn(plan, v, out)
    times = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(plan, v, out)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    if profile:
        flush.zero_()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        fn(plan, v, out)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    es = v.element_size()
    nbytes = 2 * 4 * (N + 1) * es                     # read v, write B v
    flops = 4 * 2 * 2.5 * N * math.log2(N)             # two DCT-I per component
    plan.close()
    return ms, nbytes, flops


def apply_sweep(lgs=range(10, 25), reps=5):
    """B and B^T on 4 components for N = 2^10..2^24 in FP64 and FP32, cold L2: median ms and
    algorithmic GB/s (read v + write the product)."""
    import torch
    out = {}
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        rows = {}
        for lg in lgs:
            fwd, nbytes, flops = measure_apply(1 << lg, dt, reps=reps)
            trn, _, _ = measure_apply(1 << lg, dt, reps=reps, trans=True)
            rows[str(lg)] = {"B_ms": round(fwd, 5), "BT_ms": round(trn, 5), "B_gbs": round(nbytes / fwd / 1e6, 2),
                             "BT_gbs": round(nbytes / trn / 1e6, 2), "B_tflops": round(flops / fwd / 1e9, 4)}
        out[name] = rows
    return out


def cufft_product(v, s):
    """Comparison only (never the product path): B v for v of shape (n_c, N + 1) with cuFFT through
    torch.fft -- the library's formulation (DCT-I = real FFT of the even extension of length 2N,
    the integration stencil with the aliasing fold, DCT-I back, minus the node-0 value) written
    with torch ops."""
    import torch
    N = v.shape[-1] - 1

    def dct1(x):
        ext = torch.cat([x, x[..., 1:N].flip(-1)], dim=-1)
        return torch.fft.rfft(ext, dim=-1).real[..., :N + 1]

    Y = dct1(v)
    g = torch.zeros_like(Y)
    k = torch.arange(2, N - 1, dtype=v.dtype, device=v.device)
    g[..., 1] = (Y[..., 2] - Y[..., 0]) / (4.0 * N)
    g[..., 2:N - 1] = (Y[..., 3:N] - Y[..., 1:N - 2]) / (4.0 * k * N)
    g[..., N - 1] = ((0.5 * Y[..., N] - Y[..., N - 2]) / (2.0 * (N - 1) * N) - 0.5 * Y[..., N] / (2.0 * (N + 1) * N)) / 2.0
    g[..., N] = -Y[..., N - 1] / (2.0 * N * N)
    y = dct1(g)
    return s * (y - y[..., :1])


def cufft_comparison(lgs=(16, 20, 22), reps=9):
    """cuFFT-based product (torch.fft) against the library's product on 4 components, cold L2:
    median ms of each and their relative difference (a comparison; the product path uses only
    the library's own kernels)."""
    import torch
    from paper_2509_01855_gb300 import api
    rows = {}
    for lg in lgs:
        N = 1 << lg
        for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
            g = torch.Generator(device="cuda")
            g.manual_seed(2509_01855)
            v = torch.randn(4, N + 1, dtype=dt, device="cuda", generator=g)
            plan = api.Plan(N, n_comp=4, max_batch=1, dtype=dt, t0=0.0, tf=TF)
            vp = plan.empty(1)
            vp[0, :, :N + 1] = v
            op = plan.empty(1)
            flush = l2_flush_buffer()
            res = {}
            for label, fn in (("library", lambda: api.birkhoff_apply(plan, vp, op)),
                              ("cufft", lambda: cufft_product(v, 0.5 * TF))):
                for _ in range(3):
                    fn()
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    fn()
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                res[label] = statistics.median(ts)
            ref = cufft_product(v, 0.5 * TF)
            lib_out = api.birkhoff_apply(plan, vp, op)[0, :, :N + 1]
            diff = float((lib_out - ref).norm() / ref.norm())
            rows["%s_2p%d" % (name, lg)] = {"library_ms": round(res["library"], 5), "cufft_ms": round(res["cufft"], 5),
                                            "rel_diff": diff}
            plan.close()
    return rows


def batched_apply(reps=15):
    """Uneven-N batch of products (the serving mix's sizes: one plan of each N = 2^8..2^16 in each
    precision, 4 components, one vector each): birkhoff_apply_batch against one birkhoff_apply per
    plan, back to back (warm L2: the batch is ~20 MB), median ms, and the library launches each
    takes."""
    import torch
    from paper_2509_01855_gb300 import _lib, api
    rows = {}
    lib = _lib.lib()
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        plans = [api.Plan(1 << k, n_comp=4, max_batch=1, dtype=dt, t0=0.0, tf=TF) for k in range(8, 17)]
        vs, outs = [], []
        for i, p in enumerate(plans):
            v = p.empty(1)
            g = torch.Generator(device="cuda")
            g.manual_seed(100 + i)
            v[0, :, :p.L] = torch.randn(4, p.L, dtype=dt, device="cuda", generator=g)
            vs.append(v)
            outs.append(p.empty(1))

        def seq():
            for p, v, o in zip(plans, vs, outs):
                api.birkhoff_apply(p, v, o)

        def bat():
            api.birkhoff_apply_batch(plans, vs, outs)
        res = {}
        for label, fn in (("sequential", seq), ("batched", bat)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            c0 = lib.bk_launch_count()
            fn()
            torch.cuda.synchronize()
            launches = lib.bk_launch_count() - c0
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            res[label] = {"ms": round(statistics.median(ts), 5), "launches": int(launches)}
        rows[name] = dict(res, plans=len(plans), N="2^8..2^16", paths=sorted({p.shape()["path"] for p in plans}))
        for p in plans:
            p.close()
    return rows


def dense_crossover(lgs=range(4, 11), reps=9):
    """FP32 products on 4 components, FFT chain vs the dense tensor-core product (the GPU
    analogue of the paper's Fig. BVisNlogN), cold L2: median ms of B v."""
    import torch
    rows = {}
    for lg in lgs:
        fft, _, _ = measure_apply(1 << lg, torch.float32, reps=reps, dense=False)
        dense, _, _ = measure_apply(1 << lg, torch.float32, reps=reps, dense=True)
        rows[str(lg)] = {"fft_ms": round(fft, 5), "dense_ms": round(dense, 5)}
    return rows


def min_time_table(lgs=range(10, 21), a=0.05, rf=6.0, t_seed=24.0):
    """The minimum-time orbit transfer of Eq. ot (free final time, thrust a = 0.05, r 1 -> 6) for
    N = 2^10..2^20: a minimum-energy solve at t_f = 24 seeds it (bk_min_time_seed), then the
    Newton-Krylov solve of the free-time KKT system. Per N: Newton iterations, KKT solves and
    Krylov iterations (Table tab:m's columns, with this library's outer loop), the final time T and
    the solve's device time (CUDA events, FP64; the 2^20 row also with FP32 inner solves)."""
    import torch
    from paper_2509_01855_gb300 import _lib, api, synth
    rows = {}
    cases = [(lg, torch.float64) for lg in lgs] + [(max(lgs), torch.float32)]
    for lg, dt in cases:
        N = 1 << lg
        me = api.Problem(_lib.BK_ORBIT, N, torch.float64, 0.0, t_seed, (a, rf))
        t, _ = api.Plan(N, t0=0.0, tf=t_seed).grid()
        X, U = synth.orbit_guess(t.numpy(), rf, t_seed)
        zme = me.pack(X, U)
        ime = api.newton_solve(me, zme, tol=1e-11, krylov_rtol=1e-12, max_iter=60)
        mt = api.Problem(_lib.BK_ORBIT_MT, N, dt, 0.0, t_seed, (a, rf))
        z = mt.zeros(dtype=torch.float64)
        api.min_time_seed(mt, me, zme, z)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        info = api.newton_solve(mt, z, tol=1e-10, max_iter=60, raise_on_fail=False)
        e1.record()
        torch.cuda.synchronize()
        key = str(lg) + ("" if dt == torch.float64 else "_f32inner")
        rows[key] = {"seed_newton_its": ime["iterations"], "newton_its": info["iterations"],
                     "kkt_solves": info["kkt_solves"], "krylov_its": info["krylov_iterations"],
                     "converged": bool(info["converged"]), "residual": info["residual"],
                     "T": 2.0 * z[mt.s_index].item(), "ms": round(e0.elapsed_time(e1), 3)}
        me.close()
        mt.close()
    return rows


BOUNDED_MU = (1e-4, 1e-9)   # barrier schedule of the bounded orbit transfer (scaled to its cost)


def orbit_bounds(fr=0.9, ft=0.95):
    """Thrust bounds of the bounded orbit transfer, below the unbounded optimum's peaks:
    |u_r| <= 0.9 max|u_r| and u_theta <= 0.95 max u_theta (peaks of the unbounded solve at N = 64)."""
    import torch
    from paper_2509_01855_gb300 import api
    p64, z64 = make_orbit(64, torch.float64)
    api.newton_solve(p64, z64)
    U = p64.split(z64)[1]
    a = fr * U[0].abs().max().item()
    lo, hi = [-a, -float("inf")], [a, ft * U[1].max().item()]
    p64.close()
    return lo, hi


def bounded_table(lgs=(10, 14, 17, 20)):
    """The orbit transfer of the headline solve with its thrust bounded (orbit_bounds), solved by
    newton_solve's barrier stages mu = 1e-4 .. 1e-9 in the primal and in the primal-dual form.
    Per N and form: Newton iterations over all stages, Krylov iterations, the solve's device time
    (CUDA events, FP64) and how close the solution comes to the bounds. Then the same transfer
    with the endpoint bound r(t_f) >= 1.55 in place of r(t_f) = 1.5 (no thrust bounds)."""
    import torch
    from paper_2509_01855_gb300 import api
    lo, hi = orbit_bounds()
    mu0, mu_final = BOUNDED_MU
    rows = {"bounds": {"lo": lo, "hi": hi}, "mu0": mu0, "mu_final": mu_final}
    for lg, form in [(lg, f) for lg in lgs for f in ("primal", "primal_dual")]:
        N = 1 << lg
        prob, z = make_orbit(N, torch.float64)
        prob.set_control_bounds(lo, hi)
        prob.set_barrier(mu0, mu_final, form)
        ws = api.newton_workspace(prob)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        info = api.newton_solve(prob, z, workspace=ws, raise_on_fail=False)
        e1.record()
        torch.cuda.synchronize()
        Ub = prob.split(z)[1]
        rows["%d_%s" % (lg, form)] = {"newton_its": info["iterations"], "krylov_its": info["krylov_iterations"],
                         "backtracks": info["backtracks"], "converged": bool(info["converged"]),
                         "residual": info["residual"], "ms": round(e0.elapsed_time(e1), 3),
                         "gap_ur": hi[0] - Ub[0].abs().max().item(), "gap_ut": hi[1] - Ub[1].max().item()}
        prob.close()
    # FP32 Krylov inner solves with the FP64 Newton residual (primal form), to 1e-9
    prob, z = make_orbit(1 << max(lgs), torch.float32)
    prob.set_control_bounds(lo, hi)
    prob.set_barrier(mu0, mu_final)
    ws = api.newton_workspace(prob)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    info = api.newton_solve(prob, z, tol=1e-9, workspace=ws, raise_on_fail=False)
    e1.record()
    torch.cuda.synchronize()
    rows["%d_primal_f32inner_tol1e-9" % max(lgs)] = {
        "newton_its": info["iterations"], "krylov_its": info["krylov_iterations"],
        "converged": bool(info["converged"]), "residual": info["residual"], "ms": round(e0.elapsed_time(e1), 3)}
    prob.close()
    # endpoint bound instead of the thrust bounds: r(t_f) >= 1.55 in place of r(t_f) = 1.5
    for lg in lgs:
        N = 1 << lg
        prob, z = make_orbit(N, torch.float64)
        prob.set_terminal_bounds([1.55, -float("inf"), -float("inf")], [float("inf")] * 3)
        prob.set_barrier(mu0, mu_final)
        ws = api.newton_workspace(prob)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        info = api.newton_solve(prob, z, workspace=ws, raise_on_fail=False)
        e1.record()
        torch.cuda.synchronize()
        rows["%d_endpoint_r_ge_1.55" % lg] = {
            "newton_its": info["iterations"], "krylov_its": info["krylov_iterations"],
            "converged": bool(info["converged"]), "ms": round(e0.elapsed_time(e1), 3),
            "r_tf": prob.split(z)[0][0, -1].item()}
        prob.close()
    return rows


def cpu_apply_baseline(N):
    """The oracle's FastBV chain (SciPy DCT-I, as it stands) on 4 FP64 components at N, on the
    host cores with SciPy's FFT on every core and on one; one product each, so the default run
    stays short."""
    import scipy.fft
    from oracle import birkhoff as ob
    v = np.random.default_rng(2509_01855).standard_normal((4, N + 1))
    nbytes = 2 * 4 * (N + 1) * 8
    out = {}
    for workers in (os.cpu_count() or 1, 1):
        with scipy.fft.set_workers(workers):
            ob.fastbv(v[:, :1025], 0.0, TF)        # warm-up at N = 1024 (imports, FFT set-up)
            t0 = time.perf_counter()
            ob.fastbv(v, 0.0, TF)
            sec = time.perf_counter() - t0
        out["cores_%d" % workers] = {"value": nbytes / sec / 1e9, "ms": 1e3 * sec, "cores": workers}
    best = out["cores_%d" % (os.cpu_count() or 1)]
    return {"value": best["value"], "unit": "GB/s", "ms": best["ms"], "cores": best["cores"], "kind": "oracle",
            "single_core": out.get("cores_1"),
            "sample": "oracle FastBV (SciPy DCT-I) on 4 FP64 components at N=2^%d, one product" % int(math.log2(N))}


def run_serve(n_requests, slots, rank=0, world=1, dist=None, loads=(0.8,), extra_requests=1024):
    """Serving: Poisson stream, N = 2^k with k ~ U{8..16}, r_f ~ U[1.2, 2.0], t_f ~ U[10, 30],
    FP32 Krylov with the FP64 Newton residual. The closed-loop maximum rate of this GPU is
    measured first; the stream is then offered at `loads` x that rate (the first load with
    n_requests, the others with extra_requests). Returns the first load's statistics, with the
    others under "load_sweep"."""
    import torch
    from paper_2509_01855_gb300 import synth
    from paper_2509_01855_gb300.serve import Server, combine_stats, run_schedule, shard_requests
    srv = Server(dtype=torch.float32, max_slots=slots)   # FP32 Krylov + FP64 Newton residual
    warm = [dict(id=i, arrival=0.0, N=1 << k, rf=1.5, tf=20.0) for i, k in enumerate(range(8, 17))]
    srv.run(warm, realtime=False)
    probe = shard_requests(synth.serving_requests(256, 1.0, "probe"), rank, world)
    for r in probe:
        r["arrival"] = 0.0
    _, st_closed = srv.run(probe, realtime=False)
    max_rate = max_over_ranks(-st_closed["solves_per_s"], dist)   # slowest rank sets the rate
    max_rate = -max_rate * world
    results = []
    for i, load in enumerate(loads):
        rate = load * max_rate
        n = n_requests if i == 0 else extra_requests
        reqs = shard_requests(synth.serving_requests(n, rate, "stream-%d" % i), rank, world)
        t0 = time.perf_counter()
        res = run_schedule(reqs, srv.pool, srv.solve, srv.max_slots, realtime=True)
        st = combine_stats(res, time.perf_counter() - t0, dist)
        iters = [r["newton_iterations"] for r in res if r.get("status") == "ok"]
        st.update(load=load, offered_rate=rate, newton_iterations_max=int(max(iters)) if iters else None)
        results.append(st)
    srv.close()
    st = dict(results[0])
    st.update(closed_loop_max_rate=max_rate, slots=slots, cached_slots=srv.cache_slots, slots_created=srv.pool.created,
              slots_evicted=srv.pool.evicted, dtype="f32ir",
              workload="orbit raising, N=2^k k~U{8..16}, r_f~U[1.2,2], t_f~U[10,30], Poisson arrivals")
    if len(results) > 1:
        st["load_sweep"] = [{k: r[k] for k in ("load", "offered_rate", "solves_per_s", "p50_ms", "p99_ms", "solved",
                                               "requests")} for r in results]
    return st


# ------------------------------------------------------------------------------------------
# Oracle legs (CPU)
# ------------------------------------------------------------------------------------------
def oracle_matfree_solve(N_sample, workers=1):
    """One Newton-Krylov solve of the same orbit problem by the matrix-free FP64 oracle (FastBV
    chain with SciPy's DCT-I, sequential preconditioner sweeps, plain right-preconditioned
    GMRES) at N_sample, from the same spiral guess. `workers` sets SciPy's FFT threads; the sweeps
    and the Krylov loop run on one core. Returns (seconds, info)."""
    import scipy.fft
    from oracle import problems as op
    from oracle.matfree import MatFreeKKT
    from paper_2509_01855_gb300 import synth
    M = MatFreeKKT(op.Problem(op.ORBIT, 0.0, TF, (A_NOM, RF)), N_sample)
    X, U = synth.orbit_guess(M.t, RF, TF)
    vec0 = M.pack(X, U, np.zeros((4, M.L)), np.zeros(3))
    with scipy.fft.set_workers(workers):
        t0 = time.perf_counter()
        _, info = M.newton(vec0)
        sec = time.perf_counter() - t0
    return sec, info


def cpu_baseline(N_sample=1 << 14):
    """The matrix-free oracle's solve of the orbit problem at N_sample on the host cores, with
    SciPy's FFT on every core (cpu_baseline) and on one (cpu_baseline_single_core)."""
    out = {}
    ncores = os.cpu_count() or 1
    for key, workers in (("cpu_baseline", ncores), ("cpu_baseline_single_core", 1)):
        sec, info = oracle_matfree_solve(N_sample, workers)
        out[key] = {"value": 1.0 / sec, "unit": "solves/s", "cores": workers, "kind": "oracle",
                    "N": N_sample, "seconds": sec, "newton_iterations": info["iters"],
                    "krylov_iterations": int(sum(info["krylov"])),
                    "sample": "one matrix-free FP64 oracle Newton-Krylov solve (FastBV with SciPy DCT-I on %d "
                              "FFT worker(s), sequential sweeps, GMRES) of the same orbit problem at N=2^%d; "
                              "the GPU line's value is for N=2^20" % (workers, int(math.log2(N_sample)))}
    return out


REF_N = 1 << 12


def run_reference(args):
    """Reference arm: the matrix-free FP64 oracle (test infrastructure, as it stands) on the host
    cores, one Newton-Krylov solve of the orbit problem per step at N = REF_N. The line states
    the N it ran (not the GPU arm's 2^20)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ncores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_matfree_solve(REF_N, ncores)
    times = []
    info = None
    for _ in range(args.steps):
        sec, info = oracle_matfree_solve(REF_N, ncores)
        times.append(sec)
    ms = 1000.0 * sum(times) / len(times)
    value = 1000.0 / ms
    lg = int(math.log2(REF_N))
    sample = ("one matrix-free FP64 oracle Newton-Krylov solve of the orbit problem at N=2^%d per step "
              "(%d Newton, %d Krylov iterations; FastBV with SciPy DCT-I on %d FFT workers, sequential "
              "sweeps); the GPU arm solves N=2^%d" % (lg, info["iters"], int(sum(info["krylov"])), ncores, args.N))
    cfg = config(args)
    cfg.update(N=REF_N, nodes=REF_N + 1, parallelism="host cores x%d" % ncores, l2="n/a (CPU)")
    line = {"impl": "reference", "metric": "Newton-Krylov solve rate at N=2^%d (orbit raising)" % lg,
            "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": ncores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def metric_name(args):
    if args.workload.startswith("apply"):
        return "Birkhoff apply GB/s at N=2^%d (B v on 4 components)" % args.N
    if args.workload == "newton_bounded":
        return "Newton-Krylov solve rate at N=2^%d (orbit raising, bounded thrust)" % args.N
    return "Newton-Krylov solve rate at N=2^%d (orbit raising)" % args.N


def config(args):
    prec = {"newton_f64": "f64 (double-float arithmetic in the FP64 Birkhoff transforms from N = 2^18)",
            "newton_f32ir": "f32 Krylov + f64 refinement",
            "newton_bounded": "f64 (double-float FP64 transforms from N = 2^18), control bounds by barrier",
            "apply_f64": "f64", "apply_f32": "f32", "serve": "f32ir"}[args.workload]
    c = {"workload": "orbit_raising_newton_krylov" if args.workload.startswith("newton") else "birkhoff_apply",
         "N": 1 << args.N, "nodes": (1 << args.N) + 1, "precision": prec,
         "problem": "polar orbit raising r 1->%.1f, t_f=%g, thrust-vector min-energy, x0=(1,0,0,1)" % (RF, TF),
         "initial_guess": "tangential-thrust spiral", "l2": "flushed between steps (256 MB write)",
         "parallelism": "replicas x%d" % args.gpus}
    if args.workload == "newton_bounded":
        c["workload"] = "orbit_raising_newton_krylov_bounded_thrust"
        c["bounds"] = "|u_r| <= 0.9 max|u_r|, u_theta <= 0.95 max u_theta of the unbounded optimum"
        c["barrier"] = {"mu0": BOUNDED_MU[0], "mu_final": BOUNDED_MU[1], "form": "primal"}
    return c


def tensor_rates(n=8192, reps=10):
    """Diagnostic (--workload peaks): library GEMM rates on this GPU through torch -- FP64
    (torch.matmul), INT8 with INT32 accumulation (torch._int_mm), TF32 and BF16 -- best of `reps`
    CUDA-event timings of an n x n x n product. They decide whether an FP64 dense product split
    into INT8 slices (Ozaki scheme) could beat FP64 on the CUDA cores."""
    import torch
    out = {}
    cases = [("f64", torch.float64), ("tf32", torch.float32), ("bf16", torch.bfloat16), ("int8", torch.int8)]
    for name, dt in cases:
        if dt == torch.int8:
            a = torch.randint(-100, 100, (n, n), dtype=dt, device="cuda")
            b = torch.randint(-100, 100, (n, n), dtype=dt, device="cuda")
            fn = lambda: torch._int_mm(a, b)
        else:
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            fn = lambda: a @ b
        torch.backends.cuda.matmul.allow_tf32 = name == "tf32"
        try:
            for _ in range(2):
                fn()
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            out[name] = {"ms": best, "tflops": 2.0 * n ** 3 / best / 1e9}
        except Exception as e:  # an unsupported kind on this build of torch
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
    torch.backends.cuda.matmul.allow_tf32 = False
    return {"n": n, "rates": out}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "peaks":
        print(json.dumps({"workload": "peaks", "gemm": tensor_rates()}), flush=True)
        return
    import torch
    rank, world, dist = dist_setup(args)
    hbm_peak, peak_kind = read_peaks()
    N = 1 << args.N
    dtype_name = "f64" if args.workload in ("newton_f64", "newton_bounded", "apply_f64") else "f32"
    line = {"metric": metric_name(args), "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_name, "data": "synthetic", "config": config(args)}
    if args.workload == "serve":
        from paper_2509_01855_gb300 import _lib
        lib = _lib.lib()
        c0 = lib.bk_launch_count()
        with ClockSampler(torch.cuda.current_device()) as clk:
            st = run_serve(args.serve_requests or 4096, args.serve_slots, rank, world, dist, loads=(0.8, 0.5, 0.95))
        line.update(metric="served Newton-Krylov solves/s (orbit raising, mixed N)", value=st["solves_per_s"],
                    unit="solves/s", ms_per_step=1000.0 / st["solves_per_s"] if st["solves_per_s"] else None,
                    gpu_launches=lib.bk_launch_count() - c0, clocks=clk.summary(), serve=st,
                    e2e={"value": st["solves_per_s"], "unit": "solves/s", "h2d_bytes_per_step": None,
                         "d2h_bytes_per_step": None, "note": "latency = solution on host - arrival"})
        line["config"]["workload"] = "serving"
        dt = torch.float32
    elif args.workload.startswith("newton"):
        r = run_newton(args, rank, world, dist)
        line.update(value=world * 1000.0 / r["ms"], unit="solves/s", ms_per_step=r["ms"], e2e=r["e2e"],
                    gpu_launches=r["launches"], clocks=r["clocks"], solve=r["solve"])
        dt = torch.float32 if args.workload == "newton_f32ir" else torch.float64
    else:
        dt = torch.float64 if args.workload == "apply_f64" else torch.float32
        from paper_2509_01855_gb300 import _lib
        lib = _lib.lib()
        c0 = lib.bk_launch_count()
        with ClockSampler(torch.cuda.current_device()) as clk:
            ms, nbytes, flops = measure_apply(N, dt, reps=max(args.steps, 5), profile=args.profile)
        line.update(value=world * nbytes / ms / 1e6, unit="GB/s", ms_per_step=ms,
                    gpu_launches=lib.bk_launch_count() - c0, clocks=clk.summary())
    # roofline of the dominant unit: the 4-component Birkhoff apply (four transform passes)
    ams, abytes, aflops = measure_apply(N, dt)
    if dt == torch.float64:
        peak, unit, achieved = FP64_PEAK_TFLOPS, "TFLOP/s", aflops / ams / 1e9
        bound = "alu"
    else:
        peak, unit, achieved = hbm_peak, "GB/s", abytes / ams / 1e6
        bound = "hbm"
    line["roofline"] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                        "frac": achieved / peak, "traffic": recorded_traffic(dtype_name, N),
                        "traffic_source": "profiles/traffic.json",
                        "kernel": "birkhoff_apply N=2^%d x4 components (%s)" % (args.N, dtype_name),
                        "algorithmic": {"bytes": abytes, "flops": aflops},
                        "peak_source": ("FP64 FMA nominal 1.25 TFLOP/s (2 FP64 FMA/clk/SM)" if bound == "alu"
                                        else "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind)}
    line["apply"] = {"ms": ams, "gbs": abytes / ams / 1e6, "tflops": aflops / ams / 1e9, "N": N,
                     "n_comp": 4, "dtype": dtype_name}
    if args.sweep:
        line["apply_sweep"] = apply_sweep()
        line["dense_crossover"] = dense_crossover()
        line["cufft_comparison"] = cufft_comparison()
        line["batched_apply"] = batched_apply()
        try:
            line["min_time_table"] = min_time_table()
        except Exception as e:  # the headline line must still print
            line["min_time_table"] = {"error": "%s: %s" % (type(e).__name__, e)}
        try:
            line["bounded_table"] = bounded_table()
        except Exception as e:
            line["bounded_table"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if args.workload.startswith("newton") and args.serve_requests >= 0:
        line["serve"] = run_serve(args.serve_requests or 4096, args.serve_slots, rank, world, dist,
                                  loads=(0.8, 0.5, 0.95))
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "newton_bounded":
        line["cpu_baseline"] = {"note": "not measured for the bounded workload (the oracle's bounded solve is "
                                        "dense); the default workload carries the oracle baseline"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        line.update(cpu_baseline())
        line["cpu_apply_baseline"] = cpu_apply_baseline(N)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
