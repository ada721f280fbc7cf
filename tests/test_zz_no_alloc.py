"""The allocation-free product birkhoff_apply_noalloc, through the C ABI.

It serves callers that may not allocate device memory while running (fixed-budget real-time
loops, host programs whose allocator owns the GPU): they pass their own input and output and
the library uses a statically reserved device array for tables and scratch. This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _noalloc(v, out, N, nvec, pitch, t0, tf):
    from paper_2509_01855_gb300 import _lib
    lib = _lib.lib()
    st = lib.birkhoff_apply_noalloc(ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    int(N), int(nvec), int(pitch), float(t0), float(tf),
                                    _lib.stream_ptr(None))
    return st


@pytest.mark.parametrize("calls", [[(1 << 14, 4, 0.0, 20.0), (1 << 16, 2, -1.0, 3.0)]])
def test_noalloc_matches_birkhoff_apply(calls):
    """Two calls in a row (different sizes) against the plan-based product; 1e-12 relative."""
    from paper_2509_01855_gb300 import api
    for (N, nvec, t0, tf) in calls:
        plan = api.Plan(N, n_comp=nvec, max_batch=1, dtype=torch.float64, t0=t0, tf=tf)
        L = N + 1
        v = plan.empty(1)
        v[0, :, :L] = torch.as_tensor(synth.gaussian((nvec, L), "noalloc", N))
        ref = api.birkhoff_apply(plan, v, plan.empty(1))
        out = torch.full_like(v, 5.0)
        assert _noalloc(v, out, N, nvec, plan.pitch, t0, tf) == 0
        torch.cuda.synchronize()
        a = out[0, :, :L].cpu().numpy()
        b = ref[0, :, :L].cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
        assert torch.all(out[0, :, L:] == 0)


def test_noalloc_largest_layout_matches_oracle():
    """N = 2^16 with 8 vectors (the largest layout the reserved array admits), twice in a row,
    against the oracle's FastBV chain; 1e-12 relative."""
    N, nvec, t0, tf = 1 << 16, 8, 0.0, 20.0
    L, pitch = N + 1, N + 32
    V = synth.gaussian((nvec, L), "noalloc-max")
    v = torch.zeros(nvec, pitch, dtype=torch.float64, device="cuda")
    v[:, :L] = torch.as_tensor(V)
    ref = ob.fastbv(V, t0, tf)
    for _ in range(2):
        out = torch.full_like(v, -3.0)
        assert _noalloc(v, out, N, nvec, pitch, t0, tf) == 0
        torch.cuda.synchronize()
        got = out[:, :L].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
        assert torch.all(out[:, L:] == 0)


def test_noalloc_in_a_fresh_process_without_plans():
    """The real use: a process that never creates a plan (so nothing but the entry point's own
    set-up prepares the kernels) calls it first, against the oracle."""
    code = textwrap.dedent("""
        import ctypes, sys
        import numpy as np, torch
        sys.path.insert(0, %r)
        from oracle import birkhoff as ob
        from paper_2509_01855_gb300 import _lib, synth
        N, nvec, pitch = 1 << 15, 3, (1 << 15) + 32
        V = synth.gaussian((nvec, N + 1), "noalloc-fresh")
        v = torch.zeros(nvec, pitch, dtype=torch.float64, device="cuda")
        v[:, :N + 1] = torch.as_tensor(V)
        out = torch.zeros_like(v)
        lib = _lib.lib()
        for _ in range(2):
            st = lib.birkhoff_apply_noalloc(ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            N, nvec, pitch, 1.0, 5.0, None)
            assert st == 0, lib.bk_last_error()
            torch.cuda.synchronize()
            ref = ob.fastbv(V, 1.0, 5.0)
            e = np.linalg.norm(out[:, :N + 1].cpu().numpy() - ref) / np.linalg.norm(ref)
            assert e < 1e-12, e
        print("fresh-process noalloc ok")
    """ % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "fresh-process noalloc ok" in r.stdout, r.stdout + r.stderr


def test_noalloc_rejects_sizes_beyond_its_scratch():
    v = torch.zeros(2 * ((1 << 17) + 32), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(v)
    assert _noalloc(v, out, 1 << 17, 1, (1 << 17) + 32, 0.0, 1.0) == 1     # BK_ERR_ARG
    assert _noalloc(v, out, 1 << 14, 9, (1 << 14) + 32, 0.0, 1.0) == 1     # too many vectors
    from paper_2509_01855_gb300 import _lib
    assert b"N must be" in _lib.lib().bk_last_error() or b"nvec" in _lib.lib().bk_last_error()


def test_noalloc_rejects_overlapping_vectors():
    from paper_2509_01855_gb300 import _lib
    N, pitch = 1 << 14, (1 << 14) + 32
    buf = torch.zeros(3 * pitch, dtype=torch.float64, device="cuda")
    assert _noalloc(buf, buf, N, 1, pitch, 0.0, 1.0) == 1
    assert _noalloc(buf, buf[pitch:], N, 2, pitch, 0.0, 1.0) == 1
    assert b"overlap" in _lib.lib().bk_last_error()
