"""The allocation-free product birkhoff_apply_noalloc, through the C ABI.

It serves callers that may not allocate device memory while running (fixed-budget real-time
loops, host programs whose allocator owns the GPU): they pass their own input and output and
the library uses a statically reserved device array for tables and scratch. This file is
collected last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu


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


def test_noalloc_rejects_sizes_beyond_its_scratch():
    v = torch.zeros(2 * ((1 << 17) + 32), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(v)
    assert _noalloc(v, out, 1 << 17, 1, (1 << 17) + 32, 0.0, 1.0) == 1     # BK_ERR_ARG
    assert _noalloc(v, out, 1 << 14, 9, (1 << 14) + 32, 0.0, 1.0) == 1     # too many vectors
    from paper_2509_01855_gb300 import _lib
    assert b"N must be" in _lib.lib().bk_last_error() or b"nvec" in _lib.lib().bk_last_error()
