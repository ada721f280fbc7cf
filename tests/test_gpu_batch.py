"""birkhoff_apply_batch: products of plans with different N in shared launches.

Every entry of a batch must come out bitwise equal to the plan's own birkhoff_apply(_T): the
batched kernels run each plan's pass bodies with that plan's shapes and thread count. One entry
is also checked against the FastBV oracle, so that the comparison does not rest on the per-plan
path alone. The mixes hold plans of every path: single-CTA, unsplit four-step, dense (N not a
power of two up to 1024), Bluestein, split and double-float four-step.
"""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu

MIXES = {
    torch.float32: [64, 4096, 256, 8192, 1 << 14, 100, 1 << 16, 3000, 1 << 12, 1 << 23],
    torch.float64: [64, 256, 128, 1024, 1 << 14, 1000, 1 << 16, 1 << 17, 1 << 18, 2048],
}


def _plans(dtype, Ns):
    from paper_2509_01855_gb300 import api
    plans, vs = [], []
    for i, N in enumerate(Ns):
        b = 1 + (i % 2)
        p = api.Plan(N, n_comp=2, max_batch=2, dtype=dtype, t0=0.5, tf=0.5 + 4.0 * (1 + i % 3))
        v = p.empty(b)
        v[:, :, :p.L] = torch.as_tensor(synth.gaussian((b, 2, p.L), "batch", N, i), dtype=dtype)
        v[:, :, p.L:] = 5.0
        plans.append(p)
        vs.append(v)
    return api, plans, vs


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("trans", [False, True])
def test_batch_matches_each_plan_bitwise(dtype, trans):
    api, plans, vs = _plans(dtype, MIXES[dtype])
    paths = {p.shape()["path"] for p in plans}
    assert {"single_cta", "four_step", "dense"} <= paths, paths
    ref = []
    for p, v in zip(plans, vs):
        o = p.empty(v.shape[0]).fill_(1.0)
        (api.birkhoff_apply_T if trans else api.birkhoff_apply)(p, v, o)
        ref.append(o)
    outs = [p.empty(v.shape[0]).fill_(2.0) for p, v in zip(plans, vs)]
    api.birkhoff_apply_batch(plans, vs, outs, trans=trans)
    torch.cuda.synchronize()
    for p, o, r in zip(plans, outs, ref):
        assert torch.equal(o, r), (p.N, p.shape())
    # the FastBV oracle on the second four-step entry (N = 2^14)
    k = MIXES[dtype].index(1 << 14)
    V = vs[k][:, :, :plans[k].L].double().cpu().numpy()
    f = ob.fastbv_T if trans else ob.fastbv
    want = np.stack([np.stack([f(V[b, c], plans[k].t0, plans[k].tf) for c in range(2)])
                     for b in range(V.shape[0])])
    got = outs[k][:, :, :plans[k].L].double().cpu().numpy()
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)


def test_batch_in_place_and_more_than_sixteen():
    """v == out per entry, and a batch longer than one launch's 16 plans."""
    Ns = [256 * (1 + (i % 4)) if i % 3 else 1 << (8 + i % 9) for i in range(20)]
    Ns = [n if (n & (n - 1)) == 0 else 1 << 12 for n in Ns]
    api, plans, vs = _plans(torch.float32, Ns)
    ref = []
    for p, v in zip(plans, vs):
        o = p.empty(v.shape[0])
        api.birkhoff_apply(p, v, o)
        ref.append(o)
    api.birkhoff_apply_batch(plans, vs, vs)
    torch.cuda.synchronize()
    for p, v, r in zip(plans, vs, ref):
        assert torch.equal(v, r), p.N


def test_batch_rejects_bad_batches():
    from paper_2509_01855_gb300 import _lib, api
    p1 = api.Plan(1 << 14, n_comp=1, dtype=torch.float32)
    p2 = api.Plan(1 << 12, n_comp=1, dtype=torch.float64)
    v1, o1, v1b, o1b = (p1.empty(1) for _ in range(4))
    with pytest.raises(_lib.BirkhoffError):   # a four-step plan twice: shared scratch
        api.birkhoff_apply_batch([p1, p1], [v1, v1b], [o1, o1b])
    v2, o2 = p2.empty(1), p2.empty(1)
    hp = np.array([p1.handle.value, p2.handle.value], dtype=np.uint64)   # kept alive for the call
    hv = np.array([v1.data_ptr(), v2.data_ptr()], dtype=np.uint64)
    ho = np.array([o1.data_ptr(), o2.data_ptr()], dtype=np.uint64)
    hb = np.array([1, 1], dtype=np.int32)
    with pytest.raises(_lib.BirkhoffError):   # mixed dtypes
        _lib.check(_lib.lib().birkhoff_apply_batch(hp.ctypes.data, hv.ctypes.data, ho.ctypes.data, hb.ctypes.data,
                                                   2, 0, None))
