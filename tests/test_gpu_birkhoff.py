"""GPU parity of birkhoff_apply / birkhoff_apply_T against the oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from oracle import grid as og
from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu

# FP64 products must match to 1e-12 relative (2-norm), FP32 to 1e-5.
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _api():
    from paper_2509_01855_gb300 import api
    return api


def _run(N, dtype, trans, n_comp=3, batch=2, t0=0.0, tf=3.0, V=None, pitch=0, dense=None):
    api = _api()
    plan = api.Plan(N, n_comp=n_comp, max_batch=batch, dtype=dtype, t0=t0, tf=tf, pitch=pitch)
    if dense is not None:
        plan.set_dense(dense)
    L = N + 1
    if V is None:
        V = synth.gaussian((batch, n_comp, L), "bk", N, int(trans))
    v = plan.empty(batch)
    v[:, :, :L] = torch.as_tensor(V, dtype=dtype)
    v[:, :, L:] = 7.0          # padding must be ignored
    out = plan.empty(batch)
    out.fill_(3.0)
    (api.birkhoff_apply_T if trans else api.birkhoff_apply)(plan, v, out)
    torch.cuda.synchronize()
    o = out.cpu().double().numpy()
    assert np.all(o[:, :, L:] == 0.0), "padding not zeroed"
    return o[:, :, :L], V, plan


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [4, 8, 16, 64, 256, 1024])
@pytest.mark.parametrize("trans", [False, True])
def test_apply_vs_dense_oracle(N, dtype, trans):
    got, V, _ = _run(N, dtype, trans)
    B = ob.dense_B(N, 0.0, 3.0)
    ref = V @ (B if trans else B.T)
    assert _rel(got, ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [64, 128, 256, 512, 1024])
@pytest.mark.parametrize("trans", [False, True])
def test_dense_switch_vs_dense_oracle(N, dtype, trans):
    """A power-of-two plan switched to the dense product (tensor cores in FP32, CUDA cores in
    FP64) matches the oracle at the same tolerances as its FFT chain."""
    got, V, _ = _run(N, dtype, trans, dense=True)
    B = ob.dense_B(N, 0.0, 3.0)
    assert _rel(got, V @ (B if trans else B.T)) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [2048, 4096, 8192, 16384, 1 << 16])
@pytest.mark.parametrize("trans", [False, True])
def test_apply_vs_fastbv_oracle(N, dtype, trans):
    """Sizes past the dense oracle (and across the single-CTA / four-step boundary): compare
    with the oracle's FastBV chain on a library DCT."""
    got, V, _ = _run(N, dtype, trans, n_comp=2, batch=1)
    ref = (ob.fastbv_T if trans else ob.fastbv)(V, 0.0, 3.0)
    assert _rel(got, ref) < TOL[dtype]


@pytest.fixture
def force_split(monkeypatch):
    """Plans created while this is active use the split DCT-I from N = 2^13 on (the tuning
    variable is read at plan creation)."""
    monkeypatch.setenv("BK_SPLIT_MIN_LOG2", "13")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [8192, 16384, 1 << 16])
@pytest.mark.parametrize("trans", [False, True])
def test_split_dct_vs_fastbv_oracle(N, dtype, trans, force_split):
    """The split DCT-I (even half: DCT-I of the pair sums; odd half: DCT-III of the pair
    differences by a quarter-length inverse FFT) against the oracle's FastBV chain."""
    got, V, _ = _run(N, dtype, trans, n_comp=3, batch=2)
    ref = (ob.fastbv_T if trans else ob.fastbv)(V, 0.0, 3.0)
    assert _rel(got, ref) < TOL[dtype]


@pytest.mark.parametrize("N", [1 << 14, 1 << 17])
def test_split_sparse_modes_exact(N, force_split):
    modes, alphas = synth.sparse_modes(N)
    v, Bv = ob.sparse_mode_pair(N, modes, alphas, 0.0, 20.0)
    got, _, _ = _run(N, torch.float64, False, n_comp=1, batch=1, t0=0.0, tf=20.0, V=v[None, None, :])
    assert _rel(got[0, 0], Bv) < 1e-12


@pytest.mark.parametrize("N", [64, 4096, 1 << 15, 1 << 20])
def test_apply_sparse_modes_exact(N):
    """B applied to sum_k alpha_k T_k returns the exact integrals (closed forms)."""
    modes, alphas = synth.sparse_modes(N)
    v, Bv = ob.sparse_mode_pair(N, modes, alphas, 0.0, 20.0)
    got, _, _ = _run(N, torch.float64, False, n_comp=1, batch=1, t0=0.0, tf=20.0,
                     V=v[None, None, :])
    assert _rel(got[0, 0], Bv) < 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [16, 4096, 1 << 14, 1 << 18, 1 << 20, 1 << 22])
def test_adjoint_dot(N, dtype):
    """<B x, y> = <x, B^T y> with the library's two products."""
    api = _api()
    plan = api.Plan(N, n_comp=1, max_batch=1, dtype=dtype, t0=-1.0, tf=4.0)
    L = N + 1
    x = plan.empty(1); y = plan.empty(1)
    x[0, 0, :L] = torch.as_tensor(synth.gaussian(L, "adj-x", N), dtype=dtype)
    y[0, 0, :L] = torch.as_tensor(synth.gaussian(L, "adj-y", N), dtype=dtype)
    Bx = api.birkhoff_apply(plan, x, plan.empty(1))
    BTy = api.birkhoff_apply_T(plan, y, plan.empty(1))
    lhs = float((Bx.double() * y.double()).sum())
    rhs = float((x.double() * BTy.double()).sum())
    scale = float(Bx.double().norm() * y.double().norm())
    assert abs(lhs - rhs) / scale < (1e-13 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("N", [4, 64, 4096, 1 << 15])
def test_grid_tables(N):
    """Plan nodes and Clenshaw-Curtis weights equal the oracle's (Eq. CGLpts, last row of B^a)."""
    api = _api()
    plan = api.Plan(N, n_comp=1, dtype=torch.float64, t0=0.5, tf=2.5)
    t, w = plan.grid()
    tau = og.cgl_nodes(N)
    assert np.abs(t.numpy() - (0.5 + 1.0 * (tau + 1.0))).max() < 1e-15 * 4
    wref = og.cc_weights_sum(N) if N <= 4096 else None
    if wref is not None:
        assert np.abs(w.numpy() - wref).max() < 1e-14
    assert abs(w.sum().item() - 2.0) < 1e-13
    if N % 2 == 0:
        assert abs(w[0].item() - 1.0 / (N * N - 1.0)) < 1e-14 / N


def test_ones_gives_time():
    """B 1 = t - t0 at N = 2^20 (large four-step path)."""
    api = _api()
    N = 1 << 20
    plan = api.Plan(N, n_comp=1, dtype=torch.float64, t0=0.0, tf=20.0)
    v = plan.empty(1)
    v[0, 0, :N + 1] = 1.0
    out = api.birkhoff_apply(plan, v, plan.empty(1))
    t, _ = plan.grid()
    assert (out[0, 0, :N + 1].cpu() - t).abs().max().item() < 1e-11


def test_bad_arguments():
    api = _api()
    from paper_2509_01855_gb300._lib import BirkhoffError
    with pytest.raises(BirkhoffError):
        api.Plan((1 << 22) + 3)  # not a power of two and above the Bluestein limit of FP64
    with pytest.raises(BirkhoffError):
        api.Plan(2)              # too small
    with pytest.raises(BirkhoffError):
        api.Plan(1 << 25)        # above 2^24
    plan = api.Plan(64, n_comp=1, max_batch=1)
    v = plan.empty(2)
    with pytest.raises(BirkhoffError):
        api.birkhoff_apply(plan, v, plan.empty(2), batch=2)   # batch > max_batch


def _apply_with(plan, V, trans=False):
    api = _api()
    L = plan.N + 1
    v = plan.empty(V.shape[0])
    v[:, :, :L] = torch.as_tensor(V, dtype=plan.dtype)
    out = plan.empty(V.shape[0])
    (api.birkhoff_apply_T if trans else api.birkhoff_apply)(plan, v, out)
    torch.cuda.synchronize()
    return out.cpu().double().numpy()[:, :, :L]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_autotuned_tiles(dtype, monkeypatch):
    """The tile autotuner picks a valid four-step shape, plans of one size share it (cached),
    and the tuned and the heuristic shapes both match the oracle."""
    api = _api()
    N = 1 << 16
    p1 = api.Plan(N, n_comp=4, dtype=dtype, t0=0.0, tf=3.0)
    s1 = p1.shape()
    assert s1["path"] in ("four_step", "split_four_step")
    assert s1["N1"] * s1["N2"] in (N, N // 2, N // 4)
    assert s1["elems"] >= max(s1["N1"], 2 * s1["N2"]) and s1["elems"] & (s1["elems"] - 1) == 0
    p2 = api.Plan(N, n_comp=4, dtype=dtype, t0=0.0, tf=3.0)
    assert p2.shape() == s1
    monkeypatch.setenv("BK_AUTOTUNE", "0")
    p3 = api.Plan(N, n_comp=4, dtype=dtype, t0=0.0, tf=3.0)
    V = synth.gaussian((1, 4, N + 1), "tune", N)
    ref = ob.fastbv(V, 0.0, 3.0)
    refT = ob.fastbv_T(V, 0.0, 3.0)
    for p in (p1, p3):
        assert _rel(_apply_with(p, V), ref) < TOL[dtype]
        assert _rel(_apply_with(p, V, True), refT) < TOL[dtype]


def test_plan_shapes():
    api = _api()
    assert api.Plan(32, dtype=torch.float64).shape()["path"] == "single_cta"
    assert api.Plan(512, dtype=torch.float64).shape()["path"] == "four_step"
    assert api.Plan(100, dtype=torch.float64).shape()["path"] == "dense"
    assert api.Plan(1 << 19, n_comp=1, dtype=torch.float64).shape()["path"] == "split_four_step"
    assert api.Plan(256, n_comp=4, dtype=torch.float32).shape()["path"] == "single_cta"
    assert api.Plan(32, n_comp=4, dtype=torch.float32).shape()["path"] == "single_cta"
