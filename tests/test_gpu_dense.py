"""GPU parity of the dense tensor-core product (tcgen05, 3xTF32) against the oracle's dense B^a.

The dense path multiplies by B^a itself, so the reference is the oracle's matrix of integrated
Lagrange polynomials (Eq. manyDefs with B = s B^a); the tolerance is the FP32 product bound,
1e-5 relative in the 2-norm, as for the FP32 FFT chain.
"""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _api():
    from paper_2509_01855_gb300 import api
    return api


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dense_run(N, trans, n_comp, batch, t0=0.0, tf=3.0, dense=True):
    api = _api()
    plan = api.Plan(N, n_comp=n_comp, max_batch=batch, dtype=torch.float32, t0=t0, tf=tf)
    plan.set_dense(dense)
    L = N + 1
    V = synth.gaussian((batch, n_comp, L), "dense", N, int(trans))
    v = plan.empty(batch)
    v[:, :, :L] = torch.as_tensor(V, dtype=torch.float32)
    v[:, :, L:] = 7.0          # padding must be ignored
    out = plan.empty(batch)
    out.fill_(3.0)
    (api.birkhoff_apply_T if trans else api.birkhoff_apply)(plan, v, out)
    torch.cuda.synchronize()
    o = out.cpu().double().numpy()
    assert np.all(o[:, :, L:] == 0.0), "padding not zeroed"
    if dense:
        assert plan.dense_check() == 0, "dense kernel reported a timeout"
    return o[:, :, :L], V


@pytest.mark.parametrize("N", [4, 8, 16, 64, 128, 256, 512, 1024])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("n_comp,batch", [(1, 1), (3, 2), (17, 1), (4, 10)])
def test_dense_vs_dense_oracle(N, trans, n_comp, batch):
    """1, 6, 17 and 40 vectors: one 16-vector tile, a ragged tile, and several tiles."""
    got, V = _dense_run(N, trans, n_comp, batch)
    B = ob.dense_B(N, 0.0, 3.0)
    ref = V @ (B if trans else B.T)
    assert _rel(got, ref) < TOL32


@pytest.mark.parametrize("N", [16, 256, 1024])
def test_dense_matches_fft_chain(N):
    """The two FP32 paths of one plan agree to FP32 rounding."""
    a, V = _dense_run(N, False, 4, 2, dense=True)
    b, V2 = _dense_run(N, False, 4, 2, dense=False)
    assert np.array_equal(V, V2)
    assert _rel(a, b) < 2 * TOL32


def test_dense_constant_and_row0():
    """B 1 = t - t0 at every node and row 0 of B is zero (Eq. birk-conditions)."""
    api = _api()
    N = 512
    plan = api.Plan(N, n_comp=1, dtype=torch.float32, t0=1.0, tf=4.0)
    plan.set_dense(True)
    t, _ = plan.grid()
    v = plan.empty(1)
    v[:, :, :N + 1] = 1.0
    out = plan.empty(1)
    api.birkhoff_apply(plan, v, out)
    torch.cuda.synchronize()
    o = out[0, 0, :N + 1].cpu().double().numpy()
    assert o[0] == 0.0 or abs(o[0]) < 1e-6
    assert np.max(np.abs(o - (t.numpy() - 1.0))) < 1e-5 * 3.0


@pytest.mark.parametrize("ksplit", ["1", "3", "8", "16"])
@pytest.mark.parametrize("N", [64, 1024])
def test_dense_k_splits(N, ksplit, monkeypatch):
    """Unsplit tiles, an uneven split (chunks per CTA differ) and the largest splits give the
    same product (partials are added in a fixed order)."""
    monkeypatch.setenv("BK_DENSE_KSPLIT", ksplit)
    got, V = _dense_run(N, False, 4, 5)
    B = ob.dense_B(N, 0.0, 3.0)
    assert _rel(got, V @ B.T) < TOL32


def test_dense_repeat_is_bitwise():
    """Repeated products of one plan (counters reset by the last CTA of each tile) are
    bit-identical."""
    api = _api()
    N = 512
    plan = api.Plan(N, n_comp=4, max_batch=3, dtype=torch.float32, t0=0.0, tf=3.0)
    plan.set_dense(True)
    v = plan.empty(3)
    v[:, :, :N + 1] = torch.as_tensor(synth.gaussian((3, 4, N + 1), "dense-rep"), dtype=torch.float32)
    outs = []
    for _ in range(3):
        o = plan.empty(3)
        api.birkhoff_apply(plan, v, o)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    assert plan.dense_check() == 0


def test_dense_default_policy(monkeypatch):
    """Power-of-two plans start on the FFT chain; BK_DENSE=1 starts those with N <= 1024 and at
    most 16 vectors on the dense path; other N are always dense."""
    api = _api()
    for dt in (torch.float32, torch.float64):
        assert not api.Plan(256, n_comp=4, dtype=dt).is_dense()
        assert api.Plan(100, n_comp=4, dtype=dt).is_dense()
    monkeypatch.setenv("BK_DENSE", "1")
    for N, n_comp, batch, want in [(64, 4, 1, True), (1024, 4, 4, True), (1024, 4, 5, False), (2048, 4, 1, False)]:
        for dt in (torch.float32, torch.float64):
            assert api.Plan(N, n_comp=n_comp, max_batch=batch, dtype=dt).is_dense() == want, (N, dt)


def _run_any(N, dtype, trans, n_comp, batch, dense=None):
    api = _api()
    plan = api.Plan(N, n_comp=n_comp, max_batch=batch, dtype=dtype, t0=0.0, tf=3.0)
    if dense is not None:
        plan.set_dense(dense)
    L = N + 1
    V = synth.gaussian((batch, n_comp, L), "any", N, int(trans))
    v = plan.empty(batch)
    v[:, :, :L] = torch.as_tensor(V, dtype=dtype)
    v[:, :, L:] = 7.0
    out = plan.empty(batch)
    out.fill_(3.0)
    (api.birkhoff_apply_T if trans else api.birkhoff_apply)(plan, v, out)
    torch.cuda.synchronize()
    o = out.cpu().double().numpy()
    assert np.all(o[:, :, L:] == 0.0), "padding not zeroed"
    return o[:, :, :L], V, plan


TOL = {torch.float64: 1e-12, torch.float32: TOL32}


@pytest.mark.parametrize("N", [4, 8, 64, 256, 1024])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("n_comp,batch", [(4, 1), (5, 4)])
def test_dense_f64_vs_dense_oracle(N, trans, n_comp, batch):
    """FP64 dense product (CUDA-core FMAs, split K) against the oracle's B^a at 1e-12."""
    got, V, _ = _run_any(N, torch.float64, trans, n_comp, batch, dense=True)
    B = ob.dense_B(N, 0.0, 3.0)
    assert _rel(got, V @ (B if trans else B.T)) < 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [5, 6, 7, 12, 100, 300, 1000])
@pytest.mark.parametrize("trans", [False, True])
def test_any_N_products(N, dtype, trans):
    """N not a power of two: the plan takes the dense product, B^a formed from its definition."""
    got, V, plan = _run_any(N, dtype, trans, 3, 2)
    assert plan.shape()["path"] == "dense"
    B = ob.dense_B(N, 0.0, 3.0)
    assert _rel(got, V @ (B if trans else B.T)) < TOL[dtype]


@pytest.mark.parametrize("N", [5, 12, 100, 1000])
def test_any_N_grid(N):
    """Nodes and Clenshaw-Curtis weights (the last row of B^a) for an N that is not a power of
    two: against the oracle's nodes and closed-form weights; B 1 = t - t0."""
    from oracle import grid as og
    api = _api()
    plan = api.Plan(N, dtype=torch.float64, t0=0.0, tf=2.0)
    t, w = plan.grid()
    tau = og.cgl_nodes(N)
    assert np.max(np.abs(t.numpy() - (tau + 1.0))) < 1e-15
    assert np.max(np.abs(w.numpy() - og.cc_weights_sum(N))) < 1e-13
    v = plan.empty(1)
    v[:, :, :N + 1] = 1.0
    out = plan.empty(1)
    api.birkhoff_apply(plan, v, out)
    torch.cuda.synchronize()
    assert np.max(np.abs(out[0, 0, :N + 1].cpu().numpy() - t.numpy())) < 1e-13


def test_dense_switch_back_and_unsupported():
    api = _api()
    from paper_2509_01855_gb300._lib import BirkhoffError
    big = api.Plan(2048, dtype=torch.float32)
    with pytest.raises(BirkhoffError):
        big.set_dense(True)
    odd = api.Plan(100, dtype=torch.float64)
    with pytest.raises(BirkhoffError):
        odd.set_dense(False)
    a, V = _dense_run(64, True, 2, 1, dense=True)
    B = ob.dense_B(64, 0.0, 3.0)
    assert _rel(a, V @ B) < TOL32


def test_dense_timeout_path_reports_and_recovers():
    """The dense kernel's bounded-wait failure path, made to run by the test mode (a wait on a
    barrier nothing signals): the error word reports it, the context stays usable, and with the
    mode off the same plan computes the right product again."""
    from oracle import birkhoff as ob
    from paper_2509_01855_gb300 import _lib, api
    N = 100
    plan = api.Plan(N, n_comp=2, max_batch=1, dtype=torch.float32, t0=0.0, tf=2.0)
    assert plan.is_dense()
    V = synth.gaussian((2, N + 1), "dense-timeout")
    v = plan.empty(1)
    v[0, :, :N + 1] = torch.as_tensor(V)
    assert _lib.lib().bk_plan_dense_test_timeout(plan.handle, 1) == 0
    api.birkhoff_apply(plan, v, plan.empty(1))
    assert plan.dense_check() in (1, 2)     # the copy wait gave up (2 if a warp saw it first)
    assert _lib.lib().bk_plan_dense_test_timeout(plan.handle, 0) == 0
    out = api.birkhoff_apply(plan, v, plan.empty(1))
    assert plan.dense_check() == 0
    ref = V @ ob.dense_B(N, 0.0, 2.0).T
    assert np.linalg.norm(out[0, :, :N + 1].cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5


def test_dense_timeout_fails_the_krylov_and_newton_solves(monkeypatch):
    """A solve on a dense FP32 problem whose products time out returns BK_ERR_TIMEOUT (5)."""
    from paper_2509_01855_gb300 import _lib, api
    N = 100
    monkeypatch.setenv("BK_DENSE_TEST_TIMEOUT", "1")
    prob = api.Problem(_lib.BK_DBL_INT, N, torch.float32, 0.0, 1.0)
    monkeypatch.delenv("BK_DENSE_TEST_TIMEOUT")
    t, _ = api.Plan(N, t0=0.0, tf=1.0).grid()
    X, U = synth.double_integrator_guess(t.numpy())
    z = prob.pack(X, U)
    prob.linearize(z)
    rhs = prob.zeros(_lib.BK_OP_KKT)
    rhs[: prob.L] = 1.0
    sol = torch.zeros_like(rhs)
    info = api.krylov_solve(prob, _lib.BK_OP_KKT, rhs, sol, rtol=1e-4, raise_on_fail=False)
    assert info["status"] == 5
    res = api.newton_solve(prob, z, max_iter=2, raise_on_fail=False)
    assert res["status"] == 5
