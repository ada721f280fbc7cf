"""Full-size parity of the orbit-raising Newton-Krylov solve (the benchmark's problem: r 1 -> 1.5,
t_f = 20, minimum-energy thrust vector) against the oracle.

N = 2^14: the GPU solve against the matrix-free oracle's solve on the same grid (the same
discretisation, so the two agree to rounding and the solve tolerance). N = 2^20: the GPU solve
against the dense oracle's solution at N_ref = 1024, evaluated on the fine nodes by barycentric
interpolation. The oracle's own self-convergence (tests/test_oracle_matfree.py) puts the
discrete solution at N_ref within 5e-13 of finer grids in the states and 3e-10 in the controls
(quadrature norm). Both precisions: FP64, and FP32 Krylov with the FP64 Newton residual.

Tolerances: states 1e-9 max-abs; controls 1e-9 in the quadrature norm sqrt(sum s w u^2); the
multipliers through the costate p = (B^a)^T lambda / w in the same norm (the discrete lambda
carries the terminal multiplier nu as an atom at the last node, so lambda / w itself has no
limit there), and nu itself 1e-9. The Newton count with tight inner solves and the merit
history ||F_k||_W equal the oracle's (mesh independence, Table tab:m).
"""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from oracle import problems as op
from oracle.grid import interpolate
from oracle.kkt import DenseKKT
from oracle.matfree import MatFreeKKT
from paper_2509_01855_gb300 import synth
from tests.helpers import from_packed, to_packed

pytestmark = pytest.mark.gpu

RF, TF, A = 1.5, 20.0, 0.01
N_REF = 1024


def _guess(K):
    X, U = synth.orbit_guess(K.t, RF, TF)
    return K.pack(X, U, np.zeros((4, K.L)), np.zeros(3))


@pytest.fixture(scope="module")
def dense_ref():
    K = DenseKKT(op.Problem(op.ORBIT, 0.0, TF, (A, RF)), N_REF)
    vec, info = K.newton(_guess(K), tol=1e-12)
    assert info["converged"]
    return K, vec, info


@pytest.fixture(scope="module")
def matfree_ref_2p14():
    M = MatFreeKKT(op.Problem(op.ORBIT, 0.0, TF, (A, RF)), 1 << 14)
    vec, info = M.newton(_guess(M), tol=1e-12)
    assert info["converged"]
    return M, vec, info


def _gpu_solve(N, dtype, **kw):
    from paper_2509_01855_gb300 import _lib, api
    prob = api.Problem(_lib.BK_ORBIT, N, dtype, 0.0, TF, (A, RF))
    t, w = api.Plan(N, t0=0.0, tf=TF).grid()
    X, U = synth.orbit_guess(t.numpy(), RF, TF)
    z = prob.pack(X, U)
    ws = api.newton_workspace(prob)
    info = api.newton_solve(prob, z, workspace=ws, **kw)
    return prob, z, info, ws


def _costate(lam, w):
    return ob.fastbv_T(lam) / w


def _compare(X, U, lam, nu, w, s, Xr, Ur, pr, nur):
    wq = s * w
    p = _costate(lam, w)
    e_x = float(np.abs(X - Xr).max())
    e_u = float(np.sqrt(np.sum(wq * (U - Ur) ** 2)))
    e_p = float(np.sqrt(np.sum(wq * (p - pr) ** 2)))
    e_n = float(np.abs(nu - nur).max())
    return dict(state=e_x, control=e_u, costate=e_p, nu=e_n)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_orbit_2p14_matches_oracle_on_the_same_grid(dtype, matfree_ref_2p14):
    M, ref, rinfo = matfree_ref_2p14
    N = 1 << 14
    kw = dict(tol=1e-11, krylov_rtol=1e-12) if dtype == torch.float64 else dict(tol=1e-11)
    prob, z, info, _ = _gpu_solve(N, dtype, **kw)
    assert info["converged"], info
    # the same start point: the initial merit agrees to rounding
    assert abs(info["residual0"] - rinfo["norms"][0]) <= 1e-12 * rinfo["norms"][0]
    if dtype == torch.float64:
        assert info["iterations"] == rinfo["iters"]
    got = to_packed(prob, z)
    X, U, lam, nu = M.split(got)
    Xr, Ur, lr, nr = M.split(ref)
    err = _compare(X, U, lam, nu, M.w, M.s, Xr, Ur, _costate(lr, M.w), nr)
    print("N=2^14 %s vs oracle (same grid):" % dtype, err)
    assert err["state"] < 1e-9 and err["control"] < 1e-9 and err["nu"] < 1e-9
    assert err["costate"] < 1e-9 * max(1.0, float(np.abs(_costate(lr, M.w)).max()))
    # the discrete multipliers themselves, in the dual quadrature norm
    wq = M.s * M.w
    assert np.sqrt(np.sum((lam - lr) ** 2 / wq)) < 1e-9 * max(1.0, np.sqrt(np.sum(lr ** 2 / wq)))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_orbit_2p20_matches_oracle_interpolant(dtype, dense_ref):
    from paper_2509_01855_gb300 import api
    K, ref, rinfo = dense_ref
    N = 1 << 20
    kw = dict(tol=1e-11, krylov_rtol=1e-12) if dtype == torch.float64 else dict(tol=1e-11)
    prob, z, info, ws = _gpu_solve(N, dtype, **kw)
    assert info["converged"], info
    Xg, Ug, lg, ng = [a.detach().cpu().numpy() for a in prob.split(z)]
    tau = np.sin(np.pi * (2.0 * np.arange(N + 1) - N) / (2.0 * N))     # fine CGL nodes
    eN = np.zeros(N + 1); eN[N] = 1.0
    w = ob.fastbv_T(eN)                                                  # fine CC weights
    s = 0.5 * TF
    Xr, Ur, lr, nr = K.split(ref)
    vals = interpolate(np.concatenate([Xr, Ur, _costate(lr, K.w)]), N_REF, tau)
    err = _compare(Xg, Ug, lg, ng, w, s, vals[:4], vals[4:6], vals[6:], nr)
    print("N=2^20 %s vs oracle N_ref=%d interpolant:" % (dtype, N_REF), err)
    assert err["state"] < 1e-9 and err["control"] < 1e-9 and err["nu"] < 1e-9
    assert err["costate"] < 1e-9 * max(1.0, float(np.abs(vals[6:]).max()))
    if dtype == torch.float64:
        # mesh independence: the Newton count and the merit history of the oracle at N_ref
        assert info["iterations"] == rinfo["iters"]
        assert abs(info["residual0"] - rinfo["norms"][0]) < 1e-9 * rinfo["norms"][0]
        t, _ = api.Plan(N, t0=0.0, tf=TF).grid()
        X0, U0 = synth.orbit_guess(t.numpy(), RF, TF)
        for k in range(1, rinfo["iters"]):
            zk = prob.pack(X0, U0)
            ik = api.newton_solve(prob, zk, workspace=ws, max_iter=k, raise_on_fail=False, **kw)
            assert ik["iterations"] == k
            # the inner solves stop at 1e-12 (2-norm), so late steps agree to ~1e-12 absolute
            assert abs(ik["residual"] - rinfo["norms"][k]) < 1e-5 * rinfo["norms"][k] + 1e-12, (k, ik, rinfo["norms"])
