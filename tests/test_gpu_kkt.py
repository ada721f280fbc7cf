"""GPU parity of kkt_apply, precond_apply, krylov_solve and newton_solve against the dense oracle."""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from oracle import problems as op
from oracle.kkt import DenseKKT
from paper_2509_01855_gb300 import synth
from tests.helpers import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _api():
    from paper_2509_01855_gb300 import _lib, api
    return api, _lib


def _setup(kind, N, dtype, seed=0):
    """Library problem, oracle DenseKKT and a linearisation point (packed, oracle order)."""
    api, lib = _api()
    if kind == op.ORBIT:
        t0, tf, params = 0.0, 20.0, (0.01, 1.5)
    elif kind == op.DBL_INT:
        t0, tf, params = 0.0, 1.0, ()
    else:
        t0, tf, params = 0.0, 2.0, (1.0,)
    oprob = op.Problem(kind, t0, tf, params)
    K = DenseKKT(oprob, N)
    prob = api.Problem({op.DBL_INT: lib.BK_DBL_INT, op.ORBIT: lib.BK_ORBIT,
                        op.BILINEAR: lib.BK_BILINEAR}[kind], N, dtype, t0, tf, params)
    g = synth.rng("kkt-lin", kind, N, seed)
    if kind == op.ORBIT:
        X, U = synth.orbit_guess(K.t, 1.5, tf)
        X = X + 0.01 * g.standard_normal(X.shape)
        U = U + 0.001 * g.standard_normal(U.shape)
    elif kind == op.DBL_INT:
        X, U = synth.double_integrator_guess(K.t)
        X = X + 0.1 * g.standard_normal(X.shape)
        U = g.standard_normal(U.shape)
    else:
        X = 1.0 + 0.1 * g.standard_normal((1, K.L))
        U = synth.smooth_coefficient(K.t, t0, tf, N)[None, :]
    lam = 0.01 * g.standard_normal((oprob.n_x, K.L))
    nu = 0.01 * g.standard_normal(oprob.n_e)
    vec = K.pack(X, U, lam, nu)
    z = from_packed(prob, vec)
    prob.linearize(z)
    return api, lib, prob, K, vec


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind,N", [(op.ORBIT, 16), (op.ORBIT, 64), (op.DBL_INT, 32), (op.BILINEAR, 64),
                                    (op.ORBIT, 256)])
def test_state_operator_and_preconditioner(kind, N, dtype):
    api, lib, prob, K, vec = _setup(kind, N, dtype)
    g = synth.rng("state-in", kind, N)
    chi = g.standard_normal(K.nc)
    x = from_packed(prob, chi, dtype, op_kkt=False)
    out = torch.zeros_like(x)
    api.kkt_apply(prob, lib.BK_OP_STATE, x, out)
    Gx = K.state_matrix(vec)
    assert rel(to_packed(prob, out, False), Gx @ chi) < TOL[dtype]
    # Reference: the oracle's sequential forward / backward substitution through the rows of P
    # (pinned to the dense P in the oracle tests). A dense LU solve of P loses ~cond(P) * eps
    # (2e-11 at N = 256 for the orbit), more than the sweep itself.
    X, U, _, _ = K.split(vec)
    Jx, _ = K.prob.jac(X, U)
    Y = chi.reshape(K.prob.n_x, K.L)
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    api.precond_apply(prob, lib.BK_OP_STATE, x, out, transpose=False)
    assert rel(to_packed(prob, out, False), ob.fastpinvy_block(K.s * K.w, Jx, Y).ravel()) < tol
    api.precond_apply(prob, lib.BK_OP_STATE, x, out, transpose=True)
    assert rel(to_packed(prob, out, False), ob.fastpinvy_block_T(K.s * K.w, Jx, Y).ravel()) < tol
    # padding stays zero
    o = out.view(prob.n_x, prob.pitch)
    assert torch.all(o[:, prob.L:] == 0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind,N", [(op.ORBIT, 16), (op.ORBIT, 128), (op.DBL_INT, 32), (op.DBL_INT, 8),
                                    (op.ORBIT, 45), (op.DBL_INT, 100)])
def test_kkt_operator_and_preconditioner(kind, N, dtype):
    api, lib, prob, K, vec = _setup(kind, N, dtype)
    g = synth.rng("kkt-in", kind, N)
    d = g.standard_normal(K.n)
    x = from_packed(prob, d, dtype)
    out = torch.zeros_like(x)
    api.kkt_apply(prob, lib.BK_OP_KKT, x, out)
    assert rel(to_packed(prob, out), K.matrix(vec) @ d) < TOL[dtype]
    api.precond_apply(prob, lib.BK_OP_KKT, x, out)
    ref = np.linalg.solve(K.precond_matrix(vec), d)
    # K-tilde is badly scaled (H~ = s w with w_0 ~ 1/N^2): compare in the relative 2-norm
    assert rel(to_packed(prob, out), ref) < (1e-10 if dtype == torch.float64 else 1e-3)


@pytest.mark.parametrize("kind,N,opname", [(op.ORBIT, 64, "KKT"), (op.DBL_INT, 64, "KKT"),
                                           (op.BILINEAR, 128, "STATE"), (op.ORBIT, 128, "STATE")])
def test_krylov_solve_matches_dense_solve(kind, N, opname):
    api, lib, prob, K, vec = _setup(kind, N, torch.float64)
    opc = lib.BK_OP_KKT if opname == "KKT" else lib.BK_OP_STATE
    g = synth.rng("krylov-rhs", kind, N)
    if opname == "KKT":
        A = K.matrix(vec)
        b = g.standard_normal(K.n)
    else:
        A = K.state_matrix(vec)
        b = g.standard_normal(K.nc)
    rhs = from_packed(prob, b, op_kkt=opname == "KKT")
    sol = torch.zeros_like(rhs)
    info = api.krylov_solve(prob, opc, rhs, sol, rtol=1e-12, restart=40, max_iter=400)
    assert info["converged"], info
    x = to_packed(prob, sol, opname == "KKT")
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-11
    xref = np.linalg.solve(A, b)
    assert rel(x, xref) < 1e-11 * np.linalg.cond(A) + 1e-12


def test_krylov_not_converged_status():
    api, lib, prob, K, vec = _setup(op.ORBIT, 64, torch.float64)
    from paper_2509_01855_gb300._lib import BirkhoffError
    rhs = from_packed(prob, synth.gaussian(K.n, "nc"))
    sol = torch.zeros_like(rhs)
    info = api.krylov_solve(prob, lib.BK_OP_KKT, rhs, sol, rtol=1e-14, max_iter=1, raise_on_fail=False)
    assert info["status"] == 4 and not info["converged"] and info["iterations"] == 1
    with pytest.raises(BirkhoffError):
        api.krylov_solve(prob, lib.BK_OP_KKT, rhs, sol, rtol=1e-14, max_iter=1)


def test_preconditioned_iterations_fall_with_N():
    """The paper's linear-solve experiment: with the Birkhoff preconditioner the GMRES count on
    [I - B diag(d)] dX = x^a b does not grow with N (smooth d)."""
    api, lib = _api()
    counts = []
    for N in (256, 1024, 4096, 1 << 14):
        oprob = op.Problem(op.BILINEAR, 0.0, 2.0, (1.0,))
        prob = api.Problem(lib.BK_BILINEAR, N, torch.float64, 0.0, 2.0, (1.0,))
        t, _ = api.Plan(N, t0=0.0, tf=2.0).grid()
        d = synth.smooth_coefficient(t.numpy(), 0.0, 2.0, "fig6")
        z = prob.pack(np.ones((1, N + 1)), d[None, :])
        prob.linearize(z)
        rhs = prob.zeros(lib.BK_OP_STATE)
        rhs.view(1, prob.pitch)[:, :N + 1] = 1.0
        sol = torch.zeros_like(rhs)
        info = api.krylov_solve(prob, lib.BK_OP_STATE, rhs, sol, rtol=1e-12)
        counts.append(info["iterations"])
    assert all(counts[i + 1] <= counts[i] for i in range(len(counts) - 1)), counts
    assert counts[-1] <= 10, counts


@pytest.mark.parametrize("N", [4, 16, 64, 256, 6, 100, 1000])
def test_newton_double_integrator_closed_form(N):
    api, lib = _api()
    prob = api.Problem(lib.BK_DBL_INT, N, torch.float64, 0.0, 1.0)
    t, w = api.Plan(N, t0=0.0, tf=1.0).grid()
    t = t.numpy(); w = w.numpy()
    X, U = synth.double_integrator_guess(t)
    z = prob.pack(X, U)
    # linear dynamics, quadratic cost: one Newton step with a tight inner solve is exact
    info = api.newton_solve(prob, z, krylov_rtol=1e-12)
    assert info["converged"] and info["iterations"] == 1
    Xg, Ug, _, _ = [a.cpu().numpy() for a in prob.split(z)]
    assert np.abs(Xg[0] - (3 * t**2 - 2 * t**3)).max() < 1e-9
    assert np.abs(Xg[1] - (6 * t - 6 * t**2)).max() < 1e-9
    assert np.sqrt(0.5 * np.sum(w * (Ug[0] - (6 - 12 * t)) ** 2)) < 1e-9


@pytest.mark.parametrize("N", [16, 256])
def test_newton_double_integrator_forcing_term(N):
    """Default inner tolerance (forcing term): loose early steps still reach the closed form."""
    api, lib = _api()
    prob = api.Problem(lib.BK_DBL_INT, N, torch.float64, 0.0, 1.0)
    t, _ = api.Plan(N, t0=0.0, tf=1.0).grid()
    t = t.numpy()
    X, U = synth.double_integrator_guess(t)
    z = prob.pack(X, U)
    info = api.newton_solve(prob, z)
    assert info["converged"] and 1 <= info["iterations"] <= 4, info
    Xg = prob.split(z)[0].cpu().numpy()
    assert np.abs(Xg[0] - (3 * t**2 - 2 * t**3)).max() < 1e-9


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [32, 128, 48, 96])
def test_newton_orbit_matches_oracle(N, dtype):
    api, lib = _api()
    rf, tf = 1.5, 20.0
    oprob = op.Problem(op.ORBIT, 0.0, tf, (0.01, rf))
    K = DenseKKT(oprob, N)
    X, U = synth.orbit_guess(K.t, rf, tf)
    vec0 = K.pack(X, U, np.zeros((4, K.L)), np.zeros(3))
    ref, rinfo = K.newton(vec0)
    assert rinfo["converged"]
    prob = api.Problem(lib.BK_ORBIT, N, dtype, 0.0, tf, (0.01, rf))
    z = from_packed(prob, vec0)
    info = api.newton_solve(prob, z)
    assert info["converged"], info
    if dtype == torch.float64:
        assert info["iterations"] == rinfo["iters"]
    else:
        # FP32 inner solves to 1e-4 make the last Newton steps linearly convergent
        assert rinfo["iters"] <= info["iterations"] <= rinfo["iters"] + 3
    got = to_packed(prob, z)
    Xr, Ur, lr, nr = K.split(ref)
    Xg, Ug, lg, ng = K.split(got)
    assert np.abs(Xg - Xr).max() < 1e-9
    wq = K.s * K.w
    assert np.sqrt(np.sum(wq * (Ug - Ur) ** 2)) < 1e-9
    assert np.sqrt(np.sum((lg - lr) ** 2 / wq)) < 1e-9 * max(1.0, np.sqrt(np.sum(lr**2 / wq)))


@pytest.mark.parametrize("reuse", [1, 2])
def test_newton_precond_reuse_same_solution(reuse):
    """Keeping (part of) the preconditioner across steps changes the Krylov path, not the
    Newton solution: the FP64 solve reaches the same point as with rebuilds every step."""
    api, lib = _api()
    N, rf, tf = 256, 1.5, 20.0
    prob = api.Problem(lib.BK_ORBIT, N, torch.float64, 0.0, tf, (0.01, rf))
    t, _ = api.Plan(N, t0=0.0, tf=tf).grid()
    X, U = synth.orbit_guess(t.numpy(), rf, tf)
    z0 = prob.pack(X, U)
    z_ref = z0.clone()
    ref = api.newton_solve(prob, z_ref, tol=1e-12)
    z = z0.clone()
    info = api.newton_solve(prob, z, tol=1e-12, precond_reuse=reuse)
    assert ref["converged"] and info["converged"]
    assert ref["precond_builds"] == ref["iterations"]
    assert 1 <= info["precond_builds"] <= info["iterations"]
    assert (z - z_ref).abs().max().item() < 1e-9
