"""GPU parity of the free-final-time orbit transfer (BK_ORBIT_MT, Eq. ot) against the oracle:
residual with the time gradient, bordered KKT product, bordered preconditioner, the
minimum-energy seed, Newton solves, and the mesh independence of Table tab:m at large N."""
import numpy as np
import pytest
import torch
from scipy.integrate import solve_ivp
from scipy.optimize import fsolve

from oracle import problems as op
from oracle.kkt import DenseKKT
from paper_2509_01855_gb300 import synth
from tests.helpers import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu

A_THRUST, R_F, T_SEED = 0.05, 6.0, 24.0
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _api():
    from paper_2509_01855_gb300 import _lib, api
    return api, _lib


def _lin_point(K, seed):
    """A linearisation point near the seeds the solver meets: the spiral for the states, angles
    spread over (-pi, pi), multipliers of the size the minimum-time solution has, s = 6.5."""
    g = synth.rng("mt-lin", K.N, seed)
    X, _ = synth.orbit_guess(K.t, R_F, T_SEED)
    X = X + 0.01 * g.standard_normal(X.shape)
    U = g.uniform(-np.pi, np.pi, (1, K.L))
    lam = g.standard_normal((4, K.L)) * K.w[None, :]
    nu = g.standard_normal(3)
    return K.pack(X, U, lam, nu, 6.5)


def _setup(N, dtype, seed=0):
    api, lib = _api()
    K = DenseKKT(op.Problem(op.ORBIT_MT, 0.0, T_SEED, (A_THRUST, R_F)), N)
    prob = api.Problem(lib.BK_ORBIT_MT, N, dtype, 0.0, T_SEED, (A_THRUST, R_F))
    vec = _lin_point(K, seed)
    z = from_packed(prob, vec)
    return api, lib, prob, K, vec, z


@pytest.mark.parametrize("N", [64, 100, 256])
def test_residual_with_time_gradient(N):
    api, lib, prob, K, vec, z = _setup(N, torch.float64)
    F = torch.zeros_like(z)
    wn = prob.residual(z, F)
    Fo = K.residual(vec)
    got = to_packed(prob, F)
    assert rel(got, Fo) < 1e-12
    assert abs(got[-1] - Fo[-1]) < 1e-12 * max(1.0, abs(Fo[-1]))      # g_s itself
    # the gradient rows enter the norm divided by w (w_0 ~ 1/N^2): rounding shows at 1e-12
    assert abs(wn - K.weighted_norm(Fo)) < 1e-11 * K.weighted_norm(Fo)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [64, 100, 256])
def test_bordered_kkt_and_preconditioner(N, dtype):
    api, lib, prob, K, vec, z = _setup(N, dtype)
    prob.linearize(z)
    g = synth.rng("mt-in", N)
    d = g.standard_normal(K.n)
    x = from_packed(prob, d, dtype)
    out = torch.zeros_like(x)
    api.kkt_apply(prob, lib.BK_OP_KKT, x, out)
    ref = K.matrix(vec) @ d
    got = to_packed(prob, out)
    assert rel(got, ref) < TOL[dtype]
    assert abs(got[-1] - ref[-1]) < 10 * TOL[dtype] * np.abs(ref).max()   # the s row
    api.precond_apply(prob, lib.BK_OP_KKT, x, out)
    M = K.precond_matrix(vec)
    ref = np.linalg.solve(M, d)
    # the dense solve itself loses about cond(K-tilde) eps (cond ~1e7 at N = 256)
    tol = 1e-10 + 1e-15 * np.linalg.cond(M) if dtype == torch.float64 else 1e-3
    assert rel(to_packed(prob, out), ref) < tol
    # padding stays zero
    o = out[:(2 * prob.n_x + prob.n_u) * prob.pitch].view(-1, prob.pitch)
    assert torch.all(o[:, prob.L:] == 0)


def _me_solve(api, lib, N, dtype=torch.float64):
    me = api.Problem(lib.BK_ORBIT, N, dtype, 0.0, T_SEED, (A_THRUST, R_F))
    t, _ = api.Plan(N, t0=0.0, tf=T_SEED).grid()
    X, U = synth.orbit_guess(t.numpy(), R_F, T_SEED)
    z = me.pack(X, U)
    info = api.newton_solve(me, z, tol=1e-11, krylov_rtol=1e-12, max_iter=60)
    assert info["converged"], info
    return me, z


@pytest.mark.parametrize("N", [64, 128])
def test_seed_matches_oracle_seed(N):
    """The library's seed and the oracle's, both from the library's minimum-energy solution."""
    api, lib = _api()
    me, zme = _me_solve(api, lib, N)
    mt = api.Problem(lib.BK_ORBIT_MT, N, torch.float64, 0.0, T_SEED, (A_THRUST, R_F))
    zmt = mt.zeros()
    api.min_time_seed(mt, me, zme, zmt)
    Kme = DenseKKT(op.Problem(op.ORBIT, 0.0, T_SEED, (A_THRUST, R_F)), N)
    K = DenseKKT(op.Problem(op.ORBIT_MT, 0.0, T_SEED, (A_THRUST, R_F)), N, Ba=Kme.Ba)
    ref = K.min_time_seed(Kme, to_packed(me, zme))
    assert rel(to_packed(mt, zmt), ref) < 1e-12
    assert zmt[mt.s_index].item() == 0.5 * T_SEED


def _mt_solve(api, lib, N, dtype=torch.float64, tol=1e-10):
    me, zme = _me_solve(api, lib, N)
    mt = api.Problem(lib.BK_ORBIT_MT, N, dtype, 0.0, T_SEED, (A_THRUST, R_F))
    z = mt.zeros(dtype=torch.float64)
    api.min_time_seed(mt, me, zme, z)
    info = api.newton_solve(mt, z, tol=tol, max_iter=40)
    return mt, z, info


@pytest.mark.parametrize("N", [64, 128])
def test_newton_min_time_matches_oracle(N):
    api, lib = _api()
    mt, z, info = _mt_solve(api, lib, N)
    assert info["converged"], info
    Kme = DenseKKT(op.Problem(op.ORBIT, 0.0, T_SEED, (A_THRUST, R_F)), N)
    X, U = synth.orbit_guess(Kme.t, R_F, T_SEED)
    vme, _ = Kme.newton(Kme.pack(X, U, np.zeros((4, Kme.L)), np.zeros(3)))
    K = DenseKKT(op.Problem(op.ORBIT_MT, 0.0, T_SEED, (A_THRUST, R_F)), N, Ba=Kme.Ba)
    ref, rinfo = K.newton(K.min_time_seed(Kme, vme), max_iter=40)
    assert rinfo["converged"]
    got = to_packed(mt, z)
    assert abs(got[-1] - ref[-1]) < 1e-9                       # the final time
    Xg, Ug, _, _ = K.split(got)
    Xr, Ur, _, _ = K.split(ref)
    assert np.abs(Xg - Xr).max() < 1e-8
    # the steering direction (the angle is defined modulo 2 pi)
    assert np.abs(np.sin(Ug) - np.sin(Ur)).max() < 1e-6 and np.abs(np.cos(Ug) - np.cos(Ur)).max() < 1e-6


def _pmp_rhs(t, y, a):
    r, th, vr, vt, pr, pth, pvr, pvt = y
    u = np.arctan2(-pvr, -pvt)
    f = [vr, vt / r, vt * vt / r - 1 / r**2 + a * np.sin(u), -vr * vt / r + a * np.cos(u)]
    dpr = -(pth * (-vt / r**2) + pvr * (-vt * vt / r**2 + 2 / r**3) + pvt * (vr * vt / r**2))
    return f + [dpr, 0.0, -(pr - pvt * vt / r), -(pth / r + 2 * pvr * vt / r - pvt * vr / r)]


def test_mesh_independence_large_N():
    """Table tab:m in kind: from the same recipe (minimum-energy seed at t_f = 24) the Newton
    count is the same for N = 2^10, 2^12, 2^14 and 2^20, and the final time agrees with
    Pontryagin's extremal (shooting, started from the library's costate at t = 0): to 1e-4 at
    2^10, to 1e-9 from 2^12 on (the discrete optimum has converged spectrally there)."""
    api, lib = _api()
    its, T, sol = {}, {}, {}
    for N in (1 << 10, 1 << 12, 1 << 14, 1 << 20):
        mt, z, info = _mt_solve(api, lib, N)
        assert info["converged"], (N, info)
        its[N] = info["iterations"]
        T[N] = 2.0 * z[mt.s_index].item()
        sol[N] = (mt, z)
    assert len(set(its.values())) == 1, its
    # costate estimate p_0 = -(B^aT lambda)_0 / w_0 of the N = 2^10 solve seeds the shooting
    N = 1 << 10
    mt, z = sol[N]
    plan = api.Plan(N, n_comp=4, t0=-1.0, tf=1.0)
    _, w = plan.grid()
    lam = plan.empty(1)
    lam.zero_()
    lam[0, :, :N + 1] = mt.split(z)[2]
    mu = plan.empty(1)
    api.birkhoff_apply_T(plan, lam, mu)
    p0 = -(mu[0, :, 0].cpu().numpy()) / w[0].item()

    def res(v):
        y = solve_ivp(_pmp_rhs, (0.0, v[3]), [1.0, 0.0, 0.0, 1.0, v[0], 0.0, v[1], v[2]], args=(A_THRUST,),
                      rtol=1e-12, atol=1e-13).y[:, -1]
        f = _pmp_rhs(0.0, y, A_THRUST)[:4]
        return [y[0] - R_F, y[2], y[3] - R_F ** -0.5, 1.0 + np.dot(y[4:], f)]
    v, _, ier, _ = fsolve(res, [p0[0], p0[2], p0[3], T[N]], full_output=True, xtol=1e-13)
    assert ier == 1 and np.abs(res(v)).max() < 1e-10
    for n_, t_ in T.items():
        assert abs(t_ - v[3]) < (1e-4 if n_ < (1 << 12) else 1e-9), (n_, t_, v[3])


def test_fp32_inner_solves_reach_fp64_solution():
    api, lib = _api()
    N = 1 << 12
    m64, z64, i64 = _mt_solve(api, lib, N, torch.float64)
    m32, z32, i32 = _mt_solve(api, lib, N, torch.float32)
    assert i64["converged"] and i32["converged"], (i64, i32)
    assert abs(z32[m32.s_index].item() - z64[m64.s_index].item()) < 1e-9


def test_invalid_time_scale_and_seed_mismatch():
    api, lib = _api()
    from paper_2509_01855_gb300._lib import BirkhoffError
    mt = api.Problem(lib.BK_ORBIT_MT, 64, torch.float64, 0.0, T_SEED, (A_THRUST, R_F))
    z = mt.zeros()
    z[mt.s_index] = -1.0
    with pytest.raises(BirkhoffError):
        api.newton_solve(mt, z)
    F = torch.zeros_like(z)
    with pytest.raises(BirkhoffError):
        mt.residual(z, F)
    me = api.Problem(lib.BK_ORBIT, 128, torch.float64, 0.0, T_SEED, (A_THRUST, R_F))
    with pytest.raises(BirkhoffError):
        api.min_time_seed(mt, me, me.zeros(), mt.zeros())
    with pytest.raises(BirkhoffError):
        api.Problem(lib.BK_ORBIT_MT, 64, torch.float64, 0.0, T_SEED, (0.0, R_F))


def test_weighted_inner_solves():
    """Inner GMRES in the merit norm (weighted_inner): the forcing term's loose steps then descend
    ||F||_W. The minimum-energy transfer to r_f = 6 converges with it (the 2-norm forcing term
    does not, in 30 steps), and the minimum-time solve reaches the tight solve's final time."""
    api, lib = _api()
    N = 1 << 12
    me = api.Problem(lib.BK_ORBIT, N, torch.float64, 0.0, T_SEED, (A_THRUST, R_F))
    t, _ = api.Plan(N, t0=0.0, tf=T_SEED).grid()
    X, U = synth.orbit_guess(t.numpy(), R_F, T_SEED)
    zme = me.pack(X, U)
    info = api.newton_solve(me, zme, tol=1e-11, weighted_inner=True, max_iter=40)
    assert info["converged"] and info["iterations"] <= 15, info
    mt = api.Problem(lib.BK_ORBIT_MT, N, torch.float64, 0.0, T_SEED, (A_THRUST, R_F))
    z = mt.zeros(dtype=torch.float64)
    api.min_time_seed(mt, me, zme, z)
    z_ref = z.clone()
    ref = api.newton_solve(mt, z_ref, tol=1e-10, max_iter=40)
    got = api.newton_solve(mt, z, tol=1e-10, max_iter=40, weighted_inner=True)
    assert ref["converged"] and got["converged"], (ref, got)
    assert abs(z[mt.s_index].item() - z_ref[mt.s_index].item()) < 1e-9
