"""Pins of the oracle's free-final-time orbit transfer (Eq. ot): dynamics derivatives, the
bordered KKT matrix and residual, the bordered preconditioner, and the discrete optimum against
Pontryagin's principle solved independently by shooting (scipy ODE integration + root finding).
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import fsolve

from oracle import problems as op
from oracle.kkt import DenseKKT

A_THRUST, R_F, T_SEED = 0.05, 6.0, 24.0


def _spiral(t, rf, T):
    """Tangential-thrust spiral ending at r_f at time T (the orbit seed's input recipe)."""
    ae = (1.0 - rf ** -0.5) / T
    v = 1.0 - ae * t
    X = np.stack([1 / v**2, (1 - v**4) / (4 * ae), 2 * ae / v**3, v])
    U = np.zeros((2, t.size)); U[1] = ae
    return X, U


def _solve(N, a=A_THRUST, rf=R_F, Tme=T_SEED):
    """Minimum-energy transfer at t_f = Tme, then the free-final-time solve seeded from it."""
    pme = op.Problem(op.ORBIT, 0.0, Tme, (a, rf))
    Kme = DenseKKT(pme, N)
    X, U = _spiral(Kme.t, rf, Tme)
    vme, ime = Kme.newton(Kme.pack(X, U, np.zeros((4, Kme.L)), np.zeros(3)))
    assert ime["converged"]
    K = DenseKKT(op.Problem(op.ORBIT_MT, 0.0, Tme, (a, rf)), N, Ba=Kme.Ba)
    seed = K.min_time_seed(Kme, vme)
    vec, info = K.newton(seed, max_iter=40)
    _solve.last_me = (Kme, vme)
    return K, seed, vec, info


def _random_point(K, rng):
    p = K.prob
    X = rng.uniform(0.9, 1.4, (p.n_x, K.L))
    U = rng.uniform(-1.0, 1.0, (p.n_u, K.L))
    return K.pack(X, U, rng.standard_normal((p.n_x, K.L)), rng.standard_normal(p.n_e), 1.7)


def test_min_time_dynamics_derivatives():
    """d f / d(x, u) and the Hessian of mu . f, including the angle's -a sin u, -a cos u,
    against central differences of f."""
    rng = np.random.default_rng(3)
    p = op.Problem(op.ORBIT_MT, 0.0, 1.0, (A_THRUST, R_F))
    L = 7
    X = rng.uniform(0.8, 1.3, (4, L))
    U = rng.uniform(-3.0, 3.0, (1, L))
    mu = rng.standard_normal((4, L))
    Jx, Ju = p.jac(X, U)
    H = p.hess_f(X, U, mu)
    h = 1e-6
    for j in range(5):
        dX = np.zeros_like(X); dU = np.zeros_like(U)
        if j < 4:
            dX[j] = h
        else:
            dU[0] = h
        fd = (p.f(X + dX, U + dU) - p.f(X - dX, U - dU)) / (2 * h)
        J = Jx[:, :, j] if j < 4 else Ju[:, :, 0]
        assert np.abs(fd.T - J).max() < 1e-8

        def g(Xa, Ua):
            jx, ju = p.jac(Xa, Ua)
            return np.einsum('mk,kmi->ki', mu, np.concatenate([jx, ju], axis=2))
        fdH = (g(X + dX, U + dU) - g(X - dX, U - dU)) / (2 * h)
        assert np.abs(fdH - H[:, :, j]).max() < 1e-7
    # the thrust has magnitude a whatever the angle
    f0 = p.f(X, U) - p.f(X, U + 1.0)
    assert np.abs(f0[:2]).max() == 0.0


@pytest.mark.parametrize("N", [6, 9])
def test_bordered_kkt_is_jacobian_of_residual(N):
    """The KKT matrix with its s row and column is the finite-difference Jacobian of the
    residual, and it is symmetric."""
    K = DenseKKT(op.Problem(op.ORBIT_MT, 0.0, 3.0, (A_THRUST, R_F)), N)
    vec = _random_point(K, np.random.default_rng(N))
    Km = K.matrix(vec)
    h = 1e-6
    fd = np.zeros_like(Km)
    for j in range(K.n):
        e = np.zeros(K.n); e[j] = h
        fd[:, j] = (K.residual(vec + e) - K.residual(vec - e)) / (2 * h)
    assert np.abs(fd - Km).max() < 1e-7
    assert np.abs(Km - Km.T).max() < 1e-14
    assert Km[-1, -1] == 0.0


def test_residual_is_gradient_of_lagrangian():
    """The gradient rows (X, U and s) are the derivatives of the Lagrangian value
    2 s + lambda . c + nu . e (cost T = t_f - t_0 = 2 s), computed here from c and e alone."""
    K = DenseKKT(op.Problem(op.ORBIT_MT, 0.0, 3.0, (A_THRUST, R_F)), 7)
    vec = _random_point(K, np.random.default_rng(11))
    nr = K.nc + K.prob.n_e + 1

    def lagrangian(v):
        F = K.residual(v)
        X, U, lam, nu = K.split(v)
        c = F[K.nz:K.nz + K.nc]
        e = F[K.nz + K.nc:K.nz + K.nc + K.prob.n_e]
        return 2.0 * v[-1] + lam.ravel() @ c + nu @ e

    F = K.residual(vec)
    h = 1e-6
    for j in list(range(K.nz)) + [K.n - 1]:
        e = np.zeros(K.n); e[j] = h
        g = (lagrangian(vec + e) - lagrangian(vec - e)) / (2 * h)
        assert abs(g - F[j]) < 1e-7 * max(1.0, abs(g)), j
    assert nr == K.n - K.nz


def test_seed_zeroes_time_gradient_and_keeps_thrust_direction():
    K, seed, _, _ = _solve(16)
    Kme, vme = _solve.last_me
    F = K.residual(seed)
    assert abs(F[-1]) < 1e-12
    X, U, lam, nu = K.split(seed)
    Xm, Um, lam_m, nu_m = Kme.split(vme)
    assert np.array_equal(X, Xm) and seed[-1] == 0.5 * T_SEED
    umag = np.hypot(Um[0], Um[1])
    assert np.abs(np.sin(U[0]) - Um[0] / umag).max() < 1e-14
    assert np.abs(np.cos(U[0]) - Um[1] / umag).max() < 1e-14
    kappa = lam[0, 3] / lam_m[0, 3]
    assert kappa > 0 and np.allclose(lam, kappa * lam_m, rtol=1e-14) and np.allclose(nu, kappa * nu_m, rtol=1e-14)


def test_bordered_preconditioner_eliminates_time_scale():
    """The bordered K-tilde shares the KKT matrix's s row and column, and right-preconditioned
    GMRES on the Newton system converges in a handful of iterations at the seed and at the
    solution; without the border it stalls above the tolerance."""
    import scipy.sparse.linalg as sla
    K, seed, vec, info = _solve(64)
    assert info["converged"]
    for v in (seed, vec):
        A = K.matrix(v)
        M = K.precond_matrix(v)
        assert np.array_equal(M[:, -1], A[:, -1]) and np.array_equal(M[-1], A[-1])
        Mi = np.linalg.inv(M)
        b = -K.residual(v)
        AP = sla.LinearOperator(A.shape, matvec=lambda x: A @ (Mi @ x))
        its = [0]
        y, flag = sla.gmres(AP, b, rtol=1e-10, restart=30, maxiter=1,
                            callback=lambda _: its.__setitem__(0, its[0] + 1), callback_type='pr_norm')
        assert flag == 0 and its[0] <= 15
        assert np.linalg.norm(A @ (Mi @ y) - b) <= 1e-9 * np.linalg.norm(b)
        # the border matters: with the identity in the s slot instead, the true residual stalls
        # above 1e-10 (near 5e-10 at N = 64), short of the free-time solve's inner tolerance
        Mu = M.copy()
        Mu[:, -1] = 0.0
        Mu[-1, :] = 0.0
        Mu[-1, -1] = 1.0
        Mui = np.linalg.inv(Mu)
        APu = sla.LinearOperator(A.shape, matvec=lambda x: A @ (Mui @ x))
        yu, _ = sla.gmres(APu, b, rtol=1e-10, restart=30, maxiter=2)
        assert np.linalg.norm(A @ (Mui @ yu) - b) > 1e-10 * np.linalg.norm(b)


# ---- Pontryagin's principle, solved by shooting (independent of the Birkhoff discretisation) --
def _pmp_rhs(t, y, a):
    """State and costate of H = 1 + p . f with the thrust along -p_v (minimum time)."""
    r, th, vr, vt, pr, pth, pvr, pvt = y
    u = np.arctan2(-pvr, -pvt)
    f = [vr, vt / r, vt * vt / r - 1 / r**2 + a * np.sin(u), -vr * vt / r + a * np.cos(u)]
    dpr = -(pth * (-vt / r**2) + pvr * (-vt * vt / r**2 + 2 / r**3) + pvt * (vr * vt / r**2))
    dpvr = -(pr - pvt * vt / r)
    dpvt = -(pth / r + 2 * pvr * vt / r - pvt * vr / r)
    return f + [dpr, 0.0, dpvr, dpvt]


def _shoot(p0_guess, T_guess, a, rf):
    """Roots of r(T) - r_f, v_r(T), v_theta(T) - r_f^-1/2, H(T) over (p_r, p_vr, p_vt)(0), T;
    p_theta = 0 (theta is free at T and absent from f)."""
    def res(z):
        y0 = [1.0, 0.0, 0.0, 1.0, z[0], 0.0, z[1], z[2]]
        y = solve_ivp(_pmp_rhs, (0.0, z[3]), y0, args=(a,), rtol=1e-12, atol=1e-13).y[:, -1]
        f = _pmp_rhs(0.0, y, a)[:4]
        return [y[0] - rf, y[2], y[3] - rf ** -0.5, 1.0 + np.dot(y[4:], f)]
    z, _, ier, _ = fsolve(res, list(p0_guess) + [T_guess], full_output=True, xtol=1e-13)
    assert ier == 1 and np.abs(res(z)).max() < 1e-10
    return z


@pytest.mark.slow
def test_discrete_optimum_matches_pontryagin():
    """The discrete optimum converges to the Pontryagin extremal: its final time approaches the
    shooting solution's as N grows (error below 5e-3 at N = 64, smaller at N = 128), the
    covector estimate p_k = -(B^aT lambda)_k / w_k gives a Hamiltonian 1 + p . f near 0 at the
    interior nodes and p_theta = 0, and the shooting started from the discrete costate at t = 0
    lands on the same extremal from both grids."""
    T = {}
    for N in (64, 128):
        K, _, vec, info = _solve(N)
        assert info["converged"] and info["iters"] <= 20
        X, U, lam, nu = K.split(vec)
        p = -(K.Ba.T @ lam.T).T / K.w[None, :]
        H = 1.0 + (p * K.prob.f(X, U)).sum(0)
        assert np.abs(H[1:-1]).max() < 0.05
        assert np.abs(p[1]).max() < 1e-12
        z = _shoot((p[0, 0], p[2, 0], p[3, 0]), 2 * vec[-1], A_THRUST, R_F)
        T[N] = (2 * vec[-1], z[3])
    Tstar = T[64][1]
    assert abs(T[128][1] - Tstar) < 1e-9
    assert abs(T[64][0] - Tstar) < 5e-3
    assert abs(T[128][0] - Tstar) < abs(T[64][0] - Tstar)
