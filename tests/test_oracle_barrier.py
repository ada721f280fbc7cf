"""Pins of the control-bound oracle (oracle/barrier.py) against the mathematics it restates.

- Its KKT matrix is the Jacobian of its residual (central finite differences), barrier terms
  included, for the double integrator and the orbit problem.
- With bounds far from the solution the barrier solve reproduces the unbounded optimum
  (double integrator: x = 3t^2 - 2t^3) to the barrier's O(mu) perturbation.
- With |u| <= 5 on the double integrator (the unbounded optimum 6 - 12 t reaches 6; 4 would be
  the feasibility limit, reached only by bang-bang control) the solution is the one
  Pontryagin's principle gives, computed independently here: u = clip(alpha (1 - 2t), -5, 5)
  (the costate is linear in t and the problem is antisymmetric about t = 1/2), with alpha fixed by x(1) = 1 through adaptive
  quadrature and a bracketing root finder.
- The iterates stay strictly inside the bounds and the recovered bound multipliers are
  nonnegative and vanish where the bound is inactive.
- Primal-dual form: its Newton matrix is the Jacobian of its residual (finite differences), the
  step by eliminating the multipliers (the form the library solves) equals the full solve, its
  residual on the central path is the primal one, and its solve reaches the primal solve's
  solution and multipliers in fewer Newton steps.
- Endpoint bounds: both forms' Newton matrices are their residuals' Jacobians with a bounded
  terminal row, and the double integrator with x(1) in [l, h] (v(1) = 0) reaches the closed form
  x = p (3t^2 - 2t^3) with p the admissible value nearest 0 (energy 6 p^2): 0.8 for [0.8, 1.2]
  and [0.8, inf), 0 for [-1, 2].
"""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq

from oracle import problems as op
from oracle.barrier import BarrierKKT
from oracle.kkt import DenseKKT
from paper_2509_01855_gb300 import synth


def _fd_jacobian(K, vec, h=1e-6):
    n = len(vec)
    J = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        J[:, j] = (K.residual(vec + e) - K.residual(vec - e)) / (2 * h)
    return J


@pytest.mark.parametrize("kind", [op.DBL_INT, op.ORBIT])
def test_barrier_matrix_is_residual_jacobian(kind):
    if kind == op.DBL_INT:
        prob = op.Problem(op.DBL_INT, 0.0, 1.0)
        lo, hi = [-4.0], [5.0]
    else:
        prob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
        lo, hi = [-0.05, -np.inf], [0.05, 0.04]
    N = 12
    K = BarrierKKT(prob, N, lo, hi)
    K.mu = 0.3
    g = synth.rng("barrier-fd", kind)
    if kind == op.DBL_INT:
        X, U = synth.double_integrator_guess(K.t)
        U = U + 0.5 * g.standard_normal(U.shape)
    else:
        X, U = synth.orbit_guess(K.t, 1.5, 20.0)
        U = 0.01 * g.standard_normal(U.shape)
    X = X + 0.01 * g.standard_normal(X.shape)
    vec = K.pack(X, U, 0.1 * g.standard_normal((prob.n_x, K.L)), 0.1 * g.standard_normal(prob.n_e))
    vec = K.interior(vec, margin=0.05)
    A = K.matrix(vec)
    J = _fd_jacobian(K, vec)
    assert np.max(np.abs(A - J)) < 1e-5 * max(1.0, np.max(np.abs(A)))
    # the barrier contributes: without it the matrices differ
    K.mu = 0.0
    assert np.max(np.abs(K.matrix(vec) - A)) > 1e-3


def test_inactive_bounds_give_the_unbounded_solution():
    prob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = BarrierKKT(prob, 32, [-100.0], [100.0])
    X, U = synth.double_integrator_guess(K.t)
    vec, info = K.solve(K.pack(X, U, np.zeros((2, K.L)), np.zeros(2)), mu_final=1e-10)
    assert info["converged"], info
    Xs = K.split(vec)[0]
    t = K.t
    assert np.max(np.abs(Xs[0] - (3 * t**2 - 2 * t**3))) < 1e-8
    assert np.max(np.abs(K.split(vec)[1][0] - (6 - 12 * t))) < 1e-6


def _pontryagin_bounded(umax=5.0):
    """u(t) = clip(alpha (1 - 2t), -umax, umax) with x(1) = int_0^1 (1 - t) u dt = 1."""
    def u_of(alpha):
        return lambda t: float(np.clip(alpha * (1 - 2 * t), -umax, umax))

    def x1(alpha):
        t1, t2 = 0.5 * (1 - umax / alpha), 0.5 * (1 + umax / alpha)
        return quad(lambda t: (1 - t) * u_of(alpha)(t), 0.0, 1.0, points=[t1, t2], epsabs=1e-14)[0] - 1.0
    alpha = brentq(x1, umax + 1e-9, 1e3, xtol=1e-14)
    u = u_of(alpha)

    def x(t):
        return quad(lambda tau: (t - tau) * u(tau), 0.0, t, epsabs=1e-14, limit=200)[0]
    return alpha, u, x


def test_active_bounds_match_pontryagin():
    alpha, u, x = _pontryagin_bounded(5.0)
    assert alpha > 6.0   # steeper than the unbounded optimum 6 - 12 t, clipped at +-5
    prob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = BarrierKKT(prob, 64, [-5.0], [5.0])
    X, U = synth.double_integrator_guess(K.t)
    vec, info = K.solve(K.pack(X, U, np.zeros((2, K.L)), np.zeros(2)))
    assert info["converged"], info
    Xs, Us = K.split(vec)[:2]
    t = K.t
    ue = np.array([u(tt) for tt in t])
    xe = np.array([x(tt) for tt in t])
    assert np.all(Us[0] > -5.0) and np.all(Us[0] < 5.0)
    assert np.max(np.abs(Us[0] - ue)) < 2e-2       # the kinks limit the discrete accuracy
    assert np.max(np.abs(Xs[0] - xe)) < 2e-4
    # multipliers: nonnegative, and only where the bound is (nearly) active
    zl, zh = K.bound_multipliers(vec)
    assert np.all(zl >= 0) and np.all(zh >= 0)
    inner = np.abs(ue) < 4.0
    assert np.max(np.abs(zl[0][inner]) + np.abs(zh[0][inner])) < 1e-4 * np.max(zl[0] + zh[0])   # O(mu)


def test_max_step_keeps_controls_inside():
    prob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = BarrierKKT(prob, 8, [-1.0], [1.0])
    X, U = synth.double_integrator_guess(K.t)
    vec = K.pack(X, U, np.zeros((2, K.L)), np.zeros(2))
    d = np.zeros_like(vec)
    d[2 * K.L:3 * K.L] = np.linspace(-3.0, 3.0, K.L)
    a = K.max_step(vec, d)
    Un = (vec + a * d)[2 * K.L:3 * K.L]
    assert 0 < a < 1 and np.all(np.abs(Un) < 1.0)
    assert abs(np.max(np.abs(Un)) - 0.995) < 1e-12


# ---- primal-dual form --------------------------------------------------------------------------
def _pd_point(kind, N=10):
    if kind == op.DBL_INT:
        prob = op.Problem(op.DBL_INT, 0.0, 1.0)
        lo, hi = [-4.0], [5.0]
    else:
        prob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
        lo, hi = [-0.05, -np.inf], [0.05, 0.04]
    K = BarrierKKT(prob, N, lo, hi)
    K.mu = 0.3
    g = synth.rng("barrier-pd", kind)
    if kind == op.DBL_INT:
        X, U = synth.double_integrator_guess(K.t)
        U = U + 0.5 * g.standard_normal(U.shape)
    else:
        X, U = synth.orbit_guess(K.t, 1.5, 20.0)
        U = 0.01 * g.standard_normal(U.shape)
    X = X + 0.01 * g.standard_normal(X.shape)
    vec = K.pack(X, U, 0.1 * g.standard_normal((prob.n_x, K.L)), 0.1 * g.standard_normal(prob.n_e))
    vec = K.interior(vec, margin=0.05)
    zl, zh = K.pd_init(vec)
    # off the central path
    zl = zl * np.exp(0.3 * g.standard_normal(zl.shape)) * np.isfinite(K.lo)[:, None]
    zh = zh * np.exp(0.3 * g.standard_normal(zh.shape)) * np.isfinite(K.hi)[:, None]
    return K, vec, zl, zh


@pytest.mark.parametrize("kind", [op.DBL_INT, op.ORBIT])
def test_pd_matrix_is_residual_jacobian(kind):
    K, vec, zl, zh = _pd_point(kind)
    p, L, n = K.prob, K.L, K.n
    m = p.n_u * L

    def full(x):
        F, Cl, Ch = K.pd_residual(x[:n], x[n:n + m].reshape(p.n_u, L), x[n + m:].reshape(p.n_u, L))
        return np.concatenate([F, Cl.ravel(), Ch.ravel()])
    x0 = np.concatenate([vec, zl.ravel(), zh.ravel()])
    h = 1e-6
    J = np.zeros((n + 2 * m, n + 2 * m))
    for j in range(n + 2 * m):
        e = np.zeros(n + 2 * m)
        e[j] = h
        J[:, j] = (full(x0 + e) - full(x0 - e)) / (2 * h)
    A = K.pd_matrix(vec, zl, zh)
    # rows and columns of absent bounds hold the identity in pd_matrix (the residual ignores them)
    live = np.ones(n + 2 * m, bool)
    for q in range(p.n_u):
        if not np.isfinite(K.lo[q]):
            live[n + q * L:n + (q + 1) * L] = False
        if not np.isfinite(K.hi[q]):
            live[n + m + q * L:n + m + (q + 1) * L] = False
    Al, Jl = A[np.ix_(live, live)], J[np.ix_(live, live)]
    assert np.max(np.abs(Al - Jl)) < 1e-5 * max(1.0, np.max(np.abs(Al)))
    assert np.all(A[~live][:, live] == 0) and np.all(A[live][:, ~live] == 0)


@pytest.mark.parametrize("kind", [op.DBL_INT, op.ORBIT])
def test_pd_step_by_elimination(kind):
    """The reduced form of the primal-dual step: eliminating dz_l, dz_h leaves the unbarriered KKT
    matrix with Sigma = z_l / (u - l) + z_h / (h - u) added to its control diagonal and the control
    rows of the right-hand side corrected by -C_l / (u - l) + C_h / (h - u); then
    dz_l = (-C_l - z_l du) / (u - l), dz_h = (-C_h + z_h du) / (h - u). It equals the full solve."""
    K, vec, zl, zh = _pd_point(kind)
    p, L = K.prob, K.L
    d, dzl, dzh = K.pd_step(vec, zl, zh)
    F, Cl, Ch = K.pd_residual(vec, zl, zh)
    U = K.split(vec)[1]
    ml, mh = np.isfinite(K.lo), np.isfinite(K.hi)
    dl = np.where(ml[:, None], U - np.where(ml, K.lo, 0.0)[:, None], 1.0)
    dh = np.where(mh[:, None], np.where(mh, K.hi, 0.0)[:, None] - U, 1.0)
    sig = np.where(ml[:, None], zl / dl, 0.0) + np.where(mh[:, None], zh / dh, 0.0)
    A = DenseKKT.matrix(K, vec)
    i0 = p.n_x * L
    A[i0:K.nz, i0:K.nz] += np.diag(sig.ravel())
    rhs = -F
    rhs[i0:K.nz] += (np.where(ml[:, None], -Cl / dl, 0.0) + np.where(mh[:, None], Ch / dh, 0.0)).ravel()
    dr = np.linalg.solve(A, rhs)
    dU = dr[i0:K.nz].reshape(p.n_u, L)
    assert np.max(np.abs(dr - d)) < 1e-9 * np.max(np.abs(d))
    assert np.max(np.abs(np.where(ml[:, None], (-Cl - zl * dU) / dl, 0.0) - dzl)) < 1e-9 * max(1.0, np.abs(dzl).max())
    assert np.max(np.abs(np.where(mh[:, None], (-Ch + zh * dU) / dh, 0.0) - dzh)) < 1e-9 * max(1.0, np.abs(dzh).max())


def test_pd_and_primal_forms_share_the_solution():
    """At a point on the central path (z = mu s w / distance) the primal-dual residual is the
    primal residual; solve_pd and solve reach the same barrier solution, solve_pd in fewer steps,
    and solve_pd's multipliers are the ones recovered from the primal solution."""
    K, vec, _, _ = _pd_point(op.DBL_INT, N=16)
    zl, zh = K.pd_init(vec)
    F, Cl, Ch = K.pd_residual(vec, zl, zh)
    assert np.max(np.abs(Cl)) < 1e-15 and np.max(np.abs(Ch)) < 1e-15
    assert np.max(np.abs(F - K.residual(vec))) < 1e-12 * np.max(np.abs(F))
    prob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = BarrierKKT(prob, 64, [-5.0], [5.0])
    X, U = synth.double_integrator_guess(K.t)
    v0 = K.pack(X, U, np.zeros((2, K.L)), np.zeros(2))
    vp, ip = K.solve(v0)
    vd, zl, zh, idd = K.solve_pd(v0)
    assert ip["converged"] and idd["converged"], (ip, idd)
    assert np.max(np.abs(vd - vp)) < 1e-8
    assert idd["iters"] < ip["iters"]
    zl_p, zh_p = K.bound_multipliers(vp)
    assert np.max(np.abs(zl - zl_p)) < 1e-6 * np.max(zl_p) and np.max(np.abs(zh - zh_p)) < 1e-6 * np.max(zh_p)
    assert np.all(zl > 0) and np.all(zh > 0)


# ---- endpoint bounds -------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [op.DBL_INT, op.ORBIT])
def test_endpoint_bound_matrices_are_residual_jacobians(kind):
    """Both forms, with a bounded terminal row beside control bounds (the barrier's terms in the
    terminal block included)."""
    K, vec, zl, zh = _pd_point(kind)
    if kind == op.DBL_INT:
        K.ebounds = {0: (0.7, 1.3)}
    else:
        K.ebounds = {0: (1.2, np.inf)}
    vec = K.interior(vec, margin=0.05)
    A = K.matrix(vec)
    J = _fd_jacobian(K, vec)
    assert np.max(np.abs(A - J)) < 1e-5 * max(1.0, np.max(np.abs(A)))
    p, L, n = K.prob, K.L, K.n
    m = p.n_u * L

    def full(x):
        F, Cl, Ch = K.pd_residual(x[:n], x[n:n + m].reshape(p.n_u, L), x[n + m:].reshape(p.n_u, L))
        return np.concatenate([F, Cl.ravel(), Ch.ravel()])
    x0 = np.concatenate([vec, zl.ravel(), zh.ravel()])
    h = 1e-6
    Apd = K.pd_matrix(vec, zl, zh)
    live = np.ones(n + 2 * m, bool)
    for q in range(p.n_u):
        if not np.isfinite(K.lo[q]):
            live[n + q * L:n + (q + 1) * L] = False
        if not np.isfinite(K.hi[q]):
            live[n + m + q * L:n + m + (q + 1) * L] = False
    cols = np.nonzero(live)[0]
    Jpd = np.zeros((n + 2 * m, len(cols)))
    for jj, j in enumerate(cols):
        e = np.zeros(n + 2 * m)
        e[j] = h
        Jpd[:, jj] = (full(x0 + e) - full(x0 - e)) / (2 * h)
    Al = Apd[np.ix_(live, cols)]
    assert np.max(np.abs(Al - Jpd[live])) < 1e-5 * max(1.0, np.max(np.abs(Al)))


@pytest.mark.parametrize("form", ["primal", "primal_dual"])
@pytest.mark.parametrize("bounds,p_star", [((0.8, 1.2), 0.8), ((0.8, np.inf), 0.8), ((-1.0, 2.0), 0.0)])
def test_endpoint_bounds_double_integrator_closed_form(bounds, p_star, form):
    """x(1) in [l, h] and v(1) = 0 with cost int u^2 / 2: the energy of the cubic x = p (3t^2 - 2t^3)
    is 6 p^2, so the optimum takes the admissible p nearest 0: p = 0.8 (bound active) or p = 0 for
    [-1, 2] (inactive: the barrier moves it by about mu / 24)."""
    prob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = BarrierKKT(prob, 32, [-np.inf], [np.inf], ebounds={0: bounds})
    X, U = synth.double_integrator_guess(K.t)
    v0 = K.pack(X, U, np.zeros((2, K.L)), np.zeros(2))
    if form == "primal":
        vec, info = K.solve(v0)
    else:
        vec, _, _, info = K.solve_pd(v0)
    assert info["converged"], info
    Xs, Us = K.split(vec)[:2]
    t = K.t
    assert abs(Xs[0, -1] - p_star) < 1e-6
    assert np.max(np.abs(Xs[0] - p_star * (3 * t**2 - 2 * t**3))) < 1e-6
    assert np.max(np.abs(Us[0] - p_star * (6 - 12 * t))) < 1e-5
    assert bounds[0] < Xs[0, -1] < bounds[1]
