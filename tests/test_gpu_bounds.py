"""GPU parity of control bounds (logarithmic barrier on the quadrature) against the oracle.

- At a fixed barrier parameter the residual, the KKT operator and the preconditioner of a
  bounded problem match oracle/barrier.py (BarrierKKT) at an interior point.
- The bounded Newton solve (barrier stages, fraction-to-boundary steps), in the primal and in the
  primal-dual form, reaches the oracle's barrier solution of the same form, for the double
  integrator (|u| <= 5) and for the orbit transfer with its thrust components bounded below
  their unbounded peaks.
- On the double integrator the solution is the one Pontryagin's principle gives (computed in
  tests/test_oracle_barrier.py, independently of both solvers), bounds far away give the
  unbounded closed form, and FP32 inner solves reach the FP64 solution.
- Endpoint bounds on terminal rows (one bound per row), beside control bounds or alone: the
  operators against the oracle at a fixed barrier parameter, the double integrator against its
  closed form (x(1) >= 0.8: p = 0.8; x(1) <= 1.2: p = 0) at N = 64 and 2^14, and the orbit
  transfer against the oracle's solve of the same form.
- Argument checks of bk_problem_set_control_bounds, bk_problem_set_terminal_bounds and
  bk_problem_set_barrier.
"""
import numpy as np
import pytest
import torch

from oracle import problems as op
from oracle.barrier import BarrierKKT
from oracle.kkt import DenseKKT
from paper_2509_01855_gb300 import synth
from tests.helpers import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu


def _api():
    from paper_2509_01855_gb300 import _lib, api
    return api, _lib


def _orbit_bounds(N=64, fr=0.9, ft=0.95):
    """Bounds below the unbounded optimum's peaks: |u_r| <= fr max|u_r|, u_theta <= ft max u_theta
    (the unbounded solution from the oracle's Newton solve)."""
    rf, tf = 1.5, 20.0
    oprob = op.Problem(op.ORBIT, 0.0, tf, (0.01, rf))
    K = DenseKKT(oprob, N)
    X, U = synth.orbit_guess(K.t, rf, tf)
    vec0 = K.pack(X, U, np.zeros((4, K.L)), np.zeros(3))
    ref, info = K.newton(vec0)
    assert info["converged"]
    Ur = K.split(ref)[1]
    a = fr * np.abs(Ur[0]).max()
    return oprob, vec0, [-a, -np.inf], [a, ft * Ur[1].max()]


def _problem(api, lib, kind, N, dtype, oprob):
    code = {op.DBL_INT: lib.BK_DBL_INT, op.ORBIT: lib.BK_ORBIT}[kind]
    return api.Problem(code, N, dtype, oprob.t0, oprob.tf, tuple(oprob.params) if kind == op.ORBIT else ())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind,N", [(op.DBL_INT, 32), (op.DBL_INT, 100), (op.ORBIT, 64), (op.ORBIT, 45)])
def test_barrier_operators_match_oracle(kind, N, dtype):
    api, lib = _api()
    g = synth.rng("bounds-ops", kind, N)
    if kind == op.DBL_INT:
        oprob = op.Problem(op.DBL_INT, 0.0, 1.0)
        lo, hi, mu = [-4.0], [5.0], 0.3
        K = BarrierKKT(oprob, N, lo, hi)
        X, U = synth.double_integrator_guess(K.t)
        U = U + g.standard_normal(U.shape)
        X = X + 0.1 * g.standard_normal(X.shape)
    else:
        oprob, _, lo, hi = _orbit_bounds()
        mu = 1e-6
        K = BarrierKKT(oprob, N, lo, hi)
        X, U = synth.orbit_guess(K.t, 1.5, 20.0)
        U = U + 1e-3 * g.standard_normal(U.shape)
        X = X + 0.01 * g.standard_normal(X.shape)
    K.mu = mu
    vec = K.pack(X, U, 0.01 * g.standard_normal((oprob.n_x, K.L)), 0.01 * g.standard_normal(oprob.n_e))
    vec = K.interior(vec, margin=0.05)
    prob = _problem(api, lib, kind, N, dtype, oprob)
    prob.set_control_bounds(lo, hi)
    prob.set_barrier(mu, mu)
    z = from_packed(prob, vec)
    # residual and its weighted norm (FP64 in both precisions)
    F = torch.zeros_like(z)
    wn = prob.residual(z, F)
    Fo = K.residual(vec)
    assert rel(to_packed(prob, F), Fo) < 1e-12
    assert abs(wn - K.weighted_norm(Fo)) < 1e-12 * K.weighted_norm(Fo)
    # the barrier is there: the unbounded residual differs in the control rows
    assert rel(DenseKKT.residual(K, vec), Fo) > 1e-6
    prob.linearize(z)
    d = g.standard_normal(K.n)
    x = from_packed(prob, d, dtype)
    out = torch.zeros_like(x)
    api.kkt_apply(prob, lib.BK_OP_KKT, x, out)
    assert rel(to_packed(prob, out), K.matrix(vec) @ d) < (1e-12 if dtype == torch.float64 else 1e-5)
    api.precond_apply(prob, lib.BK_OP_KKT, x, out)
    ref = np.linalg.solve(K.precond_matrix(vec), d)
    assert rel(to_packed(prob, out), ref) < (1e-10 if dtype == torch.float64 else 1e-3)
    # clearing the bounds restores the unbounded residual
    prob.set_control_bounds(None, None)
    prob.residual(z, F)
    assert rel(to_packed(prob, F), DenseKKT.residual(K, vec)) < 1e-12


FORMS = ["primal", "primal_dual"]


def _oracle_solve(K, vec0, form, **kw):
    if form == "primal":
        return K.solve(vec0, **kw)
    vec, _, _, info = K.solve_pd(vec0, **kw)
    return vec, info


def _solve_gpu(api, lib, kind, N, dtype, oprob, vec0, lo, hi, mu0, mu_final, tol=1e-10, form="primal"):
    prob = _problem(api, lib, kind, N, dtype, oprob)
    prob.set_control_bounds(lo, hi)
    prob.set_barrier(mu0, mu_final, form)
    z = from_packed(prob, vec0)
    info = api.newton_solve(prob, z, tol=tol)
    assert info["converged"], info
    return prob, z, info


@pytest.mark.parametrize("form", FORMS)
def test_bounded_double_integrator_matches_oracle(form):
    api, lib = _api()
    N = 64
    oprob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = BarrierKKT(oprob, N, [-5.0], [5.0])
    X, U = synth.double_integrator_guess(K.t)
    vec0 = K.pack(X, U, np.zeros((2, K.L)), np.zeros(2))
    ref, rinfo = _oracle_solve(K, vec0, form)
    assert rinfo["converged"]
    prob, z, info = _solve_gpu(api, lib, op.DBL_INT, N, torch.float64, oprob, vec0, [-5.0], [5.0], 0.1, 1e-6,
                               form=form)
    got = to_packed(prob, z)
    Xr, Ur = K.split(ref)[:2]
    Xg, Ug = K.split(got)[:2]
    assert np.all(np.abs(Ug) < 5.0)
    assert np.abs(Xg - Xr).max() < 1e-8, np.abs(Xg - Xr).max()
    assert np.abs(Ug - Ur).max() < 1e-6, np.abs(Ug - Ur).max()
    # inexact inner solves keep the oracle's Newton count within a few steps
    assert info["iterations"] <= rinfo["iters"] + 4, (info, rinfo)
    # the library's residual at the solution is the final stage's primal one (mu_final)
    F = torch.zeros_like(z)
    assert prob.residual(z, F) <= 1e-7


@pytest.mark.parametrize("form", FORMS)
def test_bounded_orbit_matches_oracle(form):
    api, lib = _api()
    N = 64
    oprob, vec0, lo, hi = _orbit_bounds(N)
    K = BarrierKKT(oprob, N, lo, hi)
    ref, rinfo = _oracle_solve(K, vec0, form, mu0=1e-4, mu_final=1e-9)
    assert rinfo["converged"], rinfo
    prob, z, info = _solve_gpu(api, lib, op.ORBIT, N, torch.float64, oprob, vec0, lo, hi, 1e-4, 1e-9, form=form)
    got = to_packed(prob, z)
    Xr, Ur = K.split(ref)[:2]
    Xg, Ug = K.split(got)[:2]
    assert np.all(np.abs(Ug[0]) < hi[0]) and np.all(Ug[1] < hi[1])
    # the bounds are active: the bounded optimum reaches them
    assert Ug[1].max() > hi[1] - 1e-5 and np.abs(Ug[0]).max() > hi[0] - 1e-5
    # at mu = 1e-9 the barrier problem is ill-conditioned near the active bounds: two solves that
    # both stop at merit 1e-10 differ by up to ~1e-6 in the state (the oracle's primal and
    # primal-dual solves, and a CPU model of this loop, do)
    assert np.abs(Xg - Xr).max() < 1e-5, np.abs(Xg - Xr).max()
    assert np.abs(Ug - Ur).max() < 1e-6, np.abs(Ug - Ur).max()
    assert info["iterations"] <= rinfo["iters"] + 6, (info, rinfo)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("N", [64, 256])
def test_bounded_double_integrator_pontryagin(N, form):
    from tests.test_oracle_barrier import _pontryagin_bounded
    api, lib = _api()
    alpha, u, x = _pontryagin_bounded(5.0)
    prob = api.Problem(lib.BK_DBL_INT, N, torch.float64, 0.0, 1.0)
    prob.set_control_bounds([-5.0], [5.0])
    prob.set_barrier(0.1, 1e-6, form)
    t = api.Plan(N, t0=0.0, tf=1.0).grid()[0].numpy()
    X, U = synth.double_integrator_guess(t)
    z = prob.pack(X, U)
    info = api.newton_solve(prob, z)
    assert info["converged"], info
    Xg, Ug = [a.cpu().numpy() for a in prob.split(z)[:2]]
    ue = np.array([u(tt) for tt in t])
    xe = np.array([x(tt) for tt in t])
    assert np.all(np.abs(Ug[0]) < 5.0)
    assert np.abs(Ug[0] - ue).max() < 2e-2
    assert np.abs(Xg[0] - xe).max() < 2e-4


@pytest.mark.parametrize("form", FORMS)
def test_inactive_bounds_give_the_unbounded_solution(form):
    api, lib = _api()
    N = 48
    prob = api.Problem(lib.BK_DBL_INT, N, torch.float64, 0.0, 1.0)
    prob.set_control_bounds([-100.0], [100.0])
    prob.set_barrier(0.1, 1e-6, form)
    t = api.Plan(N, t0=0.0, tf=1.0).grid()[0].numpy()
    X, U = synth.double_integrator_guess(t)
    z = prob.pack(X, U)
    info = api.newton_solve(prob, z)
    assert info["converged"], info
    Xg, Ug = [a.cpu().numpy() for a in prob.split(z)[:2]]
    assert np.abs(Xg[0] - (3 * t**2 - 2 * t**3)).max() < 1e-7
    assert np.abs(Ug[0] - (6 - 12 * t)).max() < 1e-5


@pytest.mark.parametrize("form", FORMS)
def test_bounded_fp32_reaches_the_fp64_solution(form):
    api, lib = _api()
    N = 64
    oprob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = DenseKKT(oprob, N)
    X, U = synth.double_integrator_guess(K.t)
    vec0 = K.pack(X, U, np.zeros((2, K.L)), np.zeros(2))
    p64, z64, _ = _solve_gpu(api, lib, op.DBL_INT, N, torch.float64, oprob, vec0, [-5.0], [5.0], 0.1, 1e-6, form=form)
    # FP32 inner solves (forcing floor 1e-4) converge linearly on the ill-conditioned last
    # stage: measured 1.6e-10 after 100 steps, so this solve stops at 1e-9
    p32, z32, i32 = _solve_gpu(api, lib, op.DBL_INT, N, torch.float32, oprob, vec0, [-5.0], [5.0], 0.1, 1e-6,
                               tol=1e-9, form=form)
    a, b = to_packed(p64, z64), to_packed(p32, z32)
    n = (oprob.n_x + oprob.n_u) * K.L
    assert np.abs(a[:n] - b[:n]).max() < 1e-5


def test_bounds_argument_checks():
    api, lib = _api()
    orbit = api.Problem(lib.BK_ORBIT, 16, torch.float64, 0.0, 20.0, (0.01, 1.5))
    with pytest.raises(ValueError):
        orbit.set_control_bounds([-1.0], [1.0])          # n_u = 2
    h = orbit.handle
    arr = lambda *v: (__import__("ctypes").c_double * len(v))(*v)
    assert lib.lib().bk_problem_set_control_bounds(h, arr(-1.0), arr(1.0), 1) == 1        # BK_ERR_ARG
    with pytest.raises(lib.BirkhoffError):
        orbit.set_control_bounds([1.0, 0.0], [1.0, 1.0])    # lo == hi
    with pytest.raises(lib.BirkhoffError):
        orbit.set_control_bounds([float("nan"), 0.0], [1.0, 1.0])
    with pytest.raises(lib.BirkhoffError):
        orbit.set_barrier(1e-3, 1e-2)                       # mu0 < mu_final
    with pytest.raises(lib.BirkhoffError):
        orbit.set_barrier(1e-3, 0.0)
    assert lib.lib().bk_problem_set_barrier(h, 1e-3, 1e-4, 2) == 1                          # unknown form
    orbit.set_control_bounds([-1.0, -np.inf], [1.0, 0.5])   # one-sided bounds are fine
    orbit.set_control_bounds(None, None)
    bil = api.Problem(lib.BK_BILINEAR, 16, torch.float64, 0.0, 2.0, (1.0,))
    with pytest.raises(lib.BirkhoffError) as e:
        bil.set_control_bounds([-1.0], [1.0])
    assert e.value.status == 7                              # BK_ERR_UNSUPPORTED


# ---- endpoint bounds ------------------------------------------------------------------------
def _ebounds_arrays(ne, eb):
    lo = [-np.inf] * ne
    hi = [np.inf] * ne
    for r, (a, b) in eb.items():
        lo[r], hi[r] = a, b
    return lo, hi


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind,N", [(op.DBL_INT, 32), (op.DBL_INT, 100), (op.ORBIT, 64), (op.ORBIT, 45)])
def test_endpoint_barrier_operators_match_oracle(kind, N, dtype):
    """Residual, KKT product and preconditioner with endpoint-bounded terminal rows beside
    control bounds, at a fixed barrier parameter."""
    api, lib = _api()
    g = synth.rng("bounds-end-ops", kind, N)
    if kind == op.DBL_INT:
        oprob = op.Problem(op.DBL_INT, 0.0, 1.0)
        lo, hi, mu, eb = [-4.0], [5.0], 0.3, {0: (0.7, np.inf)}
        K = BarrierKKT(oprob, N, lo, hi, ebounds=eb)
        X, U = synth.double_integrator_guess(K.t)
        U = U + g.standard_normal(U.shape)
        X = X + 0.1 * g.standard_normal(X.shape)
    else:
        oprob, _, lo, hi = _orbit_bounds()
        mu, eb = 1e-6, {0: (1.2, np.inf), 2: (-np.inf, 0.9)}
        K = BarrierKKT(oprob, N, lo, hi, ebounds=eb)
        X, U = synth.orbit_guess(K.t, 1.5, 20.0)
        U = U + 1e-3 * g.standard_normal(U.shape)
        X = X + 0.01 * g.standard_normal(X.shape)
    K.mu = mu
    vec = K.pack(X, U, 0.01 * g.standard_normal((oprob.n_x, K.L)), 0.01 * g.standard_normal(oprob.n_e))
    vec = K.interior(vec, margin=0.05)
    prob = _problem(api, lib, kind, N, dtype, oprob)
    prob.set_control_bounds(lo, hi)
    prob.set_terminal_bounds(*_ebounds_arrays(oprob.n_e, eb))
    prob.set_barrier(mu, mu)
    z = from_packed(prob, vec)
    F = torch.zeros_like(z)
    wn = prob.residual(z, F)
    Fo = K.residual(vec)
    assert rel(to_packed(prob, F), Fo) < 1e-12
    assert abs(wn - K.weighted_norm(Fo)) < 1e-12 * K.weighted_norm(Fo)
    prob.linearize(z)
    d = g.standard_normal(K.n)
    x = from_packed(prob, d, dtype)
    out = torch.zeros_like(x)
    api.kkt_apply(prob, lib.BK_OP_KKT, x, out)
    assert rel(to_packed(prob, out), K.matrix(vec) @ d) < (1e-12 if dtype == torch.float64 else 1e-5)
    api.precond_apply(prob, lib.BK_OP_KKT, x, out)
    ref = np.linalg.solve(K.precond_matrix(vec), d)
    assert rel(to_packed(prob, out), ref) < (1e-10 if dtype == torch.float64 else 1e-3)
    # removing the endpoint bounds restores the equality rows
    prob.set_terminal_bounds(None, None)
    prob.residual(z, F)
    K.ebounds = {}
    assert rel(to_packed(prob, F), K.residual(vec)) < 1e-12


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("eb,p_star", [({0: (0.8, np.inf)}, 0.8), ({0: (-np.inf, 1.2)}, 0.0)])
@pytest.mark.parametrize("N", [64, 1 << 14])
def test_endpoint_bounds_double_integrator_closed_form(N, eb, p_star, form):
    """x(1) >= 0.8 (active) or <= 1.2 (inactive), v(1) = 0: x = p (3t^2 - 2t^3) with p = 0.8 or 0
    (the energy 6 p^2 of the cubic takes the admissible p nearest 0)."""
    api, lib = _api()
    prob = api.Problem(lib.BK_DBL_INT, N, torch.float64, 0.0, 1.0)
    prob.set_terminal_bounds(*_ebounds_arrays(2, eb))
    prob.set_barrier(0.1, 1e-8, form)
    t = api.Plan(N, t0=0.0, tf=1.0).grid()[0].numpy()
    X, U = synth.double_integrator_guess(t)
    z = prob.pack(X, U)
    info = api.newton_solve(prob, z)
    assert info["converged"], info
    Xg, Ug = [a.cpu().numpy() for a in prob.split(z)[:2]]
    assert np.abs(Xg[0] - p_star * (3 * t**2 - 2 * t**3)).max() < 1e-6
    assert np.abs(Ug[0] - p_star * (6 - 12 * t)).max() < 1e-5
    a, b = eb[0]
    assert a < Xg[0, -1] < b


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", ["r_lower", "r_upper", "r_lower_thrust", "vt_upper_thrust"])
def test_endpoint_bounds_orbit_matches_oracle(case, form):
    api, lib = _api()
    N = 64
    oprob, vec0, lo, hi = _orbit_bounds(N)
    inf = np.inf
    eb, lo_, hi_ = {"r_lower": ({0: (1.55, inf)}, [-inf] * 2, [inf] * 2),
                    "r_upper": ({0: (-inf, 1.45)}, [-inf] * 2, [inf] * 2),
                    "r_lower_thrust": ({0: (1.45, inf)}, lo, hi),
                    "vt_upper_thrust": ({2: (-inf, 0.81)}, lo, hi)}[case]
    K = BarrierKKT(oprob, N, lo_, hi_, ebounds=eb)
    ref, rinfo = _oracle_solve(K, vec0, form, mu0=1e-4, mu_final=1e-9)
    assert rinfo["converged"], rinfo
    prob = _problem(api, lib, op.ORBIT, N, torch.float64, oprob)
    if np.isfinite(lo_[0]):
        prob.set_control_bounds(lo_, hi_)
    prob.set_terminal_bounds(*_ebounds_arrays(3, eb))
    prob.set_barrier(1e-4, 1e-9, form)
    z = from_packed(prob, vec0)
    info = api.newton_solve(prob, z)
    assert info["converged"], info
    got = to_packed(prob, z)
    Xr, Ur = K.split(ref)[:2]
    Xg, Ug = K.split(got)[:2]
    for r, (a, b) in eb.items():
        x = Xg[oprob.term_idx[r], -1]
        assert a < x < b
    assert np.abs(Xg - Xr).max() < 1e-5, np.abs(Xg - Xr).max()
    assert np.abs(Ug - Ur).max() < 1e-6, np.abs(Ug - Ur).max()


def test_terminal_bounds_argument_checks():
    api, lib = _api()
    orbit = api.Problem(lib.BK_ORBIT, 16, torch.float64, 0.0, 20.0, (0.01, 1.5))
    with pytest.raises(ValueError):
        orbit.set_terminal_bounds([1.0], [2.0])                       # n_e = 3
    with pytest.raises(lib.BirkhoffError) as e:
        orbit.set_terminal_bounds([1.2, -np.inf, -np.inf], [1.8, np.inf, np.inf])   # two-sided
    assert e.value.status == 7
    with pytest.raises(lib.BirkhoffError):
        orbit.set_terminal_bounds([np.nan, -np.inf, -np.inf], [np.inf] * 3)
    with pytest.raises(lib.BirkhoffError):
        orbit.set_terminal_bounds([np.inf, -np.inf, -np.inf], [np.inf] * 3)
    orbit.set_terminal_bounds([1.2, -np.inf, -np.inf], [np.inf] * 3)
    orbit.set_terminal_bounds(None, None)
    mt = api.Problem(lib.BK_ORBIT_MT, 16, torch.float64, 0.0, 20.0, (0.05, 6.0))
    with pytest.raises(lib.BirkhoffError) as e:
        mt.set_terminal_bounds([5.0, -np.inf, -np.inf], [np.inf] * 3)
    assert e.value.status == 7


@pytest.mark.parametrize("N", [64, 1 << 14])
def test_endpoint_bounds_fp32_inner(N):
    """FP32 Krylov inner solves with the FP64 Newton residual reach the closed form of
    x(1) >= 0.8 (p = 0.8) too (stopping at 1e-9, as the FP32 control-bound solve does)."""
    api, lib = _api()
    prob = api.Problem(lib.BK_DBL_INT, N, torch.float32, 0.0, 1.0)
    prob.set_terminal_bounds([0.8, -np.inf], [np.inf, np.inf])
    prob.set_barrier(0.1, 1e-8)
    t = api.Plan(N, t0=0.0, tf=1.0).grid()[0].numpy()
    X, U = synth.double_integrator_guess(t)
    z = prob.pack(X, U)
    info = api.newton_solve(prob, z, tol=1e-9)
    assert info["converged"], info
    Xg, Ug = [a.cpu().numpy() for a in prob.split(z)[:2]]
    assert np.abs(Xg[0] - 0.8 * (3 * t**2 - 2 * t**3)).max() < 1e-6
    assert 0.8 < Xg[0, -1]
