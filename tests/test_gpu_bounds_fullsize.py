"""Control bounds at the benchmark's size (N = 2^20), through properties that hold at any N.

- Double integrator with |u| <= 5 at N = 2^14 and 2^20, both barrier forms: the solution at
  sampled nodes against the one Pontryagin's principle gives, computed independently of the
  solver (tests/test_oracle_barrier.py: u = clip(alpha (1 - 2t), -5, 5), alpha from x(1) = 1 by
  quadrature and a bracketing root finder). At these N the discretisation error is negligible and
  the barrier's own perturbation remains: per node the barrier optimum of (u - a)^2 / 2 -
  mu log(5 - u) sits delta = mu / (a - 5 + delta) <= sqrt(mu) inside the bound, so with
  mu_final = 1e-6 the controls agree to 2e-3 (twice sqrt(mu_final), worst next to the kinks) and
  the states, integrals of the controls, to 1e-4.
- Orbit transfer with the endpoint bound r(t_f) >= 1.55 at N = 2^10, 2^14, 2^20: the oracle's
  Newton count and r(t_f) at N = 64.
- Residual, KKT product and preconditioner with control and endpoint bounds at N = 2^12 and
  2^14 against the matrix-free barrier oracle on the same grid.
- Orbit transfer with bounded thrust (the bench's bounded workload) at N = 2^20: the primal and
  the primal-dual form, two different Newton iterations, reach the same barrier solution; the
  controls stay strictly inside the bounds and reach them; the Newton counts are those at
  N = 2^10 (mesh independence, Table tab:m).
"""
import numpy as np
import pytest
import torch

from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu


def _api():
    from paper_2509_01855_gb300 import _lib, api
    return api, _lib


@pytest.mark.parametrize("form", ["primal", "primal_dual"])
@pytest.mark.parametrize("lg", [14, 20])
def test_bounded_double_integrator_full_size_pontryagin(lg, form):
    from tests.test_oracle_barrier import _pontryagin_bounded
    api, lib = _api()
    N = 1 << lg
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
    assert np.all(np.abs(Ug[0]) < 5.0)
    idx = np.unique(np.concatenate([np.linspace(0, N, 257).astype(int), [1, 2, N - 2, N - 1]]))
    ue = np.array([u(t[i]) for i in idx])
    xe = np.array([x(t[i]) for i in idx])
    assert np.abs(Ug[0][idx] - ue).max() < 2e-3, np.abs(Ug[0][idx] - ue).max()
    assert np.abs(Xg[0][idx] - xe).max() < 1e-4, np.abs(Xg[0][idx] - xe).max()
    prob.close()


def _orbit(api, lib, N, lo, hi, form):
    rf, tf = 1.5, 20.0
    prob = api.Problem(lib.BK_ORBIT, N, torch.float64, 0.0, tf, (0.01, rf))
    t = api.Plan(N, t0=0.0, tf=tf).grid()[0].numpy()
    X, U = synth.orbit_guess(t, rf, tf)
    z = prob.pack(X, U)
    prob.set_control_bounds(lo, hi)
    prob.set_barrier(1e-4, 1e-9, form)
    info = api.newton_solve(prob, z)
    assert info["converged"], info
    return prob, z, info


def test_bounded_orbit_full_size_forms_agree():
    from tests.test_gpu_bounds import _orbit_bounds
    api, lib = _api()
    _, _, lo, hi = _orbit_bounds()
    sols, its = {}, {}
    for form in ("primal", "primal_dual"):
        for lg in (10, 20):
            prob, z, info = _orbit(api, lib, 1 << lg, lo, hi, form)
            its[form, lg] = info["iterations"]
            if lg == 20:
                X, U = [a.cpu().numpy() for a in prob.split(z)[:2]]
                sols[form] = (X, U)
            prob.close()
    (Xp, Up), (Xd, Ud) = sols["primal"], sols["primal_dual"]
    for U in (Up, Ud):
        assert np.all(np.abs(U[0]) < hi[0]) and np.all(U[1] < hi[1])
        assert np.abs(U[0]).max() > hi[0] - 1e-5 and U[1].max() > hi[1] - 1e-5
    # the ill-conditioning of the last stage (mu = 1e-9) allows ~1e-6 between two solves that
    # both stop at merit 1e-10 (the same spread as between the oracle's two forms at N = 64)
    assert np.abs(Xp - Xd).max() < 1e-5, np.abs(Xp - Xd).max()
    assert np.abs(Up - Ud).max() < 1e-6, np.abs(Up - Ud).max()
    for form in ("primal", "primal_dual"):
        assert abs(its[form, 20] - its[form, 10]) <= 6, its


def test_endpoint_bounded_orbit_mesh_independent():
    """r(t_f) >= 1.55 in place of r(t_f) = 1.5 (no thrust bounds): the bound is active, the solves
    at N = 2^10, 2^14 and 2^20 take the Newton count of the oracle's solve at N = 64 (20, the same
    at every N in the oracle) within two steps, and r(t_f) sits the barrier's offset
    mu_final / |nu| above the bound, the value the oracle's solve gives at N = 64, to 1e-9."""
    from oracle import problems as op
    from oracle.barrier import BarrierKKT
    api, lib = _api()
    inf = float("inf")
    oprob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
    K = BarrierKKT(oprob, 64, [-inf] * 2, [inf] * 2, ebounds={0: (1.55, inf)})
    X, U = synth.orbit_guess(K.t, 1.5, 20.0)
    ref, rinfo = K.solve(K.pack(X, U, np.zeros((4, K.L)), np.zeros(3)), mu0=1e-4, mu_final=1e-9)
    assert rinfo["converged"]
    r_ref = K.split(ref)[0][0, -1]
    for lg in (10, 14, 20):
        N = 1 << lg
        prob = api.Problem(lib.BK_ORBIT, N, torch.float64, 0.0, 20.0, (0.01, 1.5))
        t = api.Plan(N, t0=0.0, tf=20.0).grid()[0].numpy()
        X, U = synth.orbit_guess(t, 1.5, 20.0)
        z = prob.pack(X, U)
        prob.set_terminal_bounds([1.55, -inf, -inf], [inf] * 3)
        prob.set_barrier(1e-4, 1e-9)
        info = api.newton_solve(prob, z)
        assert info["converged"], (lg, info)
        assert abs(info["iterations"] - rinfo["iters"]) <= 2, (lg, info, rinfo)
        r = prob.split(z)[0][0, -1].item()
        assert 1.55 < r and abs(r - r_ref) < 1e-9, (lg, r, r_ref)
        prob.close()


@pytest.mark.parametrize("lg", [12, 14])
def test_bounded_operators_match_matfree_oracle(lg):
    """Residual, KKT product and preconditioner with control bounds and endpoint bounds at
    N = 2^12 and 2^14 (multi-CTA transforms, three sweep levels) against the matrix-free barrier
    oracle on the same grid (oracle/matfree_barrier.py, pinned to the dense one)."""
    from oracle import problems as op
    from oracle.matfree_barrier import MatFreeBarrierKKT
    from tests.helpers import from_packed, rel, to_packed
    api, lib = _api()
    N = 1 << lg
    inf = float("inf")
    lo, hi, eb, mu = [-0.05, -inf], [0.05, 0.04], {0: (1.2, inf), 2: (-inf, 0.9)}, 1e-5
    oprob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
    M = MatFreeBarrierKKT(oprob, N, lo, hi, ebounds=eb)
    M.mu = mu
    g = synth.rng("bounds-matfree", lg)
    X, U = synth.orbit_guess(M.t, 1.5, 20.0)
    X = X + 0.01 * g.standard_normal(X.shape)
    U = U + 0.005 * g.standard_normal(U.shape)
    vec = M.pack(X, U, 0.1 * g.standard_normal((4, M.L)), 0.1 * g.standard_normal(3))
    vec = M.interior(vec, margin=0.05)
    prob = api.Problem(lib.BK_ORBIT, N, torch.float64, 0.0, 20.0, (0.01, 1.5))
    prob.set_control_bounds(lo, hi)
    prob.set_terminal_bounds([1.2, -inf, -inf], [inf, inf, 0.9])
    prob.set_barrier(mu, mu)
    z = from_packed(prob, vec)
    F = torch.zeros_like(z)
    prob.residual(z, F)
    Fo = M.residual(vec)
    assert rel(to_packed(prob, F), Fo) < 1e-12
    prob.linearize(z)
    d = g.standard_normal(M.n)
    x = from_packed(prob, d)
    out = torch.zeros_like(x)
    api.kkt_apply(prob, lib.BK_OP_KKT, x, out)
    assert rel(to_packed(prob, out), M.apply(vec, d)) < 1e-12
    M.linearize_precond(vec)
    api.precond_apply(prob, lib.BK_OP_KKT, x, out)
    assert rel(to_packed(prob, out), M.precond_solve(d)) < 1e-10
    prob.close()
