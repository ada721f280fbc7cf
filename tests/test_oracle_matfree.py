"""Pins of the matrix-free oracle (oracle/matfree.py).

Each matrix-free operator is checked against the dense class built from the definition of B^a
(Gauss-Legendre integrals of the Lagrange basis, Eq. manyDefs) at small N: the residual, the
KKT product, the preconditioner solve and the whole Newton iteration. The plain GMRES is pinned
to a direct solve. The self-convergence of the discrete orbit solution (the oracle at N_ref
against 2 N_ref and 4 N_ref) fixes how closely an oracle solution at N_ref stands in for the
solution at a far finer grid.
"""
import numpy as np
import pytest

from oracle import birkhoff as ob
from oracle import problems as op
from oracle.grid import cgl_nodes, interpolate, lagrange_matrix
from oracle.kkt import DenseKKT
from oracle.matfree import MatFreeKKT, btilde, btilde_T, gmres_right


def _point(kind, D, rng):
    p = D.prob
    if kind in (op.ORBIT, op.ORBIT_MT):
        rf = p.params[1]
        ae = (1.0 - rf ** -0.5) / (p.tf - p.t0)
        v = 1.0 - ae * (D.t - p.t0)
        X = np.stack([1 / v**2, (1 - v**4) / (4 * ae), 2 * ae / v**3, v])
        X = X + 0.01 * rng.standard_normal(X.shape)
        U = rng.uniform(-3, 3, (1, D.L)) if kind == op.ORBIT_MT else 0.01 * rng.standard_normal((2, D.L))
    else:
        X = rng.standard_normal((p.n_x, D.L))
        U = rng.standard_normal((p.n_u, D.L))
    lam = D.w * rng.standard_normal((p.n_x, D.L))
    nu = rng.standard_normal(p.n_e)
    return D.pack(X, U, lam, nu) if not D.free else D.pack(X, U, lam, nu, 6.5)


CASES = [(op.ORBIT, 16, (0.01, 1.5), 20.0), (op.ORBIT, 64, (0.01, 1.5), 20.0), (op.DBL_INT, 16, (), 1.0),
         (op.ORBIT_MT, 32, (0.05, 6.0), 24.0)]


def test_btilde_products_match_definition():
    rng = np.random.default_rng(3)
    w = rng.uniform(0.1, 1.0, 9)
    v = rng.standard_normal((2, 9))
    Bt = ob.dense_Btilde(w)
    assert np.abs(btilde(w, v) - v @ Bt.T).max() < 1e-14
    assert np.abs(btilde_T(w, v) - v @ Bt).max() < 1e-14
    assert np.abs(btilde(w, v[0]) - ob.fastbccv(w, v[0])).max() < 1e-14


@pytest.mark.parametrize("kind,N,params,tf", CASES)
def test_matfree_matches_dense(kind, N, params, tf):
    rng = np.random.default_rng(N + kind)
    pr = op.Problem(kind, 0.0, tf, params)
    D, M = DenseKKT(pr, N), MatFreeKKT(pr, N)
    assert np.abs(D.w - M.w).max() < 1e-14
    vec = _point(kind, D, rng)
    F = D.residual(vec)
    assert np.abs(M.residual(vec) - F).max() < 1e-13 * np.abs(F).max()
    d = rng.standard_normal(D.n)
    Kd = D.matrix(vec) @ d
    assert np.linalg.norm(M.apply(vec, d) - Kd) < 1e-13 * np.linalg.norm(Kd)
    Kt = D.precond_matrix(vec)
    M.linearize_precond(vec)
    z = M.precond_solve(d)
    zr = np.linalg.solve(Kt, d)
    assert np.linalg.norm(z - zr) < 1e-12 * np.linalg.norm(zr)
    # K-tilde z cancels (z is large where w is small): scale by |K-tilde| |z|
    assert np.linalg.norm(M.precond_apply_matrix(vec, z) - Kt @ z) < 1e-13 * np.linalg.norm(np.abs(Kt) @ np.abs(z))


def test_gmres_right_solves_and_counts():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((60, 60)) + 12 * np.eye(60)
    b = rng.standard_normal(60)
    x, its, rr = gmres_right(lambda v: A @ v, lambda v: v / 12.0, b, rtol=1e-13, restart=9)
    assert rr <= 1e-13 and np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-12 * np.linalg.norm(x)
    # with the exact inverse as preconditioner one iteration suffices
    Ai = np.linalg.inv(A)
    x, its, rr = gmres_right(lambda v: A @ v, lambda v: Ai @ v, b, rtol=1e-12)
    assert its == 1 and rr < 1e-12


@pytest.mark.parametrize("N", [32, 64])
def test_matfree_newton_follows_dense_newton(N):
    """Tight inner solves: the same Newton iterates, step lengths and merit history."""
    pr = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
    D, M = DenseKKT(pr, N), MatFreeKKT(pr, N)
    ae = (1.0 - 1.5 ** -0.5) / 20.0
    v = 1.0 - ae * D.t
    X = np.stack([1 / v**2, (1 - v**4) / (4 * ae), 2 * ae / v**3, v])
    U = np.zeros((2, D.L)); U[1] = ae
    v0 = D.pack(X, U, np.zeros((4, D.L)), np.zeros(3))
    r1, i1 = D.newton(v0)
    r2, i2 = M.newton(v0)
    assert i1["iters"] == i2["iters"] and i1["alphas"] == i2["alphas"]
    assert np.allclose(i1["norms"][:-1], i2["norms"][:-1], rtol=1e-6, atol=0)
    assert np.abs(r1 - r2).max() < 1e-11


def test_interpolate_reproduces_polynomials():
    """The barycentric interpolant of a degree-N polynomial is the polynomial itself."""
    N = 24
    c = np.random.default_rng(7).standard_normal(N + 1)
    P = np.polynomial.chebyshev.Chebyshev(c)
    xi = np.linspace(-1, 1, 1001)
    got = interpolate(P(cgl_nodes(N)), N, xi, chunk=100)
    assert np.abs(got - P(xi)).max() < 1e-12 * np.abs(c).sum()
    assert np.abs(lagrange_matrix(N, cgl_nodes(N)) - np.eye(N + 1)).max() == 0.0


def _orbit_solution(N):
    pr = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
    M = MatFreeKKT(pr, N)
    ae = (1.0 - 1.5 ** -0.5) / 20.0
    v = 1.0 - ae * M.t
    X = np.stack([1 / v**2, (1 - v**4) / (4 * ae), 2 * ae / v**3, v])
    U = np.zeros((2, M.L)); U[1] = ae
    vec, info = M.newton(M.pack(X, U, np.zeros((4, M.L)), np.zeros(3)), tol=1e-12)
    assert info["converged"]
    return M, vec, info


@pytest.mark.slow
def test_orbit_self_convergence_at_reference_grid():
    """The discrete orbit solution at N_ref = 1024 against 2 N_ref and 4 N_ref, through the
    barycentric interpolant: states within 1e-11 (max-abs), controls and the costate
    (B^aT lambda / w) within 1e-9 in the quadrature norm, the terminal multipliers within 1e-12,
    and the merit history of the Newton iteration the same on every grid (mesh independence)."""
    sols = {N: _orbit_solution(N) for N in (1024, 2048, 4096)}
    Mf, vf, inf = sols[4096]
    Xf, Uf, lf, nf = Mf.split(vf)
    pf = ob.fastbv_T(lf) / Mf.w
    wq = Mf.s * Mf.w
    for N in (1024, 2048):
        M, vec, info = sols[N]
        X, U, lam, nu = M.split(vec)
        p = ob.fastbv_T(lam) / M.w
        vals = interpolate(np.concatenate([X, U, p]), N, Mf.tau)
        Xi, Ui, pi = vals[:4], vals[4:6], vals[6:]
        assert np.abs(Xi - Xf).max() < 1e-11
        assert np.sqrt(np.sum(wq * (Ui - Uf) ** 2)) < 1e-9
        assert np.sqrt(np.sum(wq * (pi - pf) ** 2)) < 1e-9
        assert np.abs(nu - nf).max() < 1e-12
        assert info["iters"] == inf["iters"]
        assert np.allclose(info["norms"][:-1], inf["norms"][:-1], rtol=1e-7, atol=0)
