"""Pins of the matrix-free barrier oracle (oracle/matfree_barrier.py) against the dense one
(oracle/barrier.py, itself pinned by finite differences, closed forms and Pontryagin's
principle): residual, KKT product and K-tilde^-1 on random points and vectors, and the staged
solve, with control bounds and a one-sided endpoint bound, for the double integrator and the
orbit transfer."""
import numpy as np
import pytest

from oracle import problems as op
from oracle.barrier import BarrierKKT
from oracle.matfree_barrier import MatFreeBarrierKKT
from paper_2509_01855_gb300 import synth


def _case(kind, N):
    if kind == op.DBL_INT:
        prob = op.Problem(op.DBL_INT, 0.0, 1.0)
        lo, hi, eb, mu = [-4.0], [5.0], {0: (0.7, np.inf)}, 0.3
    else:
        prob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
        lo, hi, eb, mu = [-0.05, -np.inf], [0.05, 0.04], {0: (1.2, np.inf), 2: (-np.inf, 0.9)}, 1e-5
    D = BarrierKKT(prob, N, lo, hi, ebounds=eb)
    M = MatFreeBarrierKKT(prob, N, lo, hi, ebounds=eb)
    D.mu = M.mu = mu
    g = synth.rng("matfree-barrier", kind, N)
    if kind == op.DBL_INT:
        X, U = synth.double_integrator_guess(D.t)
        U = U + g.standard_normal(U.shape)
    else:
        X, U = synth.orbit_guess(D.t, 1.5, 20.0)
        U = U + 0.005 * g.standard_normal(U.shape)
    X = X + 0.01 * g.standard_normal(X.shape)
    vec = D.pack(X, U, 0.1 * g.standard_normal((prob.n_x, D.L)), 0.1 * g.standard_normal(prob.n_e))
    vec = D.interior(vec, margin=0.05)
    return D, M, vec, g


@pytest.mark.parametrize("kind,N", [(op.DBL_INT, 16), (op.DBL_INT, 64), (op.ORBIT, 16), (op.ORBIT, 32)])
def test_operators_match_the_dense_barrier_oracle(kind, N):
    D, M, vec, g = _case(kind, N)
    F = D.residual(vec)
    assert np.max(np.abs(M.residual(vec) - F)) < 1e-12 * np.max(np.abs(F))
    d = g.standard_normal(D.n)
    Kd = D.matrix(vec) @ d
    assert np.max(np.abs(M.apply(vec, d) - Kd)) < 1e-11 * np.max(np.abs(Kd))
    M.linearize_precond(vec)
    ref = np.linalg.solve(D.precond_matrix(vec), d)
    assert np.linalg.norm(M.precond_solve(d) - ref) < 1e-9 * np.linalg.norm(ref)
    z = g.standard_normal(D.n)
    Kz = D.precond_matrix(vec) @ z
    assert np.max(np.abs(M.precond_apply_matrix(vec, z) - Kz)) < 1e-11 * np.max(np.abs(Kz))


@pytest.mark.parametrize("kind", [op.DBL_INT, op.ORBIT])
def test_staged_solve_matches_the_dense_barrier_oracle(kind):
    N = 32
    if kind == op.DBL_INT:
        prob = op.Problem(op.DBL_INT, 0.0, 1.0)
        args = ([-5.0], [5.0], {0: (0.8, np.inf)})
        mu0, muf = 0.1, 1e-6
        X, U = synth.double_integrator_guess(BarrierKKT(prob, N, [-5.0], [5.0]).t)
    else:
        prob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
        args = ([-np.inf] * 2, [np.inf] * 2, {0: (1.55, np.inf)})
        mu0, muf = 1e-4, 1e-9
        X, U = synth.orbit_guess(BarrierKKT(prob, N, [-np.inf] * 2, [np.inf] * 2).t, 1.5, 20.0)
    D = BarrierKKT(prob, N, args[0], args[1], ebounds=args[2])
    M = MatFreeBarrierKKT(prob, N, args[0], args[1], ebounds=args[2])
    v0 = D.pack(X, U, np.zeros((prob.n_x, D.L)), np.zeros(prob.n_e))
    vd, idd = D.solve(v0, mu0=mu0, mu_final=muf)
    vm, im = M.solve(v0, mu0=mu0, mu_final=muf)
    assert idd["converged"] and im["converged"], (idd, im)
    assert np.max(np.abs(vm[:D.nz] - vd[:D.nz])) < 1e-7
