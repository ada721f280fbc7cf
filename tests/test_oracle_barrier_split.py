"""Pins of the two-multiplier endpoint rows (oracle/barrier_split.py).

- Its Newton matrix is the Jacobian of its residual (finite differences), the control barrier
  and a two-sided row included.
- The double integrator with x(1) in [0.8, 1.2] or [-1, 2] (v(1) = 0) reaches the closed form
  x = p (3t^2 - 2t^3), p = 0.8 or 0 (the energy 6 p^2 of the cubic).
- On the orbit transfer, an interval that holds the free-r(t_f) optimum ([1.0, 1.45]) gives the
  solution of the one-sided row r(t_f) <= 1.6 (inactive there too), and [1.4, 1.6] the one of
  r(t_f) >= 1.4 (active at 1.4): the same barrier problems up to the far side's O(mu) term.
"""
import numpy as np
import pytest

from oracle import problems as op
from oracle.barrier import BarrierKKT
from oracle.barrier_split import SplitEndpointKKT
from paper_2509_01855_gb300 import synth


def test_split_matrix_is_residual_jacobian():
    prob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
    K = SplitEndpointKKT(prob, 10, [-0.05, -np.inf], [0.05, 0.04], {0: (1.2, 1.8)}, ebounds={2: (-np.inf, 0.9)})
    K.mu = 0.01
    g = synth.rng("barrier-split-fd")
    X, U = synth.orbit_guess(K.t, 1.5, 20.0)
    X = X + 0.01 * g.standard_normal(X.shape)
    U = 0.01 * g.standard_normal(U.shape)
    vec = K.pack(X, U, 0.1 * g.standard_normal((4, K.L)), 0.1 * g.standard_normal(3), [0.2])
    vec = K.interior(vec, margin=0.05)
    A = K.matrix(vec)
    J = np.zeros_like(A)
    h = 1e-6
    for j in range(K.n):
        e = np.zeros(K.n)
        e[j] = h
        J[:, j] = (K.residual(vec + e) - K.residual(vec - e)) / (2 * h)
    assert np.max(np.abs(A - J)) < 1e-5 * max(1.0, np.max(np.abs(A)))


@pytest.mark.parametrize("bounds,p_star", [((0.8, 1.2), 0.8), ((-1.0, 2.0), 0.0)])
def test_split_double_integrator_closed_form(bounds, p_star):
    prob = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = SplitEndpointKKT(prob, 32, [-np.inf], [np.inf], {0: bounds})
    X, U = synth.double_integrator_guess(K.t)
    vec, info = K.solve(K.pack(X, U, np.zeros((2, K.L)), np.zeros(2)), mu_final=1e-8)
    assert info["converged"], info
    Xs = K.split(vec)[0]
    t = K.t
    assert np.max(np.abs(Xs[0] - p_star * (3 * t**2 - 2 * t**3))) < 1e-6
    assert bounds[0] < Xs[0, -1] < bounds[1]
    nl, nh = K.split(vec)[3][0], vec[K.nb]
    assert nl < 0 < nh


@pytest.mark.parametrize("interval,one_sided", [((1.0, 1.45), (-np.inf, 1.6)), ((1.4, 1.6), (1.4, np.inf))])
def test_split_orbit_matches_the_one_sided_solution(interval, one_sided):
    prob = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
    S = SplitEndpointKKT(prob, 64, [-np.inf] * 2, [np.inf] * 2, {0: interval})
    O = BarrierKKT(prob, 64, [-np.inf] * 2, [np.inf] * 2, ebounds={0: one_sided})
    X, U = synth.orbit_guess(S.t, 1.5, 20.0)
    vs, i_s = S.solve(S.pack(X, U, np.zeros((4, S.L)), np.zeros(3)), mu0=1e-4, mu_final=1e-9)
    vo, i_o = O.solve(O.pack(X, U, np.zeros((4, O.L)), np.zeros(3)), mu0=1e-4, mu_final=1e-9)
    assert i_s["converged"] and i_o["converged"], (i_s, i_o)
    assert i_s["iters"] <= 40, i_s
    # the far bound adds mu / (distance) to the barrier gradient: O(1e-9) at mu_final
    assert np.max(np.abs(vs[:S.nz] - vo[:O.nz])) < 1e-6, np.max(np.abs(vs[:S.nz] - vo[:O.nz]))
