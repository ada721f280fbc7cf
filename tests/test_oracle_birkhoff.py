"""Pins of the oracle's Birkhoff machinery against what the paper and the mathematics fix.

Every check here is independent of the quantity it pins: printed values from the paper,
closed forms, textbook identities or brute force on tiny inputs.
"""
import os

import numpy as np
import pytest

from oracle import birkhoff as ob
from oracle import grid as og

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


# ---- printed worked examples -------------------------------------------------------------
def test_printed_Ba10():
    """Eq. Ba=10: B^a for 10 CGL points, printed to two decimals (some entries truncated)."""
    printed = _load("ba10_printed.txt")
    B = ob.dense_Ba(9)
    assert printed.shape == (10, 10)
    assert np.abs(B - printed).max() <= 0.01 + 1e-12


def test_printed_Btilde10():
    """Second matrix of Eq. Ba=10: B-tilde for 10 CGL points; matches after rounding."""
    printed = _load("btilde10_printed.txt")
    Bt = ob.dense_Btilde(ob.cc_weights(9))
    assert np.array_equal(np.round(Bt, 2), printed)


# ---- grid, weights ------------------------------------------------------------------------
@pytest.mark.parametrize("N", [4, 9, 16, 64])
def test_nodes_closed_form(N):
    """Eq. CGLpts: tau_j = -cos(j pi / N), ascending, antisymmetric, endpoints +-1."""
    tau = og.cgl_nodes(N)
    j = np.arange(N + 1)
    assert np.allclose(tau, -np.cos(j * np.pi / N), atol=1e-15)
    assert tau[0] == -1.0 and tau[-1] == 1.0
    assert np.all(np.diff(tau) > 0)
    assert np.array_equal(tau, -tau[::-1])


@pytest.mark.parametrize("N", [4, 8, 9, 16, 32, 100])
def test_cc_weights(N):
    """Last row of B^a = Clenshaw-Curtis weights: it equals the independent cosine-sum closed
    form, sums to 2, is symmetric, integrates T_k exactly, and w_0 = 1/(N^2 - 1) for even N."""
    w = ob.cc_weights(N)
    w2 = og.cc_weights_sum(N)
    assert np.abs(w - w2).max() < 1e-14
    assert abs(w.sum() - 2.0) < 1e-14
    assert np.abs(w - w[::-1]).max() < 1e-14
    tau = og.cgl_nodes(N)
    for k in range(N + 1):
        exact = (1 + (-1) ** k) / (1.0 - k * k) if k != 1 else 0.0
        assert abs(w @ np.cos(k * np.arccos(np.clip(tau, -1, 1))) - exact) < 1e-13
    if N % 2 == 0:
        assert abs(w[0] - 1.0 / (N * N - 1.0)) < 1e-15


# ---- dense B^a from its definition ------------------------------------------------------
@pytest.mark.parametrize("N", [4, 9, 16, 33, 64])
def test_B_row0_and_ones(N):
    """Row 0 of B^a is zero (B_j^a(tau^a) = 0, Eq. birk-conditions) and B 1 = t - t_0."""
    t0, tf = 0.3, 2.1
    B = ob.dense_B(N, t0, tf)
    tau = og.cgl_nodes(N)
    t = t0 + 0.5 * (tf - t0) * (tau + 1.0)
    assert np.all(B[0] == 0.0)
    assert np.abs(B @ np.ones(N + 1) - (t - t0)).max() < 1e-13


@pytest.mark.parametrize("N", [4, 8, 17, 32])
def test_B_integrates_polynomial_derivatives(N):
    """B^a q' = q - q(-1) at the nodes for every polynomial q of degree <= N + 1 (brute force)."""
    rng = np.random.default_rng(N)
    B = ob.dense_Ba(N)
    tau = og.cgl_nodes(N)
    for _ in range(5):
        q = np.polynomial.Polynomial(rng.standard_normal(N + 2))
        got = B @ q.deriv()(tau)
        want = q(tau) - q(-1.0)
        assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max())


def test_B_conditioning_flat():
    """Fig. 3 claim: the condition number of I - B^a stays O(1) as N grows."""
    conds = [np.linalg.cond(np.eye(N + 1) - ob.dense_Ba(N)) for N in (16, 32, 64, 128)]
    assert max(conds) / min(conds) < 1.5
    assert max(conds) < 10.0


# ---- the FastBV chain --------------------------------------------------------------------
def test_dct1_convention_brute_force():
    """Eq. vm=DCT-1 written as a loop on a tiny input."""
    rng = np.random.default_rng(1)
    N = 7
    x = rng.standard_normal(N + 1)
    y = np.array([x[0] / 2 + sum(x[k] * np.cos(k * j * np.pi / N) for k in range(1, N))
                  + (-1) ** j * x[N] / 2 for j in range(N + 1)])
    assert np.abs(ob.dct1_paper(x) - y).max() < 1e-14


@pytest.mark.parametrize("N", [4, 8, 16, 64])
def test_fastv2a_coefficients(N):
    """Fastv2a returns the Chebyshev coefficients: sum_k a_k T_k(tau_i) = v_i (Eq. vi=sumT),
    checked with numpy's independent Chebyshev evaluation, and the round trip is the identity."""
    rng = np.random.default_rng(N)
    v = rng.standard_normal(N + 1)
    a = ob.fastv2a(v)
    tau = og.cgl_nodes(N)
    assert np.abs(np.polynomial.chebyshev.chebval(tau, a) - v).max() < 1e-13
    assert np.abs(ob.fasta2v(a) - v).max() < 1e-13


@pytest.mark.parametrize("N", [4, 9, 16, 63, 128, 256])
def test_fastbv_equals_dense(N):
    """FastBV reaches B^a V exactly (up to rounding) for random V."""
    rng = np.random.default_rng(100 + N)
    V = rng.standard_normal((3, N + 1))
    B = ob.dense_B(N, 0.0, 3.0)
    ref = V @ B.T
    got = ob.fastbv(V, 0.0, 3.0)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


@pytest.mark.parametrize("N", [4, 9, 16, 63, 128])
def test_fastbv_T_equals_dense_transpose(N):
    rng = np.random.default_rng(200 + N)
    U = rng.standard_normal((2, N + 1))
    B = ob.dense_B(N, -1.0, 2.0)
    ref = U @ B
    got = ob.fastbv_T(U, -1.0, 2.0)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13


def test_c0_is_minus_node0_value():
    """Eq. c_k=bydef: c_0 makes the integral vanish at tau = -1, i.e. sum_k c_k T_k(-1) = 0."""
    rng = np.random.default_rng(5)
    for N in (4, 9, 32):
        c = ob.integration_coeffs(ob.fastv2a(rng.standard_normal(N + 1)))
        sgn = (-1.0) ** np.arange(N + 2)
        assert abs(c @ sgn) < 1e-14 * max(1.0, np.abs(c).max())


@pytest.mark.parametrize("N", [4, 16, 64])
def test_sparse_modes_match_dense(N):
    """The closed-form integrals of T_k (Eq. intChebPoly=) agree with the quadrature B^a."""
    rng = np.random.default_rng(N)
    modes = sorted(set([0, 1, 2, N - 2, N - 1, N] + list(rng.integers(0, N + 1, 6))))
    alphas = rng.standard_normal(len(modes))
    v, Bv = ob.sparse_mode_pair(N, modes, alphas, 0.0, 2.0)
    assert np.abs(ob.dense_B(N, 0.0, 2.0) @ v - Bv).max() < 1e-13


def test_sparse_modes_large_N_against_fastbv():
    """At large N the closed forms and FastBV (library DCT) agree to rounding."""
    N = 1 << 14
    rng = np.random.default_rng(7)
    modes = [0, 1, 2, N - 2, N - 1, N] + list(rng.integers(3, N - 2, 10))
    alphas = rng.standard_normal(len(modes))
    v, Bv = ob.sparse_mode_pair(N, modes, alphas, 0.0, 20.0)
    got = ob.fastbv(v, 0.0, 20.0)
    assert np.linalg.norm(got - Bv) / np.linalg.norm(Bv) < 1e-13


def test_aliasing_identity():
    """Appendix C: T_{N+1}(tau_j) = T_{N-1}(tau_j) on the CGL grid."""
    for N in (4, 9, 64, 1000):
        assert np.abs(ob.cheb_T_at_nodes(N + 1, N) - ob.cheb_T_at_nodes(N - 1, N)).max() < 1e-13


# ---- B-tilde sweeps -------------------------------------------------------------------------
@pytest.mark.parametrize("N", [4, 9, 40])
def test_fastbccv(N):
    rng = np.random.default_rng(N)
    w = ob.cc_weights(N)
    v = rng.standard_normal(N + 1)
    assert np.abs(ob.fastbccv(w, v) - ob.dense_Btilde(w) @ v).max() < 1e-14


@pytest.mark.parametrize("N", [4, 16, 64])
def test_fastpinvy_inverts_P(N):
    """The corrected sweep inverts P = I - B-tilde diag(d); the sweep as printed does not."""
    rng = np.random.default_rng(N)
    w = ob.cc_weights(N)
    d = rng.standard_normal(N + 1)
    Y = rng.standard_normal(N + 1)
    P = np.eye(N + 1) - ob.dense_Btilde(w) * d[None, :]
    xi = ob.fastpinvy_scalar(w, d, Y)
    assert np.abs(P @ xi - Y).max() < 1e-13

    def as_printed(w, d, Y):
        out = np.zeros(len(Y)); s = 0.0
        for k in range(len(Y)):
            out[k] = (Y[k] - s) / (1.0 - w[k] * d[k] / 2.0)
            s = w[k] * d[k] * Y[k] + s
        return out
    assert np.abs(P @ as_printed(w, d, Y) - Y).max() > 1e-3


@pytest.mark.parametrize("N", [4, 16, 48])
def test_fastpinvy_block_and_transpose(N):
    rng = np.random.default_rng(N)
    n = 4
    w = ob.cc_weights(N)
    J = 0.7 * rng.standard_normal((N + 1, n, n))
    L = N + 1
    P = np.eye(n * L)
    Bt = ob.dense_Btilde(w)
    for m in range(n):
        for q in range(n):
            P[m * L:(m + 1) * L, q * L:(q + 1) * L] -= Bt * J[:, m, q][None, :]
    Y = rng.standard_normal((n, L))
    xi = ob.fastpinvy_block(w, J, Y)
    assert np.abs(P @ xi.ravel() - Y.ravel()).max() < 1e-12
    yT = ob.fastpinvy_block_T(w, J, Y)
    assert np.abs(P.T @ yT.ravel() - Y.ravel()).max() < 1e-12


@pytest.mark.parametrize("N", [4, 9, 16, 33])
def test_dense_Bb_definition(N):
    """The b-form matrix of Eq. manyDefs: last row zero (B^b_j(tau^b) = 0), B^b = B^a - 1 w^T
    (the two bases differ by their value at tau = 1, which for B^a is the weight w_j), and
    B^b q' = q - q(1) for polynomials q of degree <= N + 1 (brute force)."""
    from oracle.grid import cgl_nodes
    Bb = ob.dense_Bb(N)
    Ba = ob.dense_Ba(N)
    assert np.abs(Bb[N]).max() == 0.0
    assert np.abs(Bb - (Ba - np.outer(np.ones(N + 1), Ba[N]))).max() < 1e-13
    tau = cgl_nodes(N)
    q = np.polynomial.Polynomial(np.random.default_rng(N).standard_normal(N + 2))
    assert np.abs(Bb @ q.deriv()(tau) - (q(tau) - q(1.0))).max() < 1e-12 * max(1.0, np.abs(q.coef).sum())
