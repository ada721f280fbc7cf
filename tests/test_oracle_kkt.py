"""Pins of the oracle's problem definitions, dense KKT and Newton driver."""
import numpy as np
import pytest

from oracle import problems as op
from oracle.kkt import DenseKKT


def _orbit_guess(K, rf, T):
    """Tangential-thrust spiral that ends at r_f at t_f (input recipe of the orbit problem)."""
    ae = (1.0 - rf ** -0.5) / T
    v = 1.0 - ae * (K.t - K.prob.t0)
    X = np.stack([1 / v**2, (1 - v**4) / (4 * ae), 2 * ae / v**3, v])
    U = np.zeros((2, K.L)); U[1] = ae
    return X, U


@pytest.mark.parametrize("kind", [op.DBL_INT, op.ORBIT, op.BILINEAR])
def test_jacobians_and_hessians_by_finite_differences(kind):
    """d f / d(x, u) and sum_m mu_m Hess f_m against central differences of f itself."""
    rng = np.random.default_rng(kind)
    p = op.Problem(kind, 0.0, 1.0, (0.01, 1.5) if kind == op.ORBIT else ())
    L = 7
    X = rng.uniform(0.8, 1.3, (p.n_x, L))
    U = rng.uniform(-0.5, 0.5, (p.n_u, L))
    mu = rng.standard_normal((p.n_x, L))
    Jx, Ju = p.jac(X, U)
    H = p.hess_f(X, U, mu)
    h = 1e-6
    n = p.n_x + p.n_u
    for j in range(n):
        dX = np.zeros_like(X); dU = np.zeros_like(U)
        if j < p.n_x:
            dX[j] = h
        else:
            dU[j - p.n_x] = h
        fd = (p.f(X + dX, U + dU) - p.f(X - dX, U - dU)) / (2 * h)      # (n_x, L)
        J = Jx[:, :, j] if j < p.n_x else Ju[:, :, j - p.n_x]           # (L, n_x)
        assert np.abs(fd.T - J).max() < 1e-8
        # gradient of (mu . f) in direction j, differenced again
        def g(Xa, Ua):
            jx, ju = p.jac(Xa, Ua)
            full = np.concatenate([jx, ju], axis=2)                     # (L, n_x, n)
            return np.einsum('mk,kmi->ki', mu, full)                    # (L, n)
        fdH = (g(X + dX, U + dU) - g(X - dX, U - dU)) / (2 * h)         # (L, n)
        assert np.abs(fdH - H[:, :, j]).max() < 1e-7
    assert np.abs(H - np.transpose(H, (0, 2, 1))).max() == 0.0


@pytest.mark.parametrize("kind,N", [(op.DBL_INT, 8), (op.ORBIT, 8), (op.ORBIT, 13)])
def test_kkt_matrix_is_jacobian_of_residual(kind, N):
    """The assembled KKT matrix equals the finite-difference Jacobian of the KKT residual."""
    rng = np.random.default_rng(N)
    p = op.Problem(kind, 0.0, 2.0, (0.01, 1.5) if kind == op.ORBIT else ())
    K = DenseKKT(p, N)
    X = rng.uniform(0.9, 1.2, (p.n_x, K.L))
    U = rng.uniform(-0.1, 0.1, (p.n_u, K.L))
    vec = K.pack(X, U, rng.standard_normal((p.n_x, K.L)), rng.standard_normal(p.n_e))
    Km = K.matrix(vec)
    h = 1e-6
    fd = np.zeros_like(Km)
    for j in range(K.n):
        e = np.zeros(K.n); e[j] = h
        fd[:, j] = (K.residual(vec + e) - K.residual(vec - e)) / (2 * h)
    assert np.abs(fd - Km).max() < 1e-7
    assert np.abs(Km - Km.T).max() < 1e-14


@pytest.mark.parametrize("N", [4, 8, 16, 64, 256])
def test_double_integrator_closed_form(N):
    """Minimum-energy double integrator: x = 3t^2 - 2t^3, v = 6t - 6t^2, u = 6 - 12t, reached in
    one Newton step (linear-quadratic problem), for every even N >= 4."""
    p = op.Problem(op.DBL_INT, 0.0, 1.0)
    K = DenseKKT(p, N)
    lam = 0.5 * (K.tau + 1.0)
    X = np.stack([lam, np.zeros(K.L)])
    vec0 = K.pack(X, np.zeros((1, K.L)), np.zeros((2, K.L)), np.zeros(2))
    vec, info = K.newton(vec0)
    assert info["iters"] == 1 and info["converged"]
    X, U, _, _ = K.split(vec)
    t = K.t
    assert np.abs(X[0] - (3 * t**2 - 2 * t**3)).max() < 1e-13
    assert np.abs(X[1] - (6 * t - 6 * t**2)).max() < 1e-13
    werr = np.sqrt(K.s * np.sum(K.w * (U[0] - (6 - 12 * t)) ** 2))
    assert werr < 1e-9
    assert abs(K.s * np.sum(K.w * U[0] ** 2) - 12.0) < 1e-9


def test_orbit_mesh_independence():
    """Table tab:m's claim in kind: the same Newton count and residual history for every N,
    and a spectrally converged solution (theta_f to 1e-10 between N = 128 and N = 256)."""
    rf, T = 1.5, 20.0
    hist = {}
    thf = {}
    for N in (32, 64, 128, 256):
        p = op.Problem(op.ORBIT, 0.0, T, (0.01, rf))
        K = DenseKKT(p, N)
        X, U = _orbit_guess(K, rf, T)
        vec, info = K.newton(K.pack(X, U, np.zeros((4, K.L)), np.zeros(3)))
        assert info["converged"]
        hist[N] = (info["iters"], np.array(info["norms"][:3]))
        thf[N] = K.split(vec)[0][1, -1]
        Xs = K.split(vec)[0]
        assert abs(Xs[0, -1] - rf) < 1e-12 and abs(Xs[2, -1]) < 1e-12
        assert abs(Xs[3, -1] - rf ** -0.5) < 1e-12
    assert len({h[0] for h in hist.values()}) == 1
    for N in (64, 128, 256):
        assert np.allclose(hist[N][1], hist[32][1], rtol=0.05)
    assert abs(thf[256] - thf[128]) < 1e-10


def test_precond_matrix_structure():
    """K-tilde keeps the zero blocks it is defined with and reduces to the exact KKT matrix
    where B-tilde = B^a would hold (checked through its state block: P = I - s B-tilde J_x)."""
    p = op.Problem(op.ORBIT, 0.0, 20.0, (0.01, 1.5))
    K = DenseKKT(p, 16)
    X, U = _orbit_guess(K, 1.5, 20.0)
    vec = K.pack(X, U, np.zeros((4, K.L)), np.zeros(3))
    Kt = K.precond_matrix(vec)
    assert np.abs(Kt - Kt.T).max() == 0.0
    nc = K.nc
    assert np.all(Kt[:nc, :K.nz] == 0.0)
    P = K.state_precond_matrix(vec)
    for m in range(4):
        blk = P[m * K.L:(m + 1) * K.L, m * K.L:(m + 1) * K.L]
        assert np.all(np.triu(blk, 1) == 0.0)       # lower triangular per component block
