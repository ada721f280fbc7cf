"""Birkhoff matrices and the FastBV chain (oracle; test infrastructure only).

Paper sections: "Fast Computation of Birkhoff Matrix-Vector Products" (Eqs. xdot=v=sumT through
chatk=, algorithms Fasta2v and FastBV), Appendix B (Fastv2a), Appendix C (aliasing), and
"Development of a Special Birkhoff-Centric Preconditioner" (B-tilde, FastBccV, FastPinvY).

Conventions: tau-domain matrices act on a vector indexed j = 0..N over the CGL nodes in
ascending order (tau_0 = -1). The time-domain product is s * B^a v with s = (t_f - t_0)/2
(reading: the paper works on [-1, 1]; on [t_0, t_f] the chain rule gives the factor s).
"""
import numpy as np
import scipy.fft

from .grid import cgl_nodes, lagrange_matrix


# --------------------------------------------------------------------------------------------
# Dense B^a from its definition
# --------------------------------------------------------------------------------------------
def dense_Ba(N):
    """[B^a]_ij = B^a_j(tau_i) (Eq. manyDefs), with B^a_j the Birkhoff basis of Eq. birk-conditions.

    B^a_j(-1) = 0 and dB^a_j/dtau(tau_i) = delta_ij with B^a_j a polynomial of degree N+1, so
    dB^a_j/dtau is the degree-N Lagrange polynomial l_j and B^a_j(tau) = int_{-1}^{tau} l_j.
    Each row is integrated with an n-point Gauss-Legendre rule on [-1, tau_i], n = N//2 + 2,
    which is exact for the degree-N integrand. Row 0 is zero. O(N^3) work.
    """
    tau = cgl_nodes(N)
    nq = N // 2 + 2
    xg, wg = np.polynomial.legendre.leggauss(nq)
    B = np.zeros((N + 1, N + 1))
    for i in range(1, N + 1):
        half = 0.5 * (tau[i] + 1.0)
        xi = -1.0 + half * (xg + 1.0)
        B[i] = half * (wg @ lagrange_matrix(N, xi))
    return B


def dense_Bb(N):
    """[B^b]_ij = B^b_j(tau_i) (Eq. manyDefs), the b-form Birkhoff basis of Eq. birk-conditions:
    B^b_j(tau^b = 1) = 0 and dB^b_j/dtau(tau_i) = delta_ij, so B^b_j(tau) = -int_{tau}^{1} l_j.
    Each row by an n-point Gauss-Legendre rule on [tau_i, 1], n = N//2 + 2 (exact for degree N).
    Row N is zero. O(N^3) work; written from the definition, independently of dense_Ba."""
    tau = cgl_nodes(N)
    nq = N // 2 + 2
    xg, wg = np.polynomial.legendre.leggauss(nq)
    B = np.zeros((N + 1, N + 1))
    for i in range(N):
        half = 0.5 * (1.0 - tau[i])
        xi = tau[i] + half * (xg + 1.0)
        B[i] = -half * (wg @ lagrange_matrix(N, xi))
    return B


def dense_B(N, t0=-1.0, tf=1.0):
    """Time-domain Birkhoff matrix s * B^a, s = (t_f - t_0)/2, so that (B 1)_i = t_i - t_0."""
    return 0.5 * (tf - t0) * dense_Ba(N)


def cc_weights(N):
    """w^CC_j = last row of B^a (the remark after Eq. Ba=10: exactly the Clenshaw-Curtis weights)."""
    return dense_Ba(N)[N].copy()


# --------------------------------------------------------------------------------------------
# The FastBV chain, step by step in the paper's order, with a library DCT-I as the transform
# --------------------------------------------------------------------------------------------
def dct1_paper(x):
    """The paper's DCT-I (Eq. vm=DCT-1): y_j = x_0/2 + sum_{k=1}^{N-1} x_k cos(k j pi/N) + (-1)^j x_N/2.

    This is one half of SciPy's unnormalised type-1 DCT, which serves as the library primitive.
    """
    return 0.5 * scipy.fft.dct(np.asarray(x, dtype=np.float64), type=1, axis=-1)


def fastv2a(v):
    """Fastv2a (Appendix B): reverse, DCT-I times 2/N, halve the first and last coefficient."""
    v = np.asarray(v, dtype=np.float64)
    N = v.shape[-1] - 1
    at = (2.0 / N) * dct1_paper(v[..., ::-1])
    a = at.copy()
    a[..., 0] *= 0.5
    a[..., N] *= 0.5
    return a


def fasta2v(a):
    """Fasta2v (boxed algorithm after Eq. coeff2v-1): double the ends, DCT-I, reverse."""
    a = np.asarray(a, dtype=np.float64).copy()
    N = a.shape[-1] - 1
    a[..., 0] *= 2.0
    a[..., N] *= 2.0
    return dct1_paper(a)[..., ::-1].copy()


def integration_coeffs(a):
    """c_0..c_{N+1} of Eq. c_k=bydef from the Chebyshev coefficients a_0..a_N (needs N >= 2)."""
    a = np.asarray(a, dtype=np.float64)
    N = a.shape[-1] - 1
    c = np.zeros(a.shape[:-1] + (N + 2,))
    k = np.arange(2, N + 1, dtype=np.float64)
    sgn = np.where(np.arange(2, N + 1) % 2 == 0, 1.0, -1.0)
    c[..., 0] = a[..., 0] - a[..., 1] / 4.0 - (a[..., 2:] * (sgn / (k * k - 1.0))).sum(axis=-1)
    c[..., 1] = a[..., 0] - a[..., 2] / 2.0
    kk = np.arange(2, N, dtype=np.float64)
    c[..., 2:N] = (a[..., 1:N - 1] - a[..., 3:N + 1]) / (2.0 * kk)
    c[..., N] = a[..., N - 1] / (2.0 * N)
    c[..., N + 1] = a[..., N] / (2.0 * (N + 1))
    return c


def alias_fold(c):
    """c-hat of Eq. chatk=: drop c_{N+1} onto c_{N-1} (T_{N+1} = T_{N-1} on the CGL grid, App. C)."""
    c = np.asarray(c, dtype=np.float64)
    N = c.shape[-1] - 2
    ch = c[..., :N + 1].copy()
    ch[..., N - 1] += c[..., N + 1]
    return ch


def fastbv(v, t0=-1.0, tf=1.0):
    """FastBV: B v = s * Fasta2v(c-hat(Fastv2a(v))), the three boxed steps in order."""
    s = 0.5 * (tf - t0)
    return s * fasta2v(alias_fold(integration_coeffs(fastv2a(v))))


def fastbv_T(u, t0=-1.0, tf=1.0):
    """B^T u, the adjoint of the FastBV chain taken step by step in reverse order.

    Reading: the paper has no transpose product; the KKT operator needs one. Each step of
    fastbv is a linear map; its transpose is written out here:
      Fasta2v = Rev * D * E2          ->  transpose  E2 * D^T * Rev
      c-hat   = Fold * Integrate      ->  transpose  Integrate^T * Fold^T
      Fastv2a = H * (2/N) D * Rev     ->  transpose  Rev * (2/N) D^T * H
    where D is the paper's DCT-I matrix D_jk = cos(jk pi/N) * (1/2 if k in {0, N} else 1),
    so D^T x = D (Q x) with Q = diag(2 at the ends, 1 inside) and a final halving at the ends.
    """
    u = np.asarray(u, dtype=np.float64)
    N = u.shape[-1] - 1
    s = 0.5 * (tf - t0)

    def dct_T(x):
        y = x.copy()
        y[..., 0] *= 2.0
        y[..., N] *= 2.0
        z = dct1_paper(y)
        z[..., 0] *= 0.5
        z[..., N] *= 0.5
        return z

    # transpose of Fasta2v
    g = dct_T(u[..., ::-1].copy())
    g[..., 0] *= 2.0
    g[..., N] *= 2.0
    # transpose of the alias fold: (N+2)-vector with c_{N+1} receiving the (N-1) entry
    cT = np.zeros(u.shape[:-1] + (N + 2,))
    cT[..., :N + 1] = g
    cT[..., N + 1] = g[..., N - 1]
    # transpose of integration_coeffs: a_j = sum_k C_kj cT_k
    a = np.zeros(u.shape[:-1] + (N + 1,))
    k = np.arange(2, N + 1, dtype=np.float64)
    sgn = np.where(np.arange(2, N + 1) % 2 == 0, 1.0, -1.0)
    a[..., 0] += cT[..., 0] + cT[..., 1]
    a[..., 1] += -cT[..., 0] / 4.0
    a[..., 2:] += -cT[..., 0:1] * (sgn / (k * k - 1.0))
    a[..., 2] += -cT[..., 1] / 2.0
    kk = np.arange(2, N, dtype=np.float64)
    a[..., 1:N - 1] += cT[..., 2:N] / (2.0 * kk)
    a[..., 3:N + 1] += -cT[..., 2:N] / (2.0 * kk)
    a[..., N - 1] += cT[..., N] / (2.0 * N)
    a[..., N] += cT[..., N + 1] / (2.0 * (N + 1))
    # transpose of Fastv2a
    a[..., 0] *= 0.5
    a[..., N] *= 0.5
    out = (2.0 / N) * dct_T(a)
    return s * out[..., ::-1].copy()


# --------------------------------------------------------------------------------------------
# Closed forms: integrals of Chebyshev polynomials at the CGL nodes
# --------------------------------------------------------------------------------------------
def _cos_pi_int_over(r, N):
    """cos(pi r / N) for integer r, reducing r mod 2N exactly first."""
    r = np.mod(np.asarray(r, dtype=np.int64), 2 * N)
    return np.cos(np.pi * r.astype(np.float64) / N)


def cheb_T_at_nodes(k, N):
    """T_k(tau_j), j = 0..N, as cos(k (N - j) pi / N) (Eq. Tkj=coskj), exact integer reduction."""
    j = np.arange(N + 1, dtype=np.int64)
    return _cos_pi_int_over(int(k) * (N - j), N)


def cheb_integral_at_nodes(k, N):
    """int_{-1}^{tau_j} T_k(xi) dxi at every CGL node, from Eq. intChebPoly= (textbook calculus)."""
    k = int(k)
    T = lambda m: cheb_T_at_nodes(m, N)
    if k == 0:
        return T(1) + T(0)
    if k == 1:
        return T(2) / 4.0 - T(0) / 4.0
    sgn = 1.0 if k % 2 == 0 else -1.0
    return T(k + 1) / (2.0 * (k + 1)) - T(k - 1) / (2.0 * (k - 1)) - sgn * T(0) / (k * k - 1.0)


def sparse_mode_pair(N, modes, alphas, t0=-1.0, tf=1.0):
    """(v, B v) for v = sum_k alpha_k T_k sampled at the CGL nodes, any N, O(|modes| * N).

    B v is exact here: v is a polynomial of degree <= N, so it equals its own interpolant and
    the Birkhoff product is its exact integral from t_0 (Eqs. BVt-1, intChebPoly=).
    """
    s = 0.5 * (tf - t0)
    v = np.zeros(N + 1)
    Bv = np.zeros(N + 1)
    for k, a in zip(modes, alphas):
        v += a * cheb_T_at_nodes(k, N)
        Bv += a * cheb_integral_at_nodes(k, N)
    return v, s * Bv


# --------------------------------------------------------------------------------------------
# B-tilde and the O(N) sweeps of the preconditioner
# --------------------------------------------------------------------------------------------
def dense_Btilde(w):
    """[B-tilde^a]_ij = 0 (i < j), w_j / 2 (i = j), w_j (i > j) (definition after Eq. Ba=10)."""
    w = np.asarray(w, dtype=np.float64)
    L = w.shape[0]
    Bt = np.tril(np.tile(w, (L, 1)), -1)
    Bt[np.diag_indices(L)] = 0.5 * w
    return Bt


def fastbccv(w, v):
    """FastBccV as printed: xi_k = w_k v_k / 2 + s, then s <- 2 xi_k - s. Returns B-tilde v."""
    out = np.zeros(len(v))
    s = 0.0
    for k in range(len(v)):
        xi = w[k] * v[k] / 2.0 + s
        s = 2.0 * xi - s
        out[k] = xi
    return out


def fastpinvy_scalar(w, d, Y):
    """P^{-1} Y for P = I - B-tilde diag(d) by forward substitution.

    Reading: the sweep as printed (xi_k = (1 - w_k d_k/2)^{-1}(Y_k - s), s <- w_k d_k Y_k + s)
    does not invert P. Writing row k of P xi = Y out gives
      xi_k - sum_{j<k} w_j d_j xi_j - (w_k d_k / 2) xi_k = Y_k,
    so xi_k = (1 - w_k d_k / 2)^{-1} (Y_k + s) with s <- s + w_k d_k xi_k.
    """
    out = np.zeros(len(Y))
    s = 0.0
    for k in range(len(Y)):
        xi = (Y[k] + s) / (1.0 - w[k] * d[k] / 2.0)
        s = s + w[k] * d[k] * xi
        out[k] = xi
    return out


def fastpinvy_block(w, J, Y):
    """P^{-1} Y for P = I - (B-tilde kron I) blockdiag(J_k) (vector state, one n x n block per node).

    Reading: the paper's scalar state has a diagonal d/dX f; for n_x > 1 each node carries an
    n_x x n_x Jacobian block and B-tilde acts on every component. Row k of P xi = Y gives
    (I - w_k J_k / 2) xi_k = Y_k + sigma_k with sigma_k = sum_{j<k} w_j J_j xi_j.
    J has shape (L, n, n); Y and the result have shape (n, L) (component-major).
    """
    L, n, _ = J.shape
    out = np.zeros((n, L))
    sig = np.zeros(n)
    I = np.eye(n)
    for k in range(L):
        xi = np.linalg.solve(I - 0.5 * w[k] * J[k], Y[:, k] + sig)
        sig = sig + w[k] * (J[k] @ xi)
        out[:, k] = xi
    return out


def fastpinvy_block_T(w, J, R):
    """P^{-T} R for the same P: the backward sweep obtained by transposing the rows of P.

    Column j of P^T y = r reads y_j - J_j^T w_j (y_j / 2 + rho_j) = r_j with
    rho_j = sum_{k>j} y_k, so (I - w_j J_j^T / 2) y_j = r_j + w_j J_j^T rho_j.
    """
    L, n, _ = J.shape
    out = np.zeros((n, L))
    rho = np.zeros(n)
    I = np.eye(n)
    for j in range(L - 1, -1, -1):
        y = np.linalg.solve(I - 0.5 * w[j] * J[j].T, R[:, j] + w[j] * (J[j].T @ rho))
        rho = rho + y
        out[:, j] = y
    return out
