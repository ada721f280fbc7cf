"""CGL grid, Lagrange basis and Clenshaw-Curtis weights (oracle; test infrastructure only).

Paper: Eq. CGLpts (nodes), Eq. manyDefs (w_B = Clenshaw-Curtis weights), the remark after
Eq. Ba=10 (the last row of B^a equals the Clenshaw-Curtis weights).
"""
import numpy as np


def cgl_nodes(N):
    """tau_j = -cos(j*pi/N), j = 0..N, ascending from -1 to 1 (Eq. CGLpts).

    Evaluated as sin(pi*(2j-N)/(2N)), which is the same number and is exactly antisymmetric
    about the midpoint.
    """
    j = np.arange(N + 1, dtype=np.float64)
    return np.sin(np.pi * (2.0 * j - N) / (2.0 * N))


def bary_weights(N):
    """Barycentric weights of the CGL nodes: (-1)^j, halved at both ends (Berrut & Trefethen 2004)."""
    lam = np.where(np.arange(N + 1) % 2 == 0, 1.0, -1.0)
    lam[0] *= 0.5
    lam[N] *= 0.5
    return lam


def lagrange_matrix(N, xi):
    """Values l_j(xi_q) of all N+1 Lagrange basis polynomials on the CGL nodes at points xi.

    Returns an array of shape (len(xi), N+1). Second (true) barycentric formula; points that
    coincide with a node get the exact Kronecker row.
    """
    tau = cgl_nodes(N)
    lam = bary_weights(N)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    diff = xi[:, None] - tau[None, :]
    hit = diff == 0.0
    diff[hit] = 1.0
    t = lam[None, :] / diff
    out = t / t.sum(axis=1, keepdims=True)
    rows = hit.any(axis=1)
    if rows.any():
        out[rows] = hit[rows].astype(np.float64)
    return out


def cc_weights_sum(N):
    """Clenshaw-Curtis weights w_j = int_{-1}^{1} l_j(tau) dtau by the cosine-sum closed form.

    Expand l_j in Chebyshev polynomials with the discrete orthogonality of T_k on the CGL
    nodes (the coefficient formula of Eq. ak=3 applied to the unit vector e_j), then integrate
    term by term with int_{-1}^{1} T_k = (1 + (-1)^k) / (1 - k^2). O(N^2); the plain
    definition, not a fast algorithm.
    """
    k = np.arange(N + 1)
    j = np.arange(N + 1)
    # T_k(tau_j) = cos(k (N - j) pi / N); reduce k (N - j) mod 2N exactly in integers.
    r = np.mod(np.outer(N - j, k), 2 * N)
    Tkj = np.cos(np.pi * r / N)                      # [j, k]
    kf = k.astype(np.float64)
    intT = np.zeros(N + 1)
    ev = k % 2 == 0
    intT[ev] = 2.0 / (1.0 - kf[ev] ** 2)
    hk = np.ones(N + 1); hk[0] = 0.5; hk[N] = 0.5    # coefficient halving at k = 0, N
    vj = np.ones(N + 1); vj[0] = 0.5; vj[N] = 0.5    # endpoint halving of the nodal sum
    return (2.0 / N) * vj * (Tkj * (hk * intT)[None, :]).sum(axis=1)


def interpolate(values, N, xi, chunk=8192):
    """Values at the points xi of the degree-N interpolant through `values` on the CGL nodes of
    size N (last axis), by the barycentric formula of ``lagrange_matrix``; xi is processed in
    chunks so that large targets fit in memory."""
    values = np.asarray(values, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.empty(values.shape[:-1] + (xi.size,))
    for a in range(0, xi.size, chunk):
        Lm = lagrange_matrix(N, xi[a:a + chunk])
        out[..., a:a + chunk] = values @ Lm.T
    return out
