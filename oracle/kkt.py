"""Dense KKT of the a-form Birkhoff discretisation and a Newton-Lagrange driver (oracle).

Test infrastructure only. The discretisation is Eq. Prob-PNa with V eliminated (V = f(X, U))
and the initial state fixed (x^a = x0):

    c(X, U) = X - x0 (x) 1 - s (I (x) B^a) f(X, U) = 0          (n_x * L rows)
    e(X)    = X[term_idx, N] - term_val = 0                     (n_e rows)
    J       = s * sum_i w_i F(x_i, u_i)                          (Clenshaw-Curtis quadrature)

Row N of c equals the x^b row of Eq. Prob-PNa because the last row of B^a is w^CC.
Reading (the paper does not describe its outer SQP loop): Newton's method on the KKT conditions
F(z, y) = [grad J + G^T y ; c ; e] = 0 with the exact Hessian of the Lagrangian, and a
backtracking line search (alpha = 1, 1/2, ...; Armijo constant 1e-4) on the quadrature-weighted
residual norm

    ||F||_W^2 = sum_i w_i |c_i|^2 + sum_i |g_i|^2 / w_i + |e|^2,

where g are the gradient rows (X and U) and w the Clenshaw-Curtis weights. It measures c in
L2 and the gradient in the dual norm, so it does not grow with N; with it the Newton counts are
the same for every N (the mesh independence of Table tab:m).

Vector layout (component-major, matching the library): z = [X_0..X_{n_x-1}, U_0..U_{n_u-1}],
y = [lambda_0..lambda_{n_x-1}, nu], each X_m, U_q, lambda_m a length-L block.
"""
import numpy as np

from .birkhoff import dense_Ba
from .grid import cgl_nodes


class DenseKKT:
    """Dense operators of one problem at one grid size N."""

    def __init__(self, prob, N, Ba=None):
        self.prob = prob
        self.N = N
        self.L = N + 1
        self.Ba = dense_Ba(N) if Ba is None else Ba
        self.w = self.Ba[N].copy()
        self.s = 0.5 * (prob.tf - prob.t0)
        self.tau = cgl_nodes(N)
        self.t = prob.t0 + self.s * (self.tau + 1.0)
        nx, nu, L = prob.n_x, prob.n_u, self.L
        self.nz = (nx + nu) * L
        self.nc = nx * L
        self.n = self.nz + self.nc + prob.n_e

    # ---- packing --------------------------------------------------------------------------
    def split(self, vec):
        p, L = self.prob, self.L
        X = vec[:p.n_x * L].reshape(p.n_x, L)
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        lam = vec[self.nz:self.nz + self.nc].reshape(p.n_x, L)
        nu = vec[self.nz + self.nc:]
        return X, U, lam, nu

    def pack(self, X, U, lam, nu):
        return np.concatenate([X.ravel(), U.ravel(), lam.ravel(), np.asarray(nu, float).ravel()])

    # ---- residual ---------------------------------------------------------------------------
    def residual(self, vec):
        """F = [grad_z L ; c ; e] at vec = (X, U, lambda, nu)."""
        p, s, B = self.prob, self.s, self.Ba
        X, U, lam, nu = self.split(vec)
        f = p.f(X, U)
        c = X - p.x0[:, None] - s * (B @ f.T).T
        e = p.terminal_residual(X)
        Jx, Ju = p.jac(X, U)
        mu = (B.T @ lam.T).T                       # mu_m = B^T lambda_m
        gX = lam - s * np.einsum('kmp,mk->pk', Jx, mu)
        gU = s * self.w[None, :] * p.cost_grad_u(U) - s * np.einsum('kmq,mk->qk', Ju, mu)
        for r, (i, _) in enumerate(zip(p.term_idx, p.term_val)):
            gX[i, -1] += nu[r]
        return np.concatenate([gX.ravel(), gU.ravel(), c.ravel(), e])

    # ---- Jacobian of F (the KKT matrix) ---------------------------------------------------
    def matrix(self, vec):
        p, s, B, L = self.prob, self.s, self.Ba, self.L
        nx, nu_ = p.n_x, p.n_u
        X, U, lam, nu = self.split(vec)
        Jx, Ju = p.jac(X, U)
        mu = (B.T @ lam.T).T
        Hn = -s * p.hess_f(X, U, mu)              # (L, nx+nu, nx+nu)
        for q in range(nu_):
            Hn[:, nx + q, nx + q] += s * self.w * p.cost_hess_uu()
        H = np.zeros((self.nz, self.nz))
        nvar = nx + nu_
        for a in range(nvar):
            for b in range(nvar):
                H[a * L:(a + 1) * L, b * L:(b + 1) * L] = np.diag(Hn[:, a, b])
        G = np.zeros((self.nc, self.nz))
        for m in range(nx):
            for q in range(nx):
                blk = -s * B * Jx[:, m, q][None, :]
                if m == q:
                    blk = blk + np.eye(L)
                G[m * L:(m + 1) * L, q * L:(q + 1) * L] = blk
            for q in range(nu_):
                G[m * L:(m + 1) * L, (nx + q) * L:(nx + q + 1) * L] = -s * B * Ju[:, m, q][None, :]
        Ge = np.zeros((p.n_e, self.nz))
        for r, i in enumerate(p.term_idx):
            Ge[r, i * L + L - 1] = 1.0
        A = np.vstack([G, Ge])
        K = np.zeros((self.n, self.n))
        K[:self.nz, :self.nz] = H
        K[:self.nz, self.nz:] = A.T
        K[self.nz:, :self.nz] = A
        return K

    def apply(self, vec, dvec):
        """KKT matrix at vec times dvec (dense)."""
        return self.matrix(vec) @ dvec

    # ---- merit ----------------------------------------------------------------------------
    def weighted_norm(self, F):
        """||F||_W (see the module docstring)."""
        p, L, w = self.prob, self.L, self.w
        gX = F[:p.n_x * L].reshape(p.n_x, L)
        gU = F[p.n_x * L:self.nz].reshape(p.n_u, L)
        c = F[self.nz:self.nz + self.nc].reshape(p.n_x, L)
        e = F[self.nz + self.nc:]
        return float(np.sqrt((w * c * c).sum() + (gX * gX / w).sum() + (gU * gU / w).sum()
                             + (e * e).sum()))

    # ---- Newton-Lagrange ------------------------------------------------------------------
    def newton(self, vec0, tol=1e-10, max_iter=30, armijo=1e-4, max_backtrack=30):
        """Newton's method on F(z, y) = 0 with backtracking on ||F||_W; stops at ||F||_W <= tol.

        Returns (vec, info) with info = dict(iters, alphas, norms, converged).
        """
        vec = np.array(vec0, dtype=np.float64)
        F = self.residual(vec)
        norms = [self.weighted_norm(F)]
        alphas = []
        it = 0
        while norms[-1] > tol and it < max_iter:
            d = np.linalg.solve(self.matrix(vec), -F)
            alpha = 1.0
            f0 = norms[-1]
            for _ in range(max_backtrack):
                trial = vec + alpha * d
                Ft = self.residual(trial)
                if self.weighted_norm(Ft) <= (1.0 - armijo * alpha) * f0:
                    break
                alpha *= 0.5
            vec, F = trial, Ft
            alphas.append(alpha)
            norms.append(self.weighted_norm(F))
            it += 1
        return vec, dict(iters=it, alphas=alphas, norms=norms, converged=bool(norms[-1] <= tol))

    # ---- the Birkhoff KKT preconditioner (dense definition) -------------------------------
    def precond_matrix(self, vec):
        """K-tilde: the KKT matrix with B^a -> B-tilde^a in the constraint Jacobian and the
        Hessian kept only in its cost part on the controls (s w_i grad_uu F).

            [ 0      0      P^T    E^T ]
            [ 0      Huu    Pu^T   0   ]      P  = I - s (B-tilde (x) I) J_x
            [ P      Pu     0      0   ]      Pu =   - s (B-tilde (x) I) J_u
            [ E      0      0      0   ]

        Reading: the paper preconditions the state system I - B^a d_X f by P = I - B-tilde d_X f
        (Section "Development of a Special Birkhoff-Centric Preconditioner"); for the full KKT
        system of the Newton step the same substitution is made in the constraint block and
        the Lagrangian Hessian is replaced by its control-cost part, which is SPD. The
        preconditioner applied by the library is K-tilde^{-1}.
        """
        from .birkhoff import dense_Btilde
        p, s, L = self.prob, self.s, self.L
        nx, nu_ = p.n_x, p.n_u
        X, U, lam, nu = self.split(vec)
        Jx, Ju = p.jac(X, U)
        Bt = dense_Btilde(self.w)
        P = np.zeros((self.nc, self.nc))
        Pu = np.zeros((self.nc, nu_ * L))
        for m in range(nx):
            for q in range(nx):
                blk = -s * Bt * Jx[:, m, q][None, :]
                if m == q:
                    blk = blk + np.eye(L)
                P[m * L:(m + 1) * L, q * L:(q + 1) * L] = blk
            for q in range(nu_):
                Pu[m * L:(m + 1) * L, q * L:(q + 1) * L] = -s * Bt * Ju[:, m, q][None, :]
        Huu = np.diag(np.tile(s * self.w * p.cost_hess_uu(), nu_))
        E = np.zeros((p.n_e, self.nc))
        for r, i in enumerate(p.term_idx):
            E[r, i * L + L - 1] = 1.0
        nz, nc, ne = self.nz, self.nc, p.n_e
        Kt = np.zeros((self.n, self.n))
        xs, us, ls, es = slice(0, nc), slice(nc, nz), slice(nz, nz + nc), slice(nz + nc, self.n)
        Kt[xs, ls] = P.T
        Kt[xs, es] = E.T
        Kt[us, us] = Huu
        Kt[us, ls] = Pu.T
        Kt[ls, xs] = P
        Kt[ls, us] = Pu
        Kt[es, xs] = E
        return Kt

    def state_matrix(self, vec):
        """G_x = I - s (B^a (x) I) J_x: the state block of the constraint Jacobian."""
        return self.matrix(vec)[self.nz:self.nz + self.nc, :self.nc]

    def state_precond_matrix(self, vec):
        """P = I - s (B-tilde (x) I) J_x: the Birkhoff preconditioner of the state block."""
        return self.precond_matrix(vec)[self.nz:self.nz + self.nc, :self.nc]


def state_operator(Ba, s, d):
    """A = I - s B^a diag(d): the matrix of Eq. Newton-ivp / Eq. Achibetadef (scalar state)."""
    L = Ba.shape[0]
    return np.eye(L) - s * Ba * np.asarray(d)[None, :]


def preconditioner_matrix(w, s, d):
    """P = I - s B-tilde diag(d) (definition of the Birkhoff preconditioner, scalar state)."""
    from .birkhoff import dense_Btilde
    L = len(w)
    return np.eye(L) - s * dense_Btilde(w) * np.asarray(d)[None, :]
