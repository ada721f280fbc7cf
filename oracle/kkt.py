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

Free final time (ORBIT_MT, Eq. ot). The time scale s = (t_f - t_0)/2 is one more unknown, stored
after nu: vec = [X, U, lambda, nu, s]. The cost is J = t_f - t_0 = 2 s, so the Lagrangian
2 s + lambda . c + nu . e has the extra gradient row

    g_s = dL/ds = 2 - lambda . (B^a (x) I) f(X, U),

and the KKT matrix gains one row and column: d g_X / ds = -J_x^T (B^aT lambda),
d g_U / ds = -J_u^T (B^aT lambda), d c / ds = -(B^a (x) I) f, zero against nu and s. The
weighted norm adds |g_s|^2.
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
        self.free = bool(getattr(prob, 'free_time', False))
        self.n = self.nz + self.nc + prob.n_e + (1 if self.free else 0)

    # ---- packing --------------------------------------------------------------------------
    def split(self, vec):
        p, L = self.prob, self.L
        X = vec[:p.n_x * L].reshape(p.n_x, L)
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        lam = vec[self.nz:self.nz + self.nc].reshape(p.n_x, L)
        nu = vec[self.nz + self.nc:self.nz + self.nc + p.n_e]
        return X, U, lam, nu

    def s_of(self, vec):
        """Time scale at vec: the last entry for a free final time, else (t_f - t_0)/2."""
        return float(vec[-1]) if self.free else self.s

    def pack(self, X, U, lam, nu, s=None):
        parts = [X.ravel(), U.ravel(), lam.ravel(), np.asarray(nu, float).ravel()]
        if self.free:
            parts.append([self.s if s is None else float(s)])
        return np.concatenate(parts)

    def border(self, vec):
        """Free final time: the KKT matrix's s column, [d g_X/ds ; d g_U/ds ; d c/ds ; 0 ; 0]."""
        p, B = self.prob, self.Ba
        X, U, lam, nu = self.split(vec)
        Jx, Ju = p.jac(X, U)
        muh = (B.T @ lam.T).T                      # B^aT lambda, unscaled
        col = np.zeros(self.n)
        col[:p.n_x * self.L] = -np.einsum('kmp,mk->pk', Jx, muh).ravel()
        col[p.n_x * self.L:self.nz] = -np.einsum('kmq,mk->qk', Ju, muh).ravel()
        col[self.nz:self.nz + self.nc] = -(B @ p.f(X, U).T).T.ravel()
        return col

    # ---- residual ---------------------------------------------------------------------------
    def residual(self, vec):
        """F = [grad_z L ; c ; e] at vec = (X, U, lambda, nu)."""
        p, s, B = self.prob, self.s_of(vec), self.Ba
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
        tail = [e]
        if self.free:
            tail.append([2.0 - float(np.sum(lam * (B @ f.T).T))])
        return np.concatenate([gX.ravel(), gU.ravel(), c.ravel()] + tail)

    # ---- Jacobian of F (the KKT matrix) ---------------------------------------------------
    def matrix(self, vec):
        p, s, B, L = self.prob, self.s_of(vec), self.Ba, self.L
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
        ny = self.nc + p.n_e
        K[:self.nz, :self.nz] = H
        K[:self.nz, self.nz:self.nz + ny] = A.T
        K[self.nz:self.nz + ny, :self.nz] = A
        if self.free:
            col = self.border(vec)
            K[:, -1] = col
            K[-1, :] = col
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
        e = F[self.nz + self.nc:]                  # e, and g_s for a free final time
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
            accepted = False
            for _ in range(max_backtrack):
                trial = vec + alpha * d
                # a free final time must stay positive: a trial with s <= 0 is rejected
                if self.s_of(trial) > 0.0:
                    Ft = self.residual(trial)
                    if self.weighted_norm(Ft) <= (1.0 - armijo * alpha) * f0:
                        accepted = True
                        break
                alpha *= 0.5
            if not accepted:
                break                                   # line search failed: stop here
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

        Free final time (ORBIT_MT, no running cost): Huu is the per-node bound
        a |mu_v,k| + 1e-3 s w_k of the angle's Lagrangian curvature a (mu_vr sin u + mu_vt cos u),
        mu = s B^aT lambda (the two agree where the angle is stationary; the floor keeps Huu
        positive where mu_v vanishes), and K-tilde is bordered by the KKT matrix's own s row and
        column (zero diagonal), so that the preconditioner eliminates s exactly.
        """
        from .birkhoff import dense_Btilde
        p, s, L = self.prob, self.s_of(vec), self.L
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
        if self.free:
            mu = s * (self.Ba.T @ lam.T).T
            Huu = np.diag(p.a * np.hypot(mu[2], mu[3]) + 1e-3 * s * self.w)
        else:
            Huu = np.diag(np.tile(s * self.w * p.cost_hess_uu(), nu_))
        E = np.zeros((p.n_e, self.nc))
        for r, i in enumerate(p.term_idx):
            E[r, i * L + L - 1] = 1.0
        nz, nc, ne = self.nz, self.nc, p.n_e
        Kt = np.zeros((self.n, self.n))
        xs, us, ls, es = slice(0, nc), slice(nc, nz), slice(nz, nz + nc), slice(nz + nc, nz + nc + ne)
        Kt[xs, ls] = P.T
        Kt[xs, es] = E.T
        Kt[us, us] = Huu
        Kt[us, ls] = Pu.T
        Kt[ls, xs] = P
        Kt[ls, us] = Pu
        Kt[es, xs] = E
        if self.free:
            col = self.border(vec)
            Kt[:, -1] = col
            Kt[-1, :] = col
        return Kt

    def min_time_seed(self, K_me, vec_me):
        """Initial point of a free-final-time orbit solve from a solved minimum-energy transfer.

        K_me is the DenseKKT of the ORBIT problem (same N, a, r_f) at a fixed t_f and vec_me its
        solution. The states and multipliers are kept, the steering angle is the direction of
        the thrust vector, u = atan2(u_r, u_theta) (thrust a (sin u, cos u)), s is K_me's, and
        lambda, nu are scaled by kappa = 2 / (lambda . (B^a (x) I) f) so that g_s = 0. Reading:
        the paper does not say how its solve is started; the minimum-energy solution has the
        same stationarity structure (thrust along B^aT lambda), so only the scale of the
        multipliers must change.
        """
        assert self.free and K_me.N == self.N
        X, U, lam, nu = K_me.split(vec_me)
        Um = np.arctan2(U[0], U[1])[None, :]
        vec = self.pack(X.copy(), Um, lam.copy(), nu.copy(), K_me.s)
        S = 2.0 - self.residual(vec)[-1]           # lambda . (B^a (x) I) f at the seed
        if not S > 0.0:
            raise ValueError("minimum-energy multipliers give a non-positive time gradient")
        kappa = 2.0 / S
        vec[self.nz:self.n - 1] *= kappa
        return vec

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
