"""Problem kinds: dynamics f, Jacobians and Hessians (oracle; test infrastructure only).

Each kind fixes n_x, n_u, the dynamics x' = f(x, u) of Eq. probPbold / Eq. probP, the running
cost F and the endpoint conditions. All arrays are component-major: X has shape (n_x, L),
U has shape (n_u, L); per-node Jacobians have shape (L, n_x, n_x) and (L, n_x, n_u).

Kinds
-----
DBL_INT   x = (p, v), x' = (v, u); x(t0) = (0, 0), x(tf) = (1, 0); F = u^2 / 2.
          (Minimum-energy double integrator; reading: the cost is u^2/2 so that its Hessian is
          the identity; it has the same minimiser as int u^2.)
ORBIT     x = (r, theta, v_r, v_theta), u = (u_r, u_theta) thrust acceleration vector:
            r' = v_r, theta' = v_theta / r,
            v_r' = v_theta^2 / r - 1 / r^2 + u_r,  v_theta' = -v_r v_theta / r + u_theta
          (the dynamics of Eq. ot, state reordered, with the thrust a (sin u, cos u) written
          as a free vector); x(t0) = (1, 0, 0, 1); terminal r = r_f, v_r = 0,
          v_theta = 1/sqrt(r_f), theta free; F = |u|^2 / 2 (minimum-energy transfer).
          Reading: the fixed-final-time variant has no objective in the paper. With a
          fixed-magnitude steering angle, every running cost of the angle alone is degenerate
          at second order against the energy the thrust must shed, so the thrust vector is the
          control; the nominal acceleration a (params[0]) seeds the initial guess only.
BILINEAR  scalar x' = u * x with no cost and no terminal condition. Linearised at (X, U) its
          state Jacobian is diag(U), so setting U = d gives the Newton system
          [I - s B diag(d)] dX = x^a b of Eq. Newton-ivp (the paper's linear-solve experiment).
ORBIT_MT  the minimum-time orbit transfer of Eq. ot: the same state and dynamics with the
          fixed-magnitude thrust a (sin u, cos u), u the steering angle (n_u = 1), cost
          J = T = t_f - t_0 (the final time is free: s = T / 2 is one more unknown),
          x(t0) = (1, 0, 0, 1), terminal r = r_f, v_r = 0, v_theta = 1/sqrt(r_f), theta free.
          Eq. ot orders the state (r, v_r, v_theta, theta); the library keeps (r, theta, v_r,
          v_theta) for both orbit kinds. Reading: the paper does not give a; params = (a, r_f),
          with a = 0.05 and r_f = 6 (the paper's target) as the worked case. The time tf given
          to the problem is only the initial value of the free final time.
"""
import numpy as np

DBL_INT, ORBIT, BILINEAR, ORBIT_MT = 0, 1, 2, 3


class Problem:
    """Plain description of one problem instance."""

    def __init__(self, kind, t0, tf, params=()):
        self.kind = kind
        self.t0 = float(t0)
        self.tf = float(tf)
        self.params = tuple(float(p) for p in params)
        self.free_time = kind == ORBIT_MT
        if kind == DBL_INT:
            self.n_x, self.n_u = 2, 1
            self.x0 = np.array([0.0, 0.0])
            self.term_idx = [0, 1]
            self.term_val = [1.0, 0.0]
            self.has_cost = True
        elif kind == ORBIT:
            a, rf = self.params
            self.a, self.rf = a, rf
            self.n_x, self.n_u = 4, 2
            self.x0 = np.array([1.0, 0.0, 0.0, 1.0])
            self.term_idx = [0, 2, 3]
            self.term_val = [rf, 0.0, 1.0 / np.sqrt(rf)]
            self.has_cost = True
        elif kind == ORBIT_MT:
            a, rf = self.params
            self.a, self.rf = a, rf
            self.n_x, self.n_u = 4, 1
            self.x0 = np.array([1.0, 0.0, 0.0, 1.0])
            self.term_idx = [0, 2, 3]
            self.term_val = [rf, 0.0, 1.0 / np.sqrt(rf)]
            self.has_cost = True
        elif kind == BILINEAR:
            self.n_x, self.n_u = 1, 1
            self.x0 = np.array([self.params[0] if self.params else 1.0])
            self.term_idx = []
            self.term_val = []
            self.has_cost = False
        else:
            raise ValueError("unknown problem kind")
        self.n_e = len(self.term_idx)

    # ---- dynamics -----------------------------------------------------------------------
    def f(self, X, U):
        if self.kind == DBL_INT:
            return np.stack([X[1], U[0]])
        if self.kind == ORBIT:
            r, th, vr, vt = X
            return np.stack([vr, vt / r, vt * vt / r - 1.0 / (r * r) + U[0],
                             -vr * vt / r + U[1]])
        if self.kind == ORBIT_MT:
            r, th, vr, vt = X
            u = U[0]
            return np.stack([vr, vt / r, vt * vt / r - 1.0 / (r * r) + self.a * np.sin(u),
                             -vr * vt / r + self.a * np.cos(u)])
        return (U[0] * X[0])[None, :]

    def jac(self, X, U):
        """(J_x, J_u): per-node d f / d x (L, n_x, n_x) and d f / d u (L, n_x, n_u)."""
        L = X.shape[1]
        Jx = np.zeros((L, self.n_x, self.n_x))
        Ju = np.zeros((L, self.n_x, self.n_u))
        if self.kind == DBL_INT:
            Jx[:, 0, 1] = 1.0
            Ju[:, 1, 0] = 1.0
        elif self.kind in (ORBIT, ORBIT_MT):
            r, th, vr, vt = X
            Jx[:, 0, 2] = 1.0
            Jx[:, 1, 0] = -vt / r**2
            Jx[:, 1, 3] = 1.0 / r
            Jx[:, 2, 0] = -vt * vt / r**2 + 2.0 / r**3
            Jx[:, 2, 3] = 2.0 * vt / r
            Jx[:, 3, 0] = vr * vt / r**2
            Jx[:, 3, 2] = -vt / r
            Jx[:, 3, 3] = -vr / r
            if self.kind == ORBIT:
                Ju[:, 2, 0] = 1.0
                Ju[:, 3, 1] = 1.0
            else:
                Ju[:, 2, 0] = self.a * np.cos(U[0])
                Ju[:, 3, 0] = -self.a * np.sin(U[0])
        else:
            Jx[:, 0, 0] = U[0]
            Ju[:, 0, 0] = X[0]
        return Jx, Ju

    def hess_f(self, X, U, mu):
        """sum_m mu[m, k] * Hessian of f_m w.r.t. (x, u) at node k: shape (L, n, n), n = n_x + n_u."""
        L = X.shape[1]
        n = self.n_x + self.n_u
        H = np.zeros((L, n, n))
        if self.kind == DBL_INT:
            return H
        if self.kind in (ORBIT, ORBIT_MT):
            r, th, vr, vt = X
            m_th, m_vr, m_vt = mu[1], mu[2], mu[3]
            R, VR, VT = 0, 2, 3
            # f_theta = vt / r
            H[:, R, R] += m_th * 2.0 * vt / r**3
            H[:, R, VT] += m_th * (-1.0 / r**2)
            # f_vr = vt^2 / r - 1 / r^2 + a sin u
            H[:, R, R] += m_vr * (2.0 * vt * vt / r**3 - 6.0 / r**4)
            H[:, R, VT] += m_vr * (-2.0 * vt / r**2)
            H[:, VT, VT] += m_vr * (2.0 / r)
            # f_vt = -vr vt / r + a cos u
            H[:, R, R] += m_vt * (-2.0 * vr * vt / r**3)
            H[:, R, VR] += m_vt * (vt / r**2)
            H[:, R, VT] += m_vt * (vr / r**2)
            H[:, VR, VT] += m_vt * (-1.0 / r)
            # symmetrise the off-diagonal entries written above the diagonal
            for (i, j) in [(R, VT), (R, VR), (VR, VT)]:
                H[:, j, i] = H[:, i, j]
            if self.kind == ORBIT_MT:
                # a sin u and a cos u: second derivatives -a sin u, -a cos u in the angle
                u = U[0]
                H[:, 4, 4] = -self.a * (m_vr * np.sin(u) + m_vt * np.cos(u))
            return H
        # BILINEAR: f = u x
        H[:, 0, 1] = mu[0]
        H[:, 1, 0] = mu[0]
        return H

    # ---- running cost F(x, u) = |u|^2 / 2 (none for ORBIT_MT, whose cost is T) ----------------
    def running_cost(self):
        return self.has_cost and not self.free_time

    def cost_grad_u(self, U):
        return U.copy() if self.running_cost() else np.zeros_like(U)

    def cost_hess_uu(self):
        return 1.0 if self.running_cost() else 0.0

    def terminal_residual(self, X):
        return np.array([X[i, -1] - v for i, v in zip(self.term_idx, self.term_val)])


def linear_initial_guess(prob, tau):
    """Initial guess for DBL_INT: boundary states joined linearly, u = 0."""
    lam = 0.5 * (tau + 1.0)
    xf = np.array(prob.term_val)
    X = prob.x0[:, None] * (1.0 - lam)[None, :] + xf[:, None] * lam[None, :]
    U = np.zeros((prob.n_u, len(tau)))
    return X, U
