"""Control bounds by a logarithmic barrier (oracle). Test infrastructure only.

The general problem (P) of the paper (Eq. probPbold) carries path constraints h(x, u, t) <= 0,
which the paper states but gives no method for (its solver treats the equality-constrained
Prob-PNa). This module adds the simplest path constraints, constant bounds on each control,

    l_q <= u_q(t) <= h_q        (one pair per control component; +-inf: no bound),

to the a-form discretisation of DenseKKT by a primal logarithmic barrier on the quadrature of
the constraint over time (Fiacco and McCormick's barrier method, in the primal form of Nocedal
and Wright, Numerical Optimization, 2nd ed., Section 19.6):

    J_mu = J - mu * s * sum_i w_i sum_q [ log(u_qi - l_q) + log(h_q - u_qi) ].

The quadrature weight keeps the barrier a discretisation of mu * integral log(...) dt, so the
barrier problem, like the unbounded one, does not change with N. Its KKT conditions are those of
DenseKKT with, in the gradient rows of U,

    g_U += -mu s w_i (1 / (u - l) - 1 / (h - u)),

and in the control block of the Hessian the diagonal mu s w_i (1 / (u - l)^2 + 1 / (h - u)^2).
The outer loop solves the barrier problem by the Newton-Lagrange iteration for a decreasing
sequence mu_0, mu_0 / 10, ... down to mu_final, the intermediate stages to ||F_mu||_W <=
max(tol, 10 mu) and the last to tol, and keeps the controls strictly inside their bounds by the
fraction-to-boundary rule: the step length starts at min(1, 0.995 * max{alpha : l < u + alpha du
< h}). The barrier solution lies O(mu) from the bounded optimum; the barrier Hessian of an
active bound grows like 1 / mu, so mu_final is a compromise between that distance and the
conditioning of the last stage: at 1e-6 (the default) the double integrator's last stage reaches
1e-10 in 8 Newton steps, at 1e-7 it stalls near 1e-9.
The bound multipliers are recovered as z_l = mu s w / (u - l), z_h = mu s w / (h - u).

Primal-dual form (Nocedal and Wright, Section 19.2 and 19.6; the form interior-point codes such
as IPOPT take). The bound multipliers become unknowns z_l, z_h >= 0 (one per bounded control
and node, scaled like the gradient rows, i.e. with the quadrature weight in them), and the
barrier problem's KKT conditions are

    g_U - z_l + z_h = 0,    C_l = (u - l) z_l - mu s w = 0,    C_h = (h - u) z_h - mu s w = 0

beside the unchanged state, costate and terminal rows. At C_l = C_h = 0 they reduce to the
primal conditions above, so both forms have the same solution; Newton's method on the
primal-dual system linearises the complementarity products instead of 1 / (u - l), which is
what lets it take long steps near the bounds. solve_pd runs the same stages as solve with the
full primal-dual Newton system (solved densely), the fraction-to-boundary rule on u and on
z_l, z_h, and backtracking on the merit ||F||_W^2 + sum (C_l^2 + C_h^2) / w.

Endpoint bounds (problem (P)'s e^L <= e <= e^U for the terminal conditions of the library's
kinds, e_r = x_{idx_r}(t_f)): a terminal row r may hold bounds l_r < x < h_r instead of its
equality. Their barrier psi_r(x) = -mu [log(x - l_r) + log(h_r - x)] (no quadrature weight: a
point term) keeps the KKT form with nu_r as its multiplier: the gradient row of x_{idx_r}(t_f)
keeps + nu_r, and row r of the terminal block becomes nu_r = psi_r'(x) in complementarity form,

    F_r = c(x) nu_r - mu m(x),   c = (x - l)(h - x), m = 2x - l - h   (two-sided),
                                  c = x - l, m = -1;  c = h - x, m = 1   (one-sided),

its Newton row a dx + e dnu with a = c'(x) nu - mu m'(x), e = c(x). (Dividing nu = psi' by
psi'' instead would have a spurious root at the bound itself, which the fraction-to-boundary
steps approach: seen in this oracle.) The library's preconditioner keeps the row as it is: its
n_e x n_e Schur complement becomes diag(a) E Q - diag(e). The stages start nu_r on the central
path (nu_r = psi_r'(x)); the fraction-to-boundary rule covers x(t_f), and for a one-sided row
also the sign of nu_r (negative for a lower bound, positive for an upper one). Endpoint rows
read the same in both forms above. Two-sided rows are defined here (and pinned on the double
integrator), but on the orbit transfer with a start at the bound away from the optimum
(r(t_f) in [1.3, 1.45] from the spiral that ends at 1.5) this single-multiplier row stalled,
so the library takes one bound per row.
"""
import numpy as np

from .kkt import DenseKKT

TAU = 0.995     # fraction-to-boundary


class BarrierKKT(DenseKKT):
    """DenseKKT of a problem with control bounds lo, hi (length n_u, +-inf for none) and the
    barrier parameter mu (set before each stage)."""

    def __init__(self, prob, N, lo, hi, Ba=None, ebounds=None):
        super().__init__(prob, N, Ba)
        self.lo = np.asarray(lo, float).reshape(prob.n_u)
        self.hi = np.asarray(hi, float).reshape(prob.n_u)
        self.mu = 0.0
        # endpoint bounds: {terminal row r: (l_r, h_r)}, the other rows keep their equality
        self.ebounds = dict(ebounds or {})
        for r, (a, b) in self.ebounds.items():
            assert 0 <= r < prob.n_e and a < b

    # ---- endpoint bounds ---------------------------------------------------------------------
    def _cm(self, r, x):
        """c(x), c'(x), m(x), m'(x) of endpoint row r (module docstring)."""
        a, b = self.ebounds[r]
        if np.isfinite(a) and np.isfinite(b):
            return (x - a) * (b - x), a + b - 2.0 * x, 2.0 * x - a - b, 2.0
        if np.isfinite(a):
            return x - a, 1.0, -1.0, 0.0
        return b - x, -1.0, 1.0, 0.0

    def _end_x(self, vec):
        X = self.split(vec)[0]
        return {r: X[self.prob.term_idx[r], -1] for r in self.ebounds}

    def _end_coef(self, vec):
        """{r: (F_r, a_r, e_r)} at vec."""
        nu = self.split(vec)[3]
        out = {}
        for r, x in self._end_x(vec).items():
            c, dc, m, dm = self._cm(r, x)
            out[r] = (c * nu[r] - self.mu * m, dc * nu[r] - self.mu * dm, c)
        return out

    def _end_residual(self, vec, F):
        for r, (f, _, _) in self._end_coef(vec).items():
            F[self.nz + self.nc + r] = f
        return F

    def _end_matrix(self, vec, K):
        for r, (_, a, e) in self._end_coef(vec).items():
            i = self.nz + self.nc + r
            K[i, :] = 0.0
            K[i, self.prob.term_idx[r] * self.L + self.L - 1] = a
            K[i, i] = e
        return K

    def _end_precond(self, vec, Kt):
        """The preconditioner takes the endpoint rows as they are (its E rows scaled by a)."""
        for r, (_, a, e) in self._end_coef(vec).items():
            i = self.nz + self.nc + r
            Kt[i, self.prob.term_idx[r] * self.L + self.L - 1] = a
            Kt[i, i] = e
        return Kt

    def end_init(self, vec):
        """vec with nu_r of every endpoint row on the central path, nu_r = psi_r'(x)."""
        v = np.array(vec, float)
        nu = v[self.nz + self.nc:self.nz + self.nc + self.prob.n_e]
        for r, x in self._end_x(v).items():
            a, b = self.ebounds[r]
            g = 0.0
            if np.isfinite(a):
                g -= 1.0 / (x - a)
            if np.isfinite(b):
                g += 1.0 / (b - x)
            nu[r] = self.mu * g
        return v

    def _bar_terms(self, U, s):
        """Per control and node: the barrier gradient and Hessian diagonal (zero where unbounded)."""
        g = np.zeros_like(U)
        h = np.zeros_like(U)
        for q in range(self.prob.n_u):
            if np.isfinite(self.lo[q]):
                d = U[q] - self.lo[q]
                g[q] -= 1.0 / d
                h[q] += 1.0 / (d * d)
            if np.isfinite(self.hi[q]):
                d = self.hi[q] - U[q]
                g[q] += 1.0 / d
                h[q] += 1.0 / (d * d)
        c = self.mu * s * self.w[None, :]
        return c * g, c * h

    def residual(self, vec):
        F = super().residual(vec)
        p, L = self.prob, self.L
        X, U, lam, nu = self.split(vec)
        g, _ = self._bar_terms(U, self.s_of(vec))
        F[p.n_x * L:self.nz] += g.ravel()
        return self._end_residual(vec, F)

    def matrix(self, vec):
        K = super().matrix(vec)
        p, L = self.prob, self.L
        X, U, lam, nu = self.split(vec)
        _, h = self._bar_terms(U, self.s_of(vec))
        i0 = p.n_x * L
        K[i0:self.nz, i0:self.nz] += np.diag(h.ravel())
        return self._end_matrix(vec, K)

    def precond_matrix(self, vec):
        """K-tilde with the barrier's Hessian diagonal added to its control block (which stays
        diagonal, so the block elimination of the library's preconditioner is unchanged)."""
        Kt = super().precond_matrix(vec)
        p, L = self.prob, self.L
        X, U, lam, nu = self.split(vec)
        _, h = self._bar_terms(U, self.s_of(vec))
        i0 = p.n_x * L
        Kt[i0:self.nz, i0:self.nz] += np.diag(h.ravel())
        return self._end_precond(vec, Kt)

    def max_step(self, vec, d):
        """Fraction-to-boundary: TAU times the largest alpha <= 1 / TAU keeping l < u + alpha du < h."""
        p, L = self.prob, self.L
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        dU = d[p.n_x * L:self.nz].reshape(p.n_u, L)
        amax = 1.0 / TAU
        for q in range(p.n_u):
            if np.isfinite(self.lo[q]):
                m = dU[q] < 0
                if m.any():
                    amax = min(amax, float(np.min((self.lo[q] - U[q][m]) / dU[q][m])))
            if np.isfinite(self.hi[q]):
                m = dU[q] > 0
                if m.any():
                    amax = min(amax, float(np.min((self.hi[q] - U[q][m]) / dU[q][m])))
        dX, dnu = self.split(d)[0], self.split(d)[3]
        nu = self.split(vec)[3]
        for r, x in self._end_x(vec).items():
            a, b = self.ebounds[r]
            dx = dX[p.term_idx[r], -1]
            if np.isfinite(a) and dx < 0:
                amax = min(amax, (a - x) / dx)
            if np.isfinite(b) and dx > 0:
                amax = min(amax, (b - x) / dx)
            # one-sided row: nu keeps its sign (negative below a lower bound's barrier, positive
            # for an upper one)
            if np.isfinite(a) and not np.isfinite(b) and dnu[r] > 0:
                amax = min(amax, -nu[r] / dnu[r])
            if np.isfinite(b) and not np.isfinite(a) and dnu[r] < 0:
                amax = min(amax, -nu[r] / dnu[r])
        return min(1.0, TAU * amax)

    def interior(self, vec, margin=1e-3):
        """vec with its controls moved at least `margin` (relative to the bound gap, or absolute
        for one-sided bounds) inside their bounds."""
        v = np.array(vec, float)
        p, L = self.prob, self.L
        U = v[p.n_x * L:self.nz].reshape(p.n_u, L)
        for q in range(p.n_u):
            lo, hi = self.lo[q], self.hi[q]
            gap = hi - lo if np.isfinite(lo) and np.isfinite(hi) else 1.0
            if np.isfinite(lo):
                U[q] = np.maximum(U[q], lo + margin * gap)
            if np.isfinite(hi):
                U[q] = np.minimum(U[q], hi - margin * gap)
        X = v[:p.n_x * L].reshape(p.n_x, L)
        for r, (lo, hi) in self.ebounds.items():
            gap = hi - lo if np.isfinite(lo) and np.isfinite(hi) else 1.0
            i = p.term_idx[r]
            if np.isfinite(lo):
                X[i, -1] = max(X[i, -1], lo + margin * gap)
            if np.isfinite(hi):
                X[i, -1] = min(X[i, -1], hi - margin * gap)
        return v

    def newton_stage(self, vec, tol, max_iter=50, armijo=1e-4, max_backtrack=40):
        """Newton-Lagrange on F_mu = 0 with the fraction-to-boundary step cap and backtracking
        on ||F_mu||_W. Returns (vec, iterations, final norm)."""
        F = self.residual(vec)
        nrm = self.weighted_norm(F)
        it = 0
        while nrm > tol and it < max_iter:
            d = np.linalg.solve(self.matrix(vec), -F)
            alpha = self.max_step(vec, d)
            accepted = False
            for _ in range(max_backtrack):
                trial = vec + alpha * d
                Ft = self.residual(trial)
                nt = self.weighted_norm(Ft)
                if nt <= (1.0 - armijo * alpha) * nrm:
                    accepted = True
                    break
                alpha *= 0.5
            if not accepted:
                break
            vec, F, nrm = trial, Ft, nt
            it += 1
        return vec, it, nrm

    def solve(self, vec0, mu0=1e-1, mu_final=1e-6, tol=1e-10, factor=0.1):
        """The barrier outer loop (module docstring). Returns (vec, info)."""
        vec = self.interior(vec0)
        mu = mu0
        self.mu = mu
        vec = self.end_init(vec)
        total = 0
        stages = []
        while True:
            self.mu = mu
            last = mu <= mu_final * (1.0 + 1e-12)
            vec, it, nrm = self.newton_stage(vec, tol if last else max(tol, 10.0 * mu))
            total += it
            stages.append((mu, it, nrm))
            if last:
                break
            mu = max(mu * factor, mu_final)
        return vec, dict(iters=total, stages=stages, converged=bool(stages[-1][2] <= tol))

    def bound_multipliers(self, vec):
        """z_l, z_h = mu s w / (u - l), mu s w / (h - u) (zero where unbounded)."""
        p, L = self.prob, self.L
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        c = self.mu * self.s_of(vec) * self.w[None, :]
        zl = np.where(np.isfinite(self.lo)[:, None], c / (U - np.where(np.isfinite(self.lo), self.lo, 0.0)[:, None]), 0.0)
        zh = np.where(np.isfinite(self.hi)[:, None], c / (np.where(np.isfinite(self.hi), self.hi, 0.0)[:, None] - U), 0.0)
        return zl, zh

    # ---- primal-dual form ------------------------------------------------------------------
    def _bounded(self):
        return np.isfinite(self.lo), np.isfinite(self.hi)

    def pd_init(self, vec):
        """Multipliers on the central path of the current mu: z = mu s w / (distance to the bound)."""
        p, L = self.prob, self.L
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        c = self.mu * self.s_of(vec) * self.w[None, :]
        ml, mh = self._bounded()
        zl = np.zeros_like(U)
        zh = np.zeros_like(U)
        for q in range(p.n_u):
            if ml[q]:
                zl[q] = c[0] / (U[q] - self.lo[q])
            if mh[q]:
                zh[q] = c[0] / (self.hi[q] - U[q])
        return zl, zh

    def pd_residual(self, vec, zl, zh):
        """(F, C_l, C_h): F the unbarriered KKT residual with -z_l + z_h in the control rows,
        C_l, C_h the complementarity residuals (zero rows where a control has no such bound)."""
        F = DenseKKT.residual(self, vec)
        p, L = self.prob, self.L
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        c = self.mu * self.s_of(vec) * self.w
        ml, mh = self._bounded()
        Cl = np.zeros_like(U)
        Ch = np.zeros_like(U)
        G = F[p.n_x * L:self.nz].reshape(p.n_u, L)
        for q in range(p.n_u):
            if ml[q]:
                G[q] -= zl[q]
                Cl[q] = (U[q] - self.lo[q]) * zl[q] - c
            if mh[q]:
                G[q] += zh[q]
                Ch[q] = (self.hi[q] - U[q]) * zh[q] - c
        return self._end_residual(vec, F), Cl, Ch

    def pd_merit(self, F, Cl, Ch):
        """sqrt(||F||_W^2 + sum (C_l^2 + C_h^2) / w): complementarity weighted like the gradient rows."""
        return float(np.sqrt(self.weighted_norm(F) ** 2 + ((Cl * Cl + Ch * Ch) / self.w[None, :]).sum()))

    def pd_matrix(self, vec, zl, zh):
        """Jacobian of [F; C_l; C_h] with respect to [vec; z_l; z_h], the multipliers of every
        control component included (rows and columns of an absent bound: the identity, which
        keeps that multiplier at zero)."""
        p, L = self.prob, self.L
        n, m = self.n, p.n_u * L
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        ml, mh = self._bounded()
        A = np.zeros((n + 2 * m, n + 2 * m))
        A[:n, :n] = self._end_matrix(vec, DenseKKT.matrix(self, vec))
        for q in range(p.n_u):
            rows_u = p.n_x * L + q * L + np.arange(L)      # control rows / columns of u_q
            il = n + q * L + np.arange(L)                    # z_l,q
            ih = n + m + q * L + np.arange(L)                # z_h,q
            if ml[q]:
                A[rows_u, il] = -1.0
                A[il, rows_u] = zl[q]
                A[il, il] = U[q] - self.lo[q]
            else:
                A[il, il] = 1.0
            if mh[q]:
                A[rows_u, ih] = 1.0
                A[ih, rows_u] = -zh[q]
                A[ih, ih] = self.hi[q] - U[q]
            else:
                A[ih, ih] = 1.0
        return A

    def pd_step(self, vec, zl, zh):
        """Newton step of the primal-dual system: (d, dz_l, dz_h)."""
        p, L = self.prob, self.L
        F, Cl, Ch = self.pd_residual(vec, zl, zh)
        n, m = self.n, p.n_u * L
        sol = np.linalg.solve(self.pd_matrix(vec, zl, zh), -np.concatenate([F, Cl.ravel(), Ch.ravel()]))
        return sol[:n], sol[n:n + m].reshape(p.n_u, L), sol[n + m:].reshape(p.n_u, L)

    def pd_max_step(self, vec, d, zl, zh, dzl, dzh):
        """Fraction-to-boundary for u (max_step) and for z_l, z_h >= 0: TAU times the largest
        alpha <= 1 / TAU keeping z + alpha dz > 0, the smaller of the two, capped at 1."""
        a = self.max_step(vec, d)
        zmax = 1.0 / TAU
        for z, dz in ((zl, dzl), (zh, dzh)):
            m = dz < 0
            if m.any():
                zmax = min(zmax, float(np.min(-z[m] / dz[m])))
        return min(a, 1.0, TAU * zmax)

    def pd_newton_stage(self, vec, zl, zh, tol, max_iter=50, armijo=1e-4, max_backtrack=40):
        """Newton's method on the primal-dual system at the current mu, backtracking (halving)
        on pd_merit from the fraction-to-boundary step. Returns (vec, zl, zh, iterations, merit)."""
        F, Cl, Ch = self.pd_residual(vec, zl, zh)
        nrm = self.pd_merit(F, Cl, Ch)
        it = 0
        while nrm > tol and it < max_iter:
            d, dzl, dzh = self.pd_step(vec, zl, zh)
            alpha = self.pd_max_step(vec, d, zl, zh, dzl, dzh)
            accepted = False
            for _ in range(max_backtrack):
                trial = (vec + alpha * d, zl + alpha * dzl, zh + alpha * dzh)
                nt = self.pd_merit(*self.pd_residual(*trial))
                if nt <= (1.0 - armijo * alpha) * nrm:
                    accepted = True
                    break
                alpha *= 0.5
            if not accepted:
                break
            (vec, zl, zh), nrm = trial, nt
            it += 1
        return vec, zl, zh, it, nrm

    def solve_pd(self, vec0, mu0=1e-1, mu_final=1e-6, tol=1e-10, factor=0.1):
        """The stages of solve on the primal-dual system, from the interior point of solve and
        multipliers on the first stage's central path. Returns (vec, zl, zh, info)."""
        vec = self.interior(vec0)
        mu = mu0
        self.mu = mu
        vec = self.end_init(vec)
        zl, zh = self.pd_init(vec)
        total = 0
        stages = []
        while True:
            self.mu = mu
            last = mu <= mu_final * (1.0 + 1e-12)
            vec, zl, zh, it, nrm = self.pd_newton_stage(vec, zl, zh, tol if last else max(tol, 10.0 * mu))
            total += it
            stages.append((mu, it, nrm))
            if last:
                break
            mu = max(mu * factor, mu_final)
        return vec, zl, zh, dict(iters=total, stages=stages, converged=bool(stages[-1][2] <= tol))
