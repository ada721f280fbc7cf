"""Control and endpoint bounds on the matrix-free oracle (test infrastructure only).

The barrier problem of oracle/barrier.py (primal form; one bound per endpoint row) without
dense matrices, so that the library's bounded solves can be checked on the same grid at sizes
the dense oracle cannot reach (N = 2^12 and above):

    control rows    g_U += -mu s w (1 / (u - l) - 1 / (h - u)),
                    control block += mu s w (1 / (u - l)^2 + 1 / (h - u)^2)   (diagonal),
    endpoint row r  (x - l) nu_r + mu = 0   or   (h - x) nu_r - mu = 0,  x = x_{idx_r}(t_f),
                    Newton row a dx + c dnu (a = +-nu, c the distance to the bound).

K-tilde takes the barrier diagonal into its control block and the endpoint rows as they are:
with x = x0 + X_e e from the block elimination (MatFreeKKT._solve_unbordered), the terminal
system becomes (diag(a) S + diag(c)) e = d - a * (E x0). The stages, the interior start, the
fraction-to-boundary rule and the halving line search are those of BarrierKKT.solve; each
Newton step is solved by right-preconditioned GMRES to a tight tolerance.
"""
import numpy as np

from .barrier import BarrierKKT
from .matfree import MatFreeKKT, gmres_right


class MatFreeBarrierKKT(MatFreeKKT):
    """MatFreeKKT with control bounds lo, hi (length n_u, +-inf for none), endpoint bounds
    {terminal row r: (l_r, h_r)} with one finite side each, and the barrier parameter mu."""

    # bound bookkeeping shared with the dense barrier oracle (it needs no dense matrix)
    _bar_terms = BarrierKKT._bar_terms
    _cm = BarrierKKT._cm
    _end_x = BarrierKKT._end_x
    _end_coef = BarrierKKT._end_coef
    interior = BarrierKKT.interior
    max_step = BarrierKKT.max_step
    end_init = BarrierKKT.end_init

    def __init__(self, prob, N, lo, hi, ebounds=None):
        super().__init__(prob, N)
        self.lo = np.asarray(lo, float).reshape(prob.n_u)
        self.hi = np.asarray(hi, float).reshape(prob.n_u)
        self.mu = 0.0
        self.ebounds = dict(ebounds or {})
        for r, (a, b) in self.ebounds.items():
            assert 0 <= r < prob.n_e and a < b and (np.isfinite(a) != np.isfinite(b))

    def residual(self, vec):
        F = super().residual(vec)
        p, L = self.prob, self.L
        U = self.split(vec)[1]
        g, _ = self._bar_terms(U, self.s_of(vec))
        F[p.n_x * L:self.nz] += g.ravel()
        for r, (f, _, _) in self._end_coef(vec).items():
            F[self.nz + self.nc + r] = f
        return F

    def apply(self, vec, d):
        out = super().apply(vec, d)
        p, L = self.prob, self.L
        U = self.split(vec)[1]
        dX, dU, _, dn = self.split(d)
        _, h = self._bar_terms(U, self.s_of(vec))
        out[p.n_x * L:self.nz] += (h * dU).ravel()
        for r, (_, a, c) in self._end_coef(vec).items():
            out[self.nz + self.nc + r] = a * dX[p.term_idx[r], -1] + c * dn[r]
        return out

    def linearize_precond(self, vec):
        """K-tilde with the barrier diagonal in its control block: the Schur columns of
        MatFreeKKT.linearize_precond are formed with it, then the endpoint rows' coefficients."""
        p = self.prob
        U = self.split(vec)[1]
        _, h = self._bar_terms(U, self.s_of(vec))
        self._huu_extra = h
        pc = super().linearize_precond(vec)
        coef = self._end_coef(vec)
        a = np.ones(p.n_e)
        c = np.zeros(p.n_e)
        for r, (_, ar, cr) in coef.items():
            a[r], c[r] = ar, cr
        pc.update(ea=a, ec=c)
        return pc

    def _solve_unbordered(self, r):
        pc = self._pc
        if "ea" not in pc:   # during linearize_precond (no endpoint rows needed yet)
            return super()._solve_unbordered(r)
        p, L = self.prob, self.L
        nx, nu_, ne = p.n_x, p.n_u, p.n_e
        a = r[:nx * L].reshape(nx, L)
        b = r[nx * L:self.nz].reshape(nu_, L)
        c = r[self.nz:self.nz + self.nc].reshape(nx, L)
        d = r[self.nz + self.nc:self.nz + self.nc + ne]
        from .birkhoff import fastpinvy_block, fastpinvy_block_T
        l0 = fastpinvy_block_T(pc["sw"], pc["Jx"], a)
        u0 = (b - self._PuT(l0)) / pc["huu"]
        x0 = fastpinvy_block(pc["sw"], pc["Jx"], c - self._Pu(u0))
        Ex0 = np.array([x0[i, L - 1] for i in p.term_idx])
        S = pc["ea"][:, None] * pc["S"] + np.diag(pc["ec"])
        e = np.linalg.solve(S, d - pc["ea"] * Ex0) if ne else np.zeros(0)
        l = l0 - np.tensordot(e, pc["Le"], axes=1)
        u = u0 + np.tensordot(e, pc["Ue"], axes=1)
        x = x0 + np.tensordot(e, pc["Xe"], axes=1)
        return np.concatenate([x.ravel(), u.ravel(), l.ravel(), e])

    def precond_apply_matrix(self, vec, z):
        out = super().precond_apply_matrix(vec, z)
        pc = self._pc
        x, _, _, e = self.split(z)
        for r, i in enumerate(self.prob.term_idx):
            out[self.nz + self.nc + r] = pc["ea"][r] * x[i, self.L - 1] + pc["ec"][r] * e[r]
        return out

    def newton_stage(self, vec, tol, max_iter=60, armijo=1e-4, max_backtrack=40, inner_rtol=1e-12):
        """Newton on the barrier problem at the current mu: GMRES steps, fraction-to-boundary
        start, halving on ||F||_W. Returns (vec, iterations, final norm)."""
        F = self.residual(vec)
        nrm = self.weighted_norm(F)
        it = 0
        while nrm > tol and it < max_iter:
            self.linearize_precond(vec)
            d, _, _ = gmres_right(lambda x: self.apply(vec, x), self.precond_solve, -F, rtol=inner_rtol,
                                  restart=30, max_iter=600)
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
        """The stages of BarrierKKT.solve. Returns (vec, info)."""
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
