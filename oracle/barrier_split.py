"""Two-sided endpoint bounds with two multipliers (oracle; test infrastructure only).

A terminal row r with both bounds, l_r < x < h_r (x = x_{idx_r}(t_f)), takes the barrier
-mu [log(x - l_r) + log(h_r - x)] with one multiplier per side: nu_r (in the row's own slot,
the lower side) and nu'_r (appended after nu), each in complementarity form,

    (x - l_r) nu_r + mu = 0,   (h_r - x) nu'_r - mu = 0,

and the gradient row of x gains nu_r + nu'_r. The signs nu_r < 0 < nu'_r are kept by the
fraction-to-boundary rule. With one multiplier for both sides (BarrierKKT's two-sided rows) the
row reads c(x) nu = mu m(x), whose multiplier may take either sign; on the orbit transfer from
a start at the bound away from the optimum that row stalled, while these two rows converge
(tests/test_oracle_barrier_split.py). Primal form only (the controls' barrier as in BarrierKKT).

Vector layout: the BarrierKKT vector followed by nu'_r for the two-sided rows in row order.
"""
import contextlib

import numpy as np

from .barrier import TAU, BarrierKKT


class SplitEndpointKKT(BarrierKKT):
    def __init__(self, prob, N, lo, hi, two_sided, Ba=None, ebounds=None):
        super().__init__(prob, N, lo, hi, Ba=Ba, ebounds=ebounds)
        self.two = dict(two_sided)             # {terminal row r: (l_r, h_r)}, both finite
        for r, (a, b) in self.two.items():
            assert 0 <= r < prob.n_e and r not in self.ebounds and np.isfinite(a) and np.isfinite(b) and a < b
        self.rows = sorted(self.two)
        self.nb = self.n                       # size of the BarrierKKT part
        self.n = self.nb + len(self.rows)

    @contextlib.contextmanager
    def _base(self):
        n = self.n
        self.n = self.nb
        try:
            yield
        finally:
            self.n = n

    def _parts(self, vec):
        """x = x_{idx_r}(t_f), nu_r, nu'_r, the column of x and the two row indices, per two-sided row."""
        X, _, _, nu = self.split(vec)
        L = self.L
        out = []
        for j, r in enumerate(self.rows):
            i = self.prob.term_idx[r]
            out.append((r, X[i, -1], nu[r], vec[self.nb + j], i * L + L - 1, self.nz + self.nc + r, self.nb + j))
        return out

    def pack(self, X, U, lam, nu, nu2=None):
        v = super().pack(X, U, lam, nu)
        return np.concatenate([v, np.zeros(len(self.rows)) if nu2 is None else np.asarray(nu2, float)])

    def residual(self, vec):
        with self._base():
            Fb = BarrierKKT.residual(self, vec[:self.nb])
        F = np.concatenate([Fb, np.zeros(len(self.rows))])
        for r, x, nl, nh, col, il, ih in self._parts(vec):
            a, b = self.two[r]
            F[col] += nh
            F[il] = (x - a) * nl + self.mu
            F[ih] = (b - x) * nh - self.mu
        return F

    def _rows_into(self, vec, K):
        for r, x, nl, nh, col, il, ih in self._parts(vec):
            a, b = self.two[r]
            K[col, ih] = 1.0
            K[il, :] = 0.0
            K[il, col] = nl
            K[il, il] = x - a
            K[ih, col] = -nh
            K[ih, ih] = b - x
        return K

    def matrix(self, vec):
        with self._base():
            Kb = BarrierKKT.matrix(self, vec[:self.nb])
        K = np.zeros((self.n, self.n))
        K[:self.nb, :self.nb] = Kb
        return self._rows_into(vec, K)

    def precond_matrix(self, vec):
        """K-tilde with the two-sided rows as they are (their Newton rows, as for one-sided rows)."""
        with self._base():
            Kb = BarrierKKT.precond_matrix(self, vec[:self.nb])
        K = np.zeros((self.n, self.n))
        K[:self.nb, :self.nb] = Kb
        return self._rows_into(vec, K)

    def max_step(self, vec, d):
        with self._base():
            alpha = BarrierKKT.max_step(self, vec[:self.nb], d[:self.nb])
        amax = 1.0 / TAU
        X, dX, dnu = self.split(vec)[0], self.split(d)[0], self.split(d)[3]
        for r, x, nl, nh, col, il, ih in self._parts(vec):
            a, b = self.two[r]
            dx = dX[self.prob.term_idx[r], -1]
            if dx < 0:
                amax = min(amax, (a - x) / dx)
            if dx > 0:
                amax = min(amax, (b - x) / dx)
            if dnu[r] > 0:                       # nu_r < 0
                amax = min(amax, -nl / dnu[r])
            if d[ih] < 0:                        # nu'_r > 0
                amax = min(amax, -nh / d[ih])
        return min(alpha, TAU * amax)

    def interior(self, vec, margin=1e-3):
        """BarrierKKT.interior, and x_{idx_r}(t_f) of the two-sided rows moved margin (h - l) inside."""
        with self._base():
            v = BarrierKKT.interior(self, vec[:self.nb], margin)
        X = v[:self.prob.n_x * self.L].reshape(self.prob.n_x, self.L)
        for r in self.rows:
            a, b = self.two[r]
            i = self.prob.term_idx[r]
            X[i, -1] = min(max(X[i, -1], a + margin * (b - a)), b - margin * (b - a))
        return np.concatenate([v, np.asarray(vec[self.nb:], float)])

    def end_init(self, vec):
        """BarrierKKT.end_init, and both multipliers of the two-sided rows on the central path."""
        with self._base():
            v = BarrierKKT.end_init(self, vec[:self.nb])
        v = np.concatenate([v, np.asarray(vec[self.nb:], float)])
        for r, x, nl, nh, col, il, ih in self._parts(v):
            a, b = self.two[r]
            v[il] = -self.mu / (x - a)
            v[ih] = self.mu / (b - x)
        return v

    def solve_pd(self, *args, **kwargs):
        raise NotImplementedError("two-sided endpoint rows: primal form only")
