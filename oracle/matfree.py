"""Matrix-free KKT operators and Newton-Krylov solve (oracle; test infrastructure only).

The same discretisation, residual, KKT matrix, preconditioner and merit norm as ``kkt.DenseKKT``
(Eq. Prob-PNa with V = f(X, U) eliminated; see that module), but every product with B^a goes
through the FastBV chain of ``birkhoff.fastbv`` / ``birkhoff.fastbv_T`` (Section "Fast
Computation of Birkhoff Matrix-Vector Products"), every product with B-tilde^a through its
definition as a running sum (the matrix after Eq. Ba=10, what FastBccV computes), and the
preconditioner solves through the forward and backward sweeps ``fastpinvy_block`` /
``fastpinvy_block_T`` (Section "Development of a Special Birkhoff-Centric Preconditioner"). The
linear solve of each Newton step is right-preconditioned GMRES (Algorithm 2, FastLinSol),
written out below in plain NumPy. Nothing is formed densely, so grids of 2^14 nodes and more
fit; it is slow (the sweeps are Python loops over the nodes) but every step can be checked by
eye against the dense class, to which the tests pin it at small N.

Clenshaw-Curtis weights: w = (B^a)^T e_N, the last row of B^a (the remark after Eq. Ba=10),
taken with the transpose chain.

Preconditioner K-tilde (the dense definition is ``DenseKKT.precond_matrix``):

    [ 0      0      P^T    E^T ] [x]   [a]      P  = I - s (B-tilde (x) I) J_x
    [ 0      Huu    Pu^T   0   ] [u] = [b]      Pu =   - s (B-tilde (x) I) J_u
    [ P      Pu     0      0   ] [l]   [c]      E  = terminal-row selector
    [ E      0      0      0   ] [e]   [d]

is solved by block elimination: l = P^-T (a - E^T e), u = Huu^-1 (b - Pu^T l),
x = P^-1 (c - Pu u) and E x = d. Each of l, u, x is affine in e, so e solves the n_e x n_e
system (E X_e) e = E x_0 - d, where X_e = P^-1 Pu Huu^-1 Pu^T P^-T E^T has n_e columns, formed
once per linearisation point. A free final time borders K-tilde with the KKT matrix's own s
column (``DenseKKT.border``); the border is eliminated with q = K-tilde^-1 col.
"""
import numpy as np

from . import problems as op
from .birkhoff import fastbv, fastbv_T, fastpinvy_block, fastpinvy_block_T
from .grid import cgl_nodes


def btilde(w, v):
    """B-tilde^a v along the last axis: (B-tilde v)_i = sum_{j<i} w_j v_j + w_i v_i / 2 (the
    definition after Eq. Ba=10; FastBccV computes the same running sum)."""
    wv = w * v
    return np.cumsum(wv, axis=-1) - 0.5 * wv


def btilde_T(w, y):
    """(B-tilde^a)^T y along the last axis: w_j (y_j / 2 + sum_{i>j} y_i)."""
    rev = np.cumsum(y[..., ::-1], axis=-1)[..., ::-1]        # sum_{i>=j} y_i
    return w * (rev - 0.5 * y)


def gmres_right(apply_A, apply_Minv, b, rtol=1e-12, restart=30, max_iter=300):
    """Right-preconditioned restarted GMRES (Algorithm 2, FastLinSol: GMRES on A M^-1 y = b,
    then x = M^-1 y), x_0 = 0. Arnoldi with modified Gram-Schmidt; the small least-squares
    problem by numpy.linalg.lstsq. Stops when the true residual ||b - A x|| <= rtol ||b||.
    Returns (x, iterations, relative residual)."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0
    its = 0
    r = b.copy()
    while its < max_iter:
        beta = np.linalg.norm(r)
        if beta <= rtol * nb:
            break
        m = min(restart, max_iter - its)
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        y = None
        k_used = 0
        for k in range(m):
            Z[k] = apply_Minv(V[k])
            wv = apply_A(Z[k])
            for i in range(k + 1):
                H[i, k] = V[i] @ wv
                wv = wv - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(wv)
            its += 1
            k_used = k + 1
            e1 = np.zeros(k + 2)
            e1[0] = beta
            y = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)[0]
            res = np.linalg.norm(H[:k + 2, :k + 1] @ y - e1)
            if H[k + 1, k] == 0.0 or res <= rtol * nb:
                break
            V[k + 1] = wv / H[k + 1, k]
        x = x + y @ Z[:k_used]
        r = b - apply_A(x)
    return x, its, float(np.linalg.norm(r) / nb)


class MatFreeKKT:
    """Matrix-free operators of one problem at one grid size N (any N >= 4 for which the
    FastBV chain applies, i.e. the oracle's SciPy DCT-I; in practice powers of two)."""

    def __init__(self, prob, N):
        self.prob = prob
        self.N = N
        self.L = N + 1
        eN = np.zeros(self.L)
        eN[N] = 1.0
        self.w = fastbv_T(eN)                          # last row of B^a
        self.s = 0.5 * (prob.tf - prob.t0)
        self.tau = cgl_nodes(N)
        self.t = prob.t0 + self.s * (self.tau + 1.0)
        nx, nu, L = prob.n_x, prob.n_u, self.L
        self.nz = (nx + nu) * L
        self.nc = nx * L
        self.free = bool(getattr(prob, 'free_time', False))
        self.n = self.nz + self.nc + prob.n_e + (1 if self.free else 0)
        self._pc = None

    # ---- packing (the layout of DenseKKT) ---------------------------------------------------
    def split(self, vec):
        p, L = self.prob, self.L
        X = vec[:p.n_x * L].reshape(p.n_x, L)
        U = vec[p.n_x * L:self.nz].reshape(p.n_u, L)
        lam = vec[self.nz:self.nz + self.nc].reshape(p.n_x, L)
        nu = vec[self.nz + self.nc:self.nz + self.nc + p.n_e]
        return X, U, lam, nu

    def s_of(self, vec):
        return float(vec[-1]) if self.free else self.s

    def pack(self, X, U, lam, nu, s=None):
        parts = [X.ravel(), U.ravel(), lam.ravel(), np.asarray(nu, float).ravel()]
        if self.free:
            parts.append([self.s if s is None else float(s)])
        return np.concatenate(parts)

    # B^a and its transpose on the rows of a component-major array (tau domain, s = 1)
    @staticmethod
    def Ba(v):
        return fastbv(v)

    @staticmethod
    def BaT(v):
        return fastbv_T(v)

    def border(self, vec):
        """The KKT matrix's s column (free final time), as DenseKKT.border."""
        p = self.prob
        X, U, lam, nu = self.split(vec)
        Jx, Ju = p.jac(X, U)
        muh = self.BaT(lam)
        col = np.zeros(self.n)
        col[:p.n_x * self.L] = -np.einsum('kmp,mk->pk', Jx, muh).ravel()
        col[p.n_x * self.L:self.nz] = -np.einsum('kmq,mk->qk', Ju, muh).ravel()
        col[self.nz:self.nz + self.nc] = -self.Ba(p.f(X, U)).ravel()
        return col

    # ---- residual ---------------------------------------------------------------------------
    def residual(self, vec):
        """F = [grad_z L ; c ; e (; g_s)] at vec, as DenseKKT.residual."""
        p, s = self.prob, self.s_of(vec)
        X, U, lam, nu = self.split(vec)
        f = p.f(X, U)
        Bf = self.Ba(f)
        c = X - p.x0[:, None] - s * Bf
        e = p.terminal_residual(X)
        Jx, Ju = p.jac(X, U)
        mu = self.BaT(lam)
        gX = lam - s * np.einsum('kmp,mk->pk', Jx, mu)
        gU = s * self.w[None, :] * p.cost_grad_u(U) - s * np.einsum('kmq,mk->qk', Ju, mu)
        for r, i in enumerate(p.term_idx):
            gX[i, -1] += nu[r]
        tail = [e]
        if self.free:
            tail.append([2.0 - float(np.sum(lam * Bf))])
        return np.concatenate([gX.ravel(), gU.ravel(), c.ravel()] + tail)

    def weighted_norm(self, F):
        """||F||_W, as DenseKKT.weighted_norm."""
        p, L, w = self.prob, self.L, self.w
        gX = F[:p.n_x * L].reshape(p.n_x, L)
        gU = F[p.n_x * L:self.nz].reshape(p.n_u, L)
        c = F[self.nz:self.nz + self.nc].reshape(p.n_x, L)
        e = F[self.nz + self.nc:]
        return float(np.sqrt((w * c * c).sum() + (gX * gX / w).sum() + (gU * gU / w).sum()
                             + (e * e).sum()))

    # ---- KKT matrix times a vector ------------------------------------------------------------
    def apply(self, vec, d):
        """K(vec) d without forming K: [H dz + G^T dy ; G dz ; E dz] (+ the s border)."""
        p, s, L = self.prob, self.s_of(vec), self.L
        nx, nu_ = p.n_x, p.n_u
        X, U, lam, nu = self.split(vec)
        dX, dU, dl, dn = self.split(d)
        Jx, Ju = p.jac(X, U)
        mu = self.BaT(lam)
        Hn = -s * p.hess_f(X, U, mu)
        for q in range(nu_):
            Hn[:, nx + q, nx + q] += s * self.w * p.cost_hess_uu()
        dz = np.concatenate([dX, dU])                     # (nx + nu, L)
        Hdz = np.einsum('kab,bk->ak', Hn, dz)
        BTdl = self.BaT(dl)
        gx = Hdz[:nx] + dl - s * np.einsum('kmp,mk->pk', Jx, BTdl)
        gu = Hdz[nx:] - s * np.einsum('kmq,mk->qk', Ju, BTdl)
        for r, i in enumerate(p.term_idx):
            gx[i, -1] += dn[r]
        Jd = np.einsum('kmp,pk->mk', Jx, dX) + np.einsum('kmq,qk->mk', Ju, dU)
        gc = dX - s * self.Ba(Jd)
        ge = np.array([dX[i, -1] for i in p.term_idx])
        out = np.concatenate([gx.ravel(), gu.ravel(), gc.ravel(), ge])
        if self.free:
            col = self.border(vec)
            ds = float(d[-1])
            out = np.concatenate([out, [col[:-1] @ d[:-1]]])
            out = out + col * ds
        return out

    # ---- the preconditioner K-tilde and its solve ----------------------------------------------
    def linearize_precond(self, vec):
        """Per-linearisation data of K-tilde^-1: Jacobians, Huu and the terminal Schur columns."""
        p, s, L = self.prob, self.s_of(vec), self.L
        nx, nu_, ne = p.n_x, p.n_u, p.n_e
        if nu_ == 0 or (not p.running_cost() and not self.free):
            raise ValueError("K-tilde needs a control-cost (or free-time) block")
        X, U, lam, nu = self.split(vec)
        Jx, Ju = p.jac(X, U)
        sw = s * self.w
        if self.free:
            mu = s * self.BaT(lam)
            huu = np.tile(p.a * np.hypot(mu[2], mu[3]) + 1e-3 * sw, (nu_, 1))
        else:
            huu = np.tile(sw * p.cost_hess_uu(), (nu_, 1))
        huu = huu + getattr(self, "_huu_extra", 0.0)   # a barrier's diagonal (matfree_barrier.py)
        pc = dict(vec=vec, s=s, sw=sw, Jx=Jx, Ju=Ju, huu=huu)
        self._pc = pc
        # Schur columns: for each terminal row r, E^T e_r -> l_r, u_r, x_r
        Le = np.zeros((ne, nx, L))
        Ue = np.zeros((ne, nu_, L))
        Xe = np.zeros((ne, nx, L))
        for r, i in enumerate(p.term_idx):
            rhs = np.zeros((nx, L))
            rhs[i, L - 1] = 1.0
            Le[r] = fastpinvy_block_T(sw, Jx, rhs)
            Ue[r] = self._PuT(Le[r]) / huu
            Xe[r] = fastpinvy_block(sw, Jx, -self._Pu(Ue[r]))
        S = np.array([[Xe[c][i, L - 1] for c in range(ne)] for i in p.term_idx]).reshape(ne, ne)
        pc.update(Le=Le, Ue=Ue, Xe=Xe, S=S)
        if self.free:
            pc["q"] = None
            pc["col"] = self.border(vec)
            pc["q"] = self._solve_unbordered(pc["col"][:-1])
        return pc

    def _Pu(self, u):
        pc = self._pc
        return -btilde(pc["sw"], np.einsum('kmq,qk->mk', pc["Ju"], u))

    def _PuT(self, l):
        pc = self._pc
        return -np.einsum('kmq,mk->qk', pc["Ju"], btilde_T(pc["sw"], l))

    def _solve_unbordered(self, r):
        p, L, pc = self.prob, self.L, self._pc
        nx, nu_, ne = p.n_x, p.n_u, p.n_e
        a = r[:nx * L].reshape(nx, L)
        b = r[nx * L:self.nz].reshape(nu_, L)
        c = r[self.nz:self.nz + self.nc].reshape(nx, L)
        d = r[self.nz + self.nc:self.nz + self.nc + ne]
        l0 = fastpinvy_block_T(pc["sw"], pc["Jx"], a)
        u0 = (b - self._PuT(l0)) / pc["huu"]
        x0 = fastpinvy_block(pc["sw"], pc["Jx"], c - self._Pu(u0))
        Ex0 = np.array([x0[i, L - 1] for i in p.term_idx])
        # E x = E x0 + (E X_e-columns) e with X_e columns computed for +E^T e_r: x_r = P^-1(-Pu u_r)
        # and l = l0 - Le e, u = u0 + Ue e (u depends on -l), x = x0 + Xe e
        e = np.linalg.solve(pc["S"], d - Ex0) if ne else np.zeros(0)
        l = l0 - np.tensordot(e, pc["Le"], axes=1)
        u = u0 + np.tensordot(e, pc["Ue"], axes=1)
        x = x0 + np.tensordot(e, pc["Xe"], axes=1)
        return np.concatenate([x.ravel(), u.ravel(), l.ravel(), e])

    def precond_solve(self, r):
        """K-tilde^-1 r at the last linearize_precond point."""
        if not self.free:
            return self._solve_unbordered(r)
        pc = self._pc
        col, q = pc["col"], pc["q"]
        zr = self._solve_unbordered(r[:-1])
        sig = (col[:-1] @ zr - r[-1]) / (col[:-1] @ q)
        return np.concatenate([zr - sig * q, [sig]])

    def precond_apply_matrix(self, vec, z):
        """K-tilde z (matrix-free, for residual checks of precond_solve)."""
        p, L = self.prob, self.L
        nx, nu_ = p.n_x, p.n_u
        pc = self._pc if self._pc is not None and self._pc["vec"] is vec else self.linearize_precond(vec)
        x, u, l, e = self.split(z)                    # the s entry of a bordered z is not read
        PTl = l - np.einsum('kmp,mk->pk', pc["Jx"], btilde_T(pc["sw"], l))
        ra = PTl.copy()
        for r, i in enumerate(p.term_idx):
            ra[i, L - 1] += e[r]
        rb = pc["huu"] * u + self._PuT(l)
        rc = x - btilde(pc["sw"], np.einsum('kmp,pk->mk', pc["Jx"], x)) + self._Pu(u)
        rd = np.array([x[i, L - 1] for i in p.term_idx])
        out = np.concatenate([ra.ravel(), rb.ravel(), rc.ravel(), rd])
        if self.free:
            col = pc["col"]
            out = np.concatenate([out + col[:-1] * z[-1], [col[:-1] @ z[:-1]]])
        return out

    # ---- Newton-Lagrange with GMRES inner solves -----------------------------------------------
    def newton(self, vec0, tol=1e-10, max_iter=30, armijo=1e-4, max_backtrack=30, inner_rtol=1e-12,
               restart=30, max_krylov=300):
        """Newton's method on F = 0 with the step from preconditioned GMRES (K-tilde^-1) and the
        backtracking line search of DenseKKT.newton. Returns (vec, info) with info = dict(iters,
        alphas, norms, krylov, converged)."""
        vec = np.array(vec0, dtype=np.float64)
        F = self.residual(vec)
        norms = [self.weighted_norm(F)]
        alphas, kry = [], []
        it = 0
        while norms[-1] > tol and it < max_iter:
            self.linearize_precond(vec)
            d, kits, _ = gmres_right(lambda x: self.apply(vec, x), self.precond_solve, -F,
                                     rtol=inner_rtol, restart=restart, max_iter=max_krylov)
            kry.append(kits)
            alpha = 1.0
            f0 = norms[-1]
            accepted = False
            for _ in range(max_backtrack):
                trial = vec + alpha * d
                if self.s_of(trial) > 0.0:
                    Ft = self.residual(trial)
                    if self.weighted_norm(Ft) <= (1.0 - armijo * alpha) * f0:
                        accepted = True
                        break
                alpha *= 0.5
            if not accepted:
                break
            vec, F = trial, Ft
            alphas.append(alpha)
            norms.append(self.weighted_norm(F))
            it += 1
        return vec, dict(iters=it, alphas=alphas, norms=norms, krylov=kry,
                         converged=bool(norms[-1] <= tol))


def orbit_problem(rf=1.5, tf=20.0, a=0.01, t0=0.0):
    """The orbit-raising problem of the benchmark configuration (fixed t_f; see problems.ORBIT)."""
    return op.Problem(op.ORBIT, t0, tf, (a, rf))
