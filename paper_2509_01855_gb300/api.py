"""Python binding of the C ABI (include/birkhoff.h), with the same call names.

Tensors are torch CUDA tensors; the binding passes their data pointers, sizes and the current
(or given) CUDA stream to libbirkhoff.so and raises BirkhoffError on a non-zero status.
"""
import ctypes

import torch

from . import _lib as L

_TORCH_DTYPE = {L.BK_F64: torch.float64, L.BK_F32: torch.float32}


def _dtype_code(dtype):
    if dtype in (torch.float64, "f64", L.BK_F64):
        return L.BK_F64
    if dtype in (torch.float32, "f32", L.BK_F32):
        return L.BK_F32
    raise ValueError("dtype must be float64 or float32")


class Plan:
    """A bk_plan: grid tables and scratch for Birkhoff products of size N."""

    def __init__(self, N, n_comp=1, max_batch=1, dtype=torch.float64, t0=-1.0, tf=1.0,
                 pitch=0, stream=None):
        lib = L.lib()
        self._h = ctypes.c_void_p()
        self.dtype_code = _dtype_code(dtype)
        L.check(lib.bk_plan_create(ctypes.byref(self._h), int(N), int(n_comp), int(max_batch),
                                   self.dtype_code, float(t0), float(tf), int(pitch),
                                   L.stream_ptr(stream)))
        n, l, p, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        L.check(lib.bk_plan_info(self._h, ctypes.byref(n), ctypes.byref(l), ctypes.byref(p),
                                 ctypes.byref(d)))
        self.N, self.L, self.pitch = n.value, l.value, p.value
        self.n_comp, self.max_batch = int(n_comp), int(max_batch)
        self.t0, self.tf = float(t0), float(tf)
        self.dtype = _TORCH_DTYPE[self.dtype_code]

    @property
    def handle(self):
        return self._h

    def grid(self):
        """(t, w): node times and Clenshaw-Curtis weights as host float64 tensors."""
        t = torch.empty(self.L, dtype=torch.float64)
        w = torch.empty(self.L, dtype=torch.float64)
        L.check(L.lib().bk_plan_grid(self._h, L.ptr(t), L.ptr(w)))
        return t, w

    def set_dense(self, on=True, stream=None):
        """Products through the dense tensor-core path (BK_F32 plans, N <= 1024) or the FFT chain."""
        L.check(L.lib().bk_plan_set_dense(self._h, 1 if on else 0, L.stream_ptr(stream)))

    def shape(self):
        """{"path": "single_cta" | "four_step" | "split_four_step" | "dense" | "bluestein", "N1", "N2",
        "elems"}."""
        v = [ctypes.c_int(0) for _ in range(4)]
        L.check(L.lib().bk_plan_shape(self._h, *[ctypes.byref(x) for x in v]))
        names = ("single_cta", "four_step", "split_four_step", "dense", "bluestein")
        return {"path": names[v[0].value], "N1": v[1].value, "N2": v[2].value, "elems": v[3].value}

    def is_dense(self):
        """True while the plan's products take the dense tensor-core path."""
        on = ctypes.c_int(0)
        L.check(L.lib().bk_plan_dense_state(self._h, ctypes.byref(on)))
        return bool(on.value)

    def f64_mode(self):
        """1 when the plan's FP64 transforms run in double-float arithmetic, else 0."""
        m = ctypes.c_int(0)
        L.check(L.lib().bk_plan_f64_mode(self._h, ctypes.byref(m)))
        return m.value

    def dense_check(self):
        """Error word of the dense kernel since the last check (0: every product completed)."""
        e = ctypes.c_int(0)
        L.check(L.lib().bk_plan_dense_check(self._h, ctypes.byref(e)))
        return e.value

    def empty(self, batch=1, device="cuda"):
        """A zeroed [batch, n_comp, pitch] tensor of the plan's dtype."""
        return torch.zeros(batch, self.n_comp, self.pitch, dtype=self.dtype, device=device)

    def close(self):
        if self._h:
            L.lib().bk_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_f64_transform(mode):
    """Arithmetic of FP64 transforms for plans and problems created afterwards: 1 double-float,
    0 binary64, -1 the default (double-float from N = 2^18 on)."""
    L.check(L.lib().bk_set_f64_transform(int(mode)))


def set_f64_precond(mode):
    """Precision of the preconditioner of FP64 problems created afterwards: 1 FP32, 0 FP64, -1 the
    default (FP64)."""
    L.check(L.lib().bk_set_f64_precond(int(mode)))


def set_krylov_graphs(mode):
    """GMRES restart cycles as CUDA graphs: 0 or -1 (default) never, 1 for every problem of
    fixed final time."""
    L.check(L.lib().bk_set_krylov_graphs(int(mode)))


def set_krylov_wait_limit(seconds):
    """Bound (s) on the host wait for a GMRES graph cycle; <= 0 restores the default."""
    L.check(L.lib().bk_set_krylov_wait_limit(float(seconds)))


def _check_vec(plan, t, batch):
    if not t.is_cuda or t.dtype != plan.dtype:
        raise ValueError("expected a CUDA tensor of dtype %s" % plan.dtype)
    if not t.is_contiguous() or t.numel() < batch * plan.n_comp * plan.pitch:
        raise ValueError("vector must be contiguous with batch * n_comp * pitch elements")


def birkhoff_apply(plan, v, out, batch=None, stream=None):
    """out = B v (FastBV) for [batch, n_comp, pitch] tensors."""
    batch = v.shape[0] if (batch is None and v.dim() == 3) else (batch or 1)
    _check_vec(plan, v, batch)
    _check_vec(plan, out, batch)
    L.check(L.lib().birkhoff_apply(plan.handle, L.ptr(v), L.ptr(out), int(batch),
                                   L.stream_ptr(stream)))
    return out


def birkhoff_apply_T(plan, v, out, batch=None, stream=None):
    """out = B^T v for [batch, n_comp, pitch] tensors."""
    batch = v.shape[0] if (batch is None and v.dim() == 3) else (batch or 1)
    _check_vec(plan, v, batch)
    _check_vec(plan, out, batch)
    L.check(L.lib().birkhoff_apply_T(plan.handle, L.ptr(v), L.ptr(out), int(batch),
                                     L.stream_ptr(stream)))
    return out


def birkhoff_apply_batch(plans, vs, outs, batches=None, trans=False, stream=None):
    """out_i = B_i v_i (or B_i^T v_i) for plans of one dtype and any mix of N, in one call (one
    launch per pass for the plans on the single-CTA and unsplit four-step paths)."""
    n = len(plans)
    if not (len(vs) == n and len(outs) == n) or n == 0:
        raise ValueError("plans, vs and outs must have the same non-zero length")
    if batches is None:
        batches = [v.shape[0] if v.dim() == 3 else 1 for v in vs]
    for p, v, o, b in zip(plans, vs, outs, batches):
        _check_vec(p, v, b)
        _check_vec(p, o, b)
    def addr(x):
        return x.value if isinstance(x, ctypes.c_void_p) else int(x)
    arr_p = (ctypes.c_void_p * n)(*[addr(p.handle) for p in plans])
    arr_v = (ctypes.c_void_p * n)(*[v.data_ptr() for v in vs])
    arr_o = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    arr_b = (ctypes.c_int * n)(*[int(b) for b in batches])
    L.check(L.lib().birkhoff_apply_batch(arr_p, arr_v, arr_o, arr_b, n, int(bool(trans)),
                                         L.stream_ptr(stream)))
    return outs


def birkhoff_apply_b(plan, v, out, batch=None, stream=None):
    """out = B^b v (b-form Birkhoff product: the basis vanishes at the final point)."""
    batch = v.shape[0] if (batch is None and v.dim() == 3) else (batch or 1)
    _check_vec(plan, v, batch)
    _check_vec(plan, out, batch)
    L.check(L.lib().birkhoff_apply_b(plan.handle, L.ptr(v), L.ptr(out), int(batch), L.stream_ptr(stream)))
    return out


def birkhoff_apply_b_T(plan, v, out, batch=None, stream=None):
    """out = (B^b)^T v."""
    batch = v.shape[0] if (batch is None and v.dim() == 3) else (batch or 1)
    _check_vec(plan, v, batch)
    _check_vec(plan, out, batch)
    L.check(L.lib().birkhoff_apply_b_T(plan.handle, L.ptr(v), L.ptr(out), int(batch), L.stream_ptr(stream)))
    return out


class Problem:
    """A bk_problem: dynamics kind, grid and linearisation state."""

    def __init__(self, kind, N, dtype=torch.float64, t0=0.0, tf=1.0, params=(), stream=None):
        lib = L.lib()
        self._h = ctypes.c_void_p()
        self.dtype_code = _dtype_code(dtype)
        self.dtype = _TORCH_DTYPE[self.dtype_code]
        arr = (ctypes.c_double * max(1, len(params)))(*[float(x) for x in params])
        L.check(lib.bk_problem_create(ctypes.byref(self._h), int(kind), arr, len(params), int(N),
                                      self.dtype_code, float(t0), float(tf),
                                      L.stream_ptr(stream)))
        nx, nu, ne = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        pitch, klen, slen = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        L.check(lib.bk_problem_info(self._h, ctypes.byref(nx), ctypes.byref(nu), ctypes.byref(ne),
                                    ctypes.byref(pitch), ctypes.byref(klen), ctypes.byref(slen)))
        self.kind, self.N, self.L = int(kind), int(N), int(N) + 1
        self.t0, self.tf, self.params = float(t0), float(tf), tuple(params)
        self.n_x, self.n_u, self.n_e = nx.value, nu.value, ne.value
        self.pitch, self.kkt_len, self.state_len = pitch.value, klen.value, slen.value

    @property
    def handle(self):
        return self._h

    def set_params(self, t0, tf, params):
        """Reuse this problem for new parameters and interval (no allocation)."""
        arr = (ctypes.c_double * max(1, len(params)))(*[float(x) for x in params])
        L.check(L.lib().bk_problem_set_params(self._h, arr, len(params), float(t0), float(tf)))
        self.t0, self.tf, self.params = float(t0), float(tf), tuple(params)

    def set_control_bounds(self, lo=None, hi=None):
        """Bounds lo[q] <= u_q(t) <= hi[q] on the controls (sequences of length n_u, +-inf or
        None for no bound; both None clears them). newton_solve then solves the problem with a
        logarithmic barrier on the bounds (fixed-final-time kinds with a cost only)."""
        if lo is None and hi is None:
            L.check(L.lib().bk_problem_set_control_bounds(self._h, None, None, 0))
            return
        n = self.n_u
        lo = [-float("inf")] * n if lo is None else [float(x) for x in lo]
        hi = [float("inf")] * n if hi is None else [float(x) for x in hi]
        if len(lo) != n or len(hi) != n:
            raise ValueError(f"bounds need {n} entries each")
        L.check(L.lib().bk_problem_set_control_bounds(self._h, (ctypes.c_double * n)(*lo),
                                                      (ctypes.c_double * n)(*hi), n))

    def set_terminal_bounds(self, lo=None, hi=None):
        """Bounds lo[r] <= x_{idx_r}(t_f) <= hi[r] in place of terminal condition r (sequences of
        length n_e; a row whose bounds are both infinite keeps its equality; both None removes
        them). Solved by the same barrier stages as the control bounds."""
        if lo is None and hi is None:
            L.check(L.lib().bk_problem_set_terminal_bounds(self._h, None, None, 0))
            return
        n = self.n_e
        lo = [-float("inf")] * n if lo is None else [float(x) for x in lo]
        hi = [float("inf")] * n if hi is None else [float(x) for x in hi]
        if len(lo) != n or len(hi) != n:
            raise ValueError(f"terminal bounds need {n} entries each")
        L.check(L.lib().bk_problem_set_terminal_bounds(self._h, (ctypes.c_double * n)(*lo),
                                                       (ctypes.c_double * n)(*hi), n))

    def set_barrier(self, mu0=0.1, mu_final=1e-6, form="primal"):
        """Barrier schedule of a bounded solve: stages mu0, mu0/10, ... down to mu_final, in the
        "primal" or "primal_dual" form. The residual and operator calls use mu_final (primal)."""
        code = {"primal": L.BK_BARRIER_PRIMAL, "primal_dual": L.BK_BARRIER_PRIMAL_DUAL}[form]
        L.check(L.lib().bk_problem_set_barrier(self._h, float(mu0), float(mu_final), code))

    def device_bytes(self):
        return int(L.lib().bk_problem_device_bytes(self._h))

    def precond_dtype(self):
        """torch dtype of the preconditioner (float32 for FP64 problems with the FP32 preconditioner)."""
        d = ctypes.c_int(0)
        L.check(L.lib().bk_problem_precond_dtype(self._h, ctypes.byref(d)))
        return _TORCH_DTYPE[d.value]

    def vec_len(self, op):
        return self.kkt_len if op == L.BK_OP_KKT else self.state_len

    def zeros(self, op=L.BK_OP_KKT, dtype=None, device="cuda"):
        return torch.zeros(self.vec_len(op), dtype=dtype or self.dtype, device=device)

    def linearize(self, z_lin, stream=None):
        if z_lin.dtype != torch.float64 or not z_lin.is_cuda or z_lin.numel() < self.kkt_len:
            raise ValueError("z_lin must be a CUDA float64 KKT vector")
        L.check(L.lib().bk_linearize(self._h, L.ptr(z_lin), L.stream_ptr(stream)))

    def residual(self, z, F_out, stream=None):
        """KKT residual at z into F_out; returns the weighted norm (synchronous)."""
        wn = ctypes.c_double()
        L.check(L.lib().bk_kkt_residual(self._h, L.ptr(z), L.ptr(F_out), ctypes.byref(wn),
                                        L.stream_ptr(stream)))
        return wn.value

    # layout helpers (views into a KKT vector) -------------------------------------------
    def split(self, z):
        P = self.pitch
        nx, nu = self.n_x, self.n_u
        X = z[:nx * P].view(nx, P)[:, :self.L]
        U = z[nx * P:(nx + nu) * P].view(nu, P)[:, :self.L]
        lam = z[(nx + nu) * P:(2 * nx + nu) * P].view(nx, P)[:, :self.L]
        nu_ = z[(2 * nx + nu) * P:(2 * nx + nu) * P + self.n_e]
        return X, U, lam, nu_

    def pack(self, X, U, lam=None, nu=None, dtype=torch.float64, device="cuda", s=None):
        z = torch.zeros(self.kkt_len, dtype=dtype, device=device)
        Xv, Uv, lv, nv = self.split(z)
        Xv.copy_(torch.as_tensor(X))
        Uv.copy_(torch.as_tensor(U))
        if lam is not None:
            lv.copy_(torch.as_tensor(lam))
        if nu is not None and self.n_e:
            nv.copy_(torch.as_tensor(nu))
        if self.free_time:
            z[self.s_index] = 0.5 * (self.tf - self.t0) if s is None else float(s)
        return z

    @property
    def free_time(self):
        """BK_ORBIT_MT: the time scale s = (t_f - t_0)/2 is an unknown kept in the KKT vector."""
        return self.kind == L.BK_ORBIT_MT

    @property
    def s_index(self):
        """Index of s in a KKT vector (the tail slot after nu) for a free final time."""
        return (2 * self.n_x + self.n_u) * self.pitch + self.n_e

    def close(self):
        if self._h:
            L.lib().bk_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def min_time_seed(mt, me, z_me, z_mt, stream=None):
    """Seed the minimum-time problem `mt` (BK_ORBIT_MT) from the solved minimum-energy transfer
    z_me of `me` (BK_ORBIT, same N): writes z_mt (synchronous)."""
    for z, p in ((z_me, me), (z_mt, mt)):
        if z.dtype != torch.float64 or not z.is_cuda or z.numel() < p.kkt_len:
            raise ValueError("z_me and z_mt must be CUDA float64 KKT vectors of their problems")
    L.check(L.lib().bk_min_time_seed(mt.handle, me.handle, L.ptr(z_me), L.ptr(z_mt), L.stream_ptr(stream)))
    return z_mt


def kkt_apply(prob, op, x, out, stream=None):
    L.check(L.lib().kkt_apply(prob.handle, int(op), L.ptr(x), L.ptr(out), L.stream_ptr(stream)))
    return out


def precond_apply(prob, op, x, out, transpose=False, stream=None):
    L.check(L.lib().precond_apply(prob.handle, int(op), L.ptr(x), L.ptr(out), int(bool(transpose)),
                                  L.stream_ptr(stream)))
    return out


def krylov_workspace(prob, op, restart=30):
    nbytes = L.lib().bk_krylov_workspace_bytes(prob.handle, int(op), int(restart))
    return torch.empty(max(1, (nbytes + 255) // 256 * 32), dtype=torch.float64, device="cuda")


def krylov_solve(prob, op, rhs, sol, rtol=1e-10, restart=30, max_iter=300, use_precond=True,
                 workspace=None, stream=None, raise_on_fail=True):
    """Right-preconditioned GMRES(m); returns a dict of the bk_krylov_info fields."""
    if workspace is None:
        workspace = krylov_workspace(prob, op, restart)
    opts = L.KrylovOpts(float(rtol), int(restart), int(max_iter), int(bool(use_precond)))
    info = L.KrylovInfo()
    st = L.lib().krylov_solve(prob.handle, int(op), L.ptr(rhs), L.ptr(sol), ctypes.byref(opts),
                              ctypes.byref(info), L.ptr(workspace), L.stream_ptr(stream))
    out = dict(iterations=info.iterations, restarts=info.restarts, rel_resid=info.rel_resid,
               converged=bool(info.converged), status=st)
    if raise_on_fail and st != 0:
        L.check(st)
    return out


def newton_workspace(prob, restart=30):
    nbytes = L.lib().bk_newton_workspace_bytes(prob.handle, int(restart))
    return torch.empty(max(1, (nbytes + 255) // 256 * 32), dtype=torch.float64, device="cuda")


def newton_solve(prob, z, tol=1e-10, max_iter=0, krylov_rtol=0.0, restart=30, max_krylov=0,
                 ir_rtol=1e-10, max_refine=0, precond_reuse=0, workspace=None, stream=None,
                 raise_on_fail=True, weighted_inner=False):
    """Newton-Lagrange solve in place on the FP64 KKT vector z; returns the info fields.
    Zero-valued options take the library defaults for the problem's precision;
    weighted_inner runs the inner GMRES in the merit norm ||.||_W."""
    if workspace is None:
        workspace = newton_workspace(prob, restart)
    opts = L.NewtonOpts(float(tol), int(max_iter), float(krylov_rtol), int(restart),
                        int(max_krylov), float(ir_rtol), int(max_refine), int(precond_reuse),
                        int(bool(weighted_inner)))
    info = L.NewtonInfo()
    st = L.lib().newton_solve(prob.handle, L.ptr(z), ctypes.byref(opts), ctypes.byref(info),
                              L.ptr(workspace), L.stream_ptr(stream))
    out = dict(iterations=info.iterations, krylov_iterations=info.krylov_iterations,
               kkt_solves=info.kkt_solves, backtracks=info.backtracks, residual=info.residual,
               residual0=info.residual0, converged=bool(info.converged),
               precond_builds=info.precond_builds, status=st)
    if raise_on_fail and st != 0:
        L.check(st)
    return out
