"""Parity of the preconditioner sweeps at every scan level (precond_apply, state and KKT).

The library runs the sweep of FastPinvY (corrected) as an affine scan: segments of 8 nodes
(FP64) or 16 (FP32), then levels of blocks of 32 items, so the level count grows with N:
FP64 N = 2^13 and 2^16 run 3 levels, 2^18 and 2^20 run 4; FP32 N = 2^14 and 2^17 run 3,
2^19 runs 4. N = 1000 (dense products) has a ragged last segment and block. Each size is
compared with the oracle's sequential sweeps (``fastpinvy_block`` / ``_T``, pinned to the dense
P in tests/test_oracle_birkhoff.py) and, for the KKT preconditioner K-tilde^-1, with the
matrix-free oracle's block elimination (pinned to the dense K-tilde in
tests/test_oracle_matfree.py). Flexible GMRES converges even with a wrong preconditioner, so
these comparisons are the only check of the upper scan levels.
"""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from oracle import problems as op
from oracle.matfree import MatFreeKKT
from paper_2509_01855_gb300 import synth
from tests.helpers import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu

RF, TF = 1.5, 20.0


def _setup(N, dtype, pc32=False):
    """Library problem, matrix-free oracle and a linearisation point (noisy spiral, random
    multipliers) of the orbit problem. FP64 problems get the FP64 preconditioner unless pc32."""
    from paper_2509_01855_gb300 import _lib, api
    oprob = op.Problem(op.ORBIT, 0.0, TF, (0.01, RF))
    M = MatFreeKKT(oprob, N)
    api.set_f64_precond(1 if pc32 else 0)
    try:
        prob = api.Problem(_lib.BK_ORBIT, N, dtype, 0.0, TF, (0.01, RF))
    finally:
        api.set_f64_precond(-1)
    assert prob.precond_dtype() == (torch.float32 if pc32 else dtype)
    g = synth.rng("sweep-lin", N)
    X, U = synth.orbit_guess(M.t, RF, TF)
    X = X + 0.01 * g.standard_normal(X.shape)
    U = U + 0.001 * g.standard_normal(U.shape)
    lam = 0.01 * g.standard_normal((4, M.L))
    nu = 0.01 * g.standard_normal(3)
    vec = M.pack(X, U, lam, nu)
    prob.linearize(from_packed(prob, vec))
    return api, _lib, prob, M, vec


def _levels(N, dtype):
    seg = 8 if dtype == torch.float64 else 16
    n = (N + 1 + seg - 1) // seg
    lev = 1
    while n > 32:
        n = (n + 31) // 32
        lev += 1
    return lev


def _sequential_sweeps_fp32(w, J, Y):
    """Rounding model for the FP32 tolerance: the forward and backward substitutions through
    the rows of P (the recurrences of tests/test_oracle_birkhoff.py's pinned sweeps) carried out
    entirely in binary32 on binary32-rounded inputs."""
    f = np.float32
    w, J, Y = w.astype(f), J.astype(f), Y.astype(f)
    L, n, _ = J.shape
    I = np.eye(n, dtype=f)
    fw = np.zeros((n, L), f)
    sig = np.zeros(n, f)
    for k in range(L):
        xi = np.linalg.solve(I - f(0.5) * w[k] * J[k], Y[:, k] + sig)
        sig = sig + w[k] * (J[k] @ xi)
        fw[:, k] = xi
    bw = np.zeros((n, L), f)
    rho = np.zeros(n, f)
    for j in range(L - 1, -1, -1):
        y = np.linalg.solve(I - f(0.5) * w[j] * J[j].T, Y[:, j] + w[j] * (J[j].T @ rho))
        rho = rho + y
        bw[:, j] = y
    return fw.astype(np.float64), bw.astype(np.float64)


STATE_CASES = [(1 << 13, torch.float64), (1 << 16, torch.float64), (1 << 18, torch.float64),
               (1 << 20, torch.float64), (1000, torch.float64),
               (1 << 14, torch.float32), (1 << 17, torch.float32), (1 << 19, torch.float32),
               (1000, torch.float32)]


@pytest.mark.parametrize("N,dtype", STATE_CASES)
def test_state_preconditioner_every_level(N, dtype):
    api, lib, prob, M, vec = _setup(N, dtype)
    assert N == 1000 or _levels(N, dtype) >= 3
    X, U, _, _ = M.split(vec)
    Jx, _ = M.prob.jac(X, U)
    Y = synth.gaussian((4, M.L), "sweep-rhs", N)
    x = from_packed(prob, Y.ravel(), dtype, op_kkt=False)
    out = torch.zeros_like(x)
    ref = ob.fastpinvy_block(M.s * M.w, Jx, Y)
    refT = ob.fastpinvy_block_T(M.s * M.w, Jx, Y)
    if dtype == torch.float64:
        tol = tolT = 1e-12
    else:
        # An FP32 sweep carries FP32 rounding along the whole recurrence (the propagator of the
        # linearised orbit over t_f = 20), so its error grows with N. The bound is 4x the error of
        # the oracle's own sequential sweep run in FP32 on FP32-rounded inputs, and at least 2e-5.
        seq, seqT = _sequential_sweeps_fp32(M.s * M.w, Jx, Y)
        tol = max(2e-5, 4.0 * rel(seq.ravel(), ref.ravel()))
        tolT = max(2e-5, 4.0 * rel(seqT.ravel(), refT.ravel()))
    api.precond_apply(prob, lib.BK_OP_STATE, x, out, transpose=False)
    e = rel(to_packed(prob, out, False), ref.ravel())
    assert torch.all(out.view(4, prob.pitch)[:, prob.L:] == 0)
    api.precond_apply(prob, lib.BK_OP_STATE, x, out, transpose=True)
    eT = rel(to_packed(prob, out, False), refT.ravel())
    print("state sweep N=%d %s: P^-1 %.2e (bound %.2e), P^-T %.2e (bound %.2e)" % (N, dtype, e, tol, eT, tolT))
    assert e < tol and eT < tolT


KKT_CASES = [(1 << 13, torch.float64), (1 << 16, torch.float64), (1 << 14, torch.float32),
             (1 << 17, torch.float32)]


@pytest.mark.parametrize("N,dtype", KKT_CASES)
def test_kkt_preconditioner_every_level(N, dtype):
    api, lib, prob, M, vec = _setup(N, dtype)
    M.linearize_precond(vec)
    d = synth.gaussian(M.n, "kkt-pre-rhs", N)
    x = from_packed(prob, d, dtype)
    out = torch.zeros_like(x)
    api.precond_apply(prob, lib.BK_OP_KKT, x, out)
    got = to_packed(prob, out)
    ref = M.precond_solve(d)
    # K-tilde is badly scaled (its control block is s w, w_0 ~ 1/N^2): relative 2-norm
    assert rel(got, ref) < (1e-10 if dtype == torch.float64 else 1e-3)


@pytest.mark.parametrize("N", [1 << 16, 1 << 20])
def test_fp64_problem_with_fp32_preconditioner(N):
    """An FP64 problem whose preconditioner runs in FP32: precond_apply (FP64 in, FP64 out) within
    the FP32 bound of the sweeps, for P^-1 and for K-tilde^-1."""
    api, lib, prob, M, vec = _setup(N, torch.float64, pc32=True)
    X, U, _, _ = M.split(vec)
    Jx, _ = M.prob.jac(X, U)
    Y = synth.gaussian((4, M.L), "sweep-rhs", N)
    x = from_packed(prob, Y.ravel(), torch.float64, op_kkt=False)
    out = torch.zeros_like(x)
    api.precond_apply(prob, lib.BK_OP_STATE, x, out, transpose=False)
    ref = ob.fastpinvy_block(M.s * M.w, Jx, Y)
    assert rel(to_packed(prob, out, False), ref.ravel()) < 2e-5
    if N <= 1 << 16:
        M.linearize_precond(vec)
        d = synth.gaussian(M.n, "kkt-pre-rhs", N)
        xk = from_packed(prob, d, torch.float64)
        ok = torch.zeros_like(xk)
        api.precond_apply(prob, lib.BK_OP_KKT, xk, ok)
        assert rel(to_packed(prob, ok), M.precond_solve(d)) < 1e-3
