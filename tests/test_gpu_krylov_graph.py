"""GMRES with the device-resident Arnoldi step: restart cycles as CUDA graphs against the
host-launched form.

Both forms keep the Hessenberg matrix, the Givens rotations and the stopping test on the device
and run the same kernels on the same values; the graph form only routes each step's vectors
through fixed buffers and lets a conditional WHILE node repeat the step. The solutions, iteration
counts and residuals must therefore agree bit for bit. The graph wait is bounded: a test sets a
limit no cycle can meet and checks the BK_ERR_TIMEOUT status, then that the context and the
problem still work.
"""
import numpy as np
import pytest
import torch

from oracle import problems as op
from oracle.matfree import MatFreeKKT
from paper_2509_01855_gb300 import synth
from tests.helpers import from_packed

pytestmark = pytest.mark.gpu

RF, TF = 1.5, 20.0


def _setup(N, dtype, seed=0):
    from paper_2509_01855_gb300 import _lib, api
    M = MatFreeKKT(op.Problem(op.ORBIT, 0.0, TF, (0.01, RF)), N)
    prob = api.Problem(_lib.BK_ORBIT, N, dtype, 0.0, TF, (0.01, RF))
    g = synth.rng("graph-lin", N, seed)
    X, U = synth.orbit_guess(M.t, RF, TF)
    X = X + 0.01 * g.standard_normal(X.shape)
    U = U + 0.001 * g.standard_normal(U.shape)
    vec = M.pack(X, U, 0.01 * g.standard_normal((4, M.L)), 0.01 * g.standard_normal(3))
    z = from_packed(prob, vec)
    prob.linearize(z)
    return api, _lib, prob, M


def _solve(api, prob, opc, rhs, mode, **kw):
    api.set_krylov_graphs(mode)
    try:
        sol = torch.full_like(rhs, float("nan"))
        info = api.krylov_solve(prob, opc, rhs, sol, raise_on_fail=False, **kw)
        torch.cuda.synchronize()
    finally:
        api.set_krylov_graphs(-1)
    return sol, info


@pytest.mark.parametrize("N,dtype,opname,kw", [
    (256, torch.float64, "KKT", dict(rtol=1e-12, restart=30)),
    (1000, torch.float64, "KKT", dict(rtol=1e-12, restart=30)),
    (4096, torch.float32, "KKT", dict(rtol=1e-5, restart=30)),
    (2048, torch.float64, "STATE", dict(rtol=1e-12, restart=30)),
    (512, torch.float64, "KKT", dict(rtol=1e-12, restart=4, max_iter=400)),    # several restarts
    (512, torch.float64, "KKT", dict(rtol=1e-15, restart=4, max_iter=10)),     # iteration cap
    (128, torch.float64, "STATE", dict(rtol=1e-10, restart=30, use_precond=False)),
])
def test_graph_cycles_match_host_steps_bitwise(N, dtype, opname, kw):
    api, lib, prob, M = _setup(N, dtype)
    opc = lib.BK_OP_KKT if opname == "KKT" else lib.BK_OP_STATE
    n = prob.kkt_len if opname == "KKT" else prob.state_len
    g = synth.rng("graph-rhs", N, opname)
    # a right-hand side with zero padding (the layout's unused slots), as from_packed makes
    rhs = from_packed(prob, g.standard_normal(M.n if opname == "KKT" else 4 * M.L), dtype=dtype,
                      op_kkt=opname == "KKT")
    assert rhs.numel() == n
    x0, i0 = _solve(api, prob, opc, rhs, 0, **kw)
    x1, i1 = _solve(api, prob, opc, rhs, 1, **kw)
    assert i0 == i1, (i0, i1)
    assert torch.equal(x0, x1)
    assert torch.isfinite(x0).all()
    if kw.get("max_iter") == 10:
        assert i0["status"] == 4 and i0["iterations"] == 10 and i0["restarts"] >= 3
    elif kw.get("restart") == 4:
        assert i0["restarts"] >= 2 and i0["status"] in (0, 4), i0
    else:
        assert i0["converged"], i0
    # a second graph solve reuses the captured cycle and gives the same answer again
    x2, i2 = _solve(api, prob, opc, rhs, 1, **kw)
    assert i2 == i1 and torch.equal(x2, x1)


@pytest.mark.parametrize("N,dtype", [(512, torch.float64), (2048, torch.float32)])
def test_newton_graph_matches_host_bitwise(N, dtype):
    from paper_2509_01855_gb300 import _lib, api
    M = MatFreeKKT(op.Problem(op.ORBIT, 0.0, TF, (0.01, RF)), N)
    X, U = synth.orbit_guess(M.t, RF, TF)
    vec = M.pack(X, U, np.zeros((4, M.L)), np.zeros(3))
    out = []
    for mode in (0, 1):
        prob = api.Problem(_lib.BK_ORBIT, N, dtype, 0.0, TF, (0.01, RF))
        z = from_packed(prob, vec)
        api.set_krylov_graphs(mode)
        try:
            info = api.newton_solve(prob, z, tol=1e-10)
        finally:
            api.set_krylov_graphs(-1)
        torch.cuda.synchronize()
        assert info["converged"], info
        out.append((z.clone(), info))
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_params_change_recaptures():
    """bk_problem_set_params changes the time scale the captured kernels take by value: the next
    solve captures afresh and still matches the host form."""
    api, lib, prob, M = _setup(1000, torch.float64)
    rhs = from_packed(prob, synth.rng("graph-rhs-p").standard_normal(M.n))
    _solve(api, prob, lib.BK_OP_KKT, rhs, 1, rtol=1e-12)
    prob.set_params(0.0, 25.0, (0.01, 1.7))
    X, U = synth.orbit_guess(M.t, 1.7, 25.0)
    prob.linearize(from_packed(prob, M.pack(X, U, np.zeros((4, M.L)), np.zeros(3))))
    x0, i0 = _solve(api, prob, lib.BK_OP_KKT, rhs, 0, rtol=1e-12)
    x1, i1 = _solve(api, prob, lib.BK_OP_KKT, rhs, 1, rtol=1e-12)
    assert i0 == i1 and i0["converged"] and torch.equal(x0, x1)


def test_graph_wait_limit_returns_timeout():
    """A wait limit below any cycle's run time: the solve returns BK_ERR_TIMEOUT with the cycle
    possibly still running; after a stream sync the problem and the context work as before."""
    api, lib, prob, M = _setup(4096, torch.float64)
    rhs = from_packed(prob, synth.rng("graph-rhs-t").standard_normal(M.n))
    ref, iref = _solve(api, prob, lib.BK_OP_KKT, rhs, 0, rtol=1e-12)
    api.set_krylov_wait_limit(1e-9)
    try:
        _, info = _solve(api, prob, lib.BK_OP_KKT, rhs, 1, rtol=1e-12)
    finally:
        api.set_krylov_wait_limit(0)
    torch.cuda.synchronize()
    assert info["status"] == 5, info
    x, i1 = _solve(api, prob, lib.BK_OP_KKT, rhs, 1, rtol=1e-12)
    assert i1 == iref and torch.equal(x, ref)


def test_settings_reject_bad_values():
    from paper_2509_01855_gb300 import _lib, api
    with pytest.raises(_lib.BirkhoffError):
        api.set_krylov_graphs(2)
    with pytest.raises(_lib.BirkhoffError):
        api.set_krylov_wait_limit(float("nan"))
    with pytest.raises(_lib.BirkhoffError):
        api.set_krylov_wait_limit(1e7)


def test_graph_cycles_from_concurrent_threads():
    """Four host threads, each with its own problem (its own t_f), stream and workspace, solve
    with graph cycles at the same time (captures are serialised inside the library, the cycles
    run concurrently); every solution equals the host-form solution of the same problem."""
    import threading
    from paper_2509_01855_gb300 import _lib, api
    N = 512
    M = MatFreeKKT(op.Problem(op.ORBIT, 0.0, TF, (0.01, RF)), N)
    X, U = synth.orbit_guess(M.t, RF, TF)
    vec = M.pack(X, U, np.zeros((4, M.L)), np.zeros(3))
    tfs = [18.0, 20.0, 22.0, 24.0]

    def solve_all(mode):
        api.set_krylov_graphs(mode)
        out, errs = [None] * len(tfs), []

        def work(i):
            try:
                st = torch.cuda.Stream()
                with torch.cuda.stream(st):
                    prob = api.Problem(_lib.BK_ORBIT, N, torch.float64, 0.0, tfs[i], (0.01, RF))
                    ws = api.newton_workspace(prob)
                    for rep in range(2):
                        z = from_packed(prob, vec)
                        info = api.newton_solve(prob, z, tol=1e-10, workspace=ws, stream=st)
                    st.synchronize()
                    out[i] = (z.clone(), info)
            except Exception as e:  # reported below
                errs.append(e)

        threads = [threading.Thread(target=work, args=(i,)) for i in range(len(tfs))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        api.set_krylov_graphs(-1)
        assert not errs, errs
        return out

    ref = solve_all(0)
    got = solve_all(1)
    for (zr, ir), (zg, ig) in zip(ref, got):
        assert ir["converged"] and ir == ig
        assert torch.equal(zr, zg)
