"""N that is not a power of two above the dense range (1024 < N <= 2^22 in FP64, 2^23 in FP32):
each DCT-I's length-N DFT through Bluestein's convolution on the power-of-two four-step FFT.
Products against the dense oracle (B^a from its definition, N = 1100), the oracle's FastBV chain
(SciPy's DCT-I of any length, N = 3000), and the exact integrals of Chebyshev modes (N near 10^5
and 10^6); an orbit solve at N = 3000 against the matrix-free oracle on the same grid."""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from oracle import problems as op
from oracle.matfree import MatFreeKKT
from paper_2509_01855_gb300 import synth
from tests.helpers import from_packed, to_packed

pytestmark = pytest.mark.gpu


def _prod(N, dtype, V, trans, t0=0.0, tf=2.0):
    from paper_2509_01855_gb300 import api
    plan = api.Plan(N, n_comp=V.shape[0], max_batch=1, dtype=dtype, t0=t0, tf=tf)
    assert plan.shape()["path"] == "bluestein"
    v = plan.empty(1)
    v[0, :, :N + 1] = torch.as_tensor(V)
    fn = api.birkhoff_apply_T if trans else api.birkhoff_apply
    out = fn(plan, v, plan.empty(1))
    assert torch.all(out[0, :, N + 1:] == 0)
    return out[0, :, :N + 1].double().cpu().numpy()


@pytest.fixture(scope="module")
def dense_1100():
    return ob.dense_B(1100, 0.0, 2.0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("trans", [False, True])
def test_bluestein_vs_dense_oracle(dtype, trans, dense_1100):
    N = 1100
    V = synth.gaussian((3, N + 1), "anyn", N)
    got = _prod(N, dtype, V, trans)
    ref = V @ (dense_1100 if trans else dense_1100.T)
    e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print("bluestein N=%d %s %s: %.2e" % (N, dtype, "B^T" if trans else "B", e))
    # the dense quadrature oracle itself is good to ~5e-13 here
    assert e < (1e-12 if dtype == torch.float64 else 1e-5)


@pytest.mark.parametrize("N", [3000, 4095, 12345])
def test_bluestein_vs_fastbv_oracle(N):
    V = synth.gaussian((2, N + 1), "anyn-fbv", N)
    for trans, ref in ((False, ob.fastbv(V, 0.0, 2.0)), (True, ob.fastbv_T(V, 0.0, 2.0))):
        got = _prod(N, torch.float64, V, trans)
        e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print("bluestein N=%d %s vs FastBV: %.2e" % (N, "B^T" if trans else "B", e))
        assert e < 1e-12


@pytest.mark.parametrize("N", [100003, 1000003])
def test_bluestein_exact_chebyshev_integrals(N):
    """v = sum alpha_k T_k with the modes next to N: B v is the exact integral (Eq. intChebPoly=)."""
    modes, alphas = synth.sparse_modes(N, 26, "anyn-modes")
    vv, Bv = ob.sparse_mode_pair(N, modes, alphas, 0.0, 2.0)
    got = _prod(N, torch.float64, vv[None, :], False)[0]
    e = np.linalg.norm(got - Bv) / np.linalg.norm(Bv)
    print("bluestein exact modes N=%d: %.2e" % (N, e))
    assert e < 1e-12


def test_bluestein_orbit_solve_matches_oracle_same_grid():
    from paper_2509_01855_gb300 import _lib, api
    N, rf, tf = 3000, 1.5, 20.0
    M = MatFreeKKT(op.Problem(op.ORBIT, 0.0, tf, (0.01, rf)), N)
    X, U = synth.orbit_guess(M.t, rf, tf)
    v0 = M.pack(X, U, np.zeros((4, M.L)), np.zeros(3))
    ref, rinfo = M.newton(v0, tol=1e-12)
    assert rinfo["converged"]
    prob = api.Problem(_lib.BK_ORBIT, N, torch.float64, 0.0, tf, (0.01, rf))
    z = from_packed(prob, v0)
    info = api.newton_solve(prob, z, tol=1e-11, krylov_rtol=1e-12)
    assert info["converged"] and info["iterations"] == rinfo["iters"]
    Xg, Ug, _, _ = M.split(to_packed(prob, z))
    Xr, Ur, _, _ = M.split(ref)
    assert np.abs(Xg - Xr).max() < 1e-9
    assert np.sqrt(np.sum(M.s * M.w * (Ug - Ur) ** 2)) < 1e-9


def test_bluestein_limits():
    from paper_2509_01855_gb300 import _lib, api
    from paper_2509_01855_gb300._lib import BirkhoffError
    with pytest.raises(BirkhoffError):
        api.Plan((1 << 22) + 1, dtype=torch.float64)
    p = api.Plan(1025, dtype=torch.float64)
    assert p.shape()["path"] == "bluestein" and not p.is_dense()
