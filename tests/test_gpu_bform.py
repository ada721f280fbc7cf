"""b-form Birkhoff products (birkhoff_apply_b, birkhoff_apply_b_T): the basis of Eq.
birk-conditions that vanishes at the final point, B^b = B^a - 1 w^T, against the oracle's dense
B^b formed from its definition (Gauss-Legendre integrals of the Lagrange basis over [tau_i, 1])
on the product paths: one CTA (N = 64; N = 512 in FP32), dense (N = 100), four-step (N = 512 in
FP64; N = 8192 in FP32 and 2^18 with double-float arithmetic against the oracle's FastBV chain
minus its last value) and Bluestein (N = 1100). (The dense quadrature oracle itself drifts to
~5e-12 at N = 4096, so larger N are checked through FastBV.)"""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu

T0, TF = 0.0, 3.0


def _run(N, dtype, V, trans):
    from paper_2509_01855_gb300 import api
    plan = api.Plan(N, n_comp=V.shape[0], max_batch=1, dtype=dtype, t0=T0, tf=TF)
    v = plan.empty(1)
    v[0, :, :N + 1] = torch.as_tensor(V)
    fn = api.birkhoff_apply_b_T if trans else api.birkhoff_apply_b
    out = fn(plan, v, plan.empty(1))
    assert torch.all(out[0, :, N + 1:] == 0)
    return out[0, :, :N + 1].double().cpu().numpy(), plan


@pytest.mark.parametrize("N,dtype", [(64, torch.float64), (100, torch.float64), (512, torch.float64),
                                     (512, torch.float32), (1100, torch.float64)])
@pytest.mark.parametrize("trans", [False, True])
def test_bform_vs_dense_definition(N, dtype, trans):
    Bb = 0.5 * (TF - T0) * ob.dense_Bb(N)
    V = synth.gaussian((2, N + 1), "bform", N)
    got, _ = _run(N, dtype, V, trans)
    ref = V @ (Bb if trans else Bb.T)
    e = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    tol = 1e-5 if dtype == torch.float32 else (2e-12 if N > 1024 else 1e-12)
    assert e < tol, e
    if not trans:
        assert np.abs(got[:, N]).max() == 0.0


@pytest.mark.parametrize("N,dtype", [(1 << 18, torch.float64), (8192, torch.float32)])
def test_bform_large_N_and_time_identity(N, dtype):
    """B^b v = FastBV(v) - its last value (B^bT through the adjoint identity <B^b u, v> = <u, B^bT v>)
    and B^b 1 = t - tf."""
    V = synth.gaussian((2, N + 1), "bform-large", N)
    V[1] = 1.0
    got, plan = _run(N, dtype, V, False)
    if dtype == torch.float64:
        assert plan.f64_mode() == 1
    fb = ob.fastbv(V, T0, TF)
    ref = fb - fb[:, -1:]
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.linalg.norm(got[0] - ref[0]) / np.linalg.norm(ref[0]) < tol
    t, _ = plan.grid()
    assert np.abs(got[1] - (t.numpy() - TF)).max() < (1e-11 if dtype == torch.float64 else 1e-4)
    U = synth.gaussian((2, N + 1), "bform-adj", N)
    gotT, _ = _run(N, dtype, U, True)
    lhs = np.sum(U[0] * ref[0])
    rhs = np.sum(gotT[0] * V[0])
    assert abs(lhs - rhs) < (1e-11 if dtype == torch.float64 else 1e-4) * np.linalg.norm(U[0]) * np.linalg.norm(ref[0])
