"""Double-float FP64 transforms (bk_set_f64_transform): products of four-step FP64 plans computed
in double-float arithmetic against the oracle's FastBV chain (SciPy DCT-I in binary64) and
against the library's binary64 transforms, at the FP64 tolerance of the products (1e-12 relative
2-norm), for forward and transposed products and every four-step layout (unsplit, split,
two-level split)."""
import numpy as np
import pytest
import torch

from oracle import birkhoff as ob
from paper_2509_01855_gb300 import synth

pytestmark = pytest.mark.gpu


def _plan(N, mode, nvec=4):
    from paper_2509_01855_gb300 import api
    api.set_f64_transform(mode)
    try:
        plan = api.Plan(N, n_comp=nvec, max_batch=1, dtype=torch.float64, t0=0.0, tf=20.0)
    finally:
        api.set_f64_transform(-1)
    return plan


@pytest.mark.parametrize("N", [256, 1 << 12, 1 << 14, 1 << 16, 1 << 17, 1 << 18, 1 << 20])
def test_df_products_match_oracle(N):
    from paper_2509_01855_gb300 import api
    plan = _plan(N, 1)
    assert plan.f64_mode() == 1
    V = synth.gaussian((4, N + 1), "df", N)
    v = plan.empty(1)
    v[0, :, :N + 1] = torch.as_tensor(V)
    out = api.birkhoff_apply(plan, v, plan.empty(1))
    outT = api.birkhoff_apply_T(plan, v, plan.empty(1))
    ref = ob.fastbv(V, 0.0, 20.0)
    refT = ob.fastbv_T(V, 0.0, 20.0)
    e = np.linalg.norm(out[0, :, :N + 1].cpu().numpy() - ref) / np.linalg.norm(ref)
    eT = np.linalg.norm(outT[0, :, :N + 1].cpu().numpy() - refT) / np.linalg.norm(refT)
    print("df N=%d: B %.2e  B^T %.2e" % (N, e, eT))
    assert e < 1e-12 and eT < 1e-12
    assert torch.all(out[0, :, N + 1:] == 0) and torch.all(outT[0, :, N + 1:] == 0)


@pytest.mark.parametrize("N", [1 << 14, 1 << 20])
def test_df_exact_integrals_of_chebyshev_modes(N):
    """v = sum alpha_k T_k (with the modes next to N that the aliasing fold touches): B v is the
    exact integral (Eq. intChebPoly=), so the double-float product's error is its own."""
    from paper_2509_01855_gb300 import api
    plan = _plan(N, 1, nvec=1)
    modes, alphas = synth.sparse_modes(N, 26, "df-modes")
    vv, Bv = ob.sparse_mode_pair(N, modes, alphas, 0.0, 20.0)
    v = plan.empty(1)
    v[0, 0, :N + 1] = torch.as_tensor(vv)
    out = api.birkhoff_apply(plan, v, plan.empty(1))
    e = np.linalg.norm(out[0, 0, :N + 1].cpu().numpy() - Bv) / np.linalg.norm(Bv)
    print("df exact modes N=%d: %.2e" % (N, e))
    assert e < 1e-12


def test_binary64_mode_still_available():
    from paper_2509_01855_gb300 import api
    N = 1 << 16
    p64, pdf = _plan(N, 0), _plan(N, 1)
    assert p64.f64_mode() == 0 and pdf.f64_mode() == 1
    V = synth.gaussian((4, N + 1), "df-vs-64")
    v = p64.empty(1)
    v[0, :, :N + 1] = torch.as_tensor(V)
    a = api.birkhoff_apply(p64, v, p64.empty(1))[0, :, :N + 1].cpu().numpy()
    b = api.birkhoff_apply(pdf, v, pdf.empty(1))[0, :, :N + 1].cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12
    from paper_2509_01855_gb300 import _lib
    assert _lib.lib().bk_set_f64_transform(7) == 1
