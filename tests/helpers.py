"""Layout helpers shared by the GPU tests: convert between the library's pitched KKT vectors and
the oracle's packed ones. No arithmetic of the method lives here."""
import numpy as np
import torch


def _ntail(prob):
    """Tail entries of a KKT vector: nu, and s for a free final time (right after nu)."""
    return prob.n_e + (1 if getattr(prob, "free_time", False) else 0)


def to_packed(prob, vec, op_kkt=True):
    """Pitched device vector -> packed float64 numpy vector in the oracle's ordering."""
    v = vec.detach().double().cpu().numpy()
    P, L = prob.pitch, prob.L
    nb = (2 * prob.n_x + prob.n_u) if op_kkt else prob.n_x
    blocks = [v[b * P:b * P + L] for b in range(nb)]
    out = np.concatenate(blocks)
    if op_kkt:
        out = np.concatenate([out, v[nb * P:nb * P + _ntail(prob)]])
    return out


def from_packed(prob, x, dtype=torch.float64, op_kkt=True):
    P, L = prob.pitch, prob.L
    nb = (2 * prob.n_x + prob.n_u) if op_kkt else prob.n_x
    n = prob.kkt_len if op_kkt else prob.state_len
    out = torch.zeros(n, dtype=torch.float64)
    for b in range(nb):
        out[b * P:b * P + L] = torch.as_tensor(x[b * L:(b + 1) * L])
    if op_kkt:
        nt = _ntail(prob)
        out[nb * P:nb * P + nt] = torch.as_tensor(x[nb * L:nb * L + nt])
    return out.to(dtype).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
