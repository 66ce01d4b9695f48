"""Oracle WENO step at run time: candidates, smoothness, split weights, Gauss values (Section 3.4).

Test infrastructure only (see oracle/__init__.py).

For one cell type group, with state W of shape (nv, n_cells):

1. dW of the two non-centre members of each candidate, g_j = grad_op_j dW,
   P^1_j(x_G) = W_0 + g_j . (x_G - c0).
2. beta_j = sum_{|alpha|=1} |Omega|^0 int (D^alpha P^1_j)^2 = |Omega| |g_j|^2
   (K = 1 for linear candidates).
3. Splitting with theta: gt+ = (gamma + theta|gamma|)/2, gt- = gt+ - gamma,
   sigma+- = sum gt+-, gamma+- = gt+- / sigma+-.
4. New indicator bt+- = beta (1 + gamma+- beta + (gamma+- beta)^2),
   alpha+- = gamma+- / (bt+- + eps)^2, delta+- = alpha+- / sum alpha+-.
5. R(x_G) = sigma+ sum delta+_j P^1_j - sigma- sum delta-_j P^1_j.
   Reading: the printed final formula drops sigma+-; with it a constant
   state would map to 0, so the splitting identity R = sigma+ R+ - sigma- R-
   of the same section is used.
In linear mode R(x_G) = sum_j gamma_j P^1_j(x_G).
"""
from __future__ import annotations

import numpy as np

__all__ = ["gauss_values_group"]


def gauss_values_group(t, W: np.ndarray, params) -> np.ndarray:
    """Reconstructed values at the G Gauss points of every cell of the group: (nv, N, G)."""
    W0 = W[:, t.cells]                                              # (nv, N)
    dW = np.stack([W[:, t.members[..., 0]] - W0[:, :, None],
                   W[:, t.members[..., 1]] - W0[:, :, None]], axis=-1)  # (nv, N, M, 2)
    g = np.einsum("nmab,vnmb->vnma", t.grad_op, dW)                  # (nv, N, M, 2)
    P = W0[:, :, None, None] + np.einsum("vnma,nga->vngm", g, t.dG)  # (nv, N, G, M)
    gam = t.gamma[None]                                             # (1, N, G, M)
    if params.linear:
        return (gam * P).sum(-1)
    beta = t.area[None, :, None] * (g ** 2).sum(-1)                 # (nv, N, M)
    beta = beta[:, :, None, :]                                      # (nv, N, 1, M)
    gt_p = 0.5 * (gam + params.theta * np.abs(gam))
    gt_m = gt_p - gam
    sig_p = gt_p.sum(-1, keepdims=True)
    sig_m = gt_m.sum(-1, keepdims=True)
    gam_p = gt_p / sig_p
    gam_m = gt_m / sig_m
    out = 0.0
    for gs, sig, sign in ((gam_p, sig_p, 1.0), (gam_m, sig_m, -1.0)):
        q = gs * beta
        bt = beta * (1.0 + q + q * q)
        alpha = gs / (bt + params.eps) ** 2
        delta = alpha / alpha.sum(-1, keepdims=True)
        out = out + sign * sig[..., 0] * (delta * P).sum(-1)
    return out
