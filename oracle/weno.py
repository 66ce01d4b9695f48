"""Oracle WENO step at run time: candidates, smoothness, split weights, Gauss values (Section 3.4).

Test infrastructure only (see oracle/__init__.py).

Mirror images across reflective walls carry the mirrored cell's average with
the momentum component normal to the wall reversed.

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

Characteristic variables (Euler, Section 4): for the Gauss points of local
face k the normal flux Jacobian n_x dF/dW + n_y dG/dW is taken at the Roe
average of the cell averages of the cell and its neighbour across face k
(reading: the cell itself at an outflow boundary face, its mirror image with
the normal momentum reversed at a wall); its right eigenvector
matrix R diagonalises it, the stencil averages are projected, U = R^-1 W,
steps 1-5 run on each component of U, and W(x_G) = R U(x_G).
"""
from __future__ import annotations

import numpy as np

from .flux import pressure

__all__ = ["gauss_values_group", "roe_eigenvectors"]


def _weno_points(t, W0, Wm, params, gsel):
    """Steps 1-5 at the Gauss points gsel from the cell values W0 (nv, N) and the candidates'
    member values Wm (nv, N, M, 2): (nv, N, len(gsel))."""
    dW = Wm - W0[:, :, None, None]                                  # (nv, N, M, 2)
    g = np.einsum("nmab,vnmb->vnma", t.grad_op, dW)                  # (nv, N, M, 2)
    P = W0[:, :, None, None] + np.einsum("vnma,nga->vngm", g, t.dG[:, gsel])  # (nv, N, g, M)
    gam = t.gamma[None][:, :, gsel]                                 # (1, N, g, M)
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


def roe_eigenvectors(Wl, Wr, nx, ny, gamma):
    """Right eigenvectors (columns, eigenvalues q_n - a, q_n, q_n, q_n + a) of the Euler normal
    flux Jacobian at the Roe average of the states Wl, Wr (4, ...): (..., 4, 4)."""
    rl, rr = Wl[0], Wr[0]
    sl, sr = np.sqrt(rl), np.sqrt(rr)
    hl = (Wl[3] + pressure(Wl, gamma)) / rl
    hr = (Wr[3] + pressure(Wr, gamma)) / rr
    w = sl + sr
    u = (Wl[1] / sl + Wr[1] / sr) / w                                # (sqrt(rho) u)_l + (..)_r over w
    v = (Wl[2] / sl + Wr[2] / sr) / w
    H = (sl * hl + sr * hr) / w
    a = np.sqrt((gamma - 1.0) * (H - 0.5 * (u * u + v * v)))
    qn = u * nx + v * ny
    qt = -u * ny + v * nx
    one, zero = np.ones_like(u), np.zeros_like(u)
    rows = [[one, one, zero, one],
            [u - a * nx, u, -ny * one, u + a * nx],
            [v - a * ny, v, nx * one, v + a * ny],
            [H - a * qn, 0.5 * (u * u + v * v), qt, H + a * qn]]
    return np.stack([np.stack(r, axis=-1) for r in rows], axis=-2)


def _face_frames(t, W, mesh, gamma, k):
    """R and R^-1 of local face k of every cell of the group: (N, 4, 4) each."""
    nb = np.array([mesh.neighbour(int(c), k)[0] for c in t.cells])
    wall = np.array([mesh.face_wall[mesh.cell_face[int(c)][k]] for c in t.cells])
    side = np.array([mesh.face_side[mesh.cell_face[int(c)][k]] for c in t.cells])
    nb = np.where(nb < 0, t.cells, nb)
    p = np.array([mesh.nodes[mesh.cells[c][k]] for c in t.cells])
    q = np.array([mesh.nodes[mesh.cells[c][(k + 1) % len(mesh.cells[c])]] for c in t.cells])
    d = q - p
    ln = np.hypot(d[:, 0], d[:, 1])
    nx, ny = d[:, 1] / ln, -d[:, 0] / ln                            # outward unit normal
    # across a wall the neighbour is the cell's mirror image, momentum reversed across the wall
    Wn = mesh.reflect_momentum(W[:, nb], wall & (side < 2), wall & (side >= 2))
    R = roe_eigenvectors(W[:, t.cells], Wn, nx, ny, gamma)
    return R, np.linalg.inv(R)


def gauss_values_group(t, W: np.ndarray, params, mesh=None) -> np.ndarray:
    """Reconstructed values at the G Gauss points of every cell of the group: (nv, N, G).
    Characteristic reconstruction needs the mesh (neighbours and face normals)."""
    W0 = W[:, t.cells]                                              # (nv, N)
    Wm = W[:, t.members]                                            # (nv, N, M, 2)
    if W.shape[0] == 4 and t.member_flip.any():                     # mirror images across walls
        Wm[1] = np.where(t.member_flip[..., 0], -Wm[1], Wm[1])
        Wm[2] = np.where(t.member_flip[..., 1], -Wm[2], Wm[2])
    if not getattr(params, "characteristic", False):
        return _weno_points(t, W0, Wm, params, np.arange(t.G))
    assert W.shape[0] == 4 and mesh is not None
    out = np.empty((4, len(t.cells), t.G))
    for k in range(t.G // 2):
        R, L = _face_frames(t, W, mesh, params.gas_gamma, k)
        U0 = np.einsum("nfv,vn->fn", L, W0)
        Um = np.einsum("nfv,vnmb->fnmb", L, Wm)
        Uk = _weno_points(t, U0, Um, params, np.array([2 * k, 2 * k + 1]))
        out[:, :, 2 * k:2 * k + 2] = np.einsum("nvf,fng->vng", R, Uk)
    return out
