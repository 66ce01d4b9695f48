"""Oracle precompute: quadratic reconstruction, candidates and linear weights (Sections 3.1-3.3).

Test infrastructure only (see oracle/__init__.py).

For every cell i0 and each of its Gauss points x_G (2 per edge):

1. Basis of Eq. (9), written in cell-scaled coordinates xi = (x - c0)/sqrt|Omega_0|
   (reading: the least-squares problems are posed in these coordinates so
   that the matrix entries are O(1)); p^k = m^k - avg_{Omega_0} m^k with the
   monomials m = (xi_x, xi_y, xi_x^2, xi_y^2, xi_x xi_y).
2. A_jk = E_j avg_{Omega_ij} p^k (Eq. 10), the least-squares solve for a
   (Eqs. 11-12) and eta_j, the coefficient of W_ij in P^2(x_G) (Eq. 13);
   eta_0 = 1 - sum_j eta_j because P^2 has the cell mean W_i0 built in.
3. Candidates P^1_j on S_j = {i0, S_j1, S_j2}: P^1_j = W_0 + g_j.(x - c0),
   the cell-average constraints on S_j1, S_j2 give the 2x2 system
   [c_{S_j1} - c0; c_{S_j2} - c0] g_j = [W_{S_j1} - W_0; W_{S_j2} - W_0]
   (the average of a linear function over a cell is its centroid value).
   Missing members use the replacement cell (Sections 3.1/3.2 rewrite rules).
4. B (rows: stencil slots 0..M, columns: candidates) from the coefficients
   b_jk of P^1_j(x_G) (Eq. 14), and gamma from B gamma = eta (Eq. 15).
5. Weighting parameters d_j from |gamma| (Section 3.3), the weighted system
   d_j A_jk a_k = d_j (W_ij - W_i0) -> eta^opt -> gamma^opt from B gamma = eta^opt.

Reading of the regularised solves (zeta I + M^T M) x = M^T r with
zeta = 1e-14 (Eqs. 12 and the gamma solve): their zeta -> 0+ limit, the
Moore-Penrose minimum-norm least-squares solution, computed with
numpy.linalg.pinv (singular values below rcond * sigma_max dropped).  The
paper notes the two differ by O(zeta); the limit is what two independent
implementations can agree on, since the B system is rank deficient.
Reading of d_j: computed per Gauss point from that point's gamma.
The weights used at run time are divided by their sum, which the paper's
identity sum_j gamma_j = 1 (Section 3.1) makes 1 up to the solve's rounding.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .mesh import (QUAD_SUBSTENCILS, TRI_SUBSTENCILS, SLOT_MISSING, OracleMesh)

__all__ = ["Params", "precompute", "GroupTables", "monomials"]


@dataclass
class Params:
    # epsilon of the nonlinear weights (Section 3.4 gives no value): 1e-3 reproduces the paper's
    # Table 3 (density wave, regular quads) to about 1 %, 1e-6 misses it by up to 35x
    eps: float = 1e-3
    theta: float = 3.0       # splitting parameter of Section 3.4
    rcond: float = 1e-12     # relative singular-value cut of the minimum-norm solves
    optimize: bool = True    # Section 3.3 optimisation of large linear weights
    linear: bool = False     # True: R = sum gamma_j P^1_j (the linear scheme, Eq. 14)
    eqn: str = "euler"       # "euler" or "scalar"
    gas_gamma: float = 1.4
    adv: tuple = (1.0, 1.0)  # advection velocity of the scalar equation
    characteristic: bool = False  # Euler: reconstruct characteristic variables (Section 4)
    # prescribed outer state of inflow faces (Euler): primitive (rho, u, v, p) inflow_a at the
    # Gauss points x with n . x < c0 + s t, inflow_b elsewhere; inflow_line = (n_x, n_y, c0, s)
    inflow_a: tuple | None = None
    inflow_b: tuple | None = None
    inflow_line: tuple = (1.0, 0.0, 0.0, 0.0)

    def __post_init__(self):
        # sigma- = sum (theta |gamma| - gamma) / 2 vanishes for theta = 1 when every gamma_j >= 0,
        # and gamma- = gt- / sigma- is then undefined (Section 3.4 uses theta = 3)
        if not self.theta > 1.0:
            raise ValueError("the splitting of Section 3.4 needs theta > 1")


@dataclass
class GroupTables:
    """Runtime tables of all cells of one type (quad: M=12, G=8; triangle: M=9, G=6)."""
    cells: np.ndarray      # (N,) cell ids
    M: int
    G: int
    area: np.ndarray       # (N,)
    members: np.ndarray    # (N, M, 2) cells whose averages candidate j reads (S_j1, S_j2)
    member_flip: np.ndarray  # (N, M, 2, 2) momentum components (x, y) reversed in those values (walls)
    grad_op: np.ndarray    # (N, M, 2, 2) g_j = grad_op[j] @ (dW_S1, dW_S2)
    dG: np.ndarray         # (N, G, 2) x_G - c0
    gamma: np.ndarray      # (N, G, M) linear weights used at run time
    gamma_raw: np.ndarray  # (N, G, M) before optimisation
    eta: np.ndarray        # (N, G, M+1) P^2 coefficients (optimised if optimize)
    eta_raw: np.ndarray    # (N, G, M+1)
    B: np.ndarray          # (N, G, M+1, M)
    slot_cells: np.ndarray  # (N, M+1) cell read for each slot
    E: np.ndarray          # (N, M+1)
    A: np.ndarray          # (N, M, 5) least-squares matrix of Eq. (10)


def monomials(xi_x, xi_y):
    """m = (xi_x, xi_y, xi_x^2, xi_y^2, xi_x xi_y): the non-constant monomials of Eq. (9)."""
    return np.stack([xi_x, xi_y, xi_x * xi_x, xi_y * xi_y, xi_x * xi_y], axis=-1)


def _polygon_monomial_averages(verts, cnt, c0, s):
    """Averages of the 5 monomials over polygons (..., 4, 2) with cnt vertices.

    Fan triangles (v0, vk, vk+1), each with the edge-midpoint rule (exact for
    degree <= 2).  Coordinates are first mapped to xi = (x - c0)/s.
    """
    xi = (verts - c0[..., None, :]) / s[..., None, None]
    total = 0.0
    area = 0.0
    for k in (1, 2):
        a = xi[..., 0, :]
        b = xi[..., k, :]
        c = xi[..., k + 1, :]
        use = (cnt == 4) if k == 2 else np.ones(cnt.shape, bool)
        t = 0.5 * ((b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1]) - (b[..., 1] - a[..., 1]) * (c[..., 0] - a[..., 0]))
        t = np.where(use, t, 0.0)
        mids = ((a + b) / 2.0, (b + c) / 2.0, (c + a) / 2.0)
        f = sum(monomials(m[..., 0], m[..., 1]) for m in mids)
        total = total + (t / 3.0)[..., None] * f
        area = area + t
    return total / area[..., None]


def _d_weights(gamma, quad: bool):
    """Weighting parameters of Section 3.3 from gamma (..., M); returns d (..., M) for slots 1..M."""
    a = np.abs(gamma)
    d = np.ones_like(gamma)
    if quad:
        for j in range(5, 13):
            d[..., j - 1] = 1.0 / np.maximum(1.0, a[..., j - 1])
    else:
        for j, k in ((4, 8), (8, 4), (5, 9), (9, 5), (6, 7), (7, 6)):
            d[..., j - 1] = 1.0 / np.maximum(np.maximum(1.0, a[..., j - 1]), a[..., k - 1])
    return d


def _group(mesh: OracleMesh, cells: np.ndarray, quad: bool, params: Params) -> GroupTables:
    M = 12 if quad else 9
    G = 8 if quad else 6
    sub = QUAD_SUBSTENCILS if quad else TRI_SUBSTENCILS
    N = cells.shape[0]
    verts = np.zeros((N, M + 1, 4, 2))
    cnt = np.zeros((N, M + 1), dtype=np.int64)
    E = np.zeros((N, M + 1))
    resolved = np.zeros((N, M + 1), dtype=np.int64)
    slot_cells = np.zeros((N, M + 1), dtype=np.int64)
    for n, c in enumerate(cells):
        for j in range(M + 1):
            p = mesh.slot_polygon(c, j)
            verts[n, j, :len(p)] = p
            verts[n, j, len(p):] = p[-1]
            cnt[n, j] = len(p)
            E[n, j] = 0.0 if mesh.slots[c][j][0] == SLOT_MISSING else 1.0
            resolved[n, j] = mesh.resolve(c, j)
            slot_cells[n, j] = mesh.slot_value_cell(c, j)
    c0 = mesh.centroid[cells]
    s = np.sqrt(mesh.area[cells])
    avg = _polygon_monomial_averages(verts, cnt, c0[:, None, :].repeat(M + 1, 1), s[:, None].repeat(M + 1, 1))
    # p^k = m^k - avg_{Omega_0} m^k  (Eq. 9); A_jk = E_j avg_{Omega_ij} p^k  (Eq. 10)
    A = E[:, 1:, None] * (avg[:, 1:, :] - avg[:, :1, :])
    xG = mesh.cell_gauss[cells, :G, :]
    xiG = (xG - c0[:, None, :]) / s[:, None, None]
    pG = monomials(xiG[..., 0], xiG[..., 1]) - avg[:, None, 0, :]
    A_pinv = np.linalg.pinv(A, rcond=params.rcond)                    # (N, 5, M)
    eta_nb = np.einsum("ngk,nkm->ngm", pG, A_pinv)                      # (N, G, M)
    eta = np.concatenate([1.0 - eta_nb.sum(-1, keepdims=True), eta_nb], axis=-1)

    # candidate gradients: centroid offsets of the (resolved) members
    cen = c0[:, None, :] + s[:, None, None] * avg[..., 0:2]             # (N, M+1, 2)
    s1 = np.array([resolved[:, a] for a, _ in sub]).T                   # (N, M)
    s2 = np.array([resolved[:, b] for _, b in sub]).T
    rows = np.arange(N)[:, None]
    D = np.stack([cen[rows, s1] - c0[:, None, :], cen[rows, s2] - c0[:, None, :]], axis=-2)  # (N, M, 2, 2)
    grad_op = np.linalg.pinv(D, rcond=params.rcond)                    # (N, M, 2, 2)
    members = np.stack([slot_cells[rows, s1], slot_cells[rows, s2]], axis=-1)
    flips = np.array([[mesh.slot_flips(c, j) for j in range(M + 1)] for c in cells], dtype=np.int8).reshape(N, M + 1, 2)
    member_flip = np.stack([flips[rows, s1], flips[rows, s2]], axis=2)          # (N, M, 2, 2)

    # b_jk: P^1_j(x_G) = W0 + dG . (grad_op (W_S - W0))
    dG = xG - c0[:, None, :]
    t = np.einsum("nga,nmab->ngmb", dG, grad_op)                        # (N, G, M, 2)
    B = np.zeros((N, G, M + 1, M))
    for j in range(M):
        B[np.arange(N), :, s1[:, j], j] += t[:, :, j, 0]
        B[np.arange(N), :, s2[:, j], j] += t[:, :, j, 1]
        B[:, :, 0, j] += 1.0 - t[:, :, j, 0] - t[:, :, j, 1]
    B_pinv = np.linalg.pinv(B, rcond=params.rcond)                     # (N, G, M, M+1)
    gamma_raw = np.einsum("ngmr,ngr->ngm", B_pinv, eta)

    if params.optimize:
        d = _d_weights(gamma_raw, quad)                                  # (N, G, M)
        DA = d[..., None] * A[:, None, :, :]
        DA_pinv = np.linalg.pinv(DA, rcond=params.rcond)               # (N, G, 5, M)
        eta_opt_nb = np.einsum("ngk,ngkm->ngm", pG, DA_pinv) * d
        eta_opt = np.concatenate([1.0 - eta_opt_nb.sum(-1, keepdims=True), eta_opt_nb], axis=-1)
        gamma = np.einsum("ngmr,ngr->ngm", B_pinv, eta_opt)
    else:
        eta_opt = eta
        gamma = gamma_raw
    # sum gamma_j = 1 holds exactly for the solution of B gamma = eta (Section 3.1: P^1_j and P^2
    # reproduce constants); the solve meets it only to its rounding, so it is imposed
    gamma = gamma / gamma.sum(-1, keepdims=True)
    return GroupTables(cells=cells, M=M, G=G, area=mesh.area[cells], members=members, member_flip=member_flip,
                       grad_op=grad_op,
                       dG=dG, gamma=gamma, gamma_raw=gamma_raw, eta=eta_opt, eta_raw=eta, B=B,
                       slot_cells=slot_cells, E=E, A=A)


def precompute(mesh: OracleMesh, params: Params | None = None):
    """Runtime tables for the quad group and the triangle group (either may be empty)."""
    params = params or Params()
    out = []
    for quad in (True, False):
        cells = np.nonzero(mesh.cell_size == (4 if quad else 3))[0]
        if cells.size:
            out.append(_group(mesh, cells, quad, params))
    return out
