"""Initial and exact data of the accuracy and Riemann tests (Section 4), as cell averages.

Point functions follow the problem statements of Section 4.1 (density wave,
isentropic vortex) plus the scalar analogue u_t + u_x + u_y = 0 and the
four-quadrant Riemann data.  Cell averages are taken with a tensor
Gauss-Legendre rule on Duffy-collapsed triangles of each cell's fan; this is
input preparation (the FV method works on cell averages), not part of the
scheme.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["scalar_wave", "density_wave", "isentropic_vortex", "four_quadrant_states",
           "cell_average", "four_quadrant_average", "euler_prim_to_cons"]

GAMMA = 1.4


def euler_prim_to_cons(rho, u, v, p, gamma=GAMMA):
    """(rho, u, v, p) -> W = (rho, rho U, rho V, rho E), rho E = rho|U|^2/2 + p/(gamma-1) (Eq. 1)."""
    return np.stack([rho, rho * u, rho * v, 0.5 * rho * (u * u + v * v) + p / (gamma - 1.0)])


def scalar_wave(x, y, t=0.0):
    """u0 = 1 + 0.2 sin(pi (x + y)) advected with velocity (1, 1): exact u0(x - t, y - t)."""
    return (1.0 + 0.2 * np.sin(np.pi * (x + y - 2.0 * t)))[None]


def density_wave(x, y, t=0.0, gamma=GAMMA):
    """rho = 1 + 0.2 sin(pi(x + y)), u = v = 1, p = 1, translated by (t, t)."""
    rho = 1.0 + 0.2 * np.sin(np.pi * (x + y - 2.0 * t))
    one = np.ones_like(rho)
    return euler_prim_to_cons(rho, one, one, one, gamma)


def isentropic_vortex(x, y, t=0.0, strength=5.0, L=10.0, gamma=GAMMA):
    """Mean flow (1,1,1,1) plus the isentropic vortex of Section 4.1 centred at (5,5), moved by (t, t).

    The periodic image nearest to each point is used; the perturbation is
    not exactly periodic (its tail is ~6e-6 at the domain edge), as printed.
    """
    xb = x - t - 0.5 * L
    yb = y - t - 0.5 * L
    xb = xb - L * np.round(xb / L)
    yb = yb - L * np.round(yb / L)
    r2 = xb * xb + yb * yb
    du = strength / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u = 1.0 - du * yb
    v = 1.0 + du * xb
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return euler_prim_to_cons(rho, u, v, p, gamma)


def four_quadrant_states(seed: int):
    """Four seeded piecewise-constant states (rho, u, v, p), quadrants NE, NW, SW, SE."""
    rng = np.random.Generator(np.random.PCG64(int(seed) + 15485863))
    rho = rng.uniform(0.1, 1.5, 4)
    u = rng.uniform(-1.0, 1.0, 4)
    v = rng.uniform(-1.0, 1.0, 4)
    p = rng.uniform(0.03, 1.5, 4)
    return np.stack([rho, u, v, p], axis=1)


def four_quadrant_average(mesh, seed: int, gamma=GAMMA, order=5):
    """Cell averages of the four-quadrant Riemann data, split at the domain centre."""
    states = four_quadrant_states(seed)
    xc = mesh.origin[0] + 0.5 * mesh.extent[0]
    yc = mesh.origin[1] + 0.5 * mesh.extent[1]

    def f(x, y):
        q = np.where(x >= xc, np.where(y >= yc, 0, 3), np.where(y >= yc, 1, 2))
        s = states[q]
        return euler_prim_to_cons(s[..., 0], s[..., 1], s[..., 2], s[..., 3], gamma)

    return cell_average(mesh, f, order)


def _gauss_legendre01(order: int):
    x, w = np.polynomial.legendre.leggauss(order)
    return 0.5 * (x + 1.0), 0.5 * w


def cell_average(mesh, func, order: int = 5, chunk: int = 1 << 18) -> np.ndarray:
    """Average of func(x, y) -> (nv, ...) over every cell of mesh; returns (nv, n_cells).

    Each cell is cut into the fan triangles (v0, v_k, v_k+1); each triangle
    (A, B, C) is mapped from the unit square by A + u (B - A) + u w (C - B)
    with Jacobian u |det(B - A, C - B)|, and the square gets an order x order
    Gauss-Legendre rule.
    """
    cells, cnt = mesh.padded_cells()
    P = mesh.nodes
    gx, gw = _gauss_legendre01(order)
    U, Wt = np.meshgrid(gx, gx, indexing="ij")
    WU, WW = np.meshgrid(gw, gw, indexing="ij")
    U = U.ravel()
    Wt = Wt.ravel()
    wts = (WU * WW).ravel() * U  # includes the Duffy factor u
    out = None
    n = cells.shape[0]
    for s in range(0, n, chunk):
        c = cells[s:s + chunk]
        k = cnt[s:s + chunk]
        acc = None
        area = np.zeros(c.shape[0])
        for t in range(2):  # fan triangles (0,1,2) and (0,2,3)
            A = P[c[:, 0]]
            B = P[c[:, 1 + t]]
            C = P[c[:, 2 + t]]
            use = (k == 4) if t == 1 else np.ones(c.shape[0], bool)
            det = (B[:, 0] - A[:, 0]) * (C[:, 1] - B[:, 1]) - (B[:, 1] - A[:, 1]) * (C[:, 0] - B[:, 0])
            det = np.abs(det) * use
            x = A[:, None, 0] + U[None] * ((B[:, None, 0] - A[:, None, 0]) + Wt[None] * (C[:, None, 0] - B[:, None, 0]))
            y = A[:, None, 1] + U[None] * ((B[:, None, 1] - A[:, None, 1]) + Wt[None] * (C[:, None, 1] - B[:, None, 1]))
            vals = func(x, y)  # (nv, m, q)
            contrib = (vals * wts[None, None, :]).sum(-1) * det[None, :]
            acc = contrib if acc is None else acc + contrib
            area += 0.5 * det
        avg = acc / area[None, :]
        if out is None:
            out = np.empty((avg.shape[0], n))
        out[:, s:s + chunk] = avg
    return out
