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

__all__ = ["scalar_wave", "density_wave", "isentropic_vortex", "four_quadrant_states", "riemann_exact",
           "shock_tube", "shock_vortex", "moving_shock", "double_mach",
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


def riemann_exact(left, right, xi, gamma=GAMMA):
    """Exact solution of the 1D Riemann problem for an ideal gas (the classical construction with
    a pressure function for each side, Newton iteration for the star pressure and sampling of
    the self-similar fan), as primitive (rho, u, p) at the similarity coordinates xi = x / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    g1, g2 = (gamma - 1) / (2 * gamma), (gamma + 1) / (2 * gamma)

    def side(p, r, pk, ak):  # f_K(p) and its derivative
        if p > pk:  # shock
            A, B = 2 / ((gamma + 1) * r), (gamma - 1) / (gamma + 1) * pk
            q = np.sqrt(A / (p + B))
            return (p - pk) * q, q * (1 - 0.5 * (p - pk) / (p + B))
        f = 2 * ak / (gamma - 1) * ((p / pk) ** g1 - 1)  # rarefaction
        return f, (p / pk) ** (-g2) / (r * ak)

    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (al + ar))
    for _ in range(100):
        fl, dl = side(p, rl, pl, al)
        fr, dr = side(p, rr, pr, ar)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(1e-10, p - dp)
        if abs(dp) < 1e-14 * p:
            break
    fl, _ = side(p, rl, pl, al)
    fr, _ = side(p, rr, pr, ar)
    us = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.empty((3,) + xi.shape)
    for k, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            r, u, pk, ak, sgn = rl, ul, pl, al, 1.0
        else:
            r, u, pk, ak, sgn = rr, ur, pr, ar, -1.0
        if p > pk:  # shock on this side
            rs = r * (p / pk + (gamma - 1) / (gamma + 1)) / ((gamma - 1) / (gamma + 1) * p / pk + 1)
            S = u - sgn * ak * np.sqrt(g2 * p / pk + g1)
            inside = (s >= S) if sgn > 0 else (s <= S)
            val = (rs, us, p) if inside else (r, u, pk)
        else:  # rarefaction: head, tail, fan between
            as_ = ak * (p / pk) ** g1
            head, tail = u - sgn * ak, us - sgn * as_
            if (sgn > 0 and s <= head) or (sgn < 0 and s >= head):
                val = (r, u, pk)
            elif (sgn > 0 and s >= tail) or (sgn < 0 and s <= tail):
                val = (r * (p / pk) ** (1 / gamma), us, p)
            else:
                c = 2 / (gamma + 1) + sgn * (gamma - 1) / ((gamma + 1) * ak) * (u - s)
                val = (r * c ** (2 / (gamma - 1)), 2 / (gamma + 1) * (sgn * ak + (gamma - 1) / 2 * u + s),
                       pk * c ** (2 * gamma / (gamma - 1)))
        out[(slice(None),) + k] = val
    return out


def shock_tube(left, right, x0=0.5, gamma=GAMMA):
    """f(x, y, t): conservative state of the exact 1D Riemann solution split at x = x0."""
    def f(x, y, t=0.0):
        x = np.asarray(x, dtype=np.float64)
        if t <= 0.0:
            lo = np.array(left)[:, None] * np.ones(x.size)
            hi = np.array(right)[:, None] * np.ones(x.size)
            prim = np.where((x.ravel() < x0)[None], lo, hi).reshape((3,) + x.shape)
        else:
            prim = riemann_exact(left, right, (x - x0) / t, gamma)
        rho, u, p = prim
        return euler_prim_to_cons(rho, u, 0 * u, p, gamma)
    return f


def shock_vortex(x, y, t=0.0, mach=1.1, x_shock=0.5, center=(0.25, 0.5), kappa=0.3, mu=0.204, rc=0.05,
                 gamma=GAMMA):
    """Initial data of the shock-vortex interaction: a stationary normal shock of Mach number
    `mach` at x = x_shock with the upstream state rho = 1, u = mach sqrt(gamma), v = 0, p = 1 and the
    downstream state from the normal-shock relations; upstream, an isentropic vortex perturbs the
    velocity by kappa eta e^{mu (1 - eta^2)} (sin theta, -cos theta) and the temperature p / rho by
    -(gamma - 1) kappa^2 / (4 mu gamma) e^{2 mu (1 - eta^2)}, eta = r / rc (t is not used)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m2 = mach * mach
    u1 = mach * np.sqrt(gamma)
    r21 = (gamma + 1) * m2 / ((gamma - 1) * m2 + 2)          # density ratio across the shock
    p21 = 1 + 2 * gamma / (gamma + 1) * (m2 - 1)             # pressure ratio
    dx, dy = x - center[0], y - center[1]
    eta = np.sqrt(dx * dx + dy * dy) / rc
    th = np.arctan2(dy, dx)
    e = np.exp(mu * (1 - eta * eta))
    T = 1.0 - (gamma - 1) * kappa ** 2 / (4 * mu * gamma) * e * e
    rho_up = T ** (1.0 / (gamma - 1))                          # isentropic: p / rho^gamma = 1
    up = x < x_shock
    rho = np.where(up, rho_up, r21)
    u = np.where(up, u1 + kappa * eta * e * np.sin(th), u1 / r21)
    v = np.where(up, -kappa * eta * e * np.cos(th), 0.0)
    p = np.where(up, rho_up * T, p21)
    return euler_prim_to_cons(rho, u, v, p, gamma)


def moving_shock(mach, x0, y0=0.0, angle_deg=90.0, pre=(1.4, 0.0, 0.0, 1.0), gamma=GAMMA):
    """A straight shock through (x0, y0) at `angle_deg` to the x axis, moving at Mach `mach` into the
    resting state `pre` (primitive rho, u, v, p), with the post-shock state of the normal-shock
    (Rankine-Hugoniot) relations behind it.  The shock moves along its unit normal
    n = (sin a, -cos a) at speed S = mach c_pre; behind it the gas moves along n at S (1 - rho1/rho2).

    Returns dict(post, pre: primitive 4-tuples, line: (n_x, n_y, c0, S) such that the post-shock state
    holds where n . x < c0 + S t, f: f(x, y, t) -> conservative state of this exact solution)."""
    r1, u1, v1, p1 = (float(q) for q in pre)
    assert u1 == 0.0 and v1 == 0.0, "the pre-shock gas is at rest"
    a = math.radians(angle_deg)
    nx, ny = math.sin(a), -math.cos(a)
    m2 = mach * mach
    c1 = math.sqrt(gamma * p1 / r1)
    S = mach * c1
    r2 = r1 * (gamma + 1) * m2 / ((gamma - 1) * m2 + 2)
    p2 = p1 * (1 + 2 * gamma / (gamma + 1) * (m2 - 1))
    w2 = S * (1 - r1 / r2)
    post = (r2, w2 * nx, w2 * ny, p2)
    c0 = nx * x0 + ny * y0

    def f(x, y, t=0.0):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        behind = nx * x + ny * y < c0 + S * t
        q = [np.where(behind, b, c) for b, c in zip(post, (r1, u1, v1, p1))]
        return euler_prim_to_cons(*q, gamma)

    return {"post": post, "pre": (r1, u1, v1, p1), "line": (nx, ny, c0, S), "f": f}


def double_mach(gamma=GAMMA):
    """The double Mach reflection set-up: a Mach 10 shock through (1/6, 0) at 60 degrees to the x axis
    moving into (1.4, 0, 0, 1); post-shock (8, 4.125 sqrt 3, -4.125, 116.5).  Domain [0, 4] x [0, 1],
    reflective wall on the bottom from x = 1/6, the exact post-shock state on the rest of the bottom
    and on the left, the exact moving shock on the top, outflow on the right."""
    return moving_shock(10.0, 1.0 / 6.0, 0.0, 60.0, gamma=gamma)


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
