"""Oracle numerical fluxes (Section 2, Eq. 6 and the HLLC solver it cites).

Test infrastructure only (see oracle/__init__.py).

Euler: rotational invariance F.n = T^{-1} F(T W) (Eq. 6); in the face frame
the HLLC solver of Toro (Riemann Solvers and Numerical Methods for Fluid
Dynamics, ch. 10).  Readings where the paper only cites the book:
wave speeds S_L = min(u_L - a_L, u~ - a~), S_R = max(u_R + a_R, u~ + a~)
with Roe averages (~); contact speed
S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R))
     / (rho_L (S_L - u_L) - rho_R (S_R - u_R));
star states U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, S*, v_K,
E_K/rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))).
Flux: F_L if S_L >= 0, else F_L + S_L (U*_L - U_L) if S* >= 0,
else F_R + S_R (U*_R - U_R) if S_R > 0, else F_R.
Scalar advection u_t + a . grad u = 0: the exact upwind (Godunov) flux.
"""
from __future__ import annotations

import numpy as np

__all__ = ["hllc_flux", "hllc_star", "upwind_flux", "euler_normal_flux", "pressure", "primitive_to_conservative"]


def primitive_to_conservative(q, gamma):
    """(rho, u, v, p) -> (rho, rho u, rho v, E) with E = p / (gamma - 1) + rho (u^2 + v^2) / 2 (Eq. 2)."""
    rho, u, v, p = (float(x) for x in q)
    return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def pressure(W, gamma):
    rho, mx, my, E = W
    return (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)


def euler_normal_flux(W, nx, ny, gamma):
    """Physical flux F(W) n_x + G(W) n_y of Eq. (1)."""
    rho, mx, my, E = W
    u = mx / rho
    v = my / rho
    p = pressure(W, gamma)
    un = u * nx + v * ny
    return np.stack([rho * un, mx * un + p * nx, my * un + p * ny, (E + p) * un])


def _x_flux(q, gamma):
    rho, m, mt, E = q
    u = m / rho
    p = pressure(q, gamma)
    return np.stack([m, m * u + p, mt * u, (E + p) * u])


def hllc_star(qL, qR, gamma):
    """Wave speeds and star states of HLLC for states (4, ...) already in the face frame
    (rho, rho u_n, rho u_t, E): dict with SL, SR, SS (contact speed), UsL, UsR (star states),
    FL, FR (physical normal fluxes of qL, qR)."""
    rL, rR = qL[0], qR[0]
    uL, uR = qL[1] / rL, qR[1] / rR
    vL, vR = qL[2] / rL, qR[2] / rR
    pL, pR = pressure(qL, gamma), pressure(qR, gamma)
    aL, aR = np.sqrt(gamma * pL / rL), np.sqrt(gamma * pR / rR)
    HL, HR = (qL[3] + pL) / rL, (qR[3] + pR) / rR
    sl, sr = np.sqrt(rL), np.sqrt(rR)
    ut = (sl * uL + sr * uR) / (sl + sr)
    vt = (sl * vL + sr * vR) / (sl + sr)
    Ht = (sl * HL + sr * HR) / (sl + sr)
    at = np.sqrt((gamma - 1.0) * (Ht - 0.5 * (ut * ut + vt * vt)))
    SL = np.minimum(uL - aL, ut - at)
    SR = np.maximum(uR + aR, ut + at)
    SS = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def star(q, r, u, v, p, S):
        f = r * (S - u) / (S - SS)
        return np.stack([f, f * SS, f * v, f * (q[3] / r + (SS - u) * (SS + p / (r * (S - u))))])

    return {"SL": SL, "SR": SR, "SS": SS, "UsL": star(qL, rL, uL, vL, pL, SL),
            "UsR": star(qR, rR, uR, vR, pR, SR), "FL": _x_flux(qL, gamma), "FR": _x_flux(qR, gamma)}


def hllc_flux(WL, WR, nx, ny, gamma):
    """HLLC flux through a face with unit normal (nx, ny), states (4, ...)."""
    # T W: rotate momenta into (normal, tangential)
    qL = np.stack([WL[0], WL[1] * nx + WL[2] * ny, -WL[1] * ny + WL[2] * nx, WL[3]])
    qR = np.stack([WR[0], WR[1] * nx + WR[2] * ny, -WR[1] * ny + WR[2] * nx, WR[3]])
    h = hllc_star(qL, qR, gamma)
    SL, SR, SS, FL, FR = h["SL"], h["SR"], h["SS"], h["FL"], h["FR"]
    FsL = FL + SL * (h["UsL"] - qL)
    FsR = FR + SR * (h["UsR"] - qR)
    F = np.where(SL >= 0.0, FL, np.where(SS >= 0.0, FsL, np.where(SR > 0.0, FsR, FR)))
    # T^{-1}: rotate the momentum flux back
    return np.stack([F[0], F[1] * nx - F[2] * ny, F[1] * ny + F[2] * nx, F[3]])


def upwind_flux(uL, uR, nx, ny, adv):
    an = adv[0] * nx + adv[1] * ny
    return (an * np.where(an >= 0.0, uL[0], uR[0]))[None]
