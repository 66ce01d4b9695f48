"""Oracle residual L(W) (Eq. 4), SSP-RK3 (Section 4) and the CFL time step.

Test infrastructure only (see oracle/__init__.py).

L(W)_i = -(1/|Omega_i|) sum_p |l_p| sum_k omega_k F(x_pk) . n_p with
omega_1 = omega_2 = 1/2 (Eq. 5).  Each face flux uses the Gauss-point values
of the two cells on its sides; at an outflow boundary face both states are
the inner cell's value (reading: ghost = copy of the cell, so HLLC returns the
physical flux of the inner state); at a reflective wall the outer state is the
inner one with its normal momentum reversed; at an inflow face it is the
prescribed state of `Params.inflow_*` at that Gauss point and time (the double
Mach reflection imposes the exact post-shock state and, on the top side, the
exact motion of the incident shock: a state that jumps across a moving line).
The residual takes the time t of its stage; the RK3 stages of Section 4 sit
at t, t + dt and t + dt/2.

Non-physical states (rho <= 0, p <= 0 or not finite at a Gauss point) raise
NonPhysicalState; the paper has no positivity limiter.

Time step (reading, the paper only states dt = 0.3 h for its accuracy runs):
dt = CFL * min_i 2|Omega_i| / sum_p (|v_i . n_p| + c_i) |l_p| with c = 0 for
scalar advection.
"""
from __future__ import annotations

import numpy as np

from .flux import hllc_flux, upwind_flux, pressure, primitive_to_conservative
from .mesh import OracleMesh
from .reconstruction import Params, precompute
from .weno import gauss_values_group

__all__ = ["OracleSolver", "NonPhysicalState"]


class NonPhysicalState(ArithmeticError):
    pass


class OracleSolver:
    def __init__(self, mesh: OracleMesh, params: Params | None = None):
        self.mesh = mesh
        self.params = params or Params()
        self.groups = precompute(mesh, self.params)
        self.nv = 4 if self.params.eqn == "euler" else 1
        m = mesh
        # Gauss points of the two sides: L uses 2kL, 2kL+1; R meets them at 2kR+1, 2kR
        self.fL = m.face_L
        self.fR = m.face_R
        self.gL = np.stack([2 * m.face_kL, 2 * m.face_kL + 1], axis=1)
        self.gR = np.stack([2 * m.face_kR + 1, 2 * m.face_kR], axis=1)
        self.boundary = m.face_R < 0
        self.inflow = None
        if m.face_inflow.any():
            p = self.params
            if self.nv != 4 or p.inflow_a is None or p.inflow_b is None:
                raise ValueError("inflow faces need the Euler equations and both prescribed states")
            self.inflow_a = primitive_to_conservative(p.inflow_a, p.gas_gamma)
            self.inflow_b = primitive_to_conservative(p.inflow_b, p.gas_gamma)
            nx, ny, c0, self.inflow_speed = (float(v) for v in p.inflow_line)
            f = np.flatnonzero(m.face_inflow)
            xg = m.cell_gauss[self.fL[f][:, None], self.gL[f]]   # (n_in, 2 points, 2)
            self.inflow = f
            self.inflow_xi = nx * xg[..., 0] + ny * xg[..., 1] - c0

    def gauss_values(self, W: np.ndarray) -> np.ndarray:
        Wg = np.full((self.nv, self.mesh.n_cells, 8), np.nan)
        for t in self.groups:
            Wg[:, t.cells, :t.G] = gauss_values_group(t, W, self.params, self.mesh)
        return Wg

    def inflow_states(self, t: float) -> np.ndarray:
        """Prescribed outer states of the inflow faces at time t: (4, n_inflow, 2 Gauss points)."""
        a = self.inflow_xi < self.inflow_speed * t
        return np.where(a[None], self.inflow_a[:, None, None], self.inflow_b[:, None, None])

    def face_fluxes(self, W: np.ndarray, t: float = 0.0) -> np.ndarray:
        """F_f = |l_f|/2 (F(x_f1) + F(x_f2)), normal pointing from L to R: (nv, n_faces)."""
        m = self.mesh
        Wg = self.gauss_values(W)
        R = np.where(self.boundary, self.fL, self.fR)
        gR = np.where(self.boundary[:, None], self.gL, self.gR)
        WL = Wg[:, self.fL[:, None], self.gL]               # (nv, Nf, 2)
        WR = Wg[:, R[:, None], gR]
        if self.nv == 4 and m.face_wall.any():
            # reflective wall: the outer state is the inner one with its normal momentum reversed
            n = m.face_normal[:, :, None]                    # (Nf, 2, 1)
            mn = WL[1] * n[:, 0] + WL[2] * n[:, 1]
            w = m.face_wall[:, None]
            WR = WR.copy()
            WR[1] = np.where(w, WL[1] - 2.0 * mn * n[:, 0], WR[1])
            WR[2] = np.where(w, WL[2] - 2.0 * mn * n[:, 1], WR[2])
        if self.inflow is not None:
            WR = WR.copy()
            WR[:, self.inflow] = self.inflow_states(t)
        self._check(WL)
        self._check(WR)
        nx = m.face_normal[:, 0][:, None]
        ny = m.face_normal[:, 1][:, None]
        if self.params.eqn == "euler":
            F = hllc_flux(WL, WR, nx, ny, self.params.gas_gamma)
        else:
            F = upwind_flux(WL, WR, nx, ny, self.params.adv)
        return 0.5 * m.face_len[None, :] * (F[..., 0] + F[..., 1])

    def _check(self, Wq):
        if not np.all(np.isfinite(Wq)):
            raise NonPhysicalState("non-finite value at a Gauss point")
        if self.params.eqn == "euler":
            if np.any(Wq[0] <= 0.0) or np.any(pressure(Wq, self.params.gas_gamma) <= 0.0):
                raise NonPhysicalState("rho <= 0 or p <= 0 at a Gauss point")

    def residual(self, W: np.ndarray, t: float = 0.0) -> np.ndarray:
        """L(W) of Eq. (4) at time t (t only enters through inflow faces): (nv, n_cells)."""
        F = self.face_fluxes(W, t)
        acc = np.zeros_like(W)
        np.add.at(acc, (slice(None), self.fL), -F)
        inner = ~self.boundary
        np.add.at(acc, (slice(None), self.fR[inner]), F[:, inner])
        return acc / self.mesh.area[None, :]

    def rk3_step(self, W: np.ndarray, dt: float, L=None, t: float = 0.0) -> np.ndarray:
        """Third-order TVD Runge-Kutta step of Section 4 from time t; its stages evaluate the
        residual (or the operator L(w, t)) at t, t + dt and t + dt/2."""
        L = L or self.residual
        W1 = W + dt * L(W, t)
        W2 = 0.75 * W + 0.25 * W1 + 0.25 * dt * L(W1, t + 1.0 * dt)
        return W / 3.0 + 2.0 / 3.0 * W2 + 2.0 / 3.0 * dt * L(W2, t + 0.5 * dt)

    def max_dt(self, W: np.ndarray, cfl: float) -> float:
        m = self.mesh
        if self.params.eqn == "euler":
            rho = W[0]
            u = W[1] / rho
            v = W[2] / rho
            c = np.sqrt(self.params.gas_gamma * pressure(W, self.params.gas_gamma) / rho)
        else:
            u = np.full(m.n_cells, self.params.adv[0])
            v = np.full(m.n_cells, self.params.adv[1])
            c = np.zeros(m.n_cells)
        nx, ny = m.face_normal[:, 0], m.face_normal[:, 1]
        s = np.zeros(m.n_cells)
        L = self.fL
        np.add.at(s, L, (np.abs(u[L] * nx + v[L] * ny) + c[L]) * m.face_len)
        inner = ~self.boundary
        R = self.fR[inner]
        np.add.at(s, R, (np.abs(u[R] * nx[inner] + v[R] * ny[inner]) + c[R]) * m.face_len[inner])
        return float(cfl * np.min(2.0 * m.area / s))

    def conservation(self, W: np.ndarray) -> np.ndarray:
        return (W * self.mesh.area[None, :]).sum(axis=1)

    def run(self, W: np.ndarray, t_end: float, cfl: float):
        """Step from t = 0 to t_end with N = ceil(t_end / dt_cfl) equal steps (dt from the initial
        state); the time after each step is the running sum of the steps."""
        dt0 = self.max_dt(W, cfl)
        n = int(np.ceil(t_end / dt0 - 1e-12))
        dt = t_end / n
        t = 0.0
        for _ in range(n):
            W = self.rk3_step(W, dt, t=t)
            t += dt
        return W, n, dt
