"""Exact / initial data of the Euler test problems, checked against their defining relations."""
import numpy as np

import synthetic as S

GAMMA = 1.4


def _prim(W):
    rho = W[0]
    u, v = W[1] / rho, W[2] / rho
    p = (GAMMA - 1) * (W[3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def test_shock_vortex_shock_satisfies_the_jump_conditions_and_the_vortex_is_isentropic():
    # far from the vortex: the stationary normal shock conserves mass, momentum and energy fluxes
    rho1, u1, _, p1 = _prim(S.shock_vortex(np.array([0.45]), np.array([0.05])))
    rho2, u2, _, p2 = _prim(S.shock_vortex(np.array([0.55]), np.array([0.05])))
    assert abs(u1[0] / np.sqrt(GAMMA * p1[0] / rho1[0]) - 1.1) < 1e-3   # upstream Mach 1.1
    H1 = GAMMA / (GAMMA - 1) * p1 / rho1 + 0.5 * u1 ** 2
    H2 = GAMMA / (GAMMA - 1) * p2 / rho2 + 0.5 * u2 ** 2
    # (the vortex tail still perturbs the upstream state by ~1e-8 there)
    assert np.allclose(rho1 * u1, rho2 * u2, rtol=1e-7)
    assert np.allclose(rho1 * u1 ** 2 + p1, rho2 * u2 ** 2 + p2, rtol=1e-7)
    assert np.allclose(H1, H2, rtol=1e-7)
    # upstream: the vortex keeps the entropy p / rho^gamma = 1 and perturbs the temperature most at its centre
    x = np.linspace(0.05, 0.45, 41)
    X, Y = np.meshgrid(x, np.linspace(0.3, 0.7, 41))
    rho, u, v, p = _prim(S.shock_vortex(X, Y))
    assert np.abs(p / rho ** GAMMA - 1).max() < 1e-12
    T = p / rho
    i = np.unravel_index(np.argmin(T), T.shape)
    assert abs(X[i] - 0.25) < 0.011 and abs(Y[i] - 0.5) < 0.011
    assert abs(T.min() - (1 - (GAMMA - 1) * 0.09 / (4 * 0.204 * GAMMA) * np.exp(2 * 0.204))) < 1e-3
