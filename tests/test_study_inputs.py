"""The study set-ups bench.py runs take the initial states the paper prints (Section 4)."""
import os

import numpy as np

import bench

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows():
    return {ln.split()[0]: [float(v) for v in ln.split()[1:]]
            for ln in open(os.path.join(GOLDEN, "tube_states.txt")) if not ln.startswith("#")}


def test_sod_and_lax_states_and_times():
    rows = _rows()
    for name in ("sod", "lax"):
        left, right, t = bench.TUBES[name]
        assert list(left) + list(right) + [t] == rows[name]


def test_shu_osher_initial_data():
    rows = _rows()
    x = np.array([0.5, 1.0, 1.5, 7.25])
    W = bench._shu_osher(x, 0.0 * x)
    rho, u = W[0], W[1] / W[0]
    p = 0.4 * (W[3] - 0.5 * W[1] ** 2 / W[0])
    r, ul, pl = rows["shu_osher_left"]
    assert np.allclose([rho[0], u[0], p[0]], [r, ul, pl], rtol=1e-14)
    assert np.allclose([rho[1], u[1], p[1]], [r, ul, pl], rtol=1e-14)     # x <= 1 is the left state
    assert np.allclose(rho[2:], 1.0 + 0.2 * np.sin(5.0 * x[2:]), rtol=1e-14)
    assert np.allclose(u[2:], 0.0) and np.allclose(p[2:], 1.0, rtol=1e-14)


def test_shock_vortex_parameters():
    import inspect

    import synthetic as S
    sig = inspect.signature(S.shock_vortex).parameters
    mach, xs, xc, yc, kappa, mu, rc = _rows()["shock_vortex"]
    assert sig["mach"].default == mach and sig["x_shock"].default == xs
    assert tuple(sig["center"].default) == (xc, yc)
    assert (sig["kappa"].default, sig["mu"].default, sig["rc"].default) == (kappa, mu, rc)
