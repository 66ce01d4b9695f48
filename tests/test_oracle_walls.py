"""Oracle reflective walls: mirror images across a wall carry the reversed normal momentum,
the wall flux sees the inner state mirrored.  Pinned by exact conservation of mass and energy
in a closed box and by the exact solution of a flow hitting a wall (by symmetry the Riemann
problem of two equal colliding flows: two shocks, the gas at rest between them)."""
import numpy as np
import pytest

import synthetic as S
from oracle import OracleMesh, OracleSolver, Params

GAMMA = 1.4


def _rect(nx, ny, Lx, Ly, walls, perturb=0.0, seed=0):
    X = np.linspace(0, Lx, nx + 1)
    Y = np.linspace(0, Ly, ny + 1)
    xx, yy = np.meshgrid(X, Y, indexing="xy")
    nodes = np.stack([xx.ravel(), yy.ravel()], 1)
    if perturb:
        rng = np.random.default_rng(seed)
        inner = (xx.ravel() > 0) & (xx.ravel() < Lx) & (yy.ravel() > 0) & (yy.ravel() < Ly)
        nodes[inner] += rng.uniform(-perturb, perturb, (inner.sum(), 2)) * np.array([Lx / nx, Ly / ny])
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    a = (i + (nx + 1) * j).ravel()
    q = np.stack([a, a + 1, a + 1 + (nx + 1), a + (nx + 1)], 1)
    return S.MeshInput(nodes, np.arange(0, 4 * len(q) + 1, 4), q.ravel(), "outflow", (0.0, 0.0), (Lx, Ly),
                       walls=tuple(walls))


def _cons(rho, u, v, p):
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])


def _run(sol, W, t_end, cfl=0.5):
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(sol.max_dt(W, cfl), t_end - t)
        W = sol.rk3_step(W, dt)
        t += dt
    return W


def test_closed_box_conserves_mass_and_energy():
    mi = _rect(8, 8, 1.0, 1.0, walls=(0, 1, 2, 3), perturb=0.2, seed=1)
    W = S.cell_average(mi, lambda x, y: _cons(1 + 0.2 * np.sin(2 * x + y), 0.5 + 0 * x, -0.3 + 0 * x,
                                              1 + 0.1 * np.cos(3 * y)), order=3)
    sol = OracleSolver(OracleMesh.from_input(mi), Params())
    m = sol.mesh
    R = sol.residual(W)
    total = (R * m.area).sum(axis=1)
    scale = np.abs(R * m.area).max()
    assert abs(total[0]) < 1e-13 * scale and abs(total[3]) < 1e-13 * scale
    # momentum is not conserved: the walls push back (the check above is not vacuous)
    assert abs(total[1]) > 1e-3 * scale


def _wall_shock_exact(rho, u, p):
    """Gas (rho, u > 0, p) hitting a wall: star pressure of two equal shocks, shock speed."""
    A, B = 2.0 / ((GAMMA + 1) * rho), (GAMMA - 1) / (GAMMA + 1) * p
    ps = p
    for _ in range(100):  # Newton on (ps - p) sqrt(A / (ps + B)) = u
        f = (ps - p) * np.sqrt(A / (ps + B)) - u
        df = np.sqrt(A / (ps + B)) * (1 - 0.5 * (ps - p) / (ps + B))
        ps -= f / df
    a = np.sqrt(GAMMA * p / rho)
    speed = u - a * np.sqrt((GAMMA + 1) / (2 * GAMMA) * ps / p + (GAMMA - 1) / (2 * GAMMA))
    r = ps / p
    rho_s = rho * (r + (GAMMA - 1) / (GAMMA + 1)) / ((GAMMA - 1) / (GAMMA + 1) * r + 1)
    return ps, rho_s, speed


@pytest.mark.parametrize("characteristic", [False, True])
def test_flow_into_a_wall_matches_the_exact_reflected_shock(characteristic):
    nx, L, T = 80, 0.5, 0.3
    mi = _rect(nx, 2, L, 2 * L / nx, walls=(1,))
    W = S.cell_average(mi, lambda x, y: _cons(1 + 0 * x, 1 + 0 * x, 0 * x, 1 + 0 * x), order=2)
    sol = OracleSolver(OracleMesh.from_input(mi), Params(characteristic=characteristic))
    W = _run(sol, W, T)
    ps, rho_s, speed = _wall_shock_exact(1.0, 1.0, 1.0)
    xs = L + speed * T                                       # shock position, moving away from the wall
    assert speed < 0 and 0.2 < xs < L
    cx = sol.mesh.centroid[:, 0]
    rho, u = W[0], W[1] / W[0]
    p = (GAMMA - 1) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])
    behind = cx > xs + 0.05                                  # gas at rest against the wall
    ahead = cx < xs - 0.05
    assert np.abs(u[behind]).max() < 2e-2
    assert np.abs(p[behind] / ps - 1).max() < 2e-2
    # density: the first cells at the wall keep the start-up entropy error ("wall heating")
    plateau = behind & (cx < L - 4 * L / nx)
    assert np.abs(rho[plateau] / rho_s - 1).max() < 2e-2
    assert np.abs(rho[ahead] - 1).max() < 1e-6 and np.abs(u[ahead] - 1).max() < 1e-6
    exact = np.where(cx > xs, rho_s, 1.0)
    assert np.abs(rho - exact).mean() < 0.02                 # smeared over a few cells at the shock
    # transverse motion stays small (the 2D candidates see the shock on the 2-cell-high strip)
    assert np.abs(W[2]).max() < 1e-3


def test_mirror_images_reverse_the_normal_momentum():
    """Momentum normal to a wall that is linear and vanishes on the wall continues linearly into the
    mirror images only if they reverse it: then the reconstruction reproduces it exactly at the Gauss
    points of cells next to the walls x = 1 and y = 0 and in their corner (double images)."""
    from oracle.mesh import SLOT_GHOST
    from oracle.weno import gauss_values_group
    from oracle import precompute
    mi = _rect(10, 10, 1.0, 1.0, walls=(0, 1, 2, 3), perturb=0.15, seed=3)
    lin = lambda x, y: np.stack([1 + 0 * x, 0.3 * (1 - x), 0.2 * y, 2.5 + 0 * x])
    W = S.cell_average(mi, lin, order=3)
    mesh = OracleMesh.from_input(mi)
    checked = corner = 0
    for t in precompute(mesh, Params()):
        got = gauss_values_group(t, W, Params(), mesh)
        xG = mesh.cell_gauss[t.cells, :t.G]
        exact = lin(xG[..., 0], xG[..., 1])
        cen = mesh.centroid[t.cells]
        near = np.array([any(s[0] == SLOT_GHOST for s in mesh.slots[c]) for c in t.cells])
        sel = near & (cen[:, 0] > 0.6) & (cen[:, 1] < 0.4)
        assert np.abs(got - exact)[:, sel].max() < 1e-11
        checked += sel.sum()
        corner += (sel & (cen[:, 0] > 0.85) & (cen[:, 1] < 0.15)).sum()
    assert checked >= 5 and corner >= 1
    # the same data without walls (zero-gradient images) is not reproduced there
    mi.walls = ()
    mesh0 = OracleMesh.from_input(mi)
    t0 = precompute(mesh0, Params())[0]
    got0 = gauss_values_group(t0, W, Params(), mesh0)
    xG = mesh0.cell_gauss[t0.cells, :t0.G]
    cen = mesh0.centroid[t0.cells]
    edge = (cen[:, 0] > 0.9) & (cen[:, 1] > 0.3) & (cen[:, 1] < 0.7)
    assert np.abs(got0[1] - lin(xG[..., 0], xG[..., 1])[1])[edge].max() > 1e-3


def test_exact_riemann_solver_reproduces_the_textbook_star_states():
    """The reference solution used for the shock tubes (synthetic.riemann_exact): Sod's problem
    (1, 0, 1 | 0.125, 0, 0.1) has p* = 0.30313, u* = 0.92745, rho*L = 0.42632, rho*R = 0.26557
    (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, ch. 4, test 1); a state
    and its mirror image give u* = 0 exactly."""
    rho, u, p = S.riemann_exact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), np.array([0.2, 1.5]))
    assert abs(p[0] - 0.30313) < 5e-6 and abs(u[0] - 0.92745) < 5e-6
    assert abs(rho[0] - 0.42632) < 5e-6 and abs(rho[1] - 0.26557) < 5e-6
    ps, rho_s, speed = _wall_shock_exact(1.0, 1.0, 1.0)
    r2, u2, p2 = S.riemann_exact((1.0, 1.0, 1.0), (1.0, -1.0, 1.0), np.array([speed + 1e-9, -1e-9]))
    assert abs(u2[0]) < 1e-12 and abs(p2[0] / ps - 1) < 1e-12 and abs(r2[0] / rho_s - 1) < 1e-12
