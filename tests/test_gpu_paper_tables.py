"""The CUDA path (FP64 and FP32C) against the paper's printed accuracy tables on the one mesh
of the paper that can be rebuilt exactly, the regular Cartesian quad mesh (needs a GB300).

Table 3: density wave on [0,2]^2, dt = 0.3 h, t = 2 (only rho varies, so characteristic and
component-wise reconstruction coincide).  Table 5: isentropic vortex on [0,10]^2, t = 2, with the
characteristic-variable reconstruction of Section 4 (component-wise reconstruction is 2-4 times
less accurate there).  Both with eps = 1e-3; L1 is sum |Omega| |rho - rho_exact| as in the paper.
"""
import os

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1712_08317_gb300.api import Mesh, Solver  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _errors(L, n, f, precision, characteristic, dt_h=None, kind="quad", delta=0.0):
    mi = S.periodic_mesh(n, L, kind, delta, seed=0)
    sol = Solver(Mesh.from_input(mi), eqn="euler", precision=precision, eps=1e-3, characteristic=characteristic)
    U, Ul = sol.to_device(S.cell_average(mi, f))
    dt0 = dt_h * L / n if dt_h else float(sol.max_dt(U, Ul, 0.5)[0])
    steps = int(np.ceil(2.0 / dt0 - 1e-12))
    for _ in range(steps):
        sol.step(U, Ul, 2.0 / steps)
    torch.cuda.synchronize()
    sol.check()
    W = sol.to_host(U, Ul)
    e = np.abs(W[0] - S.cell_average(mi, lambda x, y: f(x, y, 2.0))[0])
    cells, _ = mi.padded_cells()
    x, y = mi.nodes[cells][..., 0], mi.nodes[cells][..., 1]
    area = 0.5 * np.abs((x * np.roll(y, -1, 1) - np.roll(x, -1, 1) * y).sum(1))  # repeated vertices add 0
    return float((e * area).sum()), float(e.max())


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_density_wave_reproduces_table_3(precision):
    ref = np.loadtxt(os.path.join(GOLDEN, "table3_density_wave_quad_regular.txt"))
    got = np.array([_errors(2.0, int(round(2.0 / h)), S.density_wave, precision, False, dt_h=0.3) for h in ref[:, 0]])
    assert np.abs(got[:, 0] / ref[:, 1] - 1.0).max() < 0.05, got
    assert np.abs(got[:, 1] / ref[:, 3] - 1.0).max() < 0.05, got
    orders = np.log2(got[:-1] / got[1:])
    assert np.abs(orders[:, 0] - ref[1:, 2]).max() < 0.1 and np.abs(orders[:, 1] - ref[1:, 4]).max() < 0.1


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_vortex_with_characteristic_variables_reproduces_table_5(precision):
    ref = np.loadtxt(os.path.join(GOLDEN, "table5_vortex_quad_regular.txt"))
    got = np.array([_errors(10.0, int(round(10.0 / h)), S.isentropic_vortex, precision, True) for h in ref[:, 0]])
    assert np.abs(got[:, 0] / ref[:, 1] - 1.0).max() < 0.25, got
    assert np.abs(got[:, 1] / ref[:, 3] - 1.0).max() < 0.15, got


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_vortex_is_third_order_on_irregular_triangles(precision):
    """Table 6's setting (isentropic vortex, irregular triangles, t = 2, characteristic variables) on
    this repository's irregular split-quad meshes (delta = 0.1, h = 1/4 .. 1/16): the paper's
    meshes are figures only, so the digits differ, but third order is what it reports.  Measured
    FP64 orders 3.39 / 3.49 (L1) and 3.42 / 3.43 (Linf); FP32C within 0.3 % of FP64 in L1."""
    got = np.array([_errors(10.0, n, S.isentropic_vortex, precision, True, kind="tri", delta=0.1)
                    for n in (40, 80, 160)])
    orders = np.log2(got[:-1] / got[1:])
    assert (orders >= 2.8).all(), (got, orders)
    if precision == "fp32c":
        ref = np.array([_errors(10.0, n, S.isentropic_vortex, "fp64", True, kind="tri", delta=0.1) for n in (40, 80, 160)])
        assert (got[:, 0] / ref[:, 0] <= 1.05).all(), (got, ref)
