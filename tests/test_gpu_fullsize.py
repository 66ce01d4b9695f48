"""Full-size parity on the 4.0M-cell low-quality vortex mesh (periodic [0,10]^2, n = 1754,
stretch ratio 10, displacement 0.4h, 30 % of the quads split), in the launch configuration
the benchmark times (after weno_autotune).

The oracle cannot run 4M cells, so each sampled cell is checked one by one: the residual
of cell i (Eq. 4) depends only on the states and stencils of cells within three vertex
rings of i, so the oracle runs on the patch of cells within four vertex rings of i (node
ids kept in their global order, which fixes each cell's node 0 and therefore its stencil
labels) and only cell i of the patch is compared.  Properties that hold at any size
(conservation, no non-physical state, agreement of the two precisions) are checked on the
whole mesh.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import OracleMesh, OracleSolver, Params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1712_08317_gb300.api import Mesh, Solver  # noqa: E402
from patches import node_to_cells, patch, interior_samples  # noqa: E402

N_FULL = 1754
N_SAMPLES = 24
RINGS = 4


@pytest.fixture(scope="module")
def full():
    mi = S.stretched_vortex_mesh(N_FULL, seed=0)
    W = S.cell_average(mi, S.isentropic_vortex)
    mesh = Mesh.from_input(mi)
    return mi, W, mesh


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32c", 2e-3)])
def test_sampled_residual_matches_oracle_at_full_size(full, precision, tol):
    mi, W, mesh = full
    sol = Solver(mesh, eqn="euler", precision=precision)
    U, Ul = sol.to_device(W)
    sol.autotune(U, Ul)
    R = sol.to_host(sol.residual(U, Ul))
    sol.check()
    assert R.shape == W.shape and np.isfinite(R).all()
    scale = np.abs(R).max(axis=1)
    n2c = node_to_cells(mi)
    worst = 0.0
    for c in interior_samples(mi, N_SAMPLES, 1.5, 8.5):
        pm, k, ids = patch(mi, n2c, int(c), RINGS)
        assert ((pm.nodes > 0.0) & (pm.nodes < 10.0)).all()  # clear of the periodic seam
        osol = OracleSolver(OracleMesh.from_input(pm), Params(eqn="euler"))
        ref = osol.residual(W[:, ids])[:, k]
        worst = max(worst, float((np.abs(R[:, c] - ref) / scale).max()))
    assert worst < tol, worst


def test_full_size_steps_conserve_and_precisions_agree(full):
    mi, W, mesh = full
    s32 = Solver(mesh, eqn="euler", precision="fp32c")
    s64 = Solver(mesh, eqn="euler", precision="fp64")
    U, Ul = s32.to_device(W)
    V, _ = s64.to_device(W)
    s32.autotune(U, Ul)
    dt = float(s64.max_dt(V, None, 0.5)[0])
    c0 = s64.conservation(V, None)[0]
    for _ in range(5):
        s32.step(U, Ul, dt)
        s64.step(V, None, dt)
    torch.cuda.synchronize()
    s32.check()
    s64.check()
    c32 = s32.conservation(U, Ul)[0]
    c64 = s64.conservation(V, None)[0]
    assert np.abs(c32 - c0).max() <= 1e-12 * np.abs(c0).max()
    assert np.abs(c64 - c0).max() <= 1e-13 * np.abs(c0).max()
    a, b = s32.to_host(U, Ul), s64.to_host(V)
    assert float((np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)).max()) < 1e-6
