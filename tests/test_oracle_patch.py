"""The patch method of the full-size GPU check, verified on the oracle alone: the residual
of a cell computed on the patch of cells within four vertex rings of it equals the
residual of the whole mesh at that cell (periodic low-quality mesh and outflow mesh)."""
import numpy as np
import pytest

import synthetic as S
from oracle import OracleMesh, OracleSolver, Params
from patches import interior_samples, node_to_cells, patch


@pytest.mark.parametrize("which", ["vortex-periodic", "riemann-outflow"])
def test_patch_residual_equals_full_residual(which):
    if which == "vortex-periodic":
        mi = S.stretched_vortex_mesh(36, seed=5)
        W = S.cell_average(mi, S.isentropic_vortex, order=3)
        lo, hi = 3.5, 6.5
    else:
        mi = S.mesh_for_config(3, n=24, seed=5, kind="mixed")
        W = S.four_quadrant_average(mi, seed=5)
        lo, hi = 0.35, 0.65
    full = OracleSolver(OracleMesh.from_input(mi), Params(eqn="euler")).residual(W)
    scale = np.abs(full).max(axis=1)
    n2c = node_to_cells(mi)
    for c in interior_samples(mi, 4, lo, hi):
        pm, k, ids = patch(mi, n2c, int(c), 4)
        assert len(ids) < mi.n_cells
        ref = OracleSolver(OracleMesh.from_input(pm), Params(eqn="euler")).residual(W[:, ids])[:, k]
        assert np.abs(ref - full[:, c]).max() <= 1e-12 * scale.max(), c
