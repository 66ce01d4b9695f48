"""The patch method of the full-size GPU check, verified on the oracle alone: the residual
of a cell computed on the patch of cells within four vertex rings of it equals the
residual of the whole mesh at that cell (periodic low-quality mesh; outflow mesh, inside
and next to the boundary, where the stencils use mirror images)."""
import numpy as np
import pytest

import synthetic as S
from oracle import OracleMesh, OracleSolver, Params
from patches import interior_samples, node_to_cells, patch


@pytest.mark.parametrize("which", ["vortex-periodic", "riemann-outflow", "riemann-boundary"])
def test_patch_residual_equals_full_residual(which):
    if which == "vortex-periodic":
        mi = S.stretched_vortex_mesh(36, seed=5)
        W = S.cell_average(mi, S.isentropic_vortex, order=3)
        cells = interior_samples(mi, 4, 3.5, 6.5)
    else:
        mi = S.mesh_for_config(3, n=24, seed=5, kind="mixed")
        W = S.four_quadrant_average(mi, seed=5)
        if which == "riemann-outflow":
            cells = interior_samples(mi, 4, 0.35, 0.65)
        else:
            cen = mi.nodes[mi.padded_cells()[0]].mean(axis=1)
            near = np.flatnonzero(((cen < 2 / 24) | (cen > 1 - 2 / 24)).any(axis=1))
            cells = np.random.default_rng(0).choice(near, 6, replace=False)
    full = OracleSolver(OracleMesh.from_input(mi), Params(eqn="euler")).residual(W)
    scale = np.abs(full).max(axis=1)
    n2c = node_to_cells(mi)
    for c in cells:
        pm, k, ids = patch(mi, n2c, int(c), 4)
        assert len(ids) < mi.n_cells
        ref = OracleSolver(OracleMesh.from_input(pm), Params(eqn="euler")).residual(W[:, ids])[:, k]
        assert np.abs(ref - full[:, c]).max() <= 1e-12 * scale.max(), c
