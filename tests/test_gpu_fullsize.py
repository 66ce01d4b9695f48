"""Full-size parity on the benchmark workloads, in the launch configuration the benchmark
times (after weno_autotune):

* the 4.0M-cell low-quality vortex mesh (periodic [0,10]^2, n = 1754, stretch ratio 10,
  displacement 0.4h, 30 % of the quads split);
* the 1.0M-cell four-quadrant Riemann mesh (outflow [0,1]^2, n = 877, 30 % split);
* the density-wave mesh of 51,200 split triangles (periodic [0,2]^2, n = 160);
* the batch of 256 instances (5k-200k cells each, quad / tri / mixed, smooth or Riemann
  data), 14.2M cells in one solver.

The oracle cannot run these sizes, so sampled cells are checked one by one: the residual
of cell i (Eq. 4) depends only on cells within a few vertex rings of i, so the oracle runs
on the patch of cells within four vertex rings of i (node ids in their global order, which
fixes each cell's node 0 and so its stencil labels; outflow boundary faces of the mesh stay
boundary faces of the patch) and only cell i is compared.  Samples favour cells where the
residual is not trivially zero: near the Riemann data's quadrant lines and near outflow
boundaries (mirror-image stencils).  Properties that hold at any size (conservation, no
non-physical state, agreement of the two precisions) are checked on the whole vortex mesh.
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
from patches import node_to_cells, patch  # noqa: E402

RINGS = 4
TOL = {"fp64": 1e-11, "fp32c": 2e-3}


def _centroids(mi):
    cells, _ = mi.padded_cells()
    return mi.nodes[cells].mean(axis=1)


def _pick(rng, pool, k):
    pool = np.asarray(pool)
    return rng.choice(pool, size=min(k, len(pool)), replace=False) if len(pool) else np.zeros(0, np.int64)


def _samples(mi, rng, k=8):
    """Cells to check: near the quadrant lines and the boundary (outflow) or away from the
    periodic seam (periodic), plus a few anywhere allowed."""
    cen = _centroids(mi)
    lo, ext = np.asarray(mi.origin), np.asarray(mi.extent)
    h = float(np.sqrt(ext.prod() / mi.n_cells))
    u = (cen - lo) / ext
    if mi.bc == "outflow":
        near_lines = np.flatnonzero((np.abs(cen - (lo + 0.5 * ext)) < 3 * h).any(axis=1))
        near_bnd = np.flatnonzero(((cen - lo < 2 * h) | (lo + ext - cen < 2 * h)).any(axis=1))
        anywhere = np.arange(mi.n_cells)
        return np.concatenate([_pick(rng, near_lines, k), _pick(rng, near_bnd, k), _pick(rng, anywhere, k // 2)])
    inner = np.flatnonzero(((u > 0.15) & (u < 0.85)).all(axis=1))
    return _pick(rng, inner, 2 * k)


def _check(mi, W, R, cells, scale, eqn="euler"):
    """Worst |R_gpu - R_oracle| / scale over the sampled cells of mesh mi."""
    n2c = node_to_cells(mi)
    worst = 0.0
    for c in cells:
        pm, k, ids = patch(mi, n2c, int(c), RINGS)
        if mi.bc == "periodic":  # a patch must not reach the periodic seam
            lo, hi = np.asarray(mi.origin), np.asarray(mi.origin) + np.asarray(mi.extent)
            assert ((pm.nodes > lo) & (pm.nodes < hi)).all()
        osol = OracleSolver(OracleMesh.from_input(pm), Params(eqn=eqn))
        ref = osol.residual(W[:, ids])[:, k]
        worst = max(worst, float((np.abs(R[:, c] - ref) / scale).max()))
    return worst


def _workload(name):
    if name == "vortex4m":
        mi = S.stretched_vortex_mesh(1754, seed=0)
        return mi, S.cell_average(mi, S.isentropic_vortex)
    if name == "riemann1m":
        mi = S.mesh_for_config(3, n=877, seed=0, kind="mixed")
        return mi, S.four_quadrant_average(mi, seed=0)
    if name == "densitywave51k":
        mi = S.mesh_for_config(2, n=160, seed=0, kind="tri")
        return mi, S.cell_average(mi, S.density_wave)
    raise KeyError(name)


_cache = {}


def _get(name):
    if name not in _cache:
        _cache.clear()  # one large workload in memory at a time
        mi, W = _workload(name)
        _cache[name] = (mi, W, Mesh.from_input(mi))
    return _cache[name]


def _residual(mesh, W, precision):
    sol = Solver(mesh, eqn="euler", precision=precision)
    U, Ul = sol.to_device(W)
    sol.autotune(U, Ul)
    R = sol.to_host(sol.residual(U, Ul))
    sol.check()
    assert R.shape == W.shape and np.isfinite(R).all()
    return R


@pytest.mark.parametrize("name", ["vortex4m", "riemann1m", "densitywave51k"])
@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_sampled_residual_matches_oracle_at_full_size(name, precision):
    mi, W, mesh = _get(name)
    R = _residual(mesh, W, precision)
    scale = np.abs(R).max(axis=1)
    scale[scale == 0] = 1.0
    cells = _samples(mi, np.random.default_rng(3))
    assert len(cells) >= 12
    worst = _check(mi, W, R, cells, scale)
    assert worst < TOL[precision], worst


def test_full_size_steps_conserve_and_precisions_agree():
    mi, W, mesh = _get("vortex4m")
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


def test_batch_of_256_instances_matches_oracle_per_instance():
    from synthetic.meshes import instance_mesh
    _cache.clear()
    descs = S.batch_instances(256, seed=0)
    mis, inits = [], []
    for d in descs:
        mi = instance_mesh(d)
        mis.append(mi)
        inits.append(S.cell_average(mi, S.density_wave, order=3) if d["data"] == "smooth"
                     else S.four_quadrant_average(mi, d["seed"], order=3))
    big = Mesh.concat([Mesh.from_input(mi) for mi in mis])
    W = np.concatenate(inits, axis=1)
    offsets = np.concatenate([[0], np.cumsum([mi.n_cells for mi in mis])])
    assert big.n_cells == offsets[-1] > 13_000_000
    rng = np.random.default_rng(5)
    chosen = rng.choice(len(descs), size=16, replace=False)
    for precision in ("fp64", "fp32c"):
        R = _residual(big, W, precision)
        worst = 0.0
        for i in chosen:
            mi = mis[i]
            Ri = R[:, offsets[i]:offsets[i + 1]]
            scale = np.abs(Ri).max(axis=1)
            scale[scale == 0] = 1.0
            cells = _samples(mi, rng, k=2)
            worst = max(worst, _check(mi, inits[i], Ri, cells, scale))
        assert worst < TOL[precision], (precision, worst)
