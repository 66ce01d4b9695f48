"""Seeded synthetic meshes shaped like the test meshes of Section 4.

The paper's own meshes exist only as figures, so these generators stand in
for them: tensor grids of quadrilaterals with randomly displaced interior
nodes ("irregular" meshes), the same grids with every quad (or a fraction of
them) split into two triangles along a random diagonal, and a deliberately
low-quality stretched grid for the isentropic-vortex stress case.

Only inputs are produced here (node coordinates, cell -> node lists and the
boundary description); nothing of the WENO method is computed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = ["MeshInput", "quad_grid", "perturbed_quads", "split_quads", "stretched_vortex_mesh",
           "mesh_for_config", "batch_instances", "tube_mesh", "row_triangles"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclass
class MeshInput:
    """A polygon mesh as the C-ABI and the oracle both take it.

    nodes      (n_nodes, 2) float64 coordinates
    cell_ptr   (n_cells + 1,) int64 offsets into cell_nodes
    cell_nodes int64 node ids, 3 or 4 per cell, counter-clockwise
    bc         "periodic" (both directions, period = extent) or "outflow"
    walls      outflow meshes: box sides that are reflective walls instead of outflow
               (0: x = origin_x, 1: x = origin_x + extent_x, 2: y = origin_y, 3: y = origin_y + extent_y)
    wall_from  per side: the wall covers only the faces whose midpoint lies at least this far
               along the side from the origin corner (y for sides 0, 1; x for sides 2, 3)
    inflow     box sides whose faces that are not walls take a prescribed outer state
    """
    nodes: np.ndarray
    cell_ptr: np.ndarray
    cell_nodes: np.ndarray
    bc: str
    origin: tuple
    extent: tuple
    name: str = ""
    seed: int = 0
    meta: dict = field(default_factory=dict)
    walls: tuple = ()
    wall_from: tuple = (0.0, 0.0, 0.0, 0.0)
    inflow: tuple = ()

    @property
    def n_cells(self) -> int:
        return int(self.cell_ptr.shape[0] - 1)

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    def cell_sizes(self) -> np.ndarray:
        return np.diff(self.cell_ptr)

    def padded_cells(self) -> tuple[np.ndarray, np.ndarray]:
        """(n_cells, 4) node ids (last entry repeated for triangles) and the counts."""
        cnt = self.cell_sizes()
        idx = self.cell_ptr[:-1, None] + np.minimum(np.arange(4)[None, :], (cnt - 1)[:, None])
        return self.cell_nodes[idx], cnt


def _grid_coords(n: int, x0: float, L: float, mapping=None) -> np.ndarray:
    s = L * (np.arange(n + 1, dtype=np.float64) / n)
    s[-1] = L  # exact endpoint so periodic partners coincide bit for bit
    if mapping is not None:
        s = mapping(s)
        s[0] = 0.0
        s[-1] = L
    return x0 + s


def quad_grid(n: int, origin=(0.0, 0.0), extent=(1.0, 1.0), xmap=None, ymap=None, ny=None):
    """Tensor grid of n x ny quads (ny = n by default).  Node (i, j) has id i + (n+1) j; cells CCW."""
    ny = n if ny is None else ny
    X = _grid_coords(n, origin[0], extent[0], xmap)
    Y = _grid_coords(ny, origin[1], extent[1], ymap)
    xx, yy = np.meshgrid(X, Y, indexing="xy")
    nodes = np.stack([xx.ravel(), yy.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(n), np.arange(ny), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    a = i + (n + 1) * j
    quads = np.stack([a, a + 1, a + 1 + (n + 1), a + (n + 1)], axis=1).astype(np.int64)
    return nodes, quads, X, Y


def _local_spacing(c: np.ndarray) -> np.ndarray:
    d = np.diff(c)
    amp = np.empty_like(c)
    amp[1:-1] = np.minimum(d[:-1], d[1:])
    amp[0] = d[0]
    amp[-1] = d[-1]
    return amp


def _quads_convex(pos: np.ndarray, quads: np.ndarray, min_cross: np.ndarray) -> np.ndarray:
    p = pos[quads]  # (nq, 4, 2)
    e = np.roll(p, -1, axis=1) - p  # edge k: p_k -> p_{k+1}
    en = np.roll(e, -1, axis=1)
    cross = e[..., 0] * en[..., 1] - e[..., 1] * en[..., 0]
    return np.all(cross > min_cross[:, None], axis=1)


def perturbed_quads(n: int, origin=(0.0, 0.0), extent=(1.0, 1.0), delta=0.1, seed=0,
                    xmap=None, ymap=None, ny=None):
    """Quad grid whose interior nodes move i.i.d. uniformly in [-delta h, delta h]^2.

    h is the local minimum grid spacing in each direction.  Boundary nodes stay
    put, so opposite boundaries keep matching node positions (periodic pairing
    is exact).  Any quad with a corner triangle smaller than a tenth of the
    undisplaced cell area (a sliver, or a non-convex quad) has its interior
    nodes redrawn until no such quad is left.
    """
    ny = n if ny is None else ny
    nodes, quads, X, Y = quad_grid(n, origin, extent, xmap, ymap, ny)
    rng = _rng(seed)
    ax = delta * _local_spacing(X)
    ay = delta * _local_spacing(Y)
    AX, AY = np.meshgrid(ax, ay, indexing="xy")
    amp = np.stack([AX.ravel(), AY.ravel()], axis=1)
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(ny + 1), indexing="xy")
    interior = ((ii > 0) & (ii < n) & (jj > 0) & (jj < ny)).ravel()
    amp[~interior] = 0.0
    disp = rng.uniform(-1.0, 1.0, size=nodes.shape) * amp
    pos = nodes + disp
    # every corner triangle (and so both triangles of either diagonal split) must keep
    # at least a tenth of the undisplaced cell's area: no slivers
    dx = np.diff(X)
    dy = np.diff(Y)
    cell_area = (dx[None, :] * dy[:, None]).ravel()
    min_cross = 0.2 * cell_area
    for _ in range(200):
        ok = _quads_convex(pos, quads, min_cross)
        if ok.all():
            break
        bad_nodes = np.unique(quads[~ok].ravel())
        bad_nodes = bad_nodes[interior[bad_nodes]]
        pos[bad_nodes] = nodes[bad_nodes] + rng.uniform(-1.0, 1.0, size=(bad_nodes.size, 2)) * amp[bad_nodes]
    else:  # pragma: no cover - only with absurd delta
        raise RuntimeError("could not draw a convex perturbed mesh")
    return pos, quads


def split_quads(quads: np.ndarray, frac: float, seed: int, diagonal: int | None = None):
    """Split each quad with probability frac along a random diagonal (diagonal = 0: always the
    one through the quad's first and third nodes, 1: the other one).

    Returns (cell_ptr, cell_nodes) with cells in quad order; a split quad
    contributes its two triangles in place.
    """
    rng = _rng(seed + 7919)
    nq = quads.shape[0]
    split = rng.random(nq) < frac
    diag = rng.integers(0, 2, size=nq)
    if diagonal is not None:
        diag = np.full(nq, int(diagonal))
    a, b, c, d = quads.T
    sizes = np.where(split, 6, 4)
    ptr_q = np.concatenate([[0], np.cumsum(sizes)])
    flat = np.empty(ptr_q[-1], dtype=np.int64)
    # unsplit quads
    q = ~split
    base = ptr_q[:-1][q]
    for k in range(4):
        flat[base + k] = quads[q, k]
    # diagonal a-c: (a,b,c),(a,c,d); diagonal b-d: (a,b,d),(b,c,d)
    s0 = split & (diag == 0)
    base = ptr_q[:-1][s0]
    for k, v in enumerate((a, b, c, a, c, d)):
        flat[base + k] = v[s0]
    s1 = split & (diag == 1)
    base = ptr_q[:-1][s1]
    for k, v in enumerate((a, b, d, b, c, d)):
        flat[base + k] = v[s1]
    cell_sizes = np.repeat(np.where(split, 3, 4), np.where(split, 2, 1))
    cell_ptr = np.concatenate([[0], np.cumsum(cell_sizes)]).astype(np.int64)
    return cell_ptr, flat


def _assemble(pos, quads, frac, seed, bc, origin, extent, name, meta, diagonal=None):
    if frac <= 0.0:
        cell_ptr = np.arange(0, 4 * quads.shape[0] + 1, 4, dtype=np.int64)
        cell_nodes = quads.reshape(-1).astype(np.int64)
    else:
        cell_ptr, cell_nodes = split_quads(quads, frac, seed, diagonal)
    return MeshInput(pos, cell_ptr, cell_nodes, bc, tuple(origin), tuple(extent), name, seed, dict(meta))


def _vortex_maps(L: float, a: float = 9.0 / 11.0):
    """Node maps of the low-quality mesh: g(s) = s - (a L / 2 pi) sin(2 pi s / L).

    g' ranges over [1 - a, 1 + a], so with a = 9/11 the local spacing varies by
    a factor 10; the y map is shifted a quarter period so that the widest x
    spacing meets the narrowest y spacing (aspect ratio up to 10).
    """
    k = 2.0 * math.pi / L

    def g(s):
        return s - (a / k) * np.sin(k * s)

    phi = 0.25 * L

    def gy(s):
        return g(s + phi) - g(np.asarray(phi))

    return g, gy


def row_triangles(nx: int, ny: int, extent):
    """Box [0, Lx] x [0, Ly] of near-equilateral triangles: ny rows of height Ly / ny; the nodes of
    even rows at x = i Lx / nx, those of odd rows shifted by half a spacing, plus a node on each
    side (so every row ends on the box sides with a half-width triangle).  Counter-clockwise.
    Returns (nodes, cell_nodes (n, 3))."""
    Lx, Ly = (float(v) for v in extent)
    hx = Lx / nx
    xs_even = np.arange(nx + 1) * hx
    xs_odd = np.concatenate([[0.0], (np.arange(nx) + 0.5) * hx, [Lx]])
    nodes, rows, first = [], [], 0
    for j in range(ny + 1):
        xs = xs_even if j % 2 == 0 else xs_odd
        rows.append((xs, first + np.arange(xs.size)))
        nodes.append(np.stack([xs, np.full(xs.size, j * Ly / ny)], axis=1))
        first += xs.size
    cells = []
    for j in range(ny):
        (xa, ia), (xb, ib) = rows[j], rows[j + 1]
        a = b = 0
        while a < xa.size - 1 or b < xb.size - 1:  # sweep both rows in x: each step adds one triangle
            na = xa[a + 1] if a < xa.size - 1 else np.inf
            nb = xb[b + 1] if b < xb.size - 1 else np.inf
            if na <= nb:
                cells.append((ia[a], ia[a + 1], ib[b]))
                a += 1
            else:
                cells.append((ia[a], ib[b + 1], ib[b]))
                b += 1
    pos = np.concatenate(nodes)
    cn = np.array(cells, dtype=np.int64)
    p = pos[cn]
    cross = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    cn[cross < 0] = cn[cross < 0][:, [0, 2, 1]]
    return pos, cn


def tube_mesh(nx: int, ny: int, extent, kind="quad", delta=0.1, seed=0, walls=(), wall_from=(0.0, 0.0, 0.0, 0.0),
              inflow=(), diagonal=None):
    """Outflow box [0, Lx] x [0, Ly] of nx x ny perturbed quads (kind "quad"), all split into
    triangles ("tri") or 30 % split ("mixed"), along random diagonals or the one `diagonal` names
    (see split_quads), or of near-equilateral triangles in ny rows ("rowtri", see row_triangles;
    delta and diagonal do not apply); `walls`, `wall_from` and `inflow` name reflective and inflow
    sides (see MeshInput)."""
    if kind == "rowtri":
        pos, cn = row_triangles(nx, ny, extent)
        mi = MeshInput(pos, np.arange(0, 3 * cn.shape[0] + 1, 3, dtype=np.int64), cn.reshape(-1), "outflow",
                       (0.0, 0.0), tuple(extent), f"tube-rowtri-{nx}x{ny}", seed, {"nx": nx, "ny": ny})
        mi.walls = tuple(walls)
        mi.wall_from = tuple(float(v) for v in wall_from)
        mi.inflow = tuple(inflow)
        return mi
    frac = {"quad": 0.0, "tri": 1.0, "mixed": 0.3}[kind]
    pos, quads = perturbed_quads(nx, (0.0, 0.0), tuple(extent), delta, seed, ny=ny)
    mi = _assemble(pos, quads, frac, seed, "outflow", (0.0, 0.0), tuple(extent), f"tube-{kind}-{nx}x{ny}",
                   {"nx": nx, "ny": ny, "split": frac, "delta": delta, "diagonal": diagonal}, diagonal)
    mi.walls = tuple(walls)
    mi.wall_from = tuple(float(v) for v in wall_from)
    mi.inflow = tuple(inflow)
    return mi


def stretched_vortex_mesh(n: int, frac=0.3, delta=0.4, seed=0, L=10.0):
    g, gy = _vortex_maps(L)
    pos, quads = perturbed_quads(n, (0.0, 0.0), (L, L), delta, seed, xmap=g, ymap=gy)
    return _assemble(pos, quads, frac, seed, "periodic", (0.0, 0.0), (L, L),
                     f"vortex-lowq-n{n}", {"n": n, "split": frac, "delta": delta})


def periodic_mesh(n: int, L: float, kind: str = "quad", delta: float = 0.1, seed: int = 0,
                  diagonal: int | None = None) -> MeshInput:
    """Periodic [0, L]^2 grid of n x n quads whose interior nodes are displaced by up to delta of the
    spacing (delta = 0: regular), kept as quads ("quad"), all split into triangles ("tri") or 30 %
    split ("mixed") along random diagonals or the one `diagonal` names (see split_quads): the
    regular and irregular meshes of the accuracy tests."""
    frac = {"quad": 0.0, "tri": 1.0, "mixed": 0.3}[kind]
    pos, quads = perturbed_quads(n, (0.0, 0.0), (L, L), delta, seed)
    return _assemble(pos, quads, frac, seed, "periodic", (0.0, 0.0), (L, L), f"periodic-{kind}-n{n}-d{delta}",
                     {"n": n, "split": frac, "delta": delta, "diagonal": diagonal}, diagonal)


def mesh_for_config(config: int, n: int | None = None, seed: int = 0, kind: str | None = None) -> MeshInput:
    """The synthetic mesh of a benchmark configuration.

    1: periodic [0,2]^2 perturbed quads (default n=40, 1,600 cells), delta 0.1
    2: periodic [0,2]^2 perturbed quads all split into triangles (default n=160, 51,200 cells)
    3: outflow [0,1]^2 mixed mesh, 30% of quads split (default n=877, ~1.0M cells)
    5: periodic [0,10]^2 stretched low-quality mixed mesh (default n=1754, ~4.0M cells), delta 0.4
    kind overrides the cell type for configs 1-3: "quad", "tri" or "mixed".
    """
    if config == 1:
        n = 40 if n is None else n
        frac = {"quad": 0.0, "tri": 1.0, "mixed": 0.3}[kind or "quad"]
        pos, quads = perturbed_quads(n, (0.0, 0.0), (2.0, 2.0), 0.1, seed)
        return _assemble(pos, quads, frac, seed, "periodic", (0.0, 0.0), (2.0, 2.0),
                         f"scalar-quad-n{n}", {"n": n, "split": frac, "delta": 0.1})
    if config == 2:
        n = 160 if n is None else n
        frac = {"quad": 0.0, "tri": 1.0, "mixed": 0.3}[kind or "tri"]
        pos, quads = perturbed_quads(n, (0.0, 0.0), (2.0, 2.0), 0.1, seed)
        return _assemble(pos, quads, frac, seed, "periodic", (0.0, 0.0), (2.0, 2.0),
                         f"densitywave-{kind or 'tri'}-n{n}", {"n": n, "split": frac, "delta": 0.1})
    if config == 3:
        n = 877 if n is None else n
        frac = {"quad": 0.0, "tri": 1.0, "mixed": 0.3}[kind or "mixed"]
        pos, quads = perturbed_quads(n, (0.0, 0.0), (1.0, 1.0), 0.1, seed)
        return _assemble(pos, quads, frac, seed, "outflow", (0.0, 0.0), (1.0, 1.0),
                         f"riemann4-{kind or 'mixed'}-n{n}", {"n": n, "split": frac, "delta": 0.1})
    if config == 5:
        n = 1754 if n is None else n
        return stretched_vortex_mesh(n, 0.3, 0.4, seed)
    raise ValueError(f"no single mesh for config {config}")


def batch_instances(count: int = 256, seed: int = 0, min_cells: int = 5000, max_cells: int = 200000):
    """Instance descriptions of the batched workload.

    Each instance draws a cell count log-uniformly in [min_cells, max_cells], a
    cell type uniformly from {quad, tri, mixed(30% split)} and smooth
    (periodic density wave) or Riemann (outflow four-quadrant) data with equal
    probability.  Returns a list of dicts with keys n, kind, data, seed.
    """
    rng = _rng(seed + 104729)
    out = []
    for k in range(count):
        cells = math.exp(rng.uniform(math.log(min_cells), math.log(max_cells)))
        kind = ("quad", "tri", "mixed")[int(rng.integers(0, 3))]
        data = ("smooth", "riemann")[int(rng.integers(0, 2))]
        per_quad = {"quad": 1.0, "tri": 2.0, "mixed": 1.3}[kind]
        n = max(8, int(round(math.sqrt(cells / per_quad))))
        out.append({"n": n, "kind": kind, "data": data, "seed": seed * 1000 + k})
    return out


def instance_mesh(desc: dict) -> MeshInput:
    """Mesh of one batched instance (see batch_instances)."""
    if desc["data"] == "smooth":
        return mesh_for_config(2, desc["n"], desc["seed"], desc["kind"])
    return mesh_for_config(3, desc["n"], desc["seed"], desc["kind"])
