"""Cell patches for checking a large mesh cell by cell against the oracle (test helper).

The residual of a cell (Eq. 4) reads the Gauss-point values of the cell and of its face
neighbours, and each of those comes from the cell's stencil (Sections 3.1, 3.2): cells
sharing a vertex with it and the children across its face neighbours, i.e. cells within
two vertex rings of that neighbour, whose own face neighbours lie one ring further.  On the
patch of cells within four vertex rings of a cell every one of those cells has its full
neighbourhood, so the patch's residual at the centre cell equals the full mesh's.  Node ids
keep their global order, which keeps each cell's node 0 (smallest id) and so its stencil
labels.  A patch never crosses a periodic seam; callers pick cells far enough from it.
"""
import numpy as np

import synthetic as S


def node_to_cells(mi):
    """Node -> cells CSR (ptr, cells) of a MeshInput."""
    sizes = np.diff(mi.cell_ptr)
    owner = np.repeat(np.arange(mi.n_cells), sizes)
    order = np.argsort(mi.cell_nodes, kind="stable")
    ptr = np.zeros(mi.n_nodes + 1, dtype=np.int64)
    np.add.at(ptr, mi.cell_nodes + 1, 1)
    return np.cumsum(ptr), owner[order]


def patch(mi, n2c, cell, rings):
    """Cells within `rings` vertex rings of `cell`, as an outflow MeshInput; returns it,
    the patch index of `cell` and the global ids of the patch cells."""
    ptr, cells_of = n2c
    cp, cn = mi.cell_ptr, mi.cell_nodes
    member = {cell}
    front = [cell]
    for _ in range(rings):
        nxt = []
        for c in front:
            for v in cn[cp[c]:cp[c + 1]]:
                for x in cells_of[ptr[v]:ptr[v + 1]]:
                    if x not in member:
                        member.add(int(x))
                        nxt.append(int(x))
        front = nxt
    ids = np.array(sorted(member), dtype=np.int64)
    nodes_g = np.unique(np.concatenate([cn[cp[c]:cp[c + 1]] for c in ids]))  # sorted: global order kept
    remap = {int(g): k for k, g in enumerate(nodes_g)}
    ptr_p = [0]
    nodes_p = []
    for c in ids:
        nodes_p.extend(remap[int(v)] for v in cn[cp[c]:cp[c + 1]])
        ptr_p.append(len(nodes_p))
    pm = S.MeshInput(mi.nodes[nodes_g], np.array(ptr_p, dtype=np.int64), np.array(nodes_p, dtype=np.int64),
                     "outflow", (0.0, 0.0), (1.0, 1.0))
    return pm, int(np.searchsorted(ids, cell)), ids


def interior_samples(mi, k, lo, hi, seed=3):
    """k cells (sorted) drawn uniformly among those whose vertex mean lies in [lo, hi]^2."""
    cells, _ = mi.padded_cells()
    cen = mi.nodes[cells].mean(axis=1)
    inner = np.flatnonzero(((cen > lo) & (cen < hi)).all(axis=1))
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(inner, size=k, replace=False))
