"""Oracle stencil (Sections 3.1 and 3.2) pinned by hand-enumerated meshes and brute force."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.mesh import (OracleMesh, SLOT_CELL, SLOT_GHOST, SLOT_MISSING, QUAD_CHILDREN, TRI_CHILDREN,
                         QUAD_REPLACE, TRI_REPLACE)


def _cartesian(n, L=1.0):
    nodes, quads, _, _ = S.quad_grid(n, (0.0, 0.0), (L, L))
    return S.MeshInput(nodes, np.arange(0, 4 * n * n + 1, 4), quads.ravel(), "periodic", (0.0, 0.0), (L, L))


def test_cartesian_quad_stencil_is_the_3x3_block():
    n = 6
    m = OracleMesh.from_input(_cartesian(n))

    def cell(i, j):
        return (i % n) + n * (j % n)

    i, j = 2, 3
    c = cell(i, j)
    s = m.slots[c]
    # v0 = SW corner (smallest id); faces: 0 bottom, 1 right, 2 top, 3 left
    expect = {1: cell(i, j - 1), 2: cell(i + 1, j), 3: cell(i, j + 1), 4: cell(i - 1, j),
              5: cell(i - 1, j - 1), 6: cell(i + 1, j - 1), 7: cell(i + 1, j + 1), 8: cell(i - 1, j + 1)}
    for slot, x in expect.items():
        assert s[slot][0] == SLOT_CELL and s[slot][1] == x, slot
        assert s[slot][3] == 1
    # valence-4 nodes: the second-tier children coincide with i5..i8, so they are missing
    for slot, partner in ((9, 5), (10, 6), (11, 7), (12, 8)):
        assert s[slot][0] == SLOT_MISSING and s[slot][3] == 0
        assert m.resolve(c, slot) == partner


def test_periodic_translation_of_wrapped_neighbours():
    n = 6
    m = OracleMesh.from_input(_cartesian(n))
    c = 0  # bottom-left cell: its SW neighbour wraps in both directions
    kind, x, sh, _, _ = m.slots[c][5]
    assert x == n * n - 1
    assert np.allclose(sh, [-1.0, -1.0])
    poly = m.slot_polygon(c, 5)
    assert np.allclose(poly.min(0), [-1.0 / n, -1.0 / n]) and np.allclose(poly.max(0), [0.0, 0.0])


def _flower(n, quad):
    nodes = [[0.0, 0.0]]
    for k in range(n):
        t = 2 * math.pi * k / n
        nodes.append([math.cos(t), math.sin(t)])
    cells = []
    if quad:
        for k in range(n):
            t = 2 * math.pi * (k + 0.5) / n
            nodes.append([1.6 * math.cos(t), 1.6 * math.sin(t)])
        for k in range(n):
            cells.append([0, 1 + k, 1 + n + k, 1 + (k + 1) % n])
    else:
        for k in range(n):
            cells.append([0, 1 + k, 1 + (k + 1) % n])
    ptr = np.arange(0, len(cells) * len(cells[0]) + 1, len(cells[0]))
    return OracleMesh(np.array(nodes), ptr, np.array(cells).ravel(), "outflow")


def _face(m, c, k):
    return m.cell_face[c][k]


@pytest.mark.parametrize("valence", [3, 4, 5, 6])
def test_quad_children_at_a_node_of_given_valence(valence):
    m = _flower(valence, quad=True)
    s = m.slots[0]
    # i1 across O-P0 is the petal before, i4 across P1-O the petal after; i2, i3 mirror i0
    assert s[1][1] == valence - 1 and s[4][1] == 1
    assert s[2][0] == SLOT_GHOST and s[2][1] == 0 and s[2][4] == (_face(m, 0, 1),)
    assert s[3][0] == SLOT_GHOST and s[3][1] == 0 and s[3][4] == (_face(m, 0, 2),)
    if valence == 3:
        assert s[5][0] == SLOT_MISSING and m.resolve(0, 5) == 0
        assert s[9][0] == SLOT_MISSING and m.resolve(0, 9) == 0
    elif valence == 4:
        assert s[5][1] == 2
        assert s[9][0] == SLOT_MISSING and m.resolve(0, 9) == 5
    else:
        assert s[5][1] == valence - 2 and s[9][1] == 2 and s[5][3] == s[9][3] == 1
    # across boundary faces the stencil continues with mirror images
    p1 = valence - 1
    f_p1 = m.cell_face[p1][2]          # petal p1's face Q_{p1} - P0 lies on the boundary
    assert s[6][0] == SLOT_GHOST and s[6][1] == p1 and s[6][4] == (f_p1,)
    assert s[7][0] == SLOT_GHOST and s[7][1] == 0 and s[7][4] == (_face(m, 0, 1), _face(m, 0, 2))
    assert s[8][0] == SLOT_GHOST and s[8][1] == 1 and s[8][4] == (_face(m, 0, 2),)
    assert s[10][0] == SLOT_GHOST and s[10][1] == p1 and s[10][4] == (_face(m, 0, 1),)
    assert s[11][0] == SLOT_GHOST and s[11][1] == 0 and s[11][4] == (_face(m, 0, 2), _face(m, 0, 1))
    assert s[12][0] == SLOT_GHOST and s[12][1] == 1 and s[12][4] == (m.cell_face[1][1],)
    # a mirror image is the reflected polygon: the double mirror keeps i0's area
    poly = m.slot_polygon(0, 7)
    area = 0.5 * abs(np.sum(poly[:, 0] * np.roll(poly[:, 1], -1) - np.roll(poly[:, 0], -1) * poly[:, 1]))
    assert area == pytest.approx(m.area[0], rel=1e-13)


@pytest.mark.parametrize("valence", [3, 4, 5, 6])
def test_triangle_children_at_a_node_of_given_valence(valence):
    m = _flower(valence, quad=False)
    s = m.slots[0]
    assert s[1][1] == valence - 1 and s[3][1] == 1
    assert s[2][0] == SLOT_GHOST and s[2][1] == 0 and s[2][4] == (_face(m, 0, 1),)
    if valence == 3:
        assert s[4][0] == SLOT_MISSING and m.resolve(0, 4) == 0
        assert s[7][0] == SLOT_MISSING and m.resolve(0, 7) == 0
    elif valence == 4:
        assert s[4][1] == 2
        assert s[7][0] == SLOT_MISSING and m.resolve(0, 7) == 4
    else:
        assert s[4][1] == valence - 2 and s[7][1] == 2
    p1 = valence - 1
    assert s[8][0] == SLOT_GHOST and s[8][1] == p1 and s[8][4] == (m.cell_face[p1][1],)
    assert s[5][0] == SLOT_GHOST and s[5][1] == p1 and s[5][4] == (_face(m, 0, 1),)
    assert s[9][0] == SLOT_GHOST and s[9][1] == 1 and s[9][4] == (_face(m, 0, 1),)
    assert s[6][0] == SLOT_GHOST and s[6][1] == 1 and s[6][4] == (m.cell_face[1][1],)


def test_structured_triangles_have_full_stencils():
    n = 6
    nodes, quads, _, _ = S.quad_grid(n, (0.0, 0.0), (1.0, 1.0))
    a, b, c, d = quads.T
    tris = np.stack([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 1).reshape(-1, 3)
    mi = S.MeshInput(nodes, np.arange(0, 3 * len(tris) + 1, 3), tris.ravel(), "periodic", (0, 0), (1, 1))
    m = OracleMesh.from_input(mi)
    for cell in range(m.n_cells):
        s = m.slots[cell]
        assert all(s[j][0] == SLOT_CELL for j in range(10))
        members = {s[j][1] for j in range(10)}
        assert len(members) == 10
        # the stencil is the node-neighbourhood (12 cells) minus the cell opposite each node
        classes = set(m.node_class[m.cells[cell]])
        touching = {x for x in range(m.n_cells) if x != cell and classes & set(m.node_class[m.cells[x]])}
        assert len(touching) == 12 and members - {cell} <= touching


def _brute_child(m, c, k, at_start):
    """Cell != c, != parent, sharing a face with the parent, containing the node (brute force)."""
    ids = m.cells[c]
    parent, _ = m.neighbour(c, k)
    v = m.node_class[ids[k if at_start else (k + 1) % len(ids)]]
    found = []
    pc = [m.node_class[i] for i in m.cells[parent]]
    for x in range(m.n_cells):
        if x in (c, parent):
            continue
        xc = [m.node_class[i] for i in m.cells[x]]
        if v not in xc:
            continue
        shared = set(pc) & set(xc)
        # a shared face = a shared pair of classes that is an edge of both
        pe = {frozenset((pc[i], pc[(i + 1) % len(pc)])) for i in range(len(pc))}
        xe = {frozenset((xc[i], xc[(i + 1) % len(xc)])) for i in range(len(xc))}
        if any(v in e for e in pe & xe) and len(shared) >= 2:
            found.append(x)
    assert len(found) <= 1
    return found[0] if found else -1


@pytest.mark.parametrize("cfg,kind", [(2, "mixed"), (3, "mixed"), (3, "tri"), (1, "quad")])
def test_children_and_missing_rules_by_brute_force(cfg, kind):
    mi = S.mesh_for_config(cfg, n=7, seed=11, kind=kind)
    m = OracleMesh.from_input(mi)
    for c in range(m.n_cells):
        quad = m.cell_size[c] == 4
        children = QUAD_CHILDREN if quad else TRI_CHILDREN
        replace = QUAD_REPLACE if quad else TRI_REPLACE
        s = m.slots[c]
        taken = {(s[j][1], s[j][4]) for j in range(0, len(m.cells[c]) + 1)}
        for j, k, at_start in children:
            if s[k + 1][0] == SLOT_GHOST:
                # child of a ghost: a mirror image across i0's boundary face k
                assert s[j][0] in (SLOT_GHOST, SLOT_MISSING)
                if s[j][0] == SLOT_GHOST:
                    assert s[j][4][-1] == m.cell_face[c][k]
                continue
            raw = _brute_child(m, c, k, at_start)
            if raw < 0:
                # the parent's face at that node is a boundary face: the parent's mirror image
                assert s[j][0] in (SLOT_GHOST, SLOT_MISSING)
                if s[j][0] == SLOT_GHOST:
                    assert s[j][1] == s[k + 1][1] and len(s[j][4]) == 1
                continue
            assert raw == m.child(c, k, at_start)[0]
            ident = (raw, ())
            missing = ident in taken
            r = replace[j]
            if not missing and r != 0:
                pj = s[m.resolve(c, r)]
                missing = ident == (pj[1], pj[4])
            assert (s[j][0] == SLOT_MISSING) == missing
            if not missing:
                assert s[j][1] == raw
