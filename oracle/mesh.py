"""Oracle mesh: faces, geometry and the general WENO stencil (Sections 2, 3.1, 3.2).

Test infrastructure only (see oracle/__init__.py).

Conventions (fixed readings, shared in writing with the CUDA library):

* Cells are reoriented counter-clockwise and their node list is rotated to
  start at the node with the smallest input id; local face k joins local
  nodes k -> k+1 and its outward normal is (dy, -dx)/|l|.
* Periodic boundaries identify nodes whose coordinates agree modulo the
  period ("node classes"); a neighbour reached through a periodic face is
  translated by the period so that it sits next to the cell (the paper is
  silent; the least-squares geometry needs it).
* Outflow boundaries (reading): the stencil is continued by mirror images
  across boundary faces.  The face neighbour across a boundary face is the
  mirror image of i0 (a ghost with i0's average); a child reached through a
  boundary face of a real face neighbour is that neighbour's mirror image;
  the children of a ghost are the mirror images (across the ghost's face) of
  the cells across i0's other faces at that node (a corner gives a double
  mirror of i0).  A mirror image carries the average of the cell it mirrors
  (zero-gradient outflow).  Without them, corner stencils become so
  degenerate that the optimised linear weights reach |gamma| ~ 300.
* Box sides of an outflow mesh may instead be reflective walls, over the
  whole side or from a point along it on (the wall of the double Mach
  reflection starts at x = 1/6), or inflow sides whose faces see a
  prescribed outer state in the flux; the stencil images across an inflow
  face are the outflow ones (reading: the paper states the boundary values,
  not how the reconstruction continues across them).
* Stencil (figures of Sections 3.1 and 3.2 are missing): the "child of face
  neighbour i_m at node v" is the cell across i_m's other face incident to v.
  Quad: i1..i4 across faces 0..3; i5, i6 = children of i1 at v0, v1;
  i7, i8 = children of i3 at v2, v3; i10, i11 = children of i2 at v1, v2;
  i9, i12 = children of i4 at v0, v3.  Triangle: i1..i3 across faces 0..2;
  i4, i8 = children of i1 at v0, v1; i5, i9 = children of i2 at v1, v2;
  i6, i7 = children of i3 at v2, v0.
  A child does not exist when it is i0 or one of the face neighbours, or
  (second tier: quad i9..i12, triangle i7..i9) when it is its partner slot's
  cell; images are compared by (cell, mirror faces).  Missing first-tier cells
  are replaced by i0, missing second-tier cells by their partner
  (quad i_{j-4}, triangle i_{j-3}), and get E_j = 0.
"""
from __future__ import annotations

import numpy as np

GAUSS_A = (3.0 + np.sqrt(3.0)) / 6.0  # weight of the near endpoint, Eq. (5)
GAUSS_B = (3.0 - np.sqrt(3.0)) / 6.0

SLOT_CELL, SLOT_GHOST, SLOT_MISSING = 0, 1, 2

# (slot, face of i0 whose neighbour is the parent, node: True = start node of that face)
QUAD_CHILDREN = [(5, 0, True), (6, 0, False), (7, 2, True), (8, 2, False),
                 (10, 1, True), (11, 1, False), (9, 3, False), (12, 3, True)]
QUAD_REPLACE = {5: 0, 6: 0, 7: 0, 8: 0, 9: 5, 10: 6, 11: 7, 12: 8}
TRI_CHILDREN = [(4, 0, True), (8, 0, False), (5, 1, True), (9, 1, False), (6, 2, True), (7, 2, False)]
TRI_REPLACE = {4: 0, 5: 0, 6: 0, 7: 4, 8: 5, 9: 6}

# candidate sub-stencils S_j = {i0, S_j1, S_j2} (Sections 3.1 and 3.2)
QUAD_SUBSTENCILS = [(1, 2), (2, 3), (3, 4), (4, 1), (1, 5), (1, 6), (3, 7), (3, 8),
                    (4, 9), (2, 10), (2, 11), (4, 12)]
TRI_SUBSTENCILS = [(1, 2), (2, 3), (3, 1), (1, 4), (2, 5), (3, 6), (3, 7), (1, 8), (2, 9)]


class MeshError(ValueError):
    pass


def _signed_area(p: np.ndarray) -> float:
    x, y = p[:, 0], p[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


class OracleMesh:
    """Topology + geometry + stencils of a 2D mesh of triangles and quadrilaterals."""

    def __init__(self, nodes, cell_ptr, cell_nodes, bc="periodic", origin=(0.0, 0.0), extent=(1.0, 1.0),
                 walls=(), wall_from=(0.0, 0.0, 0.0, 0.0), inflow=()):
        self.nodes = np.asarray(nodes, dtype=np.float64)
        cell_ptr = np.asarray(cell_ptr, dtype=np.int64)
        cell_nodes = np.asarray(cell_nodes, dtype=np.int64)
        self.bc = bc
        self.origin = tuple(float(v) for v in origin)
        self.extent = tuple(float(v) for v in extent)
        self.n_cells = int(cell_ptr.shape[0] - 1)
        self.walls = frozenset(int(w) for w in walls)
        self.wall_from = tuple(float(v) for v in wall_from)
        self.inflow = frozenset(int(w) for w in inflow)
        if (self.walls or self.inflow) and bc == "periodic":
            raise MeshError("walls and inflow sides are sides of an outflow box")
        self._orient_cells(cell_ptr, cell_nodes)
        self._node_classes()
        self._faces()
        self._cell_geometry()
        self._face_sides()
        self._stencils()

    @classmethod
    def from_input(cls, m):
        return cls(m.nodes, m.cell_ptr, m.cell_nodes, m.bc, m.origin, m.extent, getattr(m, "walls", ()),
                   getattr(m, "wall_from", (0.0, 0.0, 0.0, 0.0)), getattr(m, "inflow", ()))

    def _face_sides(self):
        """Box side of every boundary face (-1 elsewhere), whether it is a reflective wall (on a wall
        side, midpoint at least wall_from[side] along the side) and whether it is an inflow face."""
        self.face_side = np.full(self.n_faces, -1, dtype=np.int64)
        lo, ext = np.array(self.origin), np.array(self.extent)
        tol = 1e-9 * ext.max()
        for f in np.flatnonzero(self.face_R < 0):
            a, b = self.face_line(f)
            m = 0.5 * (a + b)
            for side, (axis, val) in enumerate(((0, lo[0]), (0, lo[0] + ext[0]), (1, lo[1]), (1, lo[1] + ext[1]))):
                if abs(a[axis] - val) <= tol and abs(b[axis] - val) <= tol and abs(m[axis] - val) <= tol:
                    self.face_side[f] = side
        self.face_wall = np.zeros(self.n_faces, dtype=bool)
        self.face_inflow = np.zeros(self.n_faces, dtype=bool)
        for f in np.flatnonzero(self.face_side >= 0):
            side = int(self.face_side[f])
            t = 1 - side // 2                                    # axis along the side
            a, b = self.face_line(f)
            along = 0.5 * (a[t] + b[t]) - lo[t]
            self.face_wall[f] = side in self.walls and along >= self.wall_from[side]
            self.face_inflow[f] = side in self.inflow and not self.face_wall[f]

    def reflect_momentum(self, W, fx, fy):
        """State with its x (y) momentum reversed where fx (fy) is set (reflection across a wall parallel
        to the y (x) axis)."""
        W = np.array(W, dtype=np.float64, copy=True)
        W[1] = np.where(fx, -W[1], W[1])
        W[2] = np.where(fy, -W[2], W[2])
        return W

    def slot_flips(self, c: int, j: int):
        """(fx, fy): momentum components reversed in the value of slot j of cell c (mirror images
        across reflective walls; an image across two walls reverses both or, for parallel walls, none)."""
        _, _, _, _, refl = self.slots[c][self.resolve(c, j)]
        fx = fy = 0
        for f in refl:
            if self.face_wall[f]:
                if self.face_side[f] < 2:
                    fx ^= 1
                else:
                    fy ^= 1
        return fx, fy

    # ------------------------------------------------------------------ topology
    def _orient_cells(self, cell_ptr, cell_nodes):
        self.cells = []
        for c in range(self.n_cells):
            ids = [int(v) for v in cell_nodes[cell_ptr[c]:cell_ptr[c + 1]]]
            if len(ids) not in (3, 4):
                raise MeshError(f"cell {c} has {len(ids)} nodes")
            a = _signed_area(self.nodes[ids])
            if a == 0.0:
                raise MeshError(f"cell {c} has zero area")
            if a < 0.0:
                ids = ids[::-1]
            k = ids.index(min(ids))
            ids = ids[k:] + ids[:k]
            p = self.nodes[ids]
            e = np.roll(p, -1, axis=0) - p
            en = np.roll(e, -1, axis=0)
            if np.any(e[:, 0] * en[:, 1] - e[:, 1] * en[:, 0] <= 0.0):
                raise MeshError(f"cell {c} is not strictly convex")
            self.cells.append(ids)
        self.cell_size = np.array([len(c) for c in self.cells])

    def _node_classes(self):
        n = self.nodes.shape[0]
        if self.bc != "periodic":
            self.node_class = np.arange(n)
            return
        rel = (self.nodes - np.array(self.origin)) / np.array(self.extent)
        rel = rel - np.floor(rel + 1e-9)
        keys = np.round(rel * 1e8).astype(np.int64)
        keys[keys == 100000000] = 0
        table = {}
        cls = np.empty(n, dtype=np.int64)
        for i in range(n):
            k = (int(keys[i, 0]), int(keys[i, 1]))
            cls[i] = table.setdefault(k, len(table))
        self.node_class = cls

    def _faces(self):
        table = {}
        for c, ids in enumerate(self.cells):
            m = len(ids)
            for k in range(m):
                a = self.node_class[ids[k]]
                b = self.node_class[ids[(k + 1) % m]]
                if a == b:
                    raise MeshError("degenerate edge")
                table.setdefault((min(a, b), max(a, b)), []).append((c, k))
        self.face_L, self.face_kL, self.face_R, self.face_kR = [], [], [], []
        self.face_shift = []
        self.cell_face = [[-1] * len(ids) for ids in self.cells]
        for key in sorted(table):
            sides = table[key]
            if len(sides) > 2:
                raise MeshError("non-manifold edge")
            if len(sides) == 1 and self.bc == "periodic":
                raise MeshError("unpaired periodic boundary face")
            (L, kL) = sides[0]
            if len(sides) == 2:
                (R, kR) = sides[1]
                if R == L:
                    raise MeshError("cell adjacent to itself (mesh too small)")
                # R's local node kR+1 carries the class of L's local node kL
                xl = self.nodes[self.cells[L][kL]]
                xr = self.nodes[self.cells[R][(kR + 1) % len(self.cells[R])]]
                if self.node_class[self.cells[R][(kR + 1) % len(self.cells[R])]] != self.node_class[self.cells[L][kL]]:
                    raise MeshError("inconsistent orientation across a face")
                shift = xl - xr
            else:
                R, kR, shift = -1, -1, np.zeros(2)
            f = len(self.face_L)
            self.face_L.append(L)
            self.face_kL.append(kL)
            self.face_R.append(R)
            self.face_kR.append(kR)
            self.face_shift.append(shift)
            self.cell_face[L][kL] = f
            if R >= 0:
                self.cell_face[R][kR] = f
        self.face_L = np.array(self.face_L)
        self.face_kL = np.array(self.face_kL)
        self.face_R = np.array(self.face_R)
        self.face_kR = np.array(self.face_kR)
        self.face_shift = np.array(self.face_shift).reshape(-1, 2)
        self.n_faces = len(self.face_L)

    def neighbour(self, c: int, k: int):
        """(cell across local face k of c or -1, translation placing it next to c)."""
        f = self.cell_face[c][k]
        if self.face_L[f] == c and self.face_kL[f] == k:
            return int(self.face_R[f]), self.face_shift[f].copy()
        return int(self.face_L[f]), -self.face_shift[f]

    def child(self, c: int, k: int, at_start: bool):
        """Cell across the other face, incident to node k (at_start) or k+1, of c's face-k neighbour."""
        m, sh = self.neighbour(c, k)
        if m < 0:
            return -1, None
        f = self.cell_face[c][k]
        km = self.cell_face[m].index(f)
        nm = len(self.cells[m])
        # m walks the shared face backwards: its node km+1 is c's node k
        other = (km + 1) % nm if at_start else (km - 1) % nm
        x, sh2 = self.neighbour(m, other)
        if x < 0:
            return -1, None
        return x, sh + sh2

    # ------------------------------------------------------------------ geometry
    def _cell_geometry(self):
        n = self.n_cells
        self.area = np.empty(n)
        self.centroid = np.empty((n, 2))
        for c, ids in enumerate(self.cells):
            a, cen = polygon_area_centroid(self.nodes[ids])
            self.area[c] = a
            self.centroid[c] = cen
        # faces seen from the L cell
        P = np.array([self.nodes[self.cells[L][k]] for L, k in zip(self.face_L, self.face_kL)])
        Q = np.array([self.nodes[self.cells[L][(k + 1) % len(self.cells[L])]] for L, k in zip(self.face_L, self.face_kL)])
        d = Q - P
        self.face_len = np.hypot(d[:, 0], d[:, 1])
        self.face_normal = np.stack([d[:, 1], -d[:, 0]], axis=1) / self.face_len[:, None]
        # Gauss points of every cell: local point 2k near node k, 2k+1 near node k+1
        self.cell_gauss = np.zeros((n, 8, 2))
        for c, ids in enumerate(self.cells):
            p = self.nodes[ids]
            m = len(ids)
            for k in range(m):
                a, b = p[k], p[(k + 1) % m]
                self.cell_gauss[c, 2 * k] = GAUSS_A * a + GAUSS_B * b
                self.cell_gauss[c, 2 * k + 1] = GAUSS_B * a + GAUSS_A * b

    # ------------------------------------------------------------------ stencils
    def _image_across(self, c: int, k: int):
        """Image across local face k of (real) cell c: (kind, cell, shift, mirror faces)."""
        x, sh = self.neighbour(c, k)
        if x >= 0:
            return (SLOT_CELL, x, sh, ())
        return (SLOT_GHOST, c, np.zeros(2), (self.cell_face[c][k],))

    def _child_image(self, c: int, k: int, at_start: bool, parent):
        """Child of the face-k neighbour image `parent` of c at node k (at_start) or k+1."""
        kind, p, sh, refl = parent
        m = len(self.cells[c])
        if kind == SLOT_CELL:
            f = self.cell_face[c][k]
            km = self.cell_face[p].index(f)
            nm = len(self.cells[p])
            other = (km + 1) % nm if at_start else (km - 1) % nm
            x, sh2 = self.neighbour(p, other)
            if x >= 0:
                return (SLOT_CELL, x, sh + sh2, ())
            return (SLOT_GHOST, p, sh.copy(), (self.cell_face[p][other],))
        # parent = mirror of c across its face k: mirror the image across c's other face at that node
        k2 = (k - 1) % m if at_start else (k + 1) % m
        y = self._image_across(c, k2)
        return (SLOT_GHOST, y[1], y[2], y[3] + (self.cell_face[c][k],))

    @staticmethod
    def _identity(img):
        return (img[1], img[3])

    def _stencils(self):
        """slots[c] = list of (kind, cell, shift, E, mirror faces) for i0..iM."""
        self.slots = []
        for c, ids in enumerate(self.cells):
            quad = len(ids) == 4
            M = 12 if quad else 9
            children = QUAD_CHILDREN if quad else TRI_CHILDREN
            replace = QUAD_REPLACE if quad else TRI_REPLACE
            s = [None] * (M + 1)
            s[0] = (SLOT_CELL, c, np.zeros(2), 1, ())
            images = [(SLOT_CELL, c, np.zeros(2), ())]
            for k in range(len(ids)):
                img = self._image_across(c, k)
                images.append(img)
                s[k + 1] = (img[0], img[1], img[2], 1, img[3])
            taken = {self._identity(i) for i in images}
            first_tier = [j for j, r in replace.items() if r == 0]
            ordered = sorted(children, key=lambda t: (t[0] not in first_tier, t[0]))
            for (j, k, at_start) in ordered:
                parent = images[k + 1]
                img = self._child_image(c, k, at_start, parent)
                ident = self._identity(img)
                missing = ident in taken
                r = replace[j]
                if not missing and r != 0:
                    pj = s[self.resolve_partial(s, r, replace)]
                    missing = ident == (pj[1], pj[4])
                if missing:
                    s[j] = (SLOT_MISSING, -1, None, 0, ())
                else:
                    s[j] = (img[0], img[1], img[2], 1, img[3])
            self.slots.append(s)

    @staticmethod
    def resolve_partial(s, j, replace):
        while s[j][0] == SLOT_MISSING:
            j = replace[j]
        return j

    def resolve(self, c: int, j: int) -> int:
        """Slot whose cell a (possibly missing) slot j of cell c stands for."""
        quad = len(self.cells[c]) == 4
        replace = QUAD_REPLACE if quad else TRI_REPLACE
        return self.resolve_partial(self.slots[c], j, replace)

    def slot_value_cell(self, c: int, j: int) -> int:
        """Cell whose average is read for slot j (a mirror image reads the cell it mirrors)."""
        return self.slots[c][self.resolve(c, j)][1]

    def face_line(self, f: int):
        """End points of face f as seen from its L cell."""
        L, k = self.face_L[f], self.face_kL[f]
        p = self.nodes[self.cells[L]]
        return p[k], p[(k + 1) % len(p)]

    def slot_polygon(self, c: int, j: int) -> np.ndarray:
        """Vertices (translated and/or mirrored) of the cell standing in slot j of cell c."""
        kind, x, sh, _, refl = self.slots[c][self.resolve(c, j)]
        p = self.nodes[self.cells[x]] + sh
        for f in refl:  # mirror across each boundary face line in turn (outflow meshes: no shifts)
            a, b = self.face_line(f)
            t = (b - a) / np.hypot(*(b - a))
            r = p - a
            p = (a + 2.0 * (r @ t)[:, None] * t[None, :] - r)[::-1]
        return p


def polygon_area_centroid(p: np.ndarray):
    """Area and centroid of a convex polygon by its fan of triangles (v0, vk, vk+1)."""
    area = 0.0
    cx = 0.0
    cy = 0.0
    for k in range(1, len(p) - 1):
        a, b, c = p[0], p[k], p[k + 1]
        t = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
        area += t
        cx += t * (a[0] + b[0] + c[0]) / 3.0
        cy += t * (a[1] + b[1] + c[1]) / 3.0
    return area, np.array([cx / area, cy / area])


def polygon_average(p: np.ndarray, f) -> np.ndarray:
    """Average of f over a polygon: fan triangles, each with the edge-midpoint rule.

    The 3-point edge-midpoint rule integrates polynomials of degree <= 2 on a
    triangle exactly, which covers every basis function of Eq. (9).
    """
    total = 0.0
    area = 0.0
    for k in range(1, len(p) - 1):
        a, b, c = p[0], p[k], p[k + 1]
        t = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
        mids = [(a + b) / 2.0, (b + c) / 2.0, (c + a) / 2.0]
        total = total + t / 3.0 * sum(np.asarray(f(m[0], m[1]), dtype=np.float64) for m in mids)
        area += t
    return total / area
