// Host mesh builder: orientation, edge pairing (periodic by translation),
// Morton renumbering with quads first, faces and the general stencil.
//
// Stencil rules (Sections 3.1 and 3.2; their figures are not available, so
// the labelling below is the one consistent with the printed sub-stencils,
// the replacement rules and the triangle d_j pairs):
//  - local face k of a cell joins its nodes k -> k+1 (counter-clockwise,
//    node 0 = smallest input node id); i_{k+1} lies across face k.
//  - "child of face neighbour m at node v" = the cell across m's other face
//    incident to v.
//  - quad: i5, i6 = children of i1 at nodes 0, 1; i7, i8 = children of i3 at
//    nodes 2, 3; i10, i11 = children of i2 at nodes 1, 2; i9, i12 = children
//    of i4 at nodes 0, 3.  Replacements: i5..i8 -> i0, i9..i12 -> i5..i8.
//  - triangle: i4, i8 = children of i1 at nodes 0, 1; i5, i9 = children of
//    i2 at nodes 1, 2; i6, i7 = children of i3 at nodes 2, 0.
//    Replacements: i4..i6 -> i0, i7..i9 -> i4..i6.
//  - a child is missing (E_j = 0) if it is i0 or a face neighbour, or
//    (second tier) if it is its partner's cell; members are compared by
//    (cell, mirror faces).
//  - outflow boundaries continue the stencil by mirror images: the face
//    neighbour across a boundary face is i0 mirrored across it; a child
//    reached through a boundary face of a real face neighbour is that
//    neighbour mirrored across the face; a child of a mirrored i0 is the
//    mirror, across the same face, of the member across i0's other face at
//    that node (two mirrors at a corner).  A mirror image reads the average
//    of the cell it mirrors (zero-gradient outflow).
#include "host_mesh.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>

#include "weno3.h"

namespace weno {

const int8_t kQuadSub[12][2] = {{1, 2}, {2, 3}, {3, 4}, {4, 1}, {1, 5},  {1, 6},
                                {3, 7}, {3, 8}, {4, 9}, {2, 10}, {2, 11}, {4, 12}};
const int8_t kTriSub[9][2] = {{1, 2}, {2, 3}, {3, 1}, {1, 4}, {2, 5}, {3, 6}, {3, 7}, {1, 8}, {2, 9}};

namespace {

// (slot, parent face, at the start node of that face)
struct ChildRule { int8_t slot, face; bool start; int8_t partner; };
// first tier before second tier, so that partners are known
const ChildRule kQuadRules[8] = {{5, 0, true, 0},  {6, 0, false, 0}, {7, 2, true, 0},  {8, 2, false, 0},
                                 {9, 3, false, 5}, {10, 1, true, 6}, {11, 1, false, 7}, {12, 3, true, 8}};
const ChildRule kTriRules[6] = {{4, 0, true, 0}, {5, 1, true, 0}, {6, 2, true, 0},
                                {7, 2, false, 4}, {8, 0, false, 5}, {9, 1, false, 6}};

uint32_t spread16(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

struct EdgeRec {
  int64_t a, b;   // node ids, a < b
  int64_t cell;   // input cell
  int8_t k;       // local face
  int8_t fwd;     // 1 if the cell walks a -> b
};

}  // namespace

int resolve_slot(const Mesh& m, int64_t c, int j) {
  const Slot* s = &m.slots[c * kMaxSlots];
  const bool quad = m.is_quad(c);
  while (s[j].kind == SLOT_MISSING) {
    if (quad) j = (j >= 9) ? j - 4 : 0;
    else j = (j >= 7) ? j - 3 : 0;
  }
  return j;
}

int32_t slot_value_cell(const Mesh& m, int64_t c, int j) {
  return m.slots[c * kMaxSlots + resolve_slot(m, c, j)].cell;
}

int32_t slot_flip_bits(const Mesh& m, int64_t c, int j) {
  const Slot& s = m.slots[c * kMaxSlots + resolve_slot(m, c, j)];
  if (s.kind != SLOT_GHOST) return 0;
  int32_t bits = 0;
  for (int r = 0; r < s.nref; ++r) {
    const int8_t w = m.fwall[s.ref[r]];
    if (w == 0) bits ^= kFlipX;
    else if (w == 1) bits ^= kFlipY;
  }
  return bits;
}

int slot_polygon(const Mesh& m, int64_t c, int j, double out[4][2]) {
  const Slot& s = m.slots[c * kMaxSlots + resolve_slot(m, c, j)];
  const int64_t x = s.cell;
  const int inst = m.inst[c];
  const double tx = s.sx * m.inst_period[2 * inst], ty = s.sy * m.inst_period[2 * inst + 1];
  const int nv = m.nvert[x];
  double p[4][2];
  for (int i = 0; i < nv; ++i) {
    p[i][0] = m.verts[(x * 4 + i) * 2] + tx;
    p[i][1] = m.verts[(x * 4 + i) * 2 + 1] + ty;
  }
  for (int r = 0; r < (s.kind == SLOT_GHOST ? s.nref : 0); ++r) {
    // reflect across the line of boundary face ref[r] (as seen from its cell), reversing the order
    const int32_t f = s.ref[r];
    const int64_t L = m.fL[f];
    const int k = m.fkL[f], k1 = (k + 1) % m.nvert[L];
    const double ax = m.verts[L * 8 + 2 * k], ay = m.verts[L * 8 + 2 * k + 1];
    const double bx = m.verts[L * 8 + 2 * k1], by = m.verts[L * 8 + 2 * k1 + 1];
    const double len = std::hypot(bx - ax, by - ay);
    const double ux = (bx - ax) / len, uy = (by - ay) / len;
    double q[4][2];
    for (int i = 0; i < nv; ++i) {
      const double rx = p[i][0] - ax, ry = p[i][1] - ay;
      const double d = rx * ux + ry * uy;
      q[nv - 1 - i][0] = ax + 2.0 * d * ux - rx;
      q[nv - 1 - i][1] = ay + 2.0 * d * uy - ry;
    }
    for (int i = 0; i < nv; ++i) { p[i][0] = q[i][0]; p[i][1] = q[i][1]; }
  }
  for (int i = 0; i < nv; ++i) { out[i][0] = p[i][0]; out[i][1] = p[i][1]; }
  return nv;
}

namespace {

Slot cell_slot(int32_t x, int sx, int sy) { return Slot{x, SLOT_CELL, (int8_t)sx, (int8_t)sy, 0, {-1, -1}}; }

// Member across local face k of the real cell c: its neighbour, or c mirrored across the face.
Slot image_across(const Mesh& m, int64_t c, int k) {
  const int32_t x = m.nb_cell[c * 4 + k];
  if (x >= 0) return cell_slot(x, m.nb_sx[c * 4 + k], m.nb_sy[c * 4 + k]);
  return Slot{(int32_t)c, SLOT_GHOST, 0, 0, 1, {m.cell_face[c * 4 + k], -1}};
}

bool same_member(const Slot& a, const Slot& b) {
  if (a.kind == SLOT_MISSING || b.kind == SLOT_MISSING) return false;
  const int na = a.kind == SLOT_GHOST ? a.nref : 0, nb = b.kind == SLOT_GHOST ? b.nref : 0;
  if (a.cell != b.cell || na != nb) return false;
  for (int r = 0; r < na; ++r)
    if (a.ref[r] != b.ref[r]) return false;
  return true;
}

}  // namespace

int build_mesh(const double* xy, int64_t n_nodes, const int64_t* cell_ptr, const int64_t* cell_nodes,
               int64_t n_cells, int32_t bc, const double origin[2], const double extent[2], int32_t walls,
               const double wall_from[4], int32_t inflow, Mesh& out, std::string& err) {
  if ((walls || inflow) &&
      (bc != WENO_BC_OUTFLOW || (walls & ~15) || (inflow & ~15) || !(extent[0] > 0.0 && extent[1] > 0.0))) {
    err = "walls and inflow sides name sides (bits 0-3) of an outflow box with positive extent";
    return WENO_EINVAL;
  }
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(wall_from[k])) { err = "wall_from must be finite"; return WENO_EINVAL; }
  if (n_cells <= 0 || n_nodes <= 0) { err = "empty mesh"; return WENO_EINVAL; }
  if (n_cells > (int64_t)INT32_MAX / 8) { err = "too many cells for 32-bit indices"; return WENO_EINVAL; }
  if (bc == WENO_BC_PERIODIC && !(extent[0] > 0.0 && extent[1] > 0.0)) {
    err = "periodic mesh needs positive extent";
    return WENO_EINVAL;
  }
  // ---- 1. orientation, start node, convexity (input order)
  std::vector<int64_t> nodes(n_cells * 4);
  std::vector<int8_t> nv(n_cells);
  for (int64_t c = 0; c < n_cells; ++c) {
    const int64_t b = cell_ptr[c], e = cell_ptr[c + 1];
    const int k = (int)(e - b);
    if (k != 3 && k != 4) { err = "cell " + std::to_string(c) + " has " + std::to_string(k) + " nodes"; return WENO_EMESH; }
    int64_t id[4];
    for (int i = 0; i < k; ++i) {
      id[i] = cell_nodes[b + i];
      if (id[i] < 0 || id[i] >= n_nodes) { err = "node id out of range in cell " + std::to_string(c); return WENO_EINVAL; }
    }
    double a2 = 0.0;
    for (int i = 0; i < k; ++i) {
      const int j = (i + 1) % k;
      a2 += xy[2 * id[i]] * xy[2 * id[j] + 1] - xy[2 * id[j]] * xy[2 * id[i] + 1];
    }
    if (!(a2 != 0.0)) { err = "cell " + std::to_string(c) + " has zero area"; return WENO_EMESH; }
    if (a2 < 0.0) std::reverse(id, id + k);
    const int s = (int)(std::min_element(id, id + k) - id);
    std::rotate(id, id + s, id + k);
    for (int i = 0; i < k; ++i) {
      const int j = (i + 1) % k, l = (i + 2) % k;
      const double ex = xy[2 * id[j]] - xy[2 * id[i]], ey = xy[2 * id[j] + 1] - xy[2 * id[i] + 1];
      const double fx = xy[2 * id[l]] - xy[2 * id[j]], fy = xy[2 * id[l] + 1] - xy[2 * id[j] + 1];
      if (!(ex * fy - ey * fx > 0.0)) { err = "cell " + std::to_string(c) + " is not strictly convex"; return WENO_EMESH; }
    }
    for (int i = 0; i < 4; ++i) nodes[c * 4 + i] = id[i < k ? i : k - 1];
    nv[c] = (int8_t)k;
  }
  // ---- 2. pair edges by node ids
  std::vector<EdgeRec> edges;
  edges.reserve(n_cells * 4);
  for (int64_t c = 0; c < n_cells; ++c) {
    for (int k = 0; k < nv[c]; ++k) {
      const int64_t p = nodes[c * 4 + k], q = nodes[c * 4 + (k + 1) % nv[c]];
      edges.push_back({std::min(p, q), std::max(p, q), c, (int8_t)k, (int8_t)(p < q)});
    }
  }
  std::sort(edges.begin(), edges.end(), [](const EdgeRec& x, const EdgeRec& y) {
    return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.cell < y.cell);
  });
  std::vector<int64_t> adj_cell(n_cells * 4, -1);
  std::vector<int8_t> adj_face(n_cells * 4, -1), adj_sx(n_cells * 4, 0), adj_sy(n_cells * 4, 0);
  std::vector<size_t> boundary;
  for (size_t i = 0; i < edges.size();) {
    size_t j = i + 1;
    while (j < edges.size() && edges[j].a == edges[i].a && edges[j].b == edges[i].b) ++j;
    if (j - i > 2) { err = "non-manifold edge"; return WENO_EMESH; }
    if (j - i == 2) {
      const EdgeRec &x = edges[i], &y = edges[i + 1];
      if (x.fwd == y.fwd || x.cell == y.cell) { err = "inconsistent orientation across an edge"; return WENO_EMESH; }
      adj_cell[x.cell * 4 + x.k] = y.cell;
      adj_face[x.cell * 4 + x.k] = y.k;
      adj_cell[y.cell * 4 + y.k] = x.cell;
      adj_face[y.cell * 4 + y.k] = x.k;
    } else {
      boundary.push_back(i);
    }
    i = j;
  }
  // ---- 3. periodic pairing of boundary edges by translated coordinates
  if (bc == WENO_BC_PERIODIC) {
    const double Lx = extent[0], Ly = extent[1];
    const double tol = 1e-9 * std::max(Lx, Ly);
    struct BE { double mx, my; size_t e; };
    std::vector<BE> side[4];  // 0: x = x0, 1: x = x0 + Lx, 2: y = y0, 3: y = y0 + Ly
    for (size_t bi : boundary) {
      const EdgeRec& r = edges[bi];
      const double px = xy[2 * r.a], py = xy[2 * r.a + 1], qx = xy[2 * r.b], qy = xy[2 * r.b + 1];
      const double mx = 0.5 * (px + qx), my = 0.5 * (py + qy);
      int s = -1;
      if (std::fabs(px - origin[0]) < tol && std::fabs(qx - origin[0]) < tol) s = 0;
      else if (std::fabs(px - origin[0] - Lx) < tol && std::fabs(qx - origin[0] - Lx) < tol) s = 1;
      else if (std::fabs(py - origin[1]) < tol && std::fabs(qy - origin[1]) < tol) s = 2;
      else if (std::fabs(py - origin[1] - Ly) < tol && std::fabs(qy - origin[1] - Ly) < tol) s = 3;
      if (s < 0) { err = "boundary edge not on the periodic box"; return WENO_EPERIODIC; }
      side[s].push_back({mx, my, bi});
    }
    for (int pair = 0; pair < 2; ++pair) {
      std::vector<BE>& lo = side[2 * pair];
      std::vector<BE>& hi = side[2 * pair + 1];
      if (lo.size() != hi.size()) { err = "unequal numbers of faces on opposite periodic sides"; return WENO_EPERIODIC; }
      auto key = [pair](const BE& b) { return pair == 0 ? b.my : b.mx; };
      std::sort(hi.begin(), hi.end(), [&](const BE& x, const BE& y) { return key(x) < key(y); });
      std::vector<char> used(hi.size(), 0);
      for (const BE& l : lo) {
        const double kk = key(l);
        auto it = std::lower_bound(hi.begin(), hi.end(), kk - tol, [&](const BE& b, double v) { return key(b) < v; });
        bool found = false;
        for (; it != hi.end() && key(*it) <= kk + tol; ++it) {
          const size_t h = (size_t)(it - hi.begin());
          if (used[h]) continue;
          const EdgeRec &x = edges[l.e], &y = edges[it->e];
          const double tx = pair == 0 ? Lx : 0.0, ty = pair == 0 ? 0.0 : Ly;
          // endpoints must coincide after translation (in either order)
          auto same = [&](int64_t p, int64_t q) {
            return std::fabs(xy[2 * p] + tx - xy[2 * q]) < tol && std::fabs(xy[2 * p + 1] + ty - xy[2 * q + 1]) < tol;
          };
          if (!((same(x.a, y.a) && same(x.b, y.b)) || (same(x.a, y.b) && same(x.b, y.a)))) continue;
          used[h] = 1;
          found = true;
          // x lies on the low side: seen from x's cell, y's cell sits one period lower
          const int8_t sx = pair == 0 ? 1 : 0, sy = pair == 0 ? 0 : 1;
          adj_cell[x.cell * 4 + x.k] = y.cell;
          adj_face[x.cell * 4 + x.k] = y.k;
          adj_sx[x.cell * 4 + x.k] = (int8_t)-sx;
          adj_sy[x.cell * 4 + x.k] = (int8_t)-sy;
          adj_cell[y.cell * 4 + y.k] = x.cell;
          adj_face[y.cell * 4 + y.k] = x.k;
          adj_sx[y.cell * 4 + y.k] = sx;
          adj_sy[y.cell * 4 + y.k] = sy;
          if (x.cell == y.cell) { err = "cell adjacent to itself (mesh too small)"; return WENO_EPERIODIC; }
          break;
        }
        if (!found) { err = "unpaired periodic boundary face"; return WENO_EPERIODIC; }
      }
    }
  }
  // ---- 4. renumbering: quads first, then triangles; Morton order of centroids inside
  std::vector<double> area(n_cells), cx(n_cells), cy(n_cells);
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (int64_t c = 0; c < n_cells; ++c) {
    // Green's theorem: A = 1/2 sum cross_i, centroid = 1/(6A) sum (p_i + p_{i+1}) cross_i
    double A = 0.0, sx = 0.0, sy = 0.0;
    const double x0 = xy[2 * nodes[c * 4]], y0 = xy[2 * nodes[c * 4] + 1];
    for (int i = 0; i < nv[c]; ++i) {
      const int64_t p = nodes[c * 4 + i], q = nodes[c * 4 + (i + 1) % nv[c]];
      const double ax = xy[2 * p] - x0, ay = xy[2 * p + 1] - y0, bx = xy[2 * q] - x0, by = xy[2 * q + 1] - y0;
      const double cr = ax * by - bx * ay;
      A += cr;
      sx += (ax + bx) * cr;
      sy += (ay + by) * cr;
    }
    area[c] = 0.5 * A;
    cx[c] = x0 + sx / (3.0 * A);
    cy[c] = y0 + sy / (3.0 * A);
    xmin = std::min(xmin, cx[c]); xmax = std::max(xmax, cx[c]);
    ymin = std::min(ymin, cy[c]); ymax = std::max(ymax, cy[c]);
  }
  std::vector<uint64_t> key(n_cells);
  const double sxk = 65535.0 / std::max(xmax - xmin, 1e-300), syk = 65535.0 / std::max(ymax - ymin, 1e-300);
  for (int64_t c = 0; c < n_cells; ++c) {
    const uint32_t qx = (uint32_t)std::lround((cx[c] - xmin) * sxk), qy = (uint32_t)std::lround((cy[c] - ymin) * syk);
    key[c] = ((uint64_t)(nv[c] == 4 ? 0 : 1) << 32) | (uint64_t)(spread16(qx) | (spread16(qy) << 1));
  }
  std::vector<int64_t> perm(n_cells);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int64_t x, int64_t y) { return key[x] < key[y]; });
  std::vector<int64_t> inv(n_cells);
  for (int64_t i = 0; i < n_cells; ++i) inv[perm[i]] = i;

  Mesh& m = out;
  m = Mesh();
  m.n_inst = 1;
  m.inst_period = {bc == WENO_BC_PERIODIC ? extent[0] : 0.0, bc == WENO_BC_PERIODIC ? extent[1] : 0.0};
  m.inst_bc = {bc};
  m.inst_input_offset = {0};
  m.n_input_cells = n_cells;
  m.nQ = 0;
  for (int64_t c = 0; c < n_cells; ++c) m.nQ += (nv[c] == 4);
  m.nT = n_cells - m.nQ;
  m.perm = perm;
  m.inst.assign(n_cells, 0);
  m.verts.resize(n_cells * 8);
  m.nvert.resize(n_cells);
  m.area.resize(n_cells);
  m.cen.resize(n_cells * 2);
  m.nb_cell.assign(n_cells * 4, -1);
  m.nb_face.assign(n_cells * 4, -1);
  m.nb_sx.assign(n_cells * 4, 0);
  m.nb_sy.assign(n_cells * 4, 0);
  for (int64_t i = 0; i < n_cells; ++i) {
    const int64_t c = perm[i];
    m.nvert[i] = nv[c];
    m.area[i] = area[c];
    m.cen[2 * i] = cx[c];
    m.cen[2 * i + 1] = cy[c];
    for (int k = 0; k < 4; ++k) {
      m.verts[i * 8 + 2 * k] = xy[2 * nodes[c * 4 + k]];
      m.verts[i * 8 + 2 * k + 1] = xy[2 * nodes[c * 4 + k] + 1];
      if (k < nv[c]) {
        const int64_t x = adj_cell[c * 4 + k];
        m.nb_cell[i * 4 + k] = x < 0 ? -1 : (int32_t)inv[x];
        m.nb_face[i * 4 + k] = adj_face[c * 4 + k];
        m.nb_sx[i * 4 + k] = adj_sx[c * 4 + k];
        m.nb_sy[i * 4 + k] = adj_sy[c * 4 + k];
      }
    }
  }
  // ---- 5. faces in order of their first cell
  m.cell_face.assign(n_cells * 4, -1);
  for (int64_t i = 0; i < n_cells; ++i) {
    for (int k = 0; k < m.nvert[i]; ++k) {
      const int32_t x = m.nb_cell[i * 4 + k];
      if (x >= 0 && x < i) continue;  // made by the lower cell
      const int32_t f = (int32_t)m.fL.size();
      const double* v = &m.verts[i * 8];
      const int k1 = (k + 1) % m.nvert[i];
      const double dx = v[2 * k1] - v[2 * k], dy = v[2 * k1 + 1] - v[2 * k + 1];
      const double L = std::hypot(dx, dy);
      m.fL.push_back((int32_t)i);
      m.fkL.push_back((int8_t)k);
      m.fR.push_back(x);
      m.fkR.push_back(x >= 0 ? m.nb_face[i * 4 + k] : (int8_t)-1);
      m.fnx.push_back(dy / L);
      m.fny.push_back(-dx / L);
      m.flen.push_back(L);
      m.cell_face[i * 4 + k] = f;
      int8_t wall = -1, in = 0;
      if (x < 0 && (walls | inflow)) {
        // a face of a box side lies on it with both ends; on a side named in `walls` it is a wall
        // when its midpoint lies at least wall_from[side] along the side, otherwise on a side
        // named in `inflow` an inflow face
        const double tol = 1e-9 * std::max(extent[0], extent[1]);
        for (int side = 0; side < 4; ++side) {
          const int axis = side / 2, along = 1 - axis;
          const double line = origin[axis] + (side % 2 ? extent[axis] : 0.0);
          if (!(std::fabs(v[2 * k + axis] - line) <= tol && std::fabs(v[2 * k1 + axis] - line) <= tol)) continue;
          const double t = 0.5 * (v[2 * k + along] + v[2 * k1 + along]) - origin[along];
          const bool w = (walls >> side & 1) && t >= wall_from[side];
          wall = w ? (int8_t)axis : (int8_t)-1;
          in = !w && (inflow >> side & 1) ? 1 : 0;
        }
      }
      m.fwall.push_back(wall);
      m.fin.push_back(in);
      if (x >= 0) m.cell_face[(int64_t)x * 4 + m.nb_face[i * 4 + k]] = f;
      else m.n_boundary++;
    }
  }
  m.nF = (int64_t)m.fL.size();
  // ---- 6. stencils
  m.slots.assign(n_cells * kMaxSlots, Slot{-1, SLOT_MISSING, 0, 0, 0, {-1, -1}});
  for (int64_t i = 0; i < n_cells; ++i) {
    Slot* s = &m.slots[i * kMaxSlots];
    const int k_n = m.nvert[i];
    s[0] = cell_slot((int32_t)i, 0, 0);
    for (int k = 0; k < k_n; ++k) s[k + 1] = image_across(m, i, k);
    const ChildRule* rules = k_n == 4 ? kQuadRules : kTriRules;
    const int n_rules = k_n == 4 ? 8 : 6;
    for (int r = 0; r < n_rules; ++r) {
      const ChildRule& R = rules[r];
      const Slot& parent = s[R.face + 1];
      Slot child;
      if (parent.kind == SLOT_CELL) {
        const int32_t p = parent.cell;
        const int kp = m.nb_face[i * 4 + R.face];
        const int np = m.nvert[p];
        const int other = R.start ? (kp + 1) % np : (kp + np - 1) % np;
        const int32_t x = m.nb_cell[(int64_t)p * 4 + other];
        if (x >= 0)
          child = cell_slot(x, parent.sx + m.nb_sx[(int64_t)p * 4 + other], parent.sy + m.nb_sy[(int64_t)p * 4 + other]);
        else
          child = Slot{p, SLOT_GHOST, parent.sx, parent.sy, 1, {m.cell_face[(int64_t)p * 4 + other], -1}};
      } else {
        // parent = i0 mirrored across its face R.face: mirror the member across i0's other face at the node
        const int k2 = R.start ? (R.face + k_n - 1) % k_n : (R.face + 1) % k_n;
        child = image_across(m, i, k2);
        child.kind = SLOT_GHOST;
        child.ref[child.nref++] = m.cell_face[i * 4 + R.face];
      }
      bool missing = false;
      for (int k = 0; k <= k_n && !missing; ++k) missing = same_member(child, s[k]);
      if (!missing && R.partner != 0) missing = same_member(child, s[resolve_slot(m, i, R.partner)]);
      if (!missing) s[R.slot] = child;
    }
  }
  return WENO_OK;
}

int concat_meshes(const Mesh* const* meshes, int32_t n, Mesh& out, std::string& err) {
  if (n <= 0) { err = "no meshes to join"; return WENO_EINVAL; }
  Mesh m;
  m.n_inst = 0;
  int64_t NQ = 0, NT = 0, NF = 0;
  for (int i = 0; i < n; ++i) { NQ += meshes[i]->nQ; NT += meshes[i]->nT; NF += meshes[i]->nF; m.n_inst += meshes[i]->n_inst; }
  const int64_t N = NQ + NT;
  if (N > (int64_t)INT32_MAX / 8) { err = "too many cells for 32-bit indices"; return WENO_EINVAL; }
  m.nQ = NQ;
  m.nT = NT;
  m.perm.resize(N); m.inst.resize(N); m.verts.resize(N * 8); m.nvert.resize(N); m.area.resize(N);
  m.cen.resize(N * 2); m.nb_cell.resize(N * 4); m.nb_face.resize(N * 4); m.nb_sx.resize(N * 4);
  m.nb_sy.resize(N * 4); m.cell_face.resize(N * 4); m.slots.resize(N * kMaxSlots);
  int64_t offQ = 0, offT = 0, offF = 0, offIn = 0;
  int32_t offInst = 0;
  for (int i = 0; i < n; ++i) {
    const Mesh& a = *meshes[i];
    auto g = [&](int64_t c) -> int32_t {
      if (c < 0) return -1;
      return (int32_t)(c < a.nQ ? offQ + c : NQ + offT + (c - a.nQ));
    };
    for (int64_t c = 0; c < a.n(); ++c) {
      const int64_t d = g(c);
      m.perm[d] = a.perm[c] + offIn;
      m.inst[d] = a.inst[c] + offInst;
      std::copy(&a.verts[c * 8], &a.verts[c * 8] + 8, &m.verts[d * 8]);
      m.nvert[d] = a.nvert[c];
      m.area[d] = a.area[c];
      m.cen[2 * d] = a.cen[2 * c];
      m.cen[2 * d + 1] = a.cen[2 * c + 1];
      for (int k = 0; k < 4; ++k) {
        m.nb_cell[d * 4 + k] = g(a.nb_cell[c * 4 + k]);
        m.nb_face[d * 4 + k] = a.nb_face[c * 4 + k];
        m.nb_sx[d * 4 + k] = a.nb_sx[c * 4 + k];
        m.nb_sy[d * 4 + k] = a.nb_sy[c * 4 + k];
        const int32_t f = a.cell_face[c * 4 + k];
        m.cell_face[d * 4 + k] = f < 0 ? -1 : (int32_t)(f + offF);
      }
      for (int j = 0; j < kMaxSlots; ++j) {
        Slot s = a.slots[c * kMaxSlots + j];
        if (s.kind != SLOT_MISSING) s.cell = g(s.cell);
        if (s.kind == SLOT_GHOST)
          for (int r = 0; r < s.nref; ++r) s.ref[r] = (int32_t)(s.ref[r] + offF);
        m.slots[d * kMaxSlots + j] = s;
      }
    }
    for (int64_t f = 0; f < a.nF; ++f) {
      m.fL.push_back(g(a.fL[f]));
      m.fR.push_back(g(a.fR[f]));
      m.fkL.push_back(a.fkL[f]);
      m.fkR.push_back(a.fkR[f]);
      m.fnx.push_back(a.fnx[f]);
      m.fny.push_back(a.fny[f]);
      m.flen.push_back(a.flen[f]);
      m.fwall.push_back(a.fwall[f]);
      m.fin.push_back(a.fin[f]);
    }
    for (int k = 0; k < a.n_inst; ++k) {
      m.inst_period.push_back(a.inst_period[2 * k]);
      m.inst_period.push_back(a.inst_period[2 * k + 1]);
      m.inst_bc.push_back(a.inst_bc[k]);
      m.inst_input_offset.push_back(a.inst_input_offset[k] + offIn);
    }
    m.n_boundary += a.n_boundary;
    offQ += a.nQ;
    offT += a.nT;
    offF += a.nF;
    offIn += a.n_input_cells;
    offInst += a.n_inst;
  }
  m.nF = NF;
  m.n_input_cells = offIn;
  out = std::move(m);
  return WENO_OK;
}

}  // namespace weno
