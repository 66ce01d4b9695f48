// Host-side mesh: topology, renumbering, faces and WENO stencils.
//
// Everything here is plain C++17 on the host.  The GPU never sees these
// structures; the solver (solver.cu) derives flat device tables from them.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace weno {

// Slot kinds of the general stencil (Sections 3.1 and 3.2).
enum : int8_t { SLOT_CELL = 0, SLOT_GHOST = 1, SLOT_MISSING = 2 };

constexpr int kMaxSlots = 13;  // i0 .. i12

// A stencil member: a mesh cell, translated by whole periods (periodic meshes)
// or mirrored across one or two outflow boundary faces (SLOT_GHOST).
struct Slot {
  int32_t cell;     // the cell whose geometry (and average) the slot carries; -1 when missing
  int8_t kind;
  int8_t sx, sy;    // translation in periods of the owner's instance
  int8_t nref;      // SLOT_GHOST: number of mirror faces (1 or 2), applied in order
  int32_t ref[2];   // SLOT_GHOST: face ids of the boundary faces mirrored across
};

struct Mesh {
  // instances (1 unless built by concat)
  int32_t n_inst = 1;
  std::vector<double> inst_period;   // [n_inst][2]
  std::vector<int32_t> inst_bc;      // weno_bc_kind per instance
  std::vector<int64_t> inst_input_offset;  // first input id of each instance
  int64_t n_input_cells = 0;

  int64_t nQ = 0, nT = 0;            // internal ids: [0,nQ) quads, [nQ,nQ+nT) triangles
  int64_t nF = 0, n_boundary = 0;

  // per internal cell
  std::vector<int64_t> perm;         // internal -> input id
  std::vector<int32_t> inst;         // instance of the cell
  std::vector<double> verts;         // [n][4][2] CCW, first = smallest input node id
  std::vector<int8_t> nvert;         // 3 or 4
  std::vector<double> area;          // [n]
  std::vector<double> cen;           // [n][2]
  std::vector<int32_t> nb_cell;      // [n][4] cell across local face k, -1 at an outflow boundary
  std::vector<int8_t> nb_face;       // [n][4] that cell's local index of the shared face
  std::vector<int8_t> nb_sx, nb_sy;  // [n][4] its translation in periods
  std::vector<int32_t> cell_face;    // [n][4] face id of local face k
  std::vector<Slot> slots;           // [n][13]

  // faces, oriented from L (normal points from L to R)
  std::vector<int32_t> fL, fR;       // fR = -1: outflow boundary face
  std::vector<int8_t> fkL, fkR;
  std::vector<double> fnx, fny, flen;
  std::vector<int8_t> fwall;         // reflective wall faces: 0 on an x side, 1 on a y side; -1 otherwise
  std::vector<int8_t> fin;           // 1: inflow face (prescribed outer state), 0 otherwise

  int64_t n() const { return nQ + nT; }
  bool is_quad(int64_t c) const { return c < nQ; }
};

// Builds topology, renumbering, faces and stencils.  Returns a weno_status
// code and fills err on failure.
int build_mesh(const double* xy, int64_t n_nodes, const int64_t* cell_ptr, const int64_t* cell_nodes,
               int64_t n_cells, int32_t bc, const double origin[2], const double extent[2], int32_t walls,
               const double wall_from[4], int32_t inflow, Mesh& out, std::string& err);

// Disjoint union (batched instances).
int concat_meshes(const Mesh* const* meshes, int32_t n, Mesh& out, std::string& err);

// Candidate sub-stencils S_j = {i0, a, b}, j = 1..M (Sections 3.1, 3.2).
extern const int8_t kQuadSub[12][2];
extern const int8_t kTriSub[9][2];

// Slot whose cell a (possibly missing) slot stands for.
int resolve_slot(const Mesh& m, int64_t c, int j);

// Vertices (translated or mirrored) of the cell standing in slot j of c; returns the count.
int slot_polygon(const Mesh& m, int64_t c, int j, double out[4][2]);

// Cell whose average slot j reads at run time (a mirror image reads the cell it mirrors).
int32_t slot_value_cell(const Mesh& m, int64_t c, int j);

// Momentum components reversed in the value of slot j (mirror images across reflective walls):
// kFlipX | kFlipY bits, to be or-ed into the cell id of the device stencil table.
constexpr int32_t kFlipX = 1 << 30, kFlipY = 1 << 29, kSlotCell = (1 << 29) - 1;
int32_t slot_flip_bits(const Mesh& m, int64_t c, int j);

}  // namespace weno
