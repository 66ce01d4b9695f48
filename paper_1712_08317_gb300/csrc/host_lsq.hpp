// FP64 host precompute of the run-time reconstruction tables (Sections 3.1-3.3).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "host_mesh.hpp"

namespace weno {

struct LsqParams {
  double rcond = 1e-12;
  bool optimize = true;
  int n_threads = 0;
};

// Run-time tables of one cell type group, structure-of-arrays with the cell
// index fastest (entry e of cell q at [e * N + q]).
struct GroupTables {
  int M = 0, G = 0;
  int64_t N = 0;              // cells in the group
  int64_t first = 0;          // internal id of the group's first cell
  std::vector<int32_t> slot;  // [M][N]      cell read for slots 1..M (replacements resolved)
  std::vector<double> gop;    // [M][4][N]   g_j = [gop0 gop1; gop2 gop3] (dW_a, dW_b)
  std::vector<double> dg;     // [G][2][N]   x_G - c0
  std::vector<double> gam;    // [G][M][N]   linear weights used at run time
  std::vector<double> max_raw, max_opt;  // [N] diagnostics: max |gamma| before / after optimisation
};

// Precomputes both groups.  Returns a weno_status code.
int precompute_tables(const Mesh& m, const LsqParams& p, GroupTables& quads, GroupTables& tris, std::string& err);

// Moore-Penrose pseudo-inverse (exposed for the library's own self-checks).
void pinv_jacobi(const double* A, int m, int n, double rcond, double* P);

// Minimum-norm least-squares solutions X (n x k) of A X = B (A m x n, B m x k, m, n <= 16)
// by a complete orthogonal decomposition with column pivoting.
void minnorm_cod(const double* A, int m, int n, const double* B, int k, double rcond, double* X);

}  // namespace weno
