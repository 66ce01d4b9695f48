// FP64 host precompute: P^2 least squares, candidate gradients, linear
// weights and their optimisation, per cell and Gauss point.
//
// Per cell i0 (Section 3.1, triangles Section 3.2):
//   basis p^k = m^k - avg_{Omega_0} m^k of the monomials
//   m = (xi_x, xi_y, xi_x^2, xi_y^2, xi_x xi_y) in cell-scaled coordinates
//   xi = (x - c0)/sqrt|Omega_0| (reading; keeps the matrices O(1)).
//   A_jk = E_j avg_{Omega_ij} p^k (Eq. 10), cell averages from the exact
//   polygon moments of Green's theorem.
//   eta(x_G) = p(x_G)^T A^+ (Eq. 13), eta_0 = 1 - sum eta_j.
//   candidate j on {i0, a, b}: g_j = D_j^+ (dW_a, dW_b), D_j = [c_a - c0; c_b - c0].
//   B (slots x candidates) from P^1_j(x_G) = W0 + (x_G - c0) . g_j (Eq. 14),
//   gamma = B^+ eta (Eq. 15), by a complete orthogonal decomposition of B.
//   Section 3.3: d_j from |gamma| at the same Gauss point, eta^opt from the
//   weighted rows d_j A_j, gamma^opt = B^+ eta^opt.
// The zeta-regularised normal equations of Eqs. 12 and 15 are read as their
// zeta -> 0 limit, the minimum-norm least-squares solution: for the small
// A and D_j systems by one-sided Jacobi SVD (Hestenes) with singular values
// below rcond * sigma_max dropped; for B by QR with column pivoting (rank
// from |R_jj| > rcond |R_00|) completed by an RZ step.
#include "host_lsq.hpp"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "weno3.h"

namespace weno {

void pinv_jacobi(const double* A, int m, int n, double rcond, double* P) {
  double W[16 * 16], V[16 * 16];
  for (int i = 0; i < m * n; ++i) W[i] = A[i];
  for (int i = 0; i < n * n; ++i) V[i] = 0.0;
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  double fro = 0.0;
  for (int i = 0; i < m * n; ++i) fro += A[i] * A[i];
  // columns below this squared norm are rounding noise of a rank-deficient matrix
  const double noise = 1e-30 * fro;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = 0; i < m; ++i) {
          const double wp = W[i * n + p], wq = W[i * n + q];
          a += wp * wp;
          b += wq * wq;
          g += wp * wq;
        }
        if (g == 0.0 || std::fabs(g) <= 1e-15 * std::sqrt(a * b) || a <= noise || b <= noise) continue;
        rotated = true;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < m; ++i) {
          const double wp = W[i * n + p], wq = W[i * n + q];
          W[i * n + p] = c * wp - s * wq;
          W[i * n + q] = s * wp + c * wq;
        }
        for (int i = 0; i < n; ++i) {
          const double vp = V[i * n + p], vq = V[i * n + q];
          V[i * n + p] = c * vp - s * vq;
          V[i * n + q] = s * vp + c * vq;
        }
      }
    }
    if (!rotated) break;
  }
  double sig2[16], smax = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += W[i * n + j] * W[i * n + j];
    sig2[j] = s;
    smax = std::max(smax, std::sqrt(s));
  }
  const double cut = rcond * smax;
  double inv2[16];
  for (int j = 0; j < n; ++j) inv2[j] = (std::sqrt(sig2[j]) > cut && sig2[j] > 0.0) ? 1.0 / sig2[j] : 0.0;
  // A = (W / sigma) sigma V^T  ->  A^+ = V diag(1/sigma^2) W^T
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += V[k * n + j] * inv2[j] * W[i * n + j];
      P[k * m + i] = s;
    }
}

void minnorm_cod(const double* A, int m, int n, const double* Bk, int k, double rcond, double* X) {
  // Complete orthogonal decomposition (Golub & Van Loan, Sec. 5.4-5.5):
  // A P = Q [R11 R12; 0 0] with column pivoting (rank r from |R_jj| > rcond |R_00|),
  // [R11 R12] = [T 0] Z^T by Householder reflections from the right, then the
  // minimum-norm solution x = P Z [T^{-1} (Q^T b)_{1..r}; 0].
  double W[16 * 16], R[16 * 16];
  int piv[16];
  for (int i = 0; i < m * n; ++i) W[i] = A[i];
  for (int i = 0; i < m * k; ++i) R[i] = Bk[i];  // right-hand sides, m x k
  for (int j = 0; j < n; ++j) piv[j] = j;
  const int t = std::min(m, n);
  double r00 = 0.0;
  int r = 0;
  for (int j = 0; j < t; ++j) {
    // pivot: largest remaining column norm
    int best = j;
    double bn = -1.0;
    for (int c = j; c < n; ++c) {
      double s = 0.0;
      for (int i = j; i < m; ++i) s += W[i * n + c] * W[i * n + c];
      if (s > bn) { bn = s; best = c; }
    }
    if (best != j) {
      for (int i = 0; i < m; ++i) std::swap(W[i * n + j], W[i * n + best]);
      std::swap(piv[j], piv[best]);
    }
    const double nrm = std::sqrt(bn);
    if (j == 0) r00 = nrm;
    if (!(nrm > rcond * r00) || nrm == 0.0) break;
    r = j + 1;
    // Householder reflector v (v_j = x_j - alpha) zeroing W[j+1.., j]
    const double x0 = W[j * n + j];
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    double v[16];
    for (int i = j; i < m; ++i) v[i] = W[i * n + j];
    v[j] = x0 - alpha;
    double vv = 0.0;
    for (int i = j; i < m; ++i) vv += v[i] * v[i];
    if (vv > 0.0) {
      const double tau = 2.0 / vv;
      for (int c = j; c < n; ++c) {
        double d = 0.0;
        for (int i = j; i < m; ++i) d += v[i] * W[i * n + c];
        d *= tau;
        for (int i = j; i < m; ++i) W[i * n + c] -= d * v[i];
      }
      for (int c = 0; c < k; ++c) {
        double d = 0.0;
        for (int i = j; i < m; ++i) d += v[i] * R[i * k + c];
        d *= tau;
        for (int i = j; i < m; ++i) R[i * k + c] -= d * v[i];
      }
    }
    W[j * n + j] = alpha;
    for (int i = j + 1; i < m; ++i) W[i * n + j] = 0.0;
  }
  // RZ: reflect columns {i, r..n-1} of rows 0..i so that row i of R12 vanishes
  double zv[16][16];
  double ztau[16];
  for (int i = r - 1; i >= 0; --i) {
    if (r == n) { ztau[i] = 0.0; continue; }
    double a2 = W[i * n + i] * W[i * n + i];
    for (int c = r; c < n; ++c) a2 += W[i * n + c] * W[i * n + c];
    const double nrm = std::sqrt(a2);
    const double x0 = W[i * n + i];
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    double* v = zv[i];
    v[0] = x0 - alpha;  // coordinate i
    double vv = v[0] * v[0];
    for (int c = r; c < n; ++c) { v[1 + c - r] = W[i * n + c]; vv += v[1 + c - r] * v[1 + c - r]; }
    ztau[i] = vv > 0.0 ? 2.0 / vv : 0.0;
    for (int row = 0; row <= i; ++row) {
      double d = v[0] * W[row * n + i];
      for (int c = r; c < n; ++c) d += v[1 + c - r] * W[row * n + c];
      d *= ztau[i];
      W[row * n + i] -= d * v[0];
      for (int c = r; c < n; ++c) W[row * n + c] -= d * v[1 + c - r];
    }
  }
  for (int c = 0; c < k; ++c) {
    double w[16];
    for (int i = 0; i < n; ++i) w[i] = 0.0;
    // T y = (Q^T b)_{0..r-1}, T upper triangular in W[0..r-1][0..r-1]
    for (int i = r - 1; i >= 0; --i) {
      double s = R[i * k + c];
      for (int j = i + 1; j < r; ++j) s -= W[i * n + j] * w[j];
      w[i] = s / W[i * n + i];
    }
    // x~ = Z w = H_{r-1} ... H_0 w: apply H_0 first
    for (int i = 0; i < r; ++i) {
      if (ztau[i] == 0.0) continue;
      const double* v = zv[i];
      double d = v[0] * w[i];
      for (int cc = r; cc < n; ++cc) d += v[1 + cc - r] * w[cc];
      d *= ztau[i];
      w[i] -= d * v[0];
      for (int cc = r; cc < n; ++cc) w[cc] -= d * v[1 + cc - r];
    }
    for (int i = 0; i < n; ++i) X[piv[i] * k + c] = w[i];
  }
}

namespace {

// Averages of 1, xi_x, xi_y, xi_x^2, xi_y^2, xi_x xi_y over a polygon, by
// Green's theorem (exact polygon moments).
void polygon_moments(const double v[4][2], int nv, const double c0[2], double s, double avg[5], double* area_out) {
  double x[4], y[4];
  for (int i = 0; i < nv; ++i) { x[i] = (v[i][0] - c0[0]) / s; y[i] = (v[i][1] - c0[1]) / s; }
  double I0 = 0, Ix = 0, Iy = 0, Ixx = 0, Iyy = 0, Ixy = 0;
  for (int i = 0; i < nv; ++i) {
    const int j = (i + 1) % nv;
    const double cr = x[i] * y[j] - x[j] * y[i];
    I0 += cr;
    Ix += (x[i] + x[j]) * cr;
    Iy += (y[i] + y[j]) * cr;
    Ixx += (x[i] * x[i] + x[i] * x[j] + x[j] * x[j]) * cr;
    Iyy += (y[i] * y[i] + y[i] * y[j] + y[j] * y[j]) * cr;
    Ixy += (x[i] * y[j] + 2.0 * x[i] * y[i] + 2.0 * x[j] * y[j] + x[j] * y[i]) * cr;
  }
  I0 *= 0.5;
  avg[0] = Ix / (6.0 * I0);
  avg[1] = Iy / (6.0 * I0);
  avg[2] = Ixx / (12.0 * I0);
  avg[3] = Iyy / (12.0 * I0);
  avg[4] = Ixy / (24.0 * I0);
  if (area_out) *area_out = I0;
}

constexpr double kGA = 0.78867513459481288225;  // (3 + sqrt 3) / 6, Eq. (5)
constexpr double kGB = 0.21132486540518711775;  // (3 - sqrt 3) / 6

void cell_tables(const Mesh& m, const LsqParams& p, int64_t c, GroupTables& T, int64_t q) {
  const bool quad = m.is_quad(c);
  const int M = quad ? 12 : 9, G = quad ? 8 : 6, R = M + 1;
  const int8_t(*sub)[2] = quad ? kQuadSub : kTriSub;
  const int64_t N = T.N;
  const double c0[2] = {m.cen[2 * c], m.cen[2 * c + 1]};
  const double s0 = std::sqrt(m.area[c]);
  // slot geometry
  double avg[kMaxSlots][5];
  double E[kMaxSlots];
  int res[kMaxSlots];
  for (int j = 0; j < R; ++j) {
    double poly[4][2];
    const int nv = slot_polygon(m, c, j, poly);
    polygon_moments(poly, nv, c0, s0, avg[j], nullptr);
    E[j] = m.slots[c * kMaxSlots + j].kind == SLOT_MISSING ? 0.0 : 1.0;
    res[j] = resolve_slot(m, c, j);
  }
  // A (M x 5) and its pseudo-inverse
  double A[12 * 5], Ap[5 * 12];
  for (int j = 1; j < R; ++j)
    for (int k = 0; k < 5; ++k) A[(j - 1) * 5 + k] = E[j] * (avg[j][k] - avg[0][k]);
  pinv_jacobi(A, M, 5, p.rcond, Ap);
  // candidate gradient operators
  double gop[12][4];
  for (int j = 0; j < M; ++j) {
    const int a = res[sub[j][0]], b = res[sub[j][1]];
    double D[4] = {s0 * avg[a][0], s0 * avg[a][1], s0 * avg[b][0], s0 * avg[b][1]};  // centroid offsets
    pinv_jacobi(D, 2, 2, p.rcond, gop[j]);
    for (int e = 0; e < 4; ++e) T.gop[(j * 4 + e) * N + q] = gop[j][e];
    T.slot[j * N + q] = slot_value_cell(m, c, j + 1) | slot_flip_bits(m, c, j + 1);
  }
  const double* v = &m.verts[c * 8];
  const int nv0 = m.nvert[c];
  double mraw = 0.0, mopt = 0.0;
  for (int g = 0; g < G; ++g) {
    const int k = g / 2, k1 = (k + 1) % nv0;
    const double wa = (g & 1) ? kGB : kGA, wb = (g & 1) ? kGA : kGB;
    const double xg = wa * v[2 * k] + wb * v[2 * k1], yg = wa * v[2 * k + 1] + wb * v[2 * k1 + 1];
    const double dx = xg - c0[0], dy = yg - c0[1];
    T.dg[(g * 2 + 0) * N + q] = dx;
    T.dg[(g * 2 + 1) * N + q] = dy;
    const double ex = dx / s0, ey = dy / s0;
    const double pg[5] = {ex - avg[0][0], ey - avg[0][1], ex * ex - avg[0][2], ey * ey - avg[0][3], ex * ey - avg[0][4]};
    double eta[13];
    double sum = 0.0;
    for (int j = 1; j < R; ++j) {
      double s = 0.0;
      for (int kk = 0; kk < 5; ++kk) s += pg[kk] * Ap[kk * M + (j - 1)];
      eta[j] = s;
      sum += s;
    }
    eta[0] = 1.0 - sum;
    // B: rows = slots, columns = candidates
    double B[13 * 12];
    std::fill(B, B + R * M, 0.0);
    for (int j = 0; j < M; ++j) {
      const double t0 = dx * gop[j][0] + dy * gop[j][2];
      const double t1 = dx * gop[j][1] + dy * gop[j][3];
      B[res[sub[j][0]] * M + j] += t0;
      B[res[sub[j][1]] * M + j] += t1;
      B[0 * M + j] += 1.0 - t0 - t1;
    }
    double gam[12];
    minnorm_cod(B, R, M, eta, 1, p.rcond, gam);
    for (int j = 0; j < M; ++j) mraw = std::max(mraw, std::fabs(gam[j]));
    if (p.optimize) {
      double d[12];
      for (int j = 0; j < M; ++j) d[j] = 1.0;
      if (quad) {
        for (int j = 5; j <= 12; ++j) d[j - 1] = 1.0 / std::max(1.0, std::fabs(gam[j - 1]));
      } else {
        const int pr[6][2] = {{4, 8}, {8, 4}, {5, 9}, {9, 5}, {6, 7}, {7, 6}};
        for (auto& jk : pr)
          d[jk[0] - 1] = 1.0 / std::max(std::max(1.0, std::fabs(gam[jk[0] - 1])), std::fabs(gam[jk[1] - 1]));
      }
      // eta^opt_j = d_j [p^T (DA)^+]_j, and p^T (DA)^+ is the minimum-norm solution
      // y of (DA)^T y = p (the pseudo-inverse of a transpose is the transpose of it)
      double DAt[5 * 12], y[12];
      for (int j = 0; j < M; ++j)
        for (int kk = 0; kk < 5; ++kk) DAt[kk * M + j] = d[j] * A[j * 5 + kk];
      minnorm_cod(DAt, 5, M, pg, 1, p.rcond, y);
      sum = 0.0;
      for (int j = 1; j < R; ++j) {
        eta[j] = y[j - 1] * d[j - 1];
        sum += eta[j];
      }
      eta[0] = 1.0 - sum;
      minnorm_cod(B, R, M, eta, 1, p.rcond, gam);
    }
    // sum_j gamma_j = 1 (Section 3.1) holds for the exact solution; impose it on the computed one
    double gsum = 0.0;
    for (int j = 0; j < M; ++j) gsum += gam[j];
    for (int j = 0; j < M; ++j) {
      gam[j] /= gsum;
      T.gam[(g * M + j) * N + q] = gam[j];
      mopt = std::max(mopt, std::fabs(gam[j]));
    }
  }
  T.max_raw[q] = mraw;
  T.max_opt[q] = mopt;
}

void alloc_group(GroupTables& T, int M, int G, int64_t N, int64_t first) {
  T.M = M;
  T.G = G;
  T.N = N;
  T.first = first;
  T.slot.assign((size_t)M * N, 0);
  T.gop.assign((size_t)M * 4 * N, 0.0);
  T.dg.assign((size_t)G * 2 * N, 0.0);
  T.gam.assign((size_t)G * M * N, 0.0);
  T.max_raw.assign(N, 0.0);
  T.max_opt.assign(N, 0.0);
}

}  // namespace

int precompute_tables(const Mesh& m, const LsqParams& p, GroupTables& quads, GroupTables& tris, std::string& err) {
  try {
    alloc_group(quads, 12, 8, m.nQ, 0);
    alloc_group(tris, 9, 6, m.nT, m.nQ);
  } catch (const std::bad_alloc&) {
    err = "host allocation of the precompute tables failed";
    return WENO_ENOMEM;
  }
  const int64_t n = m.n();
  int nt = p.n_threads > 0 ? p.n_threads : (int)std::thread::hardware_concurrency();
  nt = std::max(1, std::min(nt, (int)std::max<int64_t>(1, n / 256)));
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    const int64_t chunk = 256;
    for (;;) {
      const int64_t b = next.fetch_add(chunk);
      if (b >= n) break;
      const int64_t e = std::min(n, b + chunk);
      for (int64_t c = b; c < e; ++c) {
        if (c < m.nQ) cell_tables(m, p, c, quads, c);
        else cell_tables(m, p, c, tris, c - m.nQ);
      }
    }
  };
  std::vector<std::thread> th;
  for (int i = 1; i < nt; ++i) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return WENO_OK;
}

}  // namespace weno
