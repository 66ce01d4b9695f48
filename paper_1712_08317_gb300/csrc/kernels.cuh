// sm_103a kernels of the WENO3 residual and the SSP-RK3 stage update.
//
//   K1 (reconstruction, Sections 3.1-3.4): candidate gradients from gathered
//                  stencil averages, smoothness indicators, split linear weights,
//                  new indicator, nonlinear weights and the Gauss-point values;
//                  one thread per (cell, variable):
//     k_reconstruct_tma       FP32C Euler, tables staged in shared memory by TMA
//     k_reconstruct_f32c      FP32C scalar advection
//     k_reconstruct           FP64
//     k_reconstruct_char_tma  FP32C Euler, characteristic variables (four lanes
//                             per cell exchange variables by shuffles)
//     k_reconstruct_char      FP64, characteristic variables
//   k_face         one thread per face: two Gauss points, rotated HLLC (Euler) or
//                  upwind (scalar) flux, |l|/2 (F1 + F2) (Eqs. 5-6); at reflective
//                  walls the outer state is the inner one mirrored, at inflow faces
//                  the prescribed state at the stage time.
//   k_gather       one thread per cell: signed gather of its face fluxes
//                  (Eq. 4, no atomics) fused with the RK3 stage (Section 4).
//   k_advance_time after the third stage of a step: t += dt per instance.
// The reconstruction kernels take WALLS = true on meshes with reflective walls:
// stencil entries then carry momentum flips for mirror images.
//
// Layouts: state U[cell][v] (cell-major), Gauss values Wg[point][v] with the
// points of a quad at 8q..8q+7 and of a triangle at 8 nQ + 6t.., face fluxes
// F[face][v]; per-cell tables are structure-of-arrays with the cell index
// fastest, so the 4 variable threads of a cell share each table sector.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda.h>
#include <cuda_runtime.h>

namespace weno {
namespace dev {

// Candidate sub-stencils S_j = {i0, a, b} (Sections 3.1 and 3.2).
template <int M> struct Sub;
template <> struct Sub<12> {
  static __device__ __forceinline__ int a(int j) { constexpr int t[12] = {1, 2, 3, 4, 1, 1, 3, 3, 4, 2, 2, 4}; return t[j]; }
  static __device__ __forceinline__ int b(int j) { constexpr int t[12] = {2, 3, 4, 1, 5, 6, 7, 8, 9, 10, 11, 12}; return t[j]; }
};
template <> struct Sub<9> {
  static __device__ __forceinline__ int a(int j) { constexpr int t[9] = {1, 2, 3, 1, 2, 3, 3, 1, 2}; return t[j]; }
  static __device__ __forceinline__ int b(int j) { constexpr int t[9] = {2, 3, 1, 4, 5, 6, 7, 8, 9}; return t[j]; }
};

template <typename T> __device__ __forceinline__ T fabs_(T x) { return x < T(0) ? -x : x; }

// Vector loads / stores of one cell's NV values.
template <typename T, int NV>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T w[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) w[v] = __ldg(p + v);
}
template <>
__device__ __forceinline__ void load_vec<float, 4>(const float* __restrict__ p, float w[4]) {
  const float4 x = __ldg(reinterpret_cast<const float4*>(p));
  w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
}
template <>
__device__ __forceinline__ void load_vec<double, 4>(const double* __restrict__ p, double w[4]) {
  const double2 x = __ldg(reinterpret_cast<const double2*>(p));
  const double2 y = __ldg(reinterpret_cast<const double2*>(p) + 1);
  w[0] = x.x; w[1] = x.y; w[2] = y.x; w[3] = y.y;
}
template <typename T, int NV>
__device__ __forceinline__ void store_vec(T* p, const T w[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) p[v] = w[v];
}
template <>
__device__ __forceinline__ void store_vec<float, 4>(float* p, const float w[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ void store_vec<double, 4>(double* p, const double w[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(w[0], w[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(w[2], w[3]);
}

// Stencil table entries: cell id in the low 29 bits; on meshes with reflective walls
// bit 30 / bit 29 mark a mirror image whose x / y momentum is reversed.
constexpr int32_t kDevFlipX = 1 << 30, kDevFlipY = 1 << 29, kDevSlotCell = (1 << 29) - 1;

// Flip mask of variable v (Euler: rho u -> bit 30, rho v -> bit 29).
template <bool WALLS, int NV>
__device__ __forceinline__ int32_t flip_mask(int v) {
  return (WALLS && NV == 4) ? (v == 1 ? kDevFlipX : (v == 2 ? kDevFlipY : 0)) : 0;
}

// Value of variable v of stencil entry `raw` (hi and, compensated, lo), momentum reversed for
// mirror images across walls.
template <typename T, int NV, bool WALLS, bool COMP>
__device__ __forceinline__ T slot_delta(const T* __restrict__ U, const T* __restrict__ Ulo, int32_t raw, int v,
                                        int32_t fm, T w0, T l0) {
  const int64_t cs = WALLS ? (raw & kDevSlotCell) : raw;
  T a = __ldg(U + cs * NV + v);
  T b = COMP ? __ldg(Ulo + cs * NV + v) : T(0);
  if (WALLS && (raw & fm)) { a = -a; b = -b; }
  return COMP ? (a - w0) + (b - l0) : a - w0;
}

// All variables of stencil entry `raw` (hi only), momentum reversed across walls.
template <typename T, bool WALLS>
__device__ __forceinline__ void slot_state4(const T* __restrict__ U, int32_t raw, T w[4]) {
  const int64_t cs = WALLS ? (raw & kDevSlotCell) : raw;
  load_vec<T, 4>(U + cs * 4, w);
  if (WALLS) {
    if (raw & kDevFlipX) w[1] = -w[1];
    if (raw & kDevFlipY) w[2] = -w[2];
  }
}

// Error-free sum (Knuth TwoSum): s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Double-float numbers (hi + lo, |lo| <= ulp(hi)/2): ~48-bit arithmetic from FP32
// error-free transformations (Dekker / Knuth; products via fused multiply-add).
struct df { float hi, lo; };

__device__ __forceinline__ df df_norm(float s, float e) {  // fast two-sum, |s| >= |e|
  const float h = __fadd_rn(s, e);
  return df{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}

// ---------------------------------------------------------------- K1
// Threads t in [0, N*NV): cell q = t / NV of the group, variable v = t % NV.
template <typename T, int NV, int M, int G, bool COMP, bool WALLS>
__global__ void __launch_bounds__(256) k_reconstruct(
    const T* __restrict__ U, const T* __restrict__ Ulo, const int32_t* __restrict__ slot,
    const T* __restrict__ gop, const T* __restrict__ dg, const T* __restrict__ gam,
    const T* __restrict__ area, int64_t N, int64_t first, int64_t gbase, T* __restrict__ Wg,
    T eps, T theta, int linear) {
  const int64_t total = N * NV;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / NV;
    const int v = (int)(t - q * NV);
    const int64_t c = first + q;
    const T w0 = __ldg(U + c * NV + v);
    const T l0 = COMP ? __ldg(Ulo + c * NV + v) : T(0);
    // differences to the stencil cells (slots 1..M), replacements already resolved
    T dW[M + 1];
    dW[0] = T(0);
    const int32_t fm = flip_mask<WALLS, NV>(v);
#pragma unroll
    for (int s = 1; s <= M; ++s)
      dW[s] = slot_delta<T, NV, WALLS, COMP>(U, Ulo, __ldg(slot + (int64_t)(s - 1) * N + q), v, fm, w0, l0);
    // candidate gradients g_j = D_j^+ (dW_a, dW_b), beta_j = |Omega| |g_j|^2
    T gx[M], gy[M], beta[M];
    const T a0 = __ldg(area + c);
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const T da = dW[Sub<M>::a(j)], db = dW[Sub<M>::b(j)];
      const T m0 = __ldg(gop + (int64_t)(j * 4 + 0) * N + q), m1 = __ldg(gop + (int64_t)(j * 4 + 1) * N + q);
      const T m2 = __ldg(gop + (int64_t)(j * 4 + 2) * N + q), m3 = __ldg(gop + (int64_t)(j * 4 + 3) * N + q);
      gx[j] = m0 * da + m1 * db;
      gy[j] = m2 * da + m3 * db;
      beta[j] = a0 * (gx[j] * gx[j] + gy[j] * gy[j]);
    }
    T* out = Wg + (gbase + q * G) * NV + v;
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
      const T dx = __ldg(dg + (int64_t)(g * 2) * N + q), dy = __ldg(dg + (int64_t)(g * 2 + 1) * N + q);
      const T* gg = gam + (int64_t)(g * M) * N + q;
      T incr;
      if (linear) {
        incr = T(0);
#pragma unroll
        for (int j = 0; j < M; ++j) incr += __ldg(gg + (int64_t)j * N) * (gx[j] * dx + gy[j] * dy);
      } else {
        // splitting of Section 3.4: gt+ = (gamma + theta |gamma|)/2, gt- = gt+ - gamma
        T sp = T(0), sm = T(0);
#pragma unroll
        for (int j = 0; j < M; ++j) {
          const T gj = __ldg(gg + (int64_t)j * N);
          const T tp = T(0.5) * (gj + theta * fabs_(gj));
          sp += tp;
          sm += tp - gj;
        }
        const T isp = T(1) / sp, ism = T(1) / sm;
        T Ap = T(0), Bp = T(0), Am = T(0), Bm = T(0);
#pragma unroll
        for (int j = 0; j < M; ++j) {
          const T gj = __ldg(gg + (int64_t)j * N);
          const T tp = T(0.5) * (gj + theta * fabs_(gj));
          const T gp = tp * isp, gm = (tp - gj) * ism;
          const T p = gx[j] * dx + gy[j] * dy;  // P^1_j(x_G) - W0
          const T qp = gp * beta[j], qm = gm * beta[j];
          const T bp = beta[j] * (T(1) + qp + qp * qp) + eps;  // new indicator + eps
          const T bm = beta[j] * (T(1) + qm + qm * qm) + eps;
          const T ap = gp / (bp * bp), am = gm / (bm * bm);
          Ap += ap;
          Bp += ap * p;
          Am += am;
          Bm += am * p;
        }
        // R - W0 = sigma+ sum delta+ p - sigma- sum delta- p
        incr = sp * (Bp / Ap) - sm * (Bm / Am);
      }
      out[(int64_t)g * NV] = COMP ? w0 + (l0 + incr) : w0 + incr;
    }
  }
}

// FP32C variant of K1 (same arithmetic in FP32 with approximate reciprocals).
// Tables: gop4[j][q] = (o0 o1 o2 o3) of D_j^+, dg2[g][q] = x_G - c0,
// gam4[g][k][q] = gamma_{4k..4k+3}, gam1[g][q] = gamma_8 (triangles).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

#ifndef WENO_K1_MIN_BLOCKS
#define WENO_K1_MIN_BLOCKS 2  // resident 256-thread blocks' worth of threads per SM the register budget is sized for
#endif

// Paired FP32 arithmetic (Blackwell f32x2): candidates j = 2k, 2k+1 share one
// instruction.  Odd M is padded with a candidate of weight 0 (it adds nothing).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 rcp2(float2 x) { return make_float2(rcp_approx(x.x), rcp_approx(x.y)); }
__device__ __forceinline__ float2 abs2(float2 x) { return make_float2(fabsf(x.x), fabsf(x.y)); }

// Per-candidate quantities of one (cell, variable) that do not depend on the
// Gauss point, as candidate pairs: gradient (gx, gy), beta and be = beta + eps.
template <int P>
struct CandPairs {
  float2 gx[P], gy[P], b[P], be[P];
};

// Increment of one Gauss point as in gauss_increment below with every step of the nonlinear
// weights in FP64 (IEEE division), from the n candidates' (beta, p = P^1_j(x_G) - W0, gamma+,
// gamma-) in v[4n]: the fallback for weights outside the FP32 range.  Not inlined and looping at
// run time, so the FP32 path keeps its registers; it runs only at Gauss points that need it.
__device__ __noinline__ float nonlinear_increment_fp64(const float* __restrict__ v, int n, float sp, float sm,
                                                      float eps_f) {
  const double eps = eps_f;
  double Ap = 0.0, Bp = 0.0, Am = 0.0, Bm = 0.0;
  for (int j = 0; j < n; ++j) {
    const double b = v[4 * j], p = v[4 * j + 1], gp = v[4 * j + 2], gn = v[4 * j + 3];
    const double qp = gp * b, qn = gn * b;
    const double dp = b * (1.0 + qp + qp * qp) + eps, dn = b * (1.0 + qn + qn * qn) + eps;
    const double ap = gp / (dp * dp), an = gn / (dn * dn);
    Ap += ap;
    Bp += ap * p;
    Am += an;
    Bm += an * p;
  }
  return (float)((double)sp * (Bp / Ap) - (double)sm * (Bm / Am));
}

constexpr float kAlphaMin = 1e-30f;  // smallest sum of alpha the FP32 weights accept (see gauss_increment)

// Nonlinear weights of one candidate pair (or, scalar, of one candidate) at one Gauss point:
// alpha+- = gamma+- / (beta~+- + eps)^2 with beta~+- = beta (1 + q + q^2), q = gamma+- beta.
__device__ __forceinline__ void pair_alpha(float2 gp, float2 gn, float2 b, float2 be, float2& ap, float2& an) {
  const float2 qp = __fmul2_rn(gp, b), qn = __fmul2_rn(gn, b);
  const float2 dp = __ffma2_rn(b, __ffma2_rn(qp, qp, qp), be);   // beta~+ + eps
  const float2 dn = __ffma2_rn(b, __ffma2_rn(qn, qn, qn), be);   // beta~- + eps
  ap = __fmul2_rn(gp, rcp2(__fmul2_rn(dp, dp)));
  an = __fmul2_rn(gn, rcp2(__fmul2_rn(dn, dn)));
}
__device__ __forceinline__ void one_alpha(float gp, float gn, float b, float be, float& ap, float& an) {
  const float qp = gp * b, qn = gn * b;
  const float dp = fmaf(b, fmaf(qp, qp, qp), be), dn = fmaf(b, fmaf(qn, qn, qn), be);
  ap = gp * rcp_approx(dp * dp);
  an = gn * rcp_approx(dn * dn);
}

// Increment R(x_G) - W0 of one Gauss point (Section 3.4, FP32) from the
// candidate pairs and the split linear weights gamma+ (gpos), gamma- (gneg)
// with their sums sigma+- (sp, sm), which depend on geometry only and are
// precomputed in FP64:
//   R - W0 = sigma+ sum delta+ p - sigma- sum delta- p,
//   delta+-_j = alpha+-_j / sum alpha+-, alpha+-_j = gamma+-_j / (beta~+-_j + eps)^2,
//   beta~+-_j = beta_j (1 + q + q^2), q = gamma+-_j beta_j.
// The linear scheme is R - W0 = sum gamma_j p_j = sigma+ sum gamma+ p - sigma- sum gamma- p.
// With M odd the last candidate (the .x lane of the last pair) is evaluated in scalar arithmetic.
template <int M>
__device__ __forceinline__ float gauss_increment(const CandPairs<(M + 1) / 2>& c, const float2* gpos,
                                                 const float2* gneg, float dx, float dy, float sp, float sm,
                                                 int linear, float& amin) {
  constexpr int P = (M + 1) / 2, FULL = M / 2;
  amin = 1.0f;
  const float2 dx2 = f2(dx, dx), dy2 = f2(dy, dy);
  if (linear) {
    float2 ap = f2(0.f, 0.f), an = f2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const float2 p = __ffma2_rn(c.gx[k], dx2, __fmul2_rn(c.gy[k], dy2));
      ap = __ffma2_rn(gpos[k], p, ap);
      an = __ffma2_rn(gneg[k], p, an);
    }
    return sp * (ap.x + ap.y) - sm * (an.x + an.y);
  }
  // sums of alpha+- and alpha+- p: pair 0 initialises them, later pairs add
  float2 Ap, Bp, Am, Bm;
#pragma unroll
  for (int k = 0; k < FULL; ++k) {
    const float2 p = __ffma2_rn(c.gx[k], dx2, __fmul2_rn(c.gy[k], dy2));  // P^1_j(x_G) - W0
    float2 ap, an;
    pair_alpha(gpos[k], gneg[k], c.b[k], c.be[k], ap, an);
    if (k == 0) {
      Ap = ap; Bp = __fmul2_rn(ap, p);
      Am = an; Bm = __fmul2_rn(an, p);
    } else {
      Ap = __fadd2_rn(Ap, ap); Bp = __ffma2_rn(ap, p, Bp);
      Am = __fadd2_rn(Am, an); Bm = __ffma2_rn(an, p, Bm);
    }
  }
  float As = Ap.x + Ap.y, Bs = Bp.x + Bp.y, Ams = Am.x + Am.y, Bms = Bm.x + Bm.y;
  if constexpr (M % 2 == 1) {
    const float p = fmaf(c.gx[P - 1].x, dx, c.gy[P - 1].x * dy);
    float ap, an;
    one_alpha(gpos[P - 1].x, gneg[P - 1].x, c.b[P - 1].x, c.be[P - 1].x, ap, an);
    As += ap; Bs = fmaf(ap, p, Bs);
    Ams += an; Bms = fmaf(an, p, Bms);
  }
  // The smaller sum of alpha of the two groups: the caller redoes the Gauss point in FP64 when it
  // falls below kAlphaMin (indicators of order 1e6 and more, whose (beta~ + eps)^2 overflows FP32
  // or whose reciprocal flushes).  Above it every candidate that matters is far from both limits;
  // the sums never exceed 1 / eps^2 <= 1e30, since eps >= 1e-15 for FP32 weights.
  amin = fminf(As, Ams);
  return sp * Bs * rcp_approx(As) - sm * Bms * rcp_approx(Ams);
}

// gauss_increment with the nonlinear weights in FP64, whose range holds every finite FP32
// beta; delta = alpha / sum alpha is the same function, so only rounding differs.
template <int P>
__device__ __forceinline__ float gauss_increment_fp64(const CandPairs<P>& c, const float2* gpos, const float2* gneg,
                                                      float dx, float dy, float sp, float sm, float eps) {
  const float2 dx2 = f2(dx, dx), dy2 = f2(dy, dy);
  float v[8 * P];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const float2 p = __ffma2_rn(c.gx[k], dx2, __fmul2_rn(c.gy[k], dy2));
    v[8 * k + 0] = c.b[k].x; v[8 * k + 1] = p.x; v[8 * k + 2] = gpos[k].x; v[8 * k + 3] = gneg[k].x;
    v[8 * k + 4] = c.b[k].y; v[8 * k + 5] = p.y; v[8 * k + 6] = gpos[k].y; v[8 * k + 7] = gneg[k].y;
  }
  return nonlinear_increment_fp64(v, 2 * P, sp, sm, eps);
}

// Candidate gradients and smoothness indicators of one (cell, variable), as
// candidate pairs (the padding candidate of odd M has g = 0, beta = 0).
template <int NV, int M, bool WALLS>
__device__ __forceinline__ void cell_gradients(const float* __restrict__ U, const float* __restrict__ Ulo,
                                               const int32_t* __restrict__ slot, int64_t slot_pitch,
                                               const float4* __restrict__ gop4, int64_t pitch, int64_t q, int64_t c,
                                               int v, float a0, float eps, float& w0, float& l0,
                                               CandPairs<(M + 1) / 2>& cp) {
  w0 = __ldg(U + c * NV + v);
  l0 = __ldg(Ulo + c * NV + v);
  float dW[M + 1];
  dW[0] = 0.0f;
  const int32_t fm = flip_mask<WALLS, NV>(v);
#pragma unroll
  for (int s = 1; s <= M; ++s)
    dW[s] = slot_delta<float, NV, WALLS, true>(U, Ulo, __ldg(slot + (int64_t)(s - 1) * slot_pitch + q), v, fm, w0, l0);
  float gx[2 * ((M + 1) / 2)], gy[2 * ((M + 1) / 2)], b[2 * ((M + 1) / 2)];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float da = dW[Sub<M>::a(j)], db = dW[Sub<M>::b(j)];
    const float4 m = __ldg(gop4 + (int64_t)j * pitch + q);
    gx[j] = fmaf(m.x, da, m.y * db);
    gy[j] = fmaf(m.z, da, m.w * db);
    b[j] = a0 * fmaf(gx[j], gx[j], gy[j] * gy[j]);
  }
  if (M % 2) { gx[M] = 0.f; gy[M] = 0.f; b[M] = 0.f; }
#pragma unroll
  for (int k = 0; k < (M + 1) / 2; ++k) {
    cp.gx[k] = f2(gx[2 * k], gx[2 * k + 1]);
    cp.gy[k] = f2(gy[2 * k], gy[2 * k + 1]);
    const float2 bb = f2(b[2 * k], b[2 * k + 1]);
    cp.b[k] = bb;
    cp.be[k] = __fadd2_rn(bb, f2(eps, eps));
  }
}

// FP32C tables (rows of `pitch` cells): gop4[j] = D_j^+ entries; dgs[g] =
// (x_G - c0, sigma+, sigma-); gpm4[g][k] = gamma+_{4k..4k+3} for k < M/4 and
// gamma-_{4(k-M/4)..} after them; g1[g] = (gamma+_8, gamma-_8) for triangles.
template <int NV, int M, int G>
__global__ void __launch_bounds__(256, WENO_K1_MIN_BLOCKS) k_reconstruct_f32c(
    const float* __restrict__ U, const float* __restrict__ Ulo, const int32_t* __restrict__ slot,
    const float4* __restrict__ gop4, const float4* __restrict__ dgs, const float4* __restrict__ gpm4,
    const float2* __restrict__ g1, const float* __restrict__ area, int64_t N, int64_t pitch, int64_t first,
    int64_t gbase, float* __restrict__ Wg, float eps, int linear) {
  constexpr int M4 = M / 4, P = (M + 1) / 2;
  const int64_t total = N * NV;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / NV;
    const int v = (int)(t - q * NV);
    const int64_t c = first + q;
    float w0, l0;
    CandPairs<P> cp;
    cell_gradients<NV, M, false>(U, Ulo, slot, N, gop4, pitch, q, c, v, __ldg(area + c), eps, w0, l0, cp);
    float* out = Wg + (gbase + q * G) * NV + v;
    // (x_G - c0, sigma+-) and the split weights of Gauss point g
    auto tables = [&](int g, float4& d, float2* gp, float2* gn) {
      d = __ldg(dgs + (int64_t)g * pitch + q);
#pragma unroll
      for (int k = 0; k < M4; ++k) {
        const float4 x = __ldg(gpm4 + (int64_t)(g * 2 * M4 + k) * pitch + q);
        const float4 y = __ldg(gpm4 + (int64_t)(g * 2 * M4 + M4 + k) * pitch + q);
        gp[2 * k] = f2(x.x, x.y); gp[2 * k + 1] = f2(x.z, x.w);
        gn[2 * k] = f2(y.x, y.y); gn[2 * k + 1] = f2(y.z, y.w);
      }
      if (M % 4) {
        const float2 e = __ldg(g1 + (int64_t)g * pitch + q);
        gp[P - 1] = f2(e.x, 0.f);
        gn[P - 1] = f2(e.y, 0.f);
      }
    };
    float amin = 1.0f;  // smallest sum of alpha over the Gauss points
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
      float4 d;
      float2 gp[P], gn[P];
      tables(g, d, gp, gn);
      float am;
      const float incr = gauss_increment<M>(cp, gp, gn, d.x, d.y, d.z, d.w, linear, am);
      amin = fminf(amin, am);
      out[(int64_t)g * NV] = w0 + (l0 + incr);
    }
    if (!(amin >= kAlphaMin)) {  // weights outside the FP32 range (rare): every point again in FP64
#pragma unroll 1
      for (int g = 0; g < G; ++g) {
        float4 d;
        float2 gp[P], gn[P];
        tables(g, d, gp, gn);
        out[(int64_t)g * NV] = w0 + (l0 + gauss_increment_fp64<P>(cp, gp, gn, d.x, d.y, d.z, d.w, eps));
      }
    }
  }
}

// ---------------------------------------------------------------- K1 with TMA-staged tables
// Euler FP32C, one block per tile or persistent: a tile is TILE consecutive cells of one type,
// one (cell, variable) per thread.  One elected thread loads the tile's split
// linear weights, Gauss offsets and gradient operators into shared memory with
// 2D TMA copies (cp.async.bulk.tensor) completing on an mbarrier; the stencil
// gathers of the tile are issued before the wait.  The next tile's copy starts
// when the block has finished reading the current one, and the other resident
// blocks hide its latency.  Every wait is bounded: on timeout the block
// records *err = 1 and exits (its one copy has completed or is abandoned with
// the block's shared memory).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s: far beyond any copy's latency
// Waits for the barrier phase; gives up after kWaitLimitNs (or 2^26 polls) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (int it = 1; it < (1 << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

#ifndef WENO_K1_TILE
#define WENO_K1_TILE 16  // cells per block tile of the TMA reconstruction (8, 16, 32 or 64)
#endif
#ifndef WENO_K1_DG_LDS
#define WENO_K1_DG_LDS 0  // 1: the TMA reconstruction re-reads the Gauss offsets from shared memory
#endif
static_assert(WENO_K1_TILE == 8 || WENO_K1_TILE == 16 || WENO_K1_TILE == 32 || WENO_K1_TILE == 64, "tile of 8, 16, 32 or 64 cells");

constexpr int kFixupChunk = 128;  // tiles a warp of a fix-up pass scans with one 4-byte load per lane

// The tiles a fix-up pass redoes, in the order it walks them: chunks blockIdx.x, + gridDim.x, ...
// of kFixupChunk one-byte marks written by the pass before it.  Every warp of the block reads the
// same words, so all warps walk the same sequence; next() returns ntiles at the end.  The marks
// are 4-byte aligned and readable up to the next multiple of 4 bytes past the last tile.
struct MarkScan {
  const uint8_t* redo;
  int64_t ntiles, chunk;
  uint32_t lanes = 0u, nib = 0u, mine = 0u;
  int cur = 0;
  __device__ MarkScan(const uint8_t* r, int64_t n) : redo(r), ntiles(n), chunk((int64_t)blockIdx.x - gridDim.x) {}
  __device__ int64_t next() {
    while (nib == 0u) {
      while (lanes == 0u) {
        chunk += gridDim.x;
        if (chunk * kFixupChunk >= ntiles) return ntiles;
        const int64_t t0 = chunk * kFixupChunk + 4 * (threadIdx.x & 31);
        const uint32_t w = t0 < ntiles ? *reinterpret_cast<const uint32_t*>(redo + t0) : 0u;
        mine = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (t0 + j < ntiles && ((w >> (8 * j)) & 0xffu)) mine |= 1u << j;
        lanes = __ballot_sync(0xffffffffu, mine != 0u);
      }
      cur = __ffs(lanes) - 1;
      lanes &= lanes - 1u;
      nib = __shfl_sync(0xffffffffu, mine, cur);
    }
    const int j = __ffs(nib) - 1;
    nib &= nib - 1u;
    return chunk * kFixupChunk + 4 * cur + j;
  }
};

// Marks of a pass whose lanes 4c..4c+3 of warp w hold cell 8w + c of a TILE-cell tile: redo[tile]
// = 1 if a lane of the tile has `bad` set, else 0; a marked tile also writes one bit per cell to
// cells[tile * TILE / 8 ...].  Called by every thread of the block.
template <int TILE>
__device__ __forceinline__ void write_marks(bool bad, int64_t tile, uint8_t* __restrict__ redo,
                                            uint8_t* __restrict__ cells) {
  const uint32_t v = __ballot_sync(0xffffffffu, bad);
  const int need = __syncthreads_or(v != 0u);
  if (need && (threadIdx.x & 31) == 0) {
    uint32_t m8 = 0u;
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) m8 |= ((v >> (4 * c8)) & 0xfu) ? 1u << c8 : 0u;
    cells[tile * (TILE / 8) + (threadIdx.x >> 5)] = (uint8_t)m8;
  }
  if (threadIdx.x == 0) redo[tile] = (uint8_t)need;
}

// Tables of the Euler FP32C reconstruction, staged per tile: the G Gauss points of a cell are taken
// as G/2 pairs (the two points of one face), whose values share a float2.  Rows of TILE float4:
//   gam [k][j]  (gamma+_j, gamma+_j', gamma-_j, gamma-_j') at points 2k and 2k+1 (split, normalised)
//   dg  [2k]    (dx, dx', dy, dy')    x_G - c0 of the two points
//   dg  [2k+1]  (sigma+, sigma+', sigma-, sigma-')
//   gop [j]     D_j^+ (the 2x2 operator from the sub-stencil's differences to the gradient)
template <int M, int G>
struct PairTile {
  static constexpr int TILE = WENO_K1_TILE;  // cells per tile; TILE x 4 threads (one per variable)
  static constexpr int THREADS = TILE * 4;
  static constexpr int NP = G / 2;
  static constexpr int GAM = NP * M * TILE * 16;
  static constexpr int DG = G * TILE * 16;
  static constexpr int GOP = M * TILE * 16;
  static constexpr int STAGE = GAM + DG + GOP;  // bytes, multiple of 128
  static constexpr int SMEM = STAGE + 16;       // one buffer + one mbarrier (padded)
};

// Indicators are clamped to kBetaMax before beta^2 and beta^3 are formed (below).  A candidate
// with beta that large has alpha = gamma / (beta~ + eps)^2 < 1e-40 whether clamped or not, i.e.
// zero in FP32; where every candidate of a group is that large, the sum of alpha is zero and the
// cell goes to the FP64 fix-up, which uses the unclamped value.
constexpr float kBetaMax = 1e12f;

// All G Gauss values of one (cell, variable) from its stencil differences dW (dW[0] = 0) and the
// tile's tables, FP32 arithmetic (Sections 3.1-3.4):
//   g_j = D_j^+ (dW_a, dW_b),  beta_j = |Omega| |g_j|^2,  p_j = g_j . (x_G - c0) = P^1_j(x_G) - W0,
//   beta~+-_j + eps = beta (1 + q + q^2) + eps, q = gamma+-_j beta, evaluated as the polynomial
//   (beta + eps) + gamma (beta^2 + gamma beta^3) in gamma,
//   alpha+-_j = gamma+-_j / (beta~+-_j + eps)^2,
//   R - W0 = sigma+ sum alpha+ p / sum alpha+  -  sigma- sum alpha- p / sum alpha-
// (the linear scheme: sigma+ sum gamma+ p - sigma- sum gamma- p).  Candidates are the outer loop,
// and the two points of a face share the paired FP32 instructions, so the per-point sums are the
// only state kept across candidates.  Returns false if a sum of alpha fell below kAlphaMin: the
// caller then has the cell redone with FP64 weights.  From finite inputs the sums are finite (the
// clamp below keeps beta^3 finite, and an overflowing square gives alpha = 0); a NaN sum comes from
// a NaN state, which FP64 weights cannot mend, and is left to the caller's state check.
template <int M, int G>
__device__ __forceinline__ bool pair_points(const float4* __restrict__ sgam, const float4* __restrict__ sdg,
                                            const float4* __restrict__ sgo, int cl, const float* dW, float a0,
                                            float eps, int linear, float w0, float l0, float* __restrict__ out) {
  constexpr int NP = G / 2, TILE = WENO_K1_TILE;
  float2 Ap[NP], Bp[NP], Am[NP], Bm[NP];
#if WENO_K1_DG_LDS
  // the offsets of face k's points, read from shared memory where they are used (fewer registers)
  auto DX = [&](int k) { const float4 r = sdg[(2 * k) * TILE + cl]; return f2(r.x, r.y); };
  auto DY = [&](int k) { const float4 r = sdg[(2 * k) * TILE + cl]; return f2(r.z, r.w); };
#else
  float2 dx[NP], dy[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float4 r = sdg[(2 * k) * TILE + cl];
    dx[k] = f2(r.x, r.y);
    dy[k] = f2(r.z, r.w);
  }
  auto DX = [&](int k) { return dx[k]; };
  auto DY = [&](int k) { return dy[k]; };
#endif
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    Ap[k] = f2(0.f, 0.f); Bp[k] = f2(0.f, 0.f);
    Am[k] = f2(0.f, 0.f); Bm[k] = f2(0.f, 0.f);
  }
  if (linear) {
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float4 m = sgo[j * TILE + cl];
      const float da = dW[Sub<M>::a(j)], db = dW[Sub<M>::b(j)];
      const float gx = fmaf(m.x, da, m.y * db), gy = fmaf(m.z, da, m.w * db);
      const float2 GX = f2(gx, gx), GY = f2(gy, gy);
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const float4 g4 = sgam[(k * M + j) * TILE + cl];
        const float2 p = __ffma2_rn(GX, DX(k), __fmul2_rn(GY, DY(k)));
        Bp[k] = __ffma2_rn(f2(g4.x, g4.y), p, Bp[k]);
        Bm[k] = __ffma2_rn(f2(g4.z, g4.w), p, Bm[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const float4 s = sdg[(2 * k + 1) * TILE + cl];
      out[(2 * k) * 4] = w0 + (l0 + (s.x * Bp[k].x - s.z * Bm[k].x));
      out[(2 * k + 1) * 4] = w0 + (l0 + (s.y * Bp[k].y - s.w * Bm[k].y));
    }
    return true;
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float4 m = sgo[j * TILE + cl];
    const float da = dW[Sub<M>::a(j)], db = dW[Sub<M>::b(j)];
    const float gx = fmaf(m.x, da, m.y * db), gy = fmaf(m.z, da, m.w * db);
    const float b0 = a0 * fmaf(gx, gx, gy * gy);
    const float b = b0 > kBetaMax ? kBetaMax : b0;  // keeps a NaN (fminf would drop it)
    const float b2 = b * b, b3 = b2 * b, be = b + eps;
    const float2 GX = f2(gx, gx), GY = f2(gy, gy), C0 = f2(be, be), C1 = f2(b2, b2), C2 = f2(b3, b3);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const float4 g4 = sgam[(k * M + j) * TILE + cl];
      const float2 gp = f2(g4.x, g4.y), gn = f2(g4.z, g4.w);
      const float2 p = __ffma2_rn(GX, DX(k), __fmul2_rn(GY, DY(k)));
      const float2 dp = __ffma2_rn(gp, __ffma2_rn(gp, C2, C1), C0);  // beta~+ + eps at both points
      const float2 dn = __ffma2_rn(gn, __ffma2_rn(gn, C2, C1), C0);
      const float2 ap = __fmul2_rn(gp, rcp2(__fmul2_rn(dp, dp)));
      const float2 an = __fmul2_rn(gn, rcp2(__fmul2_rn(dn, dn)));
      Ap[k] = __fadd2_rn(Ap[k], ap);
      Bp[k] = __ffma2_rn(ap, p, Bp[k]);
      Am[k] = __fadd2_rn(Am[k], an);
      Bm[k] = __ffma2_rn(an, p, Bm[k]);
    }
  }
  // Above kAlphaMin every candidate that matters is far from both FP32 limits; the sums never
  // exceed 1 / eps^2 <= 1e30, since eps >= 1e-15 for FP32 weights.
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float4 s = sdg[(2 * k + 1) * TILE + cl];
    ok = ok && !(Ap[k].x < kAlphaMin) && !(Ap[k].y < kAlphaMin) && !(Am[k].x < kAlphaMin) && !(Am[k].y < kAlphaMin);
    const float i0 = s.x * Bp[k].x * rcp_approx(Ap[k].x) - s.z * Bm[k].x * rcp_approx(Am[k].x);
    const float i1 = s.y * Bp[k].y * rcp_approx(Ap[k].y) - s.w * Bm[k].y * rcp_approx(Am[k].y);
    out[(2 * k) * 4] = w0 + (l0 + i0);
    out[(2 * k + 1) * 4] = w0 + (l0 + i1);
  }
  return ok;
}

// pair_points with the nonlinear weights in FP64 (IEEE division, indicators unclamped), whose
// range holds every finite FP32 beta: the fix-up of cells whose FP32 sums of alpha left the
// range.  Gauss points are the outer loop here, so only four sums are live.
template <int M, int G>
__device__ __forceinline__ void pair_points_fp64(const float4* __restrict__ sgam, const float4* __restrict__ sdg,
                                                 const float4* __restrict__ sgo, int cl, const float* dW, float a0,
                                                 float eps, float w0, float l0, float* __restrict__ out) {
  constexpr int TILE = WENO_K1_TILE;
#pragma unroll 1
  for (int g = 0; g < G; ++g) {
    const int k = g >> 1, h = g & 1;
    const float4 r = sdg[(2 * k) * TILE + cl], s = sdg[(2 * k + 1) * TILE + cl];
    const float dxg = h ? r.y : r.x, dyg = h ? r.w : r.z;
    double Ap = 0.0, Bp = 0.0, Am = 0.0, Bm = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float4 m = sgo[j * TILE + cl];
      const float da = dW[Sub<M>::a(j)], db = dW[Sub<M>::b(j)];
      const float gx = fmaf(m.x, da, m.y * db), gy = fmaf(m.z, da, m.w * db);
      const double b = (double)a0 * ((double)gx * gx + (double)gy * gy);
      const double p = fmaf(gx, dxg, gy * dyg);
      const float4 g4 = sgam[(k * M + j) * TILE + cl];
      const double gp = h ? g4.y : g4.x, gn = h ? g4.w : g4.z;
      const double qp = gp * b, qn = gn * b;
      const double dp = b * (1.0 + qp + qp * qp) + eps, dn = b * (1.0 + qn + qn * qn) + eps;
      const double ap = gp / (dp * dp), an = gn / (dn * dn);
      Ap += ap;
      Bp += ap * p;
      Am += an;
      Bm += an * p;
    }
    const double sp = h ? s.y : s.x, sm = h ? s.w : s.z;
    out[g * 4] = w0 + (l0 + (float)(sp * (Bp / Ap) - sm * (Bm / Am)));
  }
}

// FIXUP = false: the pass over every tile, FP32 weights (pair_points); each tile writes its marks
// (write_marks) for the cells whose sums of alpha left the FP32 range.  FIXUP = true: run right
// after on the marked tiles only (MarkScan), it redoes the marked cells with FP64 weights; the
// decision per cell keeps every cell's result independent of which cells share its tile.
#ifndef WENO_K1_BLOCKS_Q
#define WENO_K1_BLOCKS_Q (WENO_K1_MIN_BLOCKS * 64 / WENO_K1_TILE)  // resident blocks per SM, quads
#endif
#ifndef WENO_K1_BLOCKS_T
// triangles: 80 registers without spills, 24 warps per SM (measured 2.6 % faster per pass than at
// the quads' 16 warps, whose 122 registers spill when cut to 96)
#define WENO_K1_BLOCKS_T (WENO_K1_MIN_BLOCKS * 96 / WENO_K1_TILE)  // resident blocks per SM, triangles
#endif
// The register budget of k_reconstruct_tma<M, ...>: 65,536 / (blocks x TILE x 4) per thread.
template <int M> struct K1Blocks { static constexpr int value = M == 12 ? WENO_K1_BLOCKS_Q : WENO_K1_BLOCKS_T; };

template <int M, int G, bool WALLS, bool FIXUP>
__global__ void __launch_bounds__(WENO_K1_TILE * 4, K1Blocks<M>::value) k_reconstruct_tma(
    const __grid_constant__ CUtensorMap map_gam, const __grid_constant__ CUtensorMap map_dg,
    const __grid_constant__ CUtensorMap map_gop, const float* __restrict__ U, const float* __restrict__ Ulo,
    const int32_t* __restrict__ slot, const float* __restrict__ area, int64_t N, int64_t first, int64_t gbase,
    float* __restrict__ Wg, float eps, int linear, uint8_t* __restrict__ redo, uint8_t* __restrict__ cells,
    int* __restrict__ err, int stall) {
  using L = PairTile<M, G>;
  static_assert(L::TILE % 8 == 0, "a byte of cell marks per 8 cells");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::STAGE);
  const int tid = threadIdx.x, cl = tid >> 2, v = tid & 3;
  const int64_t ntiles = (N + L::TILE - 1) / L::TILE;
  if (tid == 0) {
    mbar_init(&bar[0], stall ? 2 : 1);  // stall != 0 (testing aid): the wait runs out
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int64_t tile) {
    mbar_expect_tx(&bar[0], L::STAGE);
    tma_load_2d(smem, &map_gam, (int)(tile * L::TILE * 4), 0, &bar[0]);
    tma_load_2d(smem + L::GAM, &map_dg, (int)(tile * L::TILE * 4), 0, &bar[0]);
    tma_load_2d(smem + L::GAM + L::DG, &map_gop, (int)(tile * L::TILE * 4), 0, &bar[0]);
  };
  MarkScan scan(redo, ntiles);
  int64_t tile = FIXUP ? scan.next() : (int64_t)blockIdx.x;
  if (!FIXUP && tid == 0 && tile < ntiles) issue(tile);
  uint32_t phase = 0u;
  const float4* sgam = reinterpret_cast<const float4*>(smem);
  const float4* sdg = reinterpret_cast<const float4*>(smem + L::GAM);
  const float4* sgo = reinterpret_cast<const float4*>(smem + L::GAM + L::DG);
  for (; tile < ntiles; tile = FIXUP ? scan.next() : tile + gridDim.x) {
    if (FIXUP && tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the previous tile's reads
      issue(tile);
    }
    const int64_t next = tile + gridDim.x;
    const int64_t q = tile * L::TILE + cl;
    const bool act = q < N && (!FIXUP || ((cells[tile * (L::TILE / 8) + (cl >> 3)] >> (cl & 7)) & 1u));
    // stencil gathers (independent of the staged tables) before the wait
    float w0 = 0.f, l0 = 0.f, a0 = 0.f, dW[M + 1];
    dW[0] = 0.f;
    if (act) {
      const int64_t c = first + q;
      w0 = __ldg(U + c * 4 + v);
      l0 = __ldg(Ulo + c * 4 + v);
      const int32_t fm = flip_mask<WALLS, 4>(v);
#pragma unroll
      for (int s = 1; s <= M; ++s)
        dW[s] = slot_delta<float, 4, WALLS, true>(U, Ulo, __ldg(slot + (int64_t)(s - 1) * N + q), v, fm, w0, l0);
      a0 = __ldg(area + c);
    }
    const bool ok = mbar_wait_bounded(&bar[0], phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) *err = 1;
      return;
    }
    bool bad = false;
    if (act) {
      float* out = Wg + (gbase + q * G) * 4 + v;
      if constexpr (FIXUP)
        pair_points_fp64<M, G>(sgam, sdg, sgo, cl, dW, a0, eps, w0, l0, out);
      else
        bad = !pair_points<M, G>(sgam, sdg, sgo, cl, dW, a0, eps, linear, w0, l0, out);
    }
    if constexpr (!FIXUP) write_marks<L::TILE>(bad, tile, redo, cells);
    __syncthreads();  // the buffer is free for the next tile's copy
    if (!FIXUP && tid == 0 && next < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(next);
    }
  }
}

// ---------------------------------------------------------------- K2
template <typename T>
struct Prm { T gas_gamma, ax, ay; };

#ifndef WENO_K2_FAST
#define WENO_K2_FAST 1  // FP32 flux with approximate reciprocal / square root (FP64 always exact); 0: IEEE-rounded
#endif

// Division and square root of the flux: IEEE-rounded, or for FP32 with WENO_K2_FAST the
// hardware approximations (rcp.approx / sqrt.approx, a few ulp), which FP32 rounding of the
// Gauss values already dominates.
template <typename T> struct FluxMath {
  static __device__ __forceinline__ T rcp(T x) { return T(1) / x; }
  static __device__ __forceinline__ T div(T a, T b) { return a / b; }
  static __device__ __forceinline__ T sqr(T x) { return sqrt(x); }
};
#if WENO_K2_FAST
template <> struct FluxMath<float> {
  static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
  static __device__ __forceinline__ float sqr(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
};
#endif

template <typename T>
__device__ __forceinline__ void euler_x_flux(T r, T un, T ut, T E, T p, T f[4]) {
  f[0] = r * un;
  f[1] = r * un * un + p;
  f[2] = r * un * ut;
  f[3] = (E + p) * un;
}

// HLLC in the frame of the unit normal (nx, ny); returns the flux rotated back.
template <typename T>
__device__ __forceinline__ void hllc(const T wl[4], const T wr[4], T nx, T ny, T gam, T out[4], bool& bad) {
  const T rl = wl[0], rr = wr[0];
  using FM = FluxMath<T>;
  const T irl = FM::rcp(rl), irr = FM::rcp(rr);
  const T ul = (wl[1] * nx + wl[2] * ny) * irl, vl = (wl[2] * nx - wl[1] * ny) * irl;
  const T ur = (wr[1] * nx + wr[2] * ny) * irr, vr = (wr[2] * nx - wr[1] * ny) * irr;
  const T pl = (gam - T(1)) * (wl[3] - T(0.5) * rl * (ul * ul + vl * vl));
  const T pr = (gam - T(1)) * (wr[3] - T(0.5) * rr * (ur * ur + vr * vr));
  bad |= !(rl > T(0)) || !(rr > T(0)) || !(pl > T(0)) || !(pr > T(0)) || !(wl[3] == wl[3]) || !(wr[3] == wr[3]);
  const T cl = FM::sqr(gam * pl * irl), cr = FM::sqr(gam * pr * irr);
  // Roe averages
  const T sl = FM::sqr(rl), sr = FM::sqr(rr), iw = FM::rcp(sl + sr);
  const T ua = (sl * ul + sr * ur) * iw, va = (sl * vl + sr * vr) * iw;
  const T Hl = (wl[3] + pl) * irl, Hr = (wr[3] + pr) * irr;
  const T Ha = (sl * Hl + sr * Hr) * iw;
  const T ca = FM::sqr((gam - T(1)) * (Ha - T(0.5) * (ua * ua + va * va)));
  const T SL = fmin(ul - cl, ua - ca), SR = fmax(ur + cr, ua + ca);
  const T ml = rl * (SL - ul), mr = rr * (SR - ur);
  const T SS = FM::div(pr - pl + ul * ml - ur * mr, ml - mr);
  T f[4];
  if (SL >= T(0)) {
    euler_x_flux(rl, ul, vl, wl[3], pl, f);
  } else if (SS >= T(0)) {
    euler_x_flux(rl, ul, vl, wl[3], pl, f);
    const T k = FM::div(ml, SL - SS);  // rho* of the left star state
    const T Es = k * (wl[3] * irl + (SS - ul) * (SS + FM::div(pl, ml)));
    f[0] += SL * (k - rl);
    f[1] += SL * (k * SS - rl * ul);
    f[2] += SL * (k * vl - rl * vl);
    f[3] += SL * (Es - wl[3]);
  } else if (SR > T(0)) {
    euler_x_flux(rr, ur, vr, wr[3], pr, f);
    const T k = FM::div(mr, SR - SS);
    const T Es = k * (wr[3] * irr + (SS - ur) * (SS + FM::div(pr, mr)));
    f[0] += SR * (k - rr);
    f[1] += SR * (k * SS - rr * ur);
    f[2] += SR * (k * vr - rr * vr);
    f[3] += SR * (Es - wr[3]);
  } else {
    euler_x_flux(rr, ur, vr, wr[3], pr, f);
  }
  out[0] = f[0];
  out[1] = f[1] * nx - f[2] * ny;
  out[2] = f[1] * ny + f[2] * nx;
  out[3] = f[3];
}


// Prescribed outer state of the inflow faces (gr = -3 - q for inflow face q): wa at
// the Gauss points whose xi = n . x_G - c0 (FP64, [q][2]) lies below speed * t_stage,
// wb elsewhere; t_stage = t[instance] + c dt[instance] with c = 0, 1, 1/2 for the
// three RK3 stages (Section 4).  The comparison is made in FP64 in both precisions.
template <typename T>
struct Inflow {
  T wa[4], wb[4];
  const double* xi;
  const double* t;
  const double* dt;
  double speed, c;
};

__device__ __forceinline__ int64_t cell_of_gauss(int64_t g, int64_t nQ) {
  return g < 8 * nQ ? g / 8 : nQ + (g - 8 * nQ) / 6;
}

// flag[instance] is set when a Gauss-point state of a face of that instance is
// non-physical; nQ and inst map the left Gauss-value index back to its cell's
// instance (inst == nullptr: a single instance).  INFLOW: the mesh has inflow faces.
template <typename T, int NV, bool INFLOW>
__global__ void __launch_bounds__(256) k_face(
    const T* __restrict__ Wg, const int32_t* __restrict__ gl, const int32_t* __restrict__ gr,
    const T* __restrict__ fnx, const T* __restrict__ fny, const T* __restrict__ flen, int64_t nF,
    T* __restrict__ F, Prm<T> prm, int* __restrict__ flag, const int32_t* __restrict__ inst, int64_t nQ,
    Inflow<T> inf) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nF; f += (int64_t)gridDim.x * blockDim.x) {
    bool bad = false;
    const int64_t il = __ldg(gl + f);
    const int64_t ir = __ldg(gr + f);
    double t_stage = 0.0;
    if constexpr (INFLOW) {
      if (ir <= -3) {
        const int i = inst ? __ldg(inst + cell_of_gauss(il, nQ)) : 0;
        t_stage = inf.t[i] + inf.c * inf.dt[i];
      }
    }
    const T nx = __ldg(fnx + f), ny = __ldg(fny + f), len = __ldg(flen + f);
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      T wl[NV], wr[NV], fk[NV];
      load_vec<T, NV>(Wg + (il + k) * NV, wl);
      // the right cell meets the left cell's point k at its point 1 - k
      if (ir >= 0) load_vec<T, NV>(Wg + (ir + 1 - k) * NV, wr);
      else {
#pragma unroll
        for (int v = 0; v < NV; ++v) wr[v] = wl[v];
        if (NV == 4 && ir == -2) {  // reflective wall: normal momentum reversed
          const T mn = wl[1] * nx + wl[2] * ny;
          wr[1] = wl[1] - T(2) * mn * nx;
          wr[2] = wl[2] - T(2) * mn * ny;
        }
        if constexpr (INFLOW && NV == 4) {
          if (ir <= -3) {
            const bool a = __ldg(inf.xi + 2 * (-3 - ir) + k) < inf.speed * t_stage;
#pragma unroll
            for (int v = 0; v < 4; ++v) wr[v] = a ? inf.wa[v] : inf.wb[v];
          }
        }
      }
      if (NV == 4) {
        hllc<T>(wl, wr, nx, ny, prm.gas_gamma, fk, bad);
      } else {
        const T an = prm.ax * nx + prm.ay * ny;
        fk[0] = an * (an >= T(0) ? wl[0] : wr[0]);
        bad |= !(fk[0] == fk[0]);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += fk[v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] *= T(0.5) * len;
    store_vec<T, NV>(F + f * NV, acc);
    if (bad) flag[inst ? __ldg(inst + cell_of_gauss(il, nQ)) : 0] = 1;  // every writer stores the same value
  }
}

// t[i] += dt[i] for every instance (after the third stage of a step).
__global__ void k_advance_time(double* __restrict__ t, const double* __restrict__ dt, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] += dt[i];
}

// ---------------------------------------------------------------- K1, characteristic variables
// Euler (Section 4): the Gauss points of local face k are reconstructed in the
// characteristic variables of the normal flux Jacobian at the Roe average of
// the cell and its neighbour across face k (stencil slot k+1; the cell itself
// at an outflow boundary).  Four consecutive lanes hold one cell; lane l
// gathers variable l of the stencil, projects the stencil differences onto
// field l with row l of R^-1 (lane shuffles bring the other variables),
// reconstructs field l, and returns variable l of W0 + R dU with row l of R.
// Reconstructing the increment dU (zero for constant data) keeps constant
// states exact whatever the rounding of R R^-1.
template <typename T> __device__ __forceinline__ T rcp_exact(T x) { return T(1) / x; }

template <typename T>
__device__ __forceinline__ T lane_sum4(const T c[4], T x, int base) {
  T r = T(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) r += c[i] * __shfl_sync(0xffffffffu, x, base + i);
  return r;
}

// Roe frame of one face for lane l: row l of R^-1 (Lr) and row l of R (Rr), fields ordered
// q_n - a, entropy, shear, q_n + a, from the two cells' averages and the outward unit normal.
template <typename T>
__device__ __forceinline__ void roe_rows(const T Wl[4], const T Wr[4], T nx, T ny, T gm1, int l, T Lr[4],
                                         T Rr[4]) {
  const T rl = Wl[0], ul = Wl[1] / rl, vl = Wl[2] / rl;
  const T hl = (Wl[3] + gm1 * (Wl[3] - T(0.5) * rl * (ul * ul + vl * vl))) / rl;
  const T rr = Wr[0], ur = Wr[1] / rr, vr = Wr[2] / rr;
  const T hr = (Wr[3] + gm1 * (Wr[3] - T(0.5) * rr * (ur * ur + vr * vr))) / rr;
  const T sl = sqrt(rl), sr = sqrt(rr), iw = T(1) / (sl + sr);
  const T u = (sl * ul + sr * ur) * iw, v = (sl * vl + sr * vr) * iw, H = (sl * hl + sr * hr) * iw;
  const T kin = T(0.5) * (u * u + v * v);
  const T a = sqrt(gm1 * (H - kin)), ia = T(1) / a;
  const T qn = u * nx + v * ny, qt = v * nx - u * ny;
  const T b1 = gm1 * ia * ia, b2 = b1 * kin;
  if (l == 0) {
    Lr[0] = T(0.5) * (b2 + qn * ia); Lr[1] = T(-0.5) * (b1 * u + nx * ia);
    Lr[2] = T(-0.5) * (b1 * v + ny * ia); Lr[3] = T(0.5) * b1;
    Rr[0] = T(1); Rr[1] = T(1); Rr[2] = T(0); Rr[3] = T(1);
  } else if (l == 1) {
    Lr[0] = T(1) - b2; Lr[1] = b1 * u; Lr[2] = b1 * v; Lr[3] = -b1;
    Rr[0] = u - a * nx; Rr[1] = u; Rr[2] = -ny; Rr[3] = u + a * nx;
  } else if (l == 2) {
    Lr[0] = -qt; Lr[1] = -ny; Lr[2] = nx; Lr[3] = T(0);
    Rr[0] = v - a * ny; Rr[1] = v; Rr[2] = nx; Rr[3] = v + a * ny;
  } else {
    Lr[0] = T(0.5) * (b2 - qn * ia); Lr[1] = T(0.5) * (nx * ia - b1 * u);
    Lr[2] = T(0.5) * (ny * ia - b1 * v); Lr[3] = T(0.5) * b1;
    Rr[0] = H - a * qn; Rr[1] = kin; Rr[2] = qt; Rr[3] = H + a * qn;
  }
}

template <typename T, int M, int G, bool COMP, bool WALLS>
__global__ void __launch_bounds__(256) k_reconstruct_char(
    const T* __restrict__ U, const T* __restrict__ Ulo, const int32_t* __restrict__ slot,
    const T* __restrict__ gop, const T* __restrict__ dg, const T* __restrict__ gam,
    const T* __restrict__ area, int64_t N, int64_t first, int64_t gbase, T* __restrict__ Wg,
    T eps, T theta, T gas_gamma, int linear) {
  const int lane = threadIdx.x & 31, base = lane & ~3, l = lane & 3;
  const int64_t total = N * 4;
  // warp-uniform loop: every lane reaches the shuffles; lanes past the end work on cell 0
  for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < total;
       t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + lane;
    const bool act = t < total;
    const int64_t q = act ? (t >> 2) : 0;
    const int64_t c = first + q;
    T W0[4];
    load_vec<T, 4>(U + c * 4, W0);
    const T w0 = W0[l];
    const T l0 = COMP ? __ldg(Ulo + c * 4 + l) : T(0);
    T dW[M + 1];
    dW[0] = T(0);
    const int32_t fm = flip_mask<WALLS, 4>(l);
#pragma unroll
    for (int s = 1; s <= M; ++s)
      dW[s] = slot_delta<T, 4, WALLS, COMP>(U, Ulo, __ldg(slot + (int64_t)(s - 1) * N + q), l, fm, w0, l0);
    const T a0 = __ldg(area + c);
#pragma unroll 1
    for (int k = 0; k < G / 2; ++k) {
      // face frame: Roe average with the neighbour, outward normal from the face's two Gauss points
      T Wn[4];
      slot_state4<T, WALLS>(U, __ldg(slot + (int64_t)k * N + q), Wn);  // slot k+1: across face k
      const T x0 = __ldg(dg + (int64_t)(4 * k) * N + q), y0 = __ldg(dg + (int64_t)(4 * k + 1) * N + q);
      const T x1 = __ldg(dg + (int64_t)(4 * k + 2) * N + q), y1 = __ldg(dg + (int64_t)(4 * k + 3) * N + q);
      const T tx = x1 - x0, ty = y1 - y0, it = T(1) / sqrt(tx * tx + ty * ty);
      T Lr[4], Rr[4];
      roe_rows<T>(W0, Wn, ty * it, -tx * it, gas_gamma - T(1), l, Lr, Rr);
      // project the stencil differences onto field l, then candidate gradients and indicators
      T dU[M + 1];
      dU[0] = T(0);
#pragma unroll
      for (int s = 1; s <= M; ++s) dU[s] = lane_sum4(Lr, dW[s], base);
      T gx[M], gy[M], beta[M];
#pragma unroll
      for (int j = 0; j < M; ++j) {
        const T da = dU[Sub<M>::a(j)], db = dU[Sub<M>::b(j)];
        const T m0 = __ldg(gop + (int64_t)(j * 4 + 0) * N + q), m1 = __ldg(gop + (int64_t)(j * 4 + 1) * N + q);
        const T m2 = __ldg(gop + (int64_t)(j * 4 + 2) * N + q), m3 = __ldg(gop + (int64_t)(j * 4 + 3) * N + q);
        gx[j] = m0 * da + m1 * db;
        gy[j] = m2 * da + m3 * db;
        beta[j] = a0 * (gx[j] * gx[j] + gy[j] * gy[j]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int g = 2 * k + h;
        const T dx = __ldg(dg + (int64_t)(g * 2) * N + q), dy = __ldg(dg + (int64_t)(g * 2 + 1) * N + q);
        const T* gg = gam + (int64_t)(g * M) * N + q;
        T incr;
        if (linear) {
          incr = T(0);
#pragma unroll
          for (int j = 0; j < M; ++j) incr += __ldg(gg + (int64_t)j * N) * (gx[j] * dx + gy[j] * dy);
        } else {
          T sp = T(0), sm = T(0);
#pragma unroll
          for (int j = 0; j < M; ++j) {
            const T gj = __ldg(gg + (int64_t)j * N);
            const T tp = T(0.5) * (gj + theta * fabs_(gj));
            sp += tp;
            sm += tp - gj;
          }
          const T isp = T(1) / sp, ism = T(1) / sm;
          T Ap = T(0), Bp = T(0), Am = T(0), Bm = T(0);
#pragma unroll
          for (int j = 0; j < M; ++j) {
            const T gj = __ldg(gg + (int64_t)j * N);
            const T tp = T(0.5) * (gj + theta * fabs_(gj));
            const T gp = tp * isp, gmn = (tp - gj) * ism;
            const T p = gx[j] * dx + gy[j] * dy;
            const T qp = gp * beta[j], qm = gmn * beta[j];
            const T bp = beta[j] * (T(1) + qp + qp * qp) + eps;
            const T bm = beta[j] * (T(1) + qm + qm * qm) + eps;
            const T ap = gp / (bp * bp), am = gmn / (bm * bm);
            Ap += ap;
            Bp += ap * p;
            Am += am;
            Bm += am * p;
          }
          incr = sp * (Bp / Ap) - sm * (Bm / Am);
        }
        const T dWl = lane_sum4(Rr, incr, base);  // variable l of R dU
        if (act) Wg[(gbase + q * G + g) * 4 + l] = COMP ? w0 + (l0 + dWl) : w0 + dWl;
      }
    }
  }
}

#ifndef WENO_KCHAR_MIN_BLOCKS
#define WENO_KCHAR_MIN_BLOCKS 2  // resident 256-thread blocks per SM the characteristic kernel's registers allow
#endif

// Increments R(x_G) - W0 of one field at the two Gauss points of face k from that field's stencil
// differences dU (dU[0] = 0) and the tile's point-pair tables (PairTile rows), FP32: the arithmetic
// of pair_points for a single face, candidates outer, both points in one paired instruction.
// Returns false if a sum of alpha fell below kAlphaMin (the cell then goes to the FP64 fix-up).
template <int M>
__device__ __forceinline__ bool face_pair(const float4* __restrict__ sgam, const float4* __restrict__ sdg,
                                          const float4* __restrict__ sgo, int cl, int k, const float* dU, float a0,
                                          float eps, int linear, float2& incr) {
  constexpr int TILE = WENO_K1_TILE;
  const float4 r = sdg[(2 * k) * TILE + cl], s = sdg[(2 * k + 1) * TILE + cl];
  const float2 dx = f2(r.x, r.y), dy = f2(r.z, r.w);
  float2 Ap = f2(0.f, 0.f), Bp = f2(0.f, 0.f), Am = f2(0.f, 0.f), Bm = f2(0.f, 0.f);
  if (linear) {
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float4 m = sgo[j * TILE + cl];
      const float da = dU[Sub<M>::a(j)], db = dU[Sub<M>::b(j)];
      const float gx = fmaf(m.x, da, m.y * db), gy = fmaf(m.z, da, m.w * db);
      const float4 g4 = sgam[(k * M + j) * TILE + cl];
      const float2 p = __ffma2_rn(f2(gx, gx), dx, __fmul2_rn(f2(gy, gy), dy));
      Bp = __ffma2_rn(f2(g4.x, g4.y), p, Bp);
      Bm = __ffma2_rn(f2(g4.z, g4.w), p, Bm);
    }
    incr = f2(s.x * Bp.x - s.z * Bm.x, s.y * Bp.y - s.w * Bm.y);
    return true;
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const float4 m = sgo[j * TILE + cl];
    const float da = dU[Sub<M>::a(j)], db = dU[Sub<M>::b(j)];
    const float gx = fmaf(m.x, da, m.y * db), gy = fmaf(m.z, da, m.w * db);
    const float b0 = a0 * fmaf(gx, gx, gy * gy);
    const float b = b0 > kBetaMax ? kBetaMax : b0;  // keeps a NaN
    const float b2 = b * b, b3 = b2 * b, be = b + eps;
    const float2 C0 = f2(be, be), C1 = f2(b2, b2), C2 = f2(b3, b3);
    const float4 g4 = sgam[(k * M + j) * TILE + cl];
    const float2 gp = f2(g4.x, g4.y), gn = f2(g4.z, g4.w);
    const float2 p = __ffma2_rn(f2(gx, gx), dx, __fmul2_rn(f2(gy, gy), dy));
    const float2 dp = __ffma2_rn(gp, __ffma2_rn(gp, C2, C1), C0);  // beta~+ + eps at both points
    const float2 dn = __ffma2_rn(gn, __ffma2_rn(gn, C2, C1), C0);
    const float2 ap = __fmul2_rn(gp, rcp2(__fmul2_rn(dp, dp)));
    const float2 an = __fmul2_rn(gn, rcp2(__fmul2_rn(dn, dn)));
    Ap = __fadd2_rn(Ap, ap);
    Bp = __ffma2_rn(ap, p, Bp);
    Am = __fadd2_rn(Am, an);
    Bm = __ffma2_rn(an, p, Bm);
  }
  incr = f2(s.x * Bp.x * rcp_approx(Ap.x) - s.z * Bm.x * rcp_approx(Am.x),
            s.y * Bp.y * rcp_approx(Ap.y) - s.w * Bm.y * rcp_approx(Am.y));
  return !(Ap.x < kAlphaMin) && !(Ap.y < kAlphaMin) && !(Am.x < kAlphaMin) && !(Am.y < kAlphaMin);
}

// face_pair with the nonlinear weights in FP64 (IEEE division, indicators unclamped): the fix-up
// of cells whose FP32 sums of alpha left the range.
template <int M>
__device__ __forceinline__ void face_pair_fp64(const float4* __restrict__ sgam, const float4* __restrict__ sdg,
                                               const float4* __restrict__ sgo, int cl, int k, const float* dU,
                                               float a0, float eps, float2& incr) {
  constexpr int TILE = WENO_K1_TILE;
  const float4 r = sdg[(2 * k) * TILE + cl], s = sdg[(2 * k + 1) * TILE + cl];
  float out[2];
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const float dxg = h ? r.y : r.x, dyg = h ? r.w : r.z;
    double Ap = 0.0, Bp = 0.0, Am = 0.0, Bm = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float4 m = sgo[j * TILE + cl];
      const float da = dU[Sub<M>::a(j)], db = dU[Sub<M>::b(j)];
      const float gx = fmaf(m.x, da, m.y * db), gy = fmaf(m.z, da, m.w * db);
      const double b = (double)a0 * ((double)gx * gx + (double)gy * gy);
      const double pj = fmaf(gx, dxg, gy * dyg);
      const float4 g4 = sgam[(k * M + j) * TILE + cl];
      const double gp = h ? g4.y : g4.x, gn = h ? g4.w : g4.z;
      const double qp = gp * b, qn = gn * b;
      const double dp = b * (1.0 + qp + qp * qp) + eps, dn = b * (1.0 + qn + qn * qn) + eps;
      const double ap = gp / (dp * dp), an = gn / (dn * dn);
      Ap += ap;
      Bp += ap * pj;
      Am += an;
      Bm += an * pj;
    }
    const double sp = h ? s.y : s.x, sm = h ? s.w : s.z;
    out[h] = (float)(sp * (Bp / Ap) - sm * (Bm / Am));
  }
  incr = f2(out[0], out[1]);
}

// FP32C characteristic reconstruction with the tile's point-pair tables (split weights, Gauss
// offsets and sigma+-, gradient operators; the PairTile layout of k_reconstruct_tma) staged in
// shared memory by TMA.  Per face, each lane builds the Roe frame, projects the stencil
// differences onto its field and evaluates the face's two Gauss points with face_pair; lanes of
// cells past the end compute on the last cell's data and store nothing.
//
// FIXUP = false: the pass, with FP32 weights; every tile writes its marks (write_marks) for the
// cells at which a Gauss point left the FP32 range of the weights.  FIXUP = true: run right after
// on the marked tiles (MarkScan), it redoes those cells with the weights in FP64 (a separate
// instance keeps that code out of the pass's register allocation); the decision per cell keeps
// every cell's result independent of which cells share its tile.
template <int M, int G, bool WALLS, bool FIXUP>
__global__ void __launch_bounds__(WENO_K1_TILE * 4, WENO_KCHAR_MIN_BLOCKS * 64 / WENO_K1_TILE)
    k_reconstruct_char_tma(const __grid_constant__ CUtensorMap map_gam, const __grid_constant__ CUtensorMap map_dg,
                           const __grid_constant__ CUtensorMap map_gop, const float* __restrict__ U,
                           const float* __restrict__ Ulo, const int32_t* __restrict__ slot,
                           const float* __restrict__ area, int64_t N, int64_t first, int64_t gbase,
                           float* __restrict__ Wg, float eps, float gas_gamma, int linear,
                           uint8_t* __restrict__ redo, uint8_t* __restrict__ cells, int* __restrict__ err,
                           int stall) {
  using L = PairTile<M, G>;
  static_assert(L::TILE % 8 == 0, "a byte of cell marks per 8 cells");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::STAGE);
  const int tid = threadIdx.x, base = (tid & 31) & ~3, l = tid & 3, cl = tid >> 2;
  const int64_t ntiles = (N + L::TILE - 1) / L::TILE;
  if (tid == 0) {
    mbar_init(&bar[0], stall ? 2 : 1);  // stall != 0 (testing aid): the wait runs out
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int64_t tile) {
    mbar_expect_tx(&bar[0], L::STAGE);
    tma_load_2d(smem, &map_gam, (int)(tile * L::TILE * 4), 0, &bar[0]);
    tma_load_2d(smem + L::GAM, &map_dg, (int)(tile * L::TILE * 4), 0, &bar[0]);
    tma_load_2d(smem + L::GAM + L::DG, &map_gop, (int)(tile * L::TILE * 4), 0, &bar[0]);
  };
  MarkScan scan(redo, ntiles);
  int64_t tile = FIXUP ? scan.next() : (int64_t)blockIdx.x;
  if (!FIXUP && tid == 0 && tile < ntiles) issue(tile);
  uint32_t phase = 0u;
  const float4* sgam = reinterpret_cast<const float4*>(smem);
  const float4* sdg = reinterpret_cast<const float4*>(smem + L::GAM);
  const float4* sgo = reinterpret_cast<const float4*>(smem + L::GAM + L::DG);
  for (; tile < ntiles; tile = FIXUP ? scan.next() : tile + gridDim.x) {
    if (FIXUP && tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the previous tile's reads
      issue(tile);
    }
    const int64_t next = tile + gridDim.x;
    const int64_t qr = tile * L::TILE + cl;
    const bool act = qr < N && (!FIXUP || ((cells[tile * (L::TILE / 8) + (cl >> 3)] >> (cl & 7)) & 1u));
    const int64_t q = act ? qr : N - 1;
    const int64_t c = first + q;
    // stencil gathers (independent of the staged tables) before the wait
    float W0[4];
    load_vec<float, 4>(U + c * 4, W0);
    const float w0 = W0[l], l0 = __ldg(Ulo + c * 4 + l);
    float dW[M + 1];
    dW[0] = 0.f;
    const int32_t fm = flip_mask<WALLS, 4>(l);
#pragma unroll
    for (int s = 1; s <= M; ++s)
      dW[s] = slot_delta<float, 4, WALLS, true>(U, Ulo, __ldg(slot + (int64_t)(s - 1) * N + q), l, fm, w0, l0);
    const float a0 = __ldg(area + c);
    const bool ok = mbar_wait_bounded(&bar[0], phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) *err = 1;
      return;
    }
    bool inrange = true;  // every sum of alpha of this lane's Gauss points within the FP32 range
#pragma unroll 1
    for (int k = 0; k < G / 2; ++k) {
      // the frame of face k: the neighbour across it (slot k + 1) and the unit normal from the
      // direction x_G' - x_G of its two Gauss points
      float Wn[4];
      slot_state4<float, WALLS>(U, __ldg(slot + (int64_t)k * N + q), Wn);
      const float4 d0 = sdg[(2 * k) * L::TILE + cl];
      const float tx = d0.y - d0.x, ty = d0.w - d0.z, it = rsqrtf(tx * tx + ty * ty);
      float Lr[4], Rr[4];
      roe_rows<float>(W0, Wn, ty * it, -tx * it, gas_gamma - 1.f, l, Lr, Rr);
      float dU[M + 1];
      dU[0] = 0.f;
#pragma unroll
      for (int s = 1; s <= M; ++s) dU[s] = lane_sum4(Lr, dW[s], base);
      float2 incr;
      if constexpr (FIXUP) {
        if (act)
          face_pair_fp64<M>(sgam, sdg, sgo, cl, k, dU, a0, eps, incr);
        else
          incr = f2(0.f, 0.f);
      } else {
        inrange = face_pair<M>(sgam, sdg, sgo, cl, k, dU, a0, eps, linear, incr) && inrange;
      }
      const float d0l = lane_sum4(Rr, incr.x, base), d1l = lane_sum4(Rr, incr.y, base);  // variable l of R dU
      if (act) {
        Wg[(gbase + q * G + 2 * k) * 4 + l] = w0 + (l0 + d0l);
        Wg[(gbase + q * G + 2 * k + 1) * 4 + l] = w0 + (l0 + d1l);
      }
    }
    // weights outside the FP32 range at a cell of the tile (rare): the fix-up pass redoes the cell
    // (any of its four lanes).  Lanes past the end read the zero fill of the tables and are left out.
    if constexpr (!FIXUP) write_marks<L::TILE>(act && !inrange, tile, redo, cells);
    __syncthreads();  // the buffer is free for the next tile's copy
    if (!FIXUP && tid == 0 && next < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(next);
    }
  }
}

// ---------------------------------------------------------------- K3
// MODE 0: R = L(U).  MODE 1..3: SSP-RK3 stage s written as
//   W(s) = W^n + c_s ((W(s-1) - W^n) + dt L(W(s-1))), c = 1, 1/4, 2/3, W(0) = W^n,
// i.e. the stages of Section 4 with the combination regrouped around W^n.
// Stages 1, 2 write the stage buffer Ws; stage 3 writes U (= W^{n+1}).
// COMP (FP32 fluxes, compensated state): the face sum is accumulated error-free
// (compensated two-sum), and 1/|Omega|, dt, the RK coefficient and the state
// update use double-float arithmetic, so that sum_i |Omega_i| dW_i telescopes
// to ~1e-14 of the fluxes and the hi + lo state keeps its ~48-bit precision.
template <typename T, int NV, int NFACE, bool COMP, int MODE>
__global__ void __launch_bounds__(256) k_gather(
    const T* __restrict__ F, const int32_t* __restrict__ cf, const T* __restrict__ inv_area,
    const T* __restrict__ inv_area_lo, int64_t N, int64_t first, T* __restrict__ U, T* __restrict__ Ulo,
    T* __restrict__ Ws, T* __restrict__ Wslo, T* __restrict__ R, const double* __restrict__ dt,
    const int32_t* __restrict__ inst) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = first + q;
    T acc[NV], comp[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { acc[v] = T(0); comp[v] = T(0); }
#pragma unroll
    for (int k = 0; k < NFACE; ++k) {
      const int32_t e = __ldg(cf + (int64_t)k * N + q);
      const int64_t f = e >= 0 ? e : ~e;
      T fv[NV];
      load_vec<T, NV>(F + f * NV, fv);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T x = e >= 0 ? -fv[v] : fv[v];  // outward flux leaves the L cell
        if (COMP) {
          float s, err;
          two_sum((float)acc[v], (float)x, s, err);
          acc[v] = s;
          comp[v] = __fadd_rn((float)comp[v], err);
        } else {
          acc[v] += x;
        }
      }
    }
    const T ia = __ldg(inv_area + c);
    if (MODE == 0) {
      T res[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) res[v] = COMP ? (acc[v] + comp[v]) * ia : acc[v] * ia;
      store_vec<T, NV>(R + c * NV, res);
    } else {
      const double dtd = dt[inst ? __ldg(inst + c) : 0];
      T un[NV], ws[NV], out[NV];
      load_vec<T, NV>(U + c * NV, un);
      if (MODE > 1) load_vec<T, NV>(Ws + c * NV, ws);
      if (!COMP) {
        const T h = (T)dtd;
        const T cs = MODE == 1 ? T(1) : (MODE == 2 ? T(0.25) : T(2.0 / 3.0));
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T d = (MODE > 1 ? ws[v] - un[v] : T(0)) + h * (acc[v] * ia);
          out[v] = un[v] + cs * d;
        }
        store_vec<T, NV>(MODE == 3 ? U + c * NV : Ws + c * NV, out);
      } else {
        const float dth = (float)dtd;
        const df h{dth, (float)(dtd - (double)dth)};
        const df iad{(float)ia, (float)__ldg(inv_area_lo + c)};
        const df cs = MODE == 1 ? df{1.0f, 0.0f} : (MODE == 2 ? df{0.25f, 0.0f} : df{0.6666667f, -1.9868216e-08f});
        T unl[NV], wsl[NV], outl[NV];
        load_vec<T, NV>(Ulo + c * NV, unl);
        if (MODE > 1) load_vec<T, NV>(Wslo + c * NV, wsl);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const df res = df_mul(df_norm((float)acc[v], (float)comp[v]), iad);
          df d = df_mul(h, res);
          if (MODE > 1) {
            float s, e;
            two_sum((float)ws[v], -(float)un[v], s, e);
            d = df_add(d, df_norm(s, __fadd_rn(e, __fsub_rn((float)wsl[v], (float)unl[v]))));
          }
          const df o = df_add(df{(float)un[v], (float)unl[v]}, df_mul(cs, d));
          out[v] = o.hi;
          outl[v] = o.lo;
        }
        store_vec<T, NV>(MODE == 3 ? U + c * NV : Ws + c * NV, out);
        store_vec<T, NV>(MODE == 3 ? Ulo + c * NV : Wslo + c * NV, outl);
      }
    }
  }
}

// ---------------------------------------------------------------- K4 (reductions, not on the hot path)
// Per-cell stable step 2|Omega| / sum_p (|v.n_p| + c)|l_p| (FP64).
template <typename T, int NV, int NFACE, bool COMP>
__global__ void k_cell_dt(const T* __restrict__ U, const T* __restrict__ Ulo, const int32_t* __restrict__ cf,
                          const double* __restrict__ fnx, const double* __restrict__ fny,
                          const double* __restrict__ flen, const double* __restrict__ area, int64_t N,
                          int64_t first, double gas_gamma, double ax, double ay, double* __restrict__ out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = first + q;
    double w[NV];
    for (int v = 0; v < NV; ++v) w[v] = (double)U[c * NV + v] + (COMP ? (double)Ulo[c * NV + v] : 0.0);
    double u = ax, vv = ay, snd = 0.0;
    if (NV == 4) {
      u = w[1] / w[0];
      vv = w[2] / w[0];
      const double p = (gas_gamma - 1.0) * (w[3] - 0.5 * w[0] * (u * u + vv * vv));
      snd = sqrt(gas_gamma * p / w[0]);
    }
    double s = 0.0;
    for (int k = 0; k < NFACE; ++k) {
      const int32_t e = cf[(int64_t)k * N + q];
      const int64_t f = e >= 0 ? e : ~e;
      s += (fabs(u * fnx[f] + vv * fny[f]) + snd) * flen[f];
    }
    out[c] = 2.0 * area[c] / s;
  }
}

// Deterministic reductions in two levels with a fixed partition, so results do
// not depend on scheduling.  Level 1: one block per chunk [c0, c1) of cells of
// one instance; mode 0: min of x[c]; mode 1: sums of area[c] * (U + U_lo)[c][v].
template <int NV>
__device__ __forceinline__ void block_reduce_store(double acc[NV], int mode, double* __restrict__ out) {
  __shared__ double sh[256 * NV];
  for (int v = 0; v < NV; ++v) sh[v * 256 + threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int v = 0; v < NV; ++v) {
        const double a = sh[v * 256 + threadIdx.x], b = sh[v * 256 + threadIdx.x + s];
        sh[v * 256 + threadIdx.x] = mode == 0 ? fmin(a, b) : a + b;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (mode == 0) out[0] = sh[0];
    else for (int v = 0; v < NV; ++v) out[v] = sh[v * 256];
  }
}

template <typename T, int NV, bool COMP>
__global__ void __launch_bounds__(256) k_chunk_reduce(const double* __restrict__ x, const T* __restrict__ U,
                                                      const T* __restrict__ Ulo, const double* __restrict__ area,
                                                      const int64_t* __restrict__ chunks, int mode,
                                                      double* __restrict__ partial) {
  const int64_t c0 = chunks[2 * blockIdx.x], c1 = chunks[2 * blockIdx.x + 1];
  double acc[NV];
  for (int v = 0; v < NV; ++v) acc[v] = mode == 0 ? 1e300 : 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    if (mode == 0) {
      acc[0] = fmin(acc[0], x[c]);
    } else {
      for (int v = 0; v < NV; ++v)
        acc[v] += area[c] * ((double)U[c * NV + v] + (COMP ? (double)Ulo[c * NV + v] : 0.0));
    }
  }
  block_reduce_store<NV>(acc, mode, partial + (int64_t)blockIdx.x * (mode == 0 ? 1 : NV));
}

// Level 2: one block per instance over its chunks' partials [k0, k1).
template <int NV>
__global__ void __launch_bounds__(256) k_instance_reduce(const double* __restrict__ partial,
                                                         const int64_t* __restrict__ chunk_off, int mode,
                                                         double* __restrict__ out) {
  const int inst = blockIdx.x;
  const int64_t k0 = chunk_off[inst], k1 = chunk_off[inst + 1];
  const int w = mode == 0 ? 1 : NV;
  double acc[NV];
  for (int v = 0; v < NV; ++v) acc[v] = mode == 0 ? 1e300 : 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x)
    for (int v = 0; v < w; ++v) acc[v] = mode == 0 ? fmin(acc[v], partial[k]) : acc[v] + partial[k * NV + v];
  block_reduce_store<NV>(acc, mode, out + (int64_t)inst * w);
}

__global__ void k_fill(double* __restrict__ p, double v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace dev
}  // namespace weno
