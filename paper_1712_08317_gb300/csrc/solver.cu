// C ABI of the library: meshes (host), solvers (device tables, launches,
// CUDA graphs of the RK3 step, autotuning, reductions).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "host_lsq.hpp"
#include "host_mesh.hpp"
#include "kernels.cuh"
#include "weno3.h"

namespace weno {
int set_error(int code, const std::string& msg);
}

using weno::GroupTables;
using weno::Mesh;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

}  // namespace

int weno::set_error(int code, const std::string& msg) { return fail(code, msg); }

namespace {

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(WENO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

struct Launch {
  int block = 256;
  int grid = 0;  // 0: one thread per work item
};

unsigned grid_of(const Launch& l, int64_t work) {
  const int64_t full = (work + l.block - 1) / l.block;
  const int64_t g = l.grid > 0 ? std::min<int64_t>(l.grid, full) : full;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 0x7fffffff));
}

// TMA reconstruction: TILE x 4 threads per block, one TILE-cell tile per iteration.
constexpr int kTile = weno::dev::PairTile<12, 8>::TILE;
unsigned tma_grid(const Launch& l, int64_t cells) {
  const int64_t tiles = (cells + kTile - 1) / kTile;
  const int64_t g = l.grid > 0 ? std::min<int64_t>(l.grid, tiles) : tiles;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 0x7fffffff));
}

}  // namespace

struct weno_mesh_s {
  Mesh m;
  // FP64 precompute of the last solver created on this mesh (same rcond / optimize reuse it)
  std::shared_ptr<std::pair<GroupTables, GroupTables>> tables;
  double tables_rcond = -1.0;
  int tables_optimize = -1;
};

struct weno_solver_s {
  int dev = 0, nsm = 0;
  weno_params prm{};
  int nv = 4;
  bool fp64 = true;
  size_t esz = 8;
  int64_t nQ = 0, nT = 0, N = 0, nF = 0, n_boundary = 0;
  int n_inst = 1;
  // device tables
  // FP64: SoA tables [entry][cell] (gop, dg, gam).  FP32C: packed rows of float4 / float2
  // with the cell fastest: gop = D_j^+ entries, dg = (x_G - c0, sigma+, sigma-),
  // gam = gamma+ then gamma- rows, gam1 = (gamma+_8, gamma-_8) of triangles.
  void *q_gop = nullptr, *q_dg = nullptr, *q_gam = nullptr, *t_gop = nullptr, *t_dg = nullptr, *t_gam = nullptr;
  void *q_gam1 = nullptr, *t_gam1 = nullptr;
  void *q_pgam = nullptr, *q_pdg = nullptr, *t_pgam = nullptr, *t_pdg = nullptr;  // point-pair tables (Euler FP32C)
  int64_t q_pitch = 0, t_pitch = 0;  // row pitch (cells) of the packed FP32C tables
  bool tma = false;                   // Euler FP32C: reconstruction with TMA-staged tables
  CUtensorMap q_map_gop{}, t_map_gop{};  // gradient operators
  CUtensorMap q_map_pgam{}, q_map_pdg{}, t_map_pgam{}, t_map_pdg{};  // point-pair tables (both FP32C Euler kernels)
  int* err = nullptr;                 // set by a kernel whose bounded wait timed out
  uint8_t* fix_marks = nullptr;       // FP32C Euler: tiles and cells whose weights left the FP32 range
  int32_t *q_slot = nullptr, *t_slot = nullptr, *q_cf = nullptr, *t_cf = nullptr;
  void *area = nullptr, *inv_area = nullptr, *inv_area_lo = nullptr;
  double* area64 = nullptr;
  int32_t *gl = nullptr, *gr = nullptr;
  void *fnx = nullptr, *fny = nullptr, *flen = nullptr;
  double *fnx64 = nullptr, *fny64 = nullptr, *flen64 = nullptr;
  int32_t* inst = nullptr;
  int64_t *chunks = nullptr, *chunk_off = nullptr;  // reduction partition: [begin, end) pairs; per-instance offsets
  int64_t n_chunks = 0;
  double* partial = nullptr;
  // scratch
  void *Wg = nullptr, *F = nullptr, *Ws = nullptr, *Wslo = nullptr;
  double *dt_dev = nullptr, *red = nullptr, *cell_dt = nullptr;
  double* t_dev = nullptr;   // time of each instance (advanced by every step)
  int64_t n_in = 0;          // inflow faces
  double* in_xi = nullptr;   // [n_in][2] n . x_G - c0 of their Gauss points
  double in_wa[4] = {}, in_wb[4] = {};  // prescribed conservative states
  int* flag = nullptr;
  int debug_stall = 0;  // weno_solver_debug_stall
  bool walls = false;   // the mesh has reflective wall faces (stencil values carry momentum flips)
  std::vector<void*> allocs;
  Launch k1q, k1t, k2, k3q, k3t;
  cudaStream_t cap = nullptr;
  struct Graph {
    const void* U;
    const void* Ulo;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;

  ~weno_solver_s() {
    DeviceGuard g(dev);
    for (auto& x : graphs) cudaGraphExecDestroy(x.exec);
    if (cap) cudaStreamDestroy(cap);
    for (void* p : allocs) cudaFree(p);
  }
  template <typename P>
  int alloc(P** p, size_t bytes) {
    void* q = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return fail(WENO_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(q);
    *p = reinterpret_cast<P*>(q);
    return WENO_OK;
  }
  void drop_graphs() {
    for (auto& x : graphs) cudaGraphExecDestroy(x.exec);
    graphs.clear();
  }
};

namespace {

using S = weno_solver_s;
static_assert(weno::dev::kDevFlipX == weno::kFlipX && weno::dev::kDevFlipY == weno::kFlipY &&
                  weno::dev::kDevSlotCell == weno::kSlotCell,
              "stencil table bit layout shared by the host tables and the kernels");

// ------------------------------------------------------------ launches
// Fix-up marks of the FP32C Euler reconstructions (component-wise and characteristic), per cell
// group (quads, then triangles): one byte per tile, then one bit per cell of the tile, each part
// padded to 16 bytes; zero bytes for every other path.
int64_t redo_part(int64_t n) {
  constexpr int64_t t = weno::dev::PairTile<12, 8>::TILE;
  const int64_t tiles = (n + t - 1) / t;
  return (tiles + 15) / 16 * 16 + (tiles * (t / 8) + 15) / 16 * 16;
}
int64_t redo_tiles_part(int64_t n) {
  constexpr int64_t t = weno::dev::PairTile<12, 8>::TILE;
  return ((n + t - 1) / t + 15) / 16 * 16;
}
int64_t redo_bytes(const S& s) {
  if (s.fp64 || s.nv != 4) return 0;
  return redo_part(s.nQ) + redo_part(s.nT);
}
// Grid of a fix-up pass over n cells: a block per kFixupChunk tiles of marks, at most 4 per SM.
unsigned fix_grid(const S& s, int64_t n) {
  constexpr int64_t t = weno::dev::PairTile<12, 8>::TILE;
  const int64_t chunks = ((n + t - 1) / t + weno::dev::kFixupChunk - 1) / weno::dev::kFixupChunk;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(chunks, 4 * s.nsm));
}

// Cell reconstruction into the Gauss-value array wg.  which: bit 0 = quad group,
// bit 1 = triangle group.
template <typename T, int NV, bool COMP, bool WALLS>
void launch_reconstruct_impl(S& s, const void* U, const void* Ulo, void* wg, cudaStream_t st, int which,
                             uint8_t* redo) {
  const T* u = static_cast<const T*>(U);
  const T* ul = static_cast<const T*>(Ulo);
  const T eps = (T)s.prm.eps, th = (T)s.prm.theta;
  if constexpr (NV == 4) {
    if (s.prm.characteristic) {
      const T gg = (T)s.prm.gas_gamma;
      if constexpr (COMP) {  // packed FP32C tables staged by TMA (setup_tma runs for every FP32C Euler solver)
        using CQ = weno::dev::PairTile<12, 8>;
        using CT = weno::dev::PairTile<9, 6>;
        // each pass is followed by its fix-up pass over the tiles it marked (a few us when none is)
        uint8_t* cells_q = redo + redo_tiles_part(s.nQ);
        uint8_t* redo_t = redo + redo_part(s.nQ);
        uint8_t* cells_t = redo_t + redo_tiles_part(s.nT);
        if (s.nQ && (which & 1)) {
          weno::dev::k_reconstruct_char_tma<12, 8, WALLS, false><<<tma_grid(s.k1q, s.nQ), CQ::THREADS, CQ::SMEM, st>>>(
              s.q_map_pgam, s.q_map_pdg, s.q_map_gop, u, ul, s.q_slot, (const float*)s.area, s.nQ, 0, 0,
              (float*)wg, eps, gg, s.prm.linear, redo, cells_q, s.err, s.debug_stall);
          weno::dev::k_reconstruct_char_tma<12, 8, WALLS, true><<<fix_grid(s, s.nQ), CQ::THREADS, CQ::SMEM, st>>>(
              s.q_map_pgam, s.q_map_pdg, s.q_map_gop, u, ul, s.q_slot, (const float*)s.area, s.nQ, 0, 0,
              (float*)wg, eps, gg, s.prm.linear, redo, cells_q, s.err, s.debug_stall);
        }
        if (s.nT && (which & 2)) {
          weno::dev::k_reconstruct_char_tma<9, 6, WALLS, false><<<tma_grid(s.k1t, s.nT), CT::THREADS, CT::SMEM, st>>>(
              s.t_map_pgam, s.t_map_pdg, s.t_map_gop, u, ul, s.t_slot, (const float*)s.area, s.nT, s.nQ,
              8 * s.nQ, (float*)wg, eps, gg, s.prm.linear, redo_t, cells_t, s.err, s.debug_stall);
          weno::dev::k_reconstruct_char_tma<9, 6, WALLS, true><<<fix_grid(s, s.nT), CT::THREADS, CT::SMEM, st>>>(
              s.t_map_pgam, s.t_map_pdg, s.t_map_gop, u, ul, s.t_slot, (const float*)s.area, s.nT, s.nQ,
              8 * s.nQ, (float*)wg, eps, gg, s.prm.linear, redo_t, cells_t, s.err, s.debug_stall);
        }
      } else {
        if (s.nQ && (which & 1))
          weno::dev::k_reconstruct_char<T, 12, 8, COMP, WALLS><<<grid_of(s.k1q, s.nQ * 4), s.k1q.block, 0, st>>>(
              u, ul, s.q_slot, (const T*)s.q_gop, (const T*)s.q_dg, (const T*)s.q_gam, (const T*)s.area, s.nQ, 0,
              0, (T*)wg, eps, th, gg, s.prm.linear);
        if (s.nT && (which & 2))
          weno::dev::k_reconstruct_char<T, 9, 6, COMP, WALLS><<<grid_of(s.k1t, s.nT * 4), s.k1t.block, 0, st>>>(
              u, ul, s.t_slot, (const T*)s.t_gop, (const T*)s.t_dg, (const T*)s.t_gam, (const T*)s.area, s.nT,
              s.nQ, 8 * s.nQ, (T*)wg, eps, th, gg, s.prm.linear);
      }
      return;
    }
  }
  if constexpr (COMP && NV == 4) {
    if (s.tma) {  // each pass is followed by its fix-up pass over the cells it marked
      using PQ = weno::dev::PairTile<12, 8>;
      using PT = weno::dev::PairTile<9, 6>;
      uint8_t* cells_q = redo + redo_tiles_part(s.nQ);
      uint8_t* redo_t = redo + redo_part(s.nQ);
      uint8_t* cells_t = redo_t + redo_tiles_part(s.nT);
      if (s.nQ && (which & 1)) {
        weno::dev::k_reconstruct_tma<12, 8, WALLS, false><<<tma_grid(s.k1q, s.nQ), PQ::THREADS, PQ::SMEM, st>>>(
            s.q_map_pgam, s.q_map_pdg, s.q_map_gop, u, ul, s.q_slot, (const float*)s.area, s.nQ, 0, 0, (float*)wg,
            eps, s.prm.linear, redo, cells_q, s.err, s.debug_stall);
        weno::dev::k_reconstruct_tma<12, 8, WALLS, true><<<fix_grid(s, s.nQ), PQ::THREADS, PQ::SMEM, st>>>(
            s.q_map_pgam, s.q_map_pdg, s.q_map_gop, u, ul, s.q_slot, (const float*)s.area, s.nQ, 0, 0, (float*)wg,
            eps, s.prm.linear, redo, cells_q, s.err, s.debug_stall);
      }
      if (s.nT && (which & 2)) {
        weno::dev::k_reconstruct_tma<9, 6, WALLS, false><<<tma_grid(s.k1t, s.nT), PT::THREADS, PT::SMEM, st>>>(
            s.t_map_pgam, s.t_map_pdg, s.t_map_gop, u, ul, s.t_slot, (const float*)s.area, s.nT, s.nQ, 8 * s.nQ,
            (float*)wg, eps, s.prm.linear, redo_t, cells_t, s.err, s.debug_stall);
        weno::dev::k_reconstruct_tma<9, 6, WALLS, true><<<fix_grid(s, s.nT), PT::THREADS, PT::SMEM, st>>>(
            s.t_map_pgam, s.t_map_pdg, s.t_map_gop, u, ul, s.t_slot, (const float*)s.area, s.nT, s.nQ, 8 * s.nQ,
            (float*)wg, eps, s.prm.linear, redo_t, cells_t, s.err, s.debug_stall);
      }
      return;
    }
  }
  if constexpr (COMP) {
    if (s.nQ && (which & 1))
      weno::dev::k_reconstruct_f32c<NV, 12, 8><<<grid_of(s.k1q, s.nQ * NV), s.k1q.block, 0, st>>>(
          u, ul, s.q_slot, (const float4*)s.q_gop, (const float4*)s.q_dg, (const float4*)s.q_gam,
          (const float2*)s.q_gam1, (const float*)s.area, s.nQ, s.q_pitch, 0, 0, (float*)wg, eps, s.prm.linear);
    if (s.nT && (which & 2))
      weno::dev::k_reconstruct_f32c<NV, 9, 6><<<grid_of(s.k1t, s.nT * NV), s.k1t.block, 0, st>>>(
          u, ul, s.t_slot, (const float4*)s.t_gop, (const float4*)s.t_dg, (const float4*)s.t_gam,
          (const float2*)s.t_gam1, (const float*)s.area, s.nT, s.t_pitch, s.nQ, 8 * s.nQ, (float*)wg, eps,
          s.prm.linear);
  } else {
    if (s.nQ && (which & 1))
      weno::dev::k_reconstruct<T, NV, 12, 8, COMP, WALLS><<<grid_of(s.k1q, s.nQ * NV), s.k1q.block, 0, st>>>(
          u, ul, s.q_slot, (const T*)s.q_gop, (const T*)s.q_dg, (const T*)s.q_gam, (const T*)s.area, s.nQ, 0, 0,
          (T*)wg, eps, th, s.prm.linear);
    if (s.nT && (which & 2))
      weno::dev::k_reconstruct<T, NV, 9, 6, COMP, WALLS><<<grid_of(s.k1t, s.nT * NV), s.k1t.block, 0, st>>>(
          u, ul, s.t_slot, (const T*)s.t_gop, (const T*)s.t_dg, (const T*)s.t_gam, (const T*)s.area, s.nT, s.nQ,
          8 * s.nQ, (T*)wg, eps, th, s.prm.linear);
  }
}

// Walls only change the stencil gathers (momentum flips of mirror images); meshes without
// walls run kernels without that code.
template <typename T, int NV, bool COMP>
void launch_reconstruct_into(S& s, const void* U, const void* Ulo, void* wg, cudaStream_t st, int which,
                             uint8_t* redo) {
  if constexpr (NV == 4) {
    if (s.walls) return launch_reconstruct_impl<T, NV, COMP, true>(s, U, Ulo, wg, st, which, redo);
  }
  launch_reconstruct_impl<T, NV, COMP, false>(s, U, Ulo, wg, st, which, redo);
}

template <typename T, int NV, bool COMP>
void launch_reconstruct(S& s, const void* U, const void* Ulo, cudaStream_t st, int which = 3) {
  launch_reconstruct_into<T, NV, COMP>(s, U, Ulo, s.Wg, st, which, s.fix_marks);
}

// Face fluxes of the Gauss values wg into fl; c places the stage in the step (time t + c dt).
template <typename T, int NV>
void launch_face_into(S& s, const void* wg, void* fl, double c, cudaStream_t st) {
  if (!s.nF) return;
  weno::dev::Prm<T> p{(T)s.prm.gas_gamma, (T)s.prm.adv[0], (T)s.prm.adv[1]};
  weno::dev::Inflow<T> in{};
  for (int v = 0; v < 4; ++v) {
    in.wa[v] = (T)s.in_wa[v];
    in.wb[v] = (T)s.in_wb[v];
  }
  in.xi = s.in_xi;
  in.t = s.t_dev;
  in.dt = s.dt_dev;
  in.speed = s.prm.inflow_line[3];
  in.c = c;
  if constexpr (NV == 4) {  // inflow faces exist for the Euler equations only
    if (s.n_in) {
      weno::dev::k_face<T, NV, true><<<grid_of(s.k2, s.nF), s.k2.block, 0, st>>>(
          (const T*)wg, s.gl, s.gr, (const T*)s.fnx, (const T*)s.fny, (const T*)s.flen, s.nF, (T*)fl, p, s.flag,
          s.inst, s.nQ, in);
      return;
    }
  }
  weno::dev::k_face<T, NV, false><<<grid_of(s.k2, s.nF), s.k2.block, 0, st>>>(
      (const T*)wg, s.gl, s.gr, (const T*)s.fnx, (const T*)s.fny, (const T*)s.flen, s.nF, (T*)fl, p, s.flag,
      s.inst, s.nQ, in);
}

template <typename T, int NV, bool COMP>
void launch_face(S& s, cudaStream_t st, double c = 0.0) {
  launch_face_into<T, NV>(s, s.Wg, s.F, c, st);
}

template <typename T, int NV, bool COMP, int MODE>
void launch_gather_mode(S& s, void* U, void* Ulo, void* R, cudaStream_t st, int which) {
  if (s.nQ && (which & 1))
    weno::dev::k_gather<T, NV, 4, COMP, MODE><<<grid_of(s.k3q, s.nQ), s.k3q.block, 0, st>>>(
        (const T*)s.F, s.q_cf, (const T*)s.inv_area, (const T*)s.inv_area_lo, s.nQ, 0, (T*)U, (T*)Ulo, (T*)s.Ws,
        (T*)s.Wslo, (T*)R,
        s.dt_dev, s.inst);
  if (s.nT && (which & 2))
    weno::dev::k_gather<T, NV, 3, COMP, MODE><<<grid_of(s.k3t, s.nT), s.k3t.block, 0, st>>>(
        (const T*)s.F, s.t_cf, (const T*)s.inv_area, (const T*)s.inv_area_lo, s.nT, s.nQ, (T*)U, (T*)Ulo, (T*)s.Ws,
        (T*)s.Wslo, (T*)R,
        s.dt_dev, s.inst);
}

template <typename T, int NV, bool COMP>
void launch_gather(S& s, int mode, void* U, void* Ulo, void* R, cudaStream_t st, int which = 3) {
  switch (mode) {
    case 0: launch_gather_mode<T, NV, COMP, 0>(s, U, Ulo, R, st, which); break;
    case 1: launch_gather_mode<T, NV, COMP, 1>(s, U, Ulo, R, st, which); break;
    case 2: launch_gather_mode<T, NV, COMP, 2>(s, U, Ulo, R, st, which); break;
    default: launch_gather_mode<T, NV, COMP, 3>(s, U, Ulo, R, st, which); break;
  }
}

template <typename T, int NV, bool COMP>
void launch_step_body(S& s, void* U, void* Ulo, cudaStream_t st) {
  // the stages of Section 4 evaluate L at t, t + dt, t + dt/2
  constexpr double kStageTime[3] = {0.0, 1.0, 0.5};
  for (int stage = 1; stage <= 3; ++stage) {
    const void* src = stage == 1 ? U : s.Ws;
    const void* srclo = stage == 1 ? Ulo : s.Wslo;
    launch_reconstruct<T, NV, COMP>(s, src, srclo, st);
    launch_face<T, NV, COMP>(s, st, kStageTime[stage - 1]);
    launch_gather<T, NV, COMP>(s, stage, U, Ulo, nullptr, st);
  }
  weno::dev::k_advance_time<<<(s.n_inst + 127) / 128, 128, 0, st>>>(s.t_dev, s.dt_dev, s.n_inst);
}

// one call per precision / variable count
#define WENO_DISPATCH(s, FN, ...)                                  \
  do {                                                             \
    if ((s).fp64) {                                                \
      if ((s).nv == 4) FN<double, 4, false>(__VA_ARGS__);          \
      else FN<double, 1, false>(__VA_ARGS__);                      \
    } else {                                                       \
      if ((s).nv == 4) FN<float, 4, true>(__VA_ARGS__);            \
      else FN<float, 1, true>(__VA_ARGS__);                        \
    }                                                              \
  } while (0)

template <typename T, int NV, bool COMP>
void launch_cell_dt(S& s, const void* U, const void* Ulo, cudaStream_t st) {
  const T* u = (const T*)U;
  const T* ul = (const T*)Ulo;
  if (s.nQ)
    weno::dev::k_cell_dt<T, NV, 4, COMP><<<(unsigned)((s.nQ + 255) / 256), 256, 0, st>>>(
        u, ul, s.q_cf, s.fnx64, s.fny64, s.flen64, s.area64, s.nQ, 0, s.prm.gas_gamma, s.prm.adv[0], s.prm.adv[1],
        s.cell_dt);
  if (s.nT)
    weno::dev::k_cell_dt<T, NV, 3, COMP><<<(unsigned)((s.nT + 255) / 256), 256, 0, st>>>(
        u, ul, s.t_cf, s.fnx64, s.fny64, s.flen64, s.area64, s.nT, s.nQ, s.prm.gas_gamma, s.prm.adv[0],
        s.prm.adv[1], s.cell_dt);
}

template <typename T, int NV, bool COMP>
void launch_reduce(S& s, const void* U, const void* Ulo, int mode, cudaStream_t st) {
  if (s.n_chunks)
    weno::dev::k_chunk_reduce<T, NV, COMP><<<(unsigned)s.n_chunks, 256, 0, st>>>(
        s.cell_dt, (const T*)U, (const T*)Ulo, s.area64, s.chunks, mode, s.partial);
  weno::dev::k_instance_reduce<NV><<<s.n_inst, 256, 0, st>>>(s.partial, s.chunk_off, mode, s.red);
}

int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(WENO_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return WENO_OK;
}

template <typename D>
int upload(S& s, D** dst, const std::vector<D>& src, cudaStream_t st) {
  int r = s.alloc(dst, src.size() * sizeof(D));
  if (r) return r;
  if (!src.empty()) CK(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(D), cudaMemcpyHostToDevice, st));
  return WENO_OK;
}

// Upload a double table in the solver's precision.
int upload_real(S& s, void** dst, const std::vector<double>& src, cudaStream_t st) {
  if (s.fp64) {
    double* d;
    int r = upload(s, &d, src, st);
    *dst = d;
    return r;
  }
  std::vector<float> f(src.size());
  for (size_t i = 0; i < src.size(); ++i) f[i] = (float)src[i];
  float* d;
  int r = upload(s, &d, f, st);
  if (r) return r;
  CK(cudaStreamSynchronize(st));  // f goes out of scope
  *dst = d;
  return WENO_OK;
}

// FP32C tables, rows of P >= N cells (padding zero, every row on a 256-byte boundary):
//   gop [j][q]        float4 D_j^+ entries
//   dg  [g][q]        float4 (x_G - c0, sigma+, sigma-)
//   gam [g][k][q]     float4 rows: gamma+_{4k..4k+3} for k < M/4, then gamma- rows
//   gam1 [g][q]       float2 (gamma+_8, gamma-_8) of triangles
// The splitting of Section 3.4 depends on the geometry only; it is evaluated
// here in FP64: gt+ = (gamma + theta|gamma|)/2, gt- = gt+ - gamma,
// sigma+- = sum gt+-, gamma+- = gt+- / sigma+-.  rows = false uploads gop only.
int upload_packed(S& s, const GroupTables& T, int64_t P, double theta, void** gop, void** dg, void** gam,
                  void** gam1, cudaStream_t st, bool rows = true) {
  const int64_t N = T.N;
  const int M = T.M, G = T.G, M4 = M / 4;
  std::vector<float> a((size_t)M * 4 * P, 0.f), b((size_t)G * 4 * P, 0.f), c((size_t)G * 2 * M4 * 4 * P, 0.f), e;
  if (M % 4) e.assign((size_t)G * 2 * P, 0.f);
  for (int j = 0; j < M; ++j)
    for (int64_t q = 0; q < N; ++q)
      for (int k = 0; k < 4; ++k) a[((size_t)j * P + q) * 4 + k] = (float)T.gop[((size_t)j * 4 + k) * N + q];
  std::vector<double> gp(M), gn(M);
  for (int g = 0; g < G; ++g) {
    for (int64_t q = 0; q < N; ++q) {
      double sp = 0.0, sm = 0.0;
      for (int j = 0; j < M; ++j) {
        const double x = T.gam[((size_t)g * M + j) * N + q];
        gp[j] = 0.5 * (x + theta * std::fabs(x));
        gn[j] = gp[j] - x;
        sp += gp[j];
        sm += gn[j];
      }
      float* d = &b[((size_t)g * P + q) * 4];
      d[0] = (float)T.dg[((size_t)g * 2 + 0) * N + q];
      d[1] = (float)T.dg[((size_t)g * 2 + 1) * N + q];
      d[2] = (float)sp;
      d[3] = (float)sm;
      for (int j = 0; j < 4 * M4; ++j) {
        c[(((size_t)g * 2 * M4 + j / 4) * P + q) * 4 + j % 4] = (float)(gp[j] / sp);
        c[(((size_t)g * 2 * M4 + M4 + j / 4) * P + q) * 4 + j % 4] = (float)(gn[j] / sm);
      }
      if (M % 4) {
        e[((size_t)g * P + q) * 2] = (float)(gp[M - 1] / sp);
        e[((size_t)g * P + q) * 2 + 1] = (float)(gn[M - 1] / sm);
      }
    }
  }
  float *pa, *pb = nullptr, *pc = nullptr, *pe = nullptr;
  int r;
  if ((r = upload(s, &pa, a, st))) return r;
  if (rows && (r = upload(s, &pb, b, st))) return r;
  if (rows && (r = upload(s, &pc, c, st))) return r;
  if (rows && M % 4 && (r = upload(s, &pe, e, st))) return r;
  CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
  *gop = pa;
  *dg = pb;
  *gam = pc;
  *gam1 = pe;
  return WENO_OK;
}

// Point-pair tables of the Euler FP32C reconstruction (k_reconstruct_tma), rows of P >= N cells
// of float4, the G Gauss points of a cell taken as G/2 pairs (points 2k, 2k+1 of face k):
//   gam [k][j][q]   (gamma+_j(2k), gamma+_j(2k+1), gamma-_j(2k), gamma-_j(2k+1))
//   dg  [2k][q]     (dx(2k), dx(2k+1), dy(2k), dy(2k+1)), (dx, dy) = x_G - c0
//   dg  [2k+1][q]   (sigma+(2k), sigma+(2k+1), sigma-(2k), sigma-(2k+1))
// with the splitting of Section 3.4 evaluated in FP64 as in upload_packed.
int upload_pairs(S& s, const GroupTables& T, int64_t P, double theta, void** gam, void** dg, cudaStream_t st) {
  const int64_t N = T.N;
  const int M = T.M, G = T.G;
  std::vector<float> a((size_t)(G / 2) * M * 4 * P, 0.f), b((size_t)G * 4 * P, 0.f);
  std::vector<double> gp(M), gn(M);
  for (int g = 0; g < G; ++g) {
    const int k = g / 2, h = g % 2;
    for (int64_t q = 0; q < N; ++q) {
      double sp = 0.0, sm = 0.0;
      for (int j = 0; j < M; ++j) {
        const double x = T.gam[((size_t)g * M + j) * N + q];
        gp[j] = 0.5 * (x + theta * std::fabs(x));
        gn[j] = gp[j] - x;
        sp += gp[j];
        sm += gn[j];
      }
      for (int j = 0; j < M; ++j) {
        float* r = &a[(((size_t)k * M + j) * P + q) * 4];
        r[h] = (float)(gp[j] / sp);
        r[2 + h] = (float)(gn[j] / sm);
      }
      float* d0 = &b[((size_t)(2 * k) * P + q) * 4];
      float* d1 = &b[((size_t)(2 * k + 1) * P + q) * 4];
      d0[h] = (float)T.dg[((size_t)g * 2 + 0) * N + q];
      d0[2 + h] = (float)T.dg[((size_t)g * 2 + 1) * N + q];
      d1[h] = (float)sp;
      d1[2 + h] = (float)sm;
    }
  }
  float *pa, *pb;
  int r;
  if ((r = upload(s, &pa, a, st))) return r;
  if ((r = upload(s, &pb, b, st))) return r;
  CK(cudaStreamSynchronize(st));  // the host vectors go out of scope
  *gam = pa;
  *dg = pb;
  return WENO_OK;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 2D float tensor map: `inner` floats per row, `rows` rows `pitch_bytes` apart, box of
// box_inner x box_rows; out-of-range elements of the last tile are filled with zeros.
int make_map_2d(EncodeTiled enc, CUtensorMap* map, void* base, uint64_t inner, uint64_t rows, uint64_t pitch_bytes,
                uint32_t box_inner, uint32_t box_rows) {
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {pitch_bytes};
  const cuuint32_t box[2] = {box_inner, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(WENO_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return WENO_OK;
}

// Tensor maps of the TMA reconstruction (Euler FP32C) and its shared-memory opt-in.
int setup_tma(S& s) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return fail(WENO_ECUDA, "cuTensorMapEncodeTiled unavailable");
  EncodeTiled enc = reinterpret_cast<EncodeTiled>(fn);
  using PQ = weno::dev::PairTile<12, 8>;
  using PT = weno::dev::PairTile<9, 6>;
  int r;
  // point-pair tables: gamma+- (G/2) * M float4 rows, offsets and sigma+- G float4 rows
  if (s.nQ) {
    if ((r = make_map_2d(enc, &s.q_map_pgam, s.q_pgam, 4 * s.q_pitch, 4 * 12, 16 * s.q_pitch, 4 * kTile, 4 * 12)))
      return r;
    if ((r = make_map_2d(enc, &s.q_map_pdg, s.q_pdg, 4 * s.q_pitch, 8, 16 * s.q_pitch, 4 * kTile, 8))) return r;
  }
  if (s.nT) {
    if ((r = make_map_2d(enc, &s.t_map_pgam, s.t_pgam, 4 * s.t_pitch, 3 * 9, 16 * s.t_pitch, 4 * kTile, 3 * 9)))
      return r;
    if ((r = make_map_2d(enc, &s.t_map_pdg, s.t_pdg, 4 * s.t_pitch, 6, 16 * s.t_pitch, 4 * kTile, 6))) return r;
  }
  for (auto fn : {weno::dev::k_reconstruct_tma<12, 8, false, false>, weno::dev::k_reconstruct_tma<12, 8, true, false>,
                  weno::dev::k_reconstruct_tma<12, 8, false, true>, weno::dev::k_reconstruct_tma<12, 8, true, true>})
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, PQ::SMEM));
  for (auto fn : {weno::dev::k_reconstruct_tma<9, 6, false, false>, weno::dev::k_reconstruct_tma<9, 6, true, false>,
                  weno::dev::k_reconstruct_tma<9, 6, false, true>, weno::dev::k_reconstruct_tma<9, 6, true, true>})
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, PT::SMEM));
  // D_j^+ rows: M float4 rows
  if (s.nQ && (r = make_map_2d(enc, &s.q_map_gop, s.q_gop, 4 * s.q_pitch, 12, 16 * s.q_pitch, 4 * kTile, 12)))
    return r;
  if (s.nT && (r = make_map_2d(enc, &s.t_map_gop, s.t_gop, 4 * s.t_pitch, 9, 16 * s.t_pitch, 4 * kTile, 9)))
    return r;
  if (s.prm.characteristic) {
    for (auto fn : {weno::dev::k_reconstruct_char_tma<12, 8, false, false>,
                    weno::dev::k_reconstruct_char_tma<12, 8, true, false>,
                    weno::dev::k_reconstruct_char_tma<12, 8, false, true>,
                    weno::dev::k_reconstruct_char_tma<12, 8, true, true>})
      CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, weno::dev::PairTile<12, 8>::SMEM));
    for (auto fn : {weno::dev::k_reconstruct_char_tma<9, 6, false, false>,
                    weno::dev::k_reconstruct_char_tma<9, 6, true, false>,
                    weno::dev::k_reconstruct_char_tma<9, 6, false, true>,
                    weno::dev::k_reconstruct_char_tma<9, 6, true, true>})
      CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, weno::dev::PairTile<9, 6>::SMEM));
  }
  s.tma = true;
  return WENO_OK;
}

int capture_step(S& s, void* U, void* Ulo);

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* weno_last_error(void) { return g_err.c_str(); }

void weno_params_default(weno_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eqn = WENO_EQN_EULER;
  p->precision = WENO_FP64;
  p->gas_gamma = 1.4;
  p->adv[0] = 1.0;
  p->adv[1] = 1.0;
  p->eps = 1e-3;
  p->theta = 3.0;
  p->rcond = 1e-12;
  p->optimize = 1;
  p->linear = 0;
  p->n_threads = 0;
}

int weno_mesh_create(const double* node_xy, int64_t n_nodes, const int64_t* cell_ptr, const int64_t* cell_nodes,
                     int64_t n_cells, const weno_mesh_opts* opts, weno_mesh_t* out) {
  if (!node_xy || !cell_ptr || !cell_nodes || !opts || !out) return fail(WENO_EINVAL, "null argument");
  if (opts->bc != WENO_BC_PERIODIC && opts->bc != WENO_BC_OUTFLOW) return fail(WENO_EINVAL, "unknown boundary kind");
  *out = nullptr;
  try {
    auto m = std::make_unique<weno_mesh_s>();
    std::string err;
    int r = weno::build_mesh(node_xy, n_nodes, cell_ptr, cell_nodes, n_cells, opts->bc, opts->origin, opts->extent,
                             opts->walls, opts->wall_from, opts->inflow, m->m, err);
    if (r) return fail(r, err);
    *out = m.release();
  } catch (const std::bad_alloc&) {
    return fail(WENO_ENOMEM, "host allocation failed while building the mesh");
  }
  return WENO_OK;
}

int weno_mesh_concat(const weno_mesh_t* meshes, int32_t n, weno_mesh_t* out) {
  if (!meshes || !out || n <= 0) return fail(WENO_EINVAL, "bad arguments to weno_mesh_concat");
  *out = nullptr;
  try {
    std::vector<const Mesh*> v(n);
    for (int i = 0; i < n; ++i) {
      if (!meshes[i]) return fail(WENO_EINVAL, "null mesh");
      v[i] = &meshes[i]->m;
    }
    auto m = std::make_unique<weno_mesh_s>();
    std::string err;
    int r = weno::concat_meshes(v.data(), n, m->m, err);
    if (r) return fail(r, err);
    *out = m.release();
  } catch (const std::bad_alloc&) {
    return fail(WENO_ENOMEM, "host allocation failed while joining meshes");
  }
  return WENO_OK;
}

int weno_mesh_get_info(weno_mesh_t mesh, weno_mesh_info* info) {
  if (!mesh || !info) return fail(WENO_EINVAL, "null argument");
  const Mesh& m = mesh->m;
  info->n_cells = m.n();
  info->n_quads = m.nQ;
  info->n_tris = m.nT;
  info->n_faces = m.nF;
  info->n_boundary = m.n_boundary;
  info->n_instances = m.n_inst;
  info->n_inflow = (int32_t)std::count(m.fin.begin(), m.fin.end(), (int8_t)1);
  return WENO_OK;
}

int weno_mesh_cell_permutation(weno_mesh_t mesh, int64_t* perm) {
  if (!mesh || !perm) return fail(WENO_EINVAL, "null argument");
  std::copy(mesh->m.perm.begin(), mesh->m.perm.end(), perm);
  return WENO_OK;
}

int weno_mesh_cell_instance(weno_mesh_t mesh, int32_t* instance) {
  if (!mesh || !instance) return fail(WENO_EINVAL, "null argument");
  std::copy(mesh->m.inst.begin(), mesh->m.inst.end(), instance);
  return WENO_OK;
}

int weno_mesh_weight_stats(weno_mesh_t mesh, const weno_params* params, double* max_raw, double* max_opt) {
  if (!mesh || !max_raw || !max_opt) return fail(WENO_EINVAL, "null argument");
  weno_params p;
  if (params) p = *params;
  else weno_params_default(&p);
  weno::LsqParams lp;
  lp.rcond = p.rcond > 0 ? p.rcond : 1e-12;
  lp.optimize = p.optimize != 0;
  lp.n_threads = p.n_threads;
  try {
    GroupTables tq, tt;
    std::string err;
    int r = weno::precompute_tables(mesh->m, lp, tq, tt, err);
    if (r) return fail(r, err);
    for (int64_t i = 0; i < tq.N; ++i) { max_raw[i] = tq.max_raw[i]; max_opt[i] = tq.max_opt[i]; }
    for (int64_t i = 0; i < tt.N; ++i) { max_raw[tq.N + i] = tt.max_raw[i]; max_opt[tq.N + i] = tt.max_opt[i]; }
  } catch (const std::bad_alloc&) {
    return fail(WENO_ENOMEM, "host allocation failed in the precompute");
  }
  return WENO_OK;
}

int weno_mesh_cell_tables(weno_mesh_t mesh, const weno_params* params, int64_t cell, int32_t* slot_cells,
                          double* grad_op, double* gauss_offset, double* gamma, int32_t* mg) {
  if (!mesh || !slot_cells || !grad_op || !gauss_offset || !gamma || !mg) return fail(WENO_EINVAL, "null argument");
  const Mesh& m = mesh->m;
  if (cell < 0 || cell >= m.n()) return fail(WENO_EINVAL, "cell out of range");
  weno_params p;
  if (params) p = *params;
  else weno_params_default(&p);
  const double rcond = p.rcond > 0 ? p.rcond : 1e-12;
  if (!mesh->tables || mesh->tables_rcond != rcond || mesh->tables_optimize != (p.optimize != 0)) {
    try {
      mesh->tables.reset();
      auto tab = std::make_shared<std::pair<GroupTables, GroupTables>>();
      weno::LsqParams lp;
      lp.rcond = rcond;
      lp.optimize = p.optimize != 0;
      lp.n_threads = p.n_threads;
      std::string err;
      int r = weno::precompute_tables(m, lp, tab->first, tab->second, err);
      if (r) return fail(r, err);
      mesh->tables = tab;
      mesh->tables_rcond = rcond;
      mesh->tables_optimize = p.optimize != 0;
    } catch (const std::bad_alloc&) {
      return fail(WENO_ENOMEM, "host allocation failed in the precompute");
    }
  }
  const bool quad = cell < m.nQ;
  const GroupTables& T = quad ? mesh->tables->first : mesh->tables->second;
  const int64_t q = quad ? cell : cell - m.nQ;
  const int64_t N = T.N;
  mg[0] = T.M;
  mg[1] = T.G;
  for (int j = 0; j < T.M; ++j) {
    slot_cells[j] = T.slot[(size_t)j * N + q] & weno::kSlotCell;
    for (int e = 0; e < 4; ++e) grad_op[j * 4 + e] = T.gop[(size_t)(j * 4 + e) * N + q];
  }
  for (int g = 0; g < T.G; ++g) {
    gauss_offset[2 * g] = T.dg[(size_t)(g * 2) * N + q];
    gauss_offset[2 * g + 1] = T.dg[(size_t)(g * 2 + 1) * N + q];
    for (int j = 0; j < T.M; ++j) gamma[g * T.M + j] = T.gam[(size_t)(g * T.M + j) * N + q];
  }
  return WENO_OK;
}

void weno_mesh_destroy(weno_mesh_t mesh) { delete mesh; }

int weno_solver_create(weno_mesh_t mesh, const weno_params* params, void* cuda_stream, weno_solver_t* out) {
  if (!mesh || !params || !out) return fail(WENO_EINVAL, "null argument");
  *out = nullptr;
  const weno_params& p = *params;
  if (p.eqn != WENO_EQN_SCALAR && p.eqn != WENO_EQN_EULER) return fail(WENO_EINVAL, "unknown equation");
  if (p.precision != WENO_FP64 && p.precision != WENO_FP32C) return fail(WENO_EINVAL, "unknown precision");
  // theta > 1 keeps sigma- = sum (theta |gamma| - gamma) / 2 > 0 (Section 3.4); at theta = 1 a Gauss
  // point whose linear weights are all >= 0 has sigma- = 0 and gamma- = 0 / 0
  if (!(p.eps > 0) || !(p.theta > 1) || (p.eqn == WENO_EQN_EULER && !(p.gas_gamma > 1)))
    return fail(WENO_EINVAL, "parameters out of range (eps > 0, theta > 1, gamma > 1)");
  // FP32 weights: alpha = gamma / (beta~ + eps)^2 <= 1 / eps^2 stays far inside the FP32 range
  if (p.precision == WENO_FP32C && !(p.eps >= 1e-15))
    return fail(WENO_EINVAL, "FP32C solvers need eps >= 1e-15 (FP32 range of the nonlinear weights); use FP64");
  if (p.characteristic && p.eqn != WENO_EQN_EULER)
    return fail(WENO_EINVAL, "characteristic variables are defined for the Euler equations only");
  const bool walls = std::any_of(mesh->m.fwall.begin(), mesh->m.fwall.end(), [](int8_t w) { return w >= 0; });
  if (walls && p.eqn != WENO_EQN_EULER) return fail(WENO_EINVAL, "reflective walls are defined for the Euler equations only");
  const int64_t n_in = std::count(mesh->m.fin.begin(), mesh->m.fin.end(), (int8_t)1);
  if (n_in && p.eqn != WENO_EQN_EULER) return fail(WENO_EINVAL, "inflow faces are defined for the Euler equations only");
  if (n_in && !(p.inflow_a[0] > 0 && p.inflow_a[3] > 0 && p.inflow_b[0] > 0 && p.inflow_b[3] > 0 &&
                std::isfinite(p.inflow_a[1] + p.inflow_a[2] + p.inflow_b[1] + p.inflow_b[2]) &&
                std::isfinite(p.inflow_line[0] + p.inflow_line[1] + p.inflow_line[2] + p.inflow_line[3])))
    return fail(WENO_EINVAL, "inflow faces need both prescribed states with rho > 0, p > 0 and a finite line");
  const Mesh& m = mesh->m;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::unique_ptr<S> s;
  try {
    s.reset(new S());
  } catch (const std::bad_alloc&) {
    return fail(WENO_ENOMEM, "host allocation failed");
  }
  CK(cudaGetDevice(&s->dev));
  CK(cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev));
  s->prm = p;
  s->walls = walls;
  s->n_in = n_in;
  if (!(s->prm.rcond > 0)) s->prm.rcond = 1e-12;
  s->nv = p.eqn == WENO_EQN_EULER ? 4 : 1;
  s->fp64 = p.precision == WENO_FP64;
  s->esz = s->fp64 ? 8 : 4;
  s->nQ = m.nQ;
  s->nT = m.nT;
  s->N = m.n();
  s->nF = m.nF;
  s->n_boundary = m.n_boundary;
  s->n_inst = m.n_inst;
  // precompute on the host (FP64), shared by solvers of the same mesh and weight options
  if (!mesh->tables || mesh->tables_rcond != s->prm.rcond || mesh->tables_optimize != (p.optimize != 0)) {
    try {
      mesh->tables.reset();
      auto tab = std::make_shared<std::pair<GroupTables, GroupTables>>();
      weno::LsqParams lp;
      lp.rcond = s->prm.rcond;
      lp.optimize = p.optimize != 0;
      lp.n_threads = p.n_threads;
      std::string err;
      int r = weno::precompute_tables(m, lp, tab->first, tab->second, err);
      if (r) return fail(r, err);
      mesh->tables = tab;
      mesh->tables_rcond = s->prm.rcond;
      mesh->tables_optimize = p.optimize != 0;
    } catch (const std::bad_alloc&) {
      return fail(WENO_ENOMEM, "host allocation failed in the precompute");
    }
  }
  const GroupTables& tq = mesh->tables->first;
  const GroupTables& tt = mesh->tables->second;
  S& d = *s;
  int r;
  if ((r = upload(d, &d.q_slot, tq.slot, st))) return r;
  if ((r = upload(d, &d.t_slot, tt.slot, st))) return r;
  if (d.fp64) {
    if ((r = upload_real(d, &d.q_gop, tq.gop, st))) return r;
    if ((r = upload_real(d, &d.q_dg, tq.dg, st))) return r;
    if ((r = upload_real(d, &d.q_gam, tq.gam, st))) return r;
    if ((r = upload_real(d, &d.t_gop, tt.gop, st))) return r;
    if ((r = upload_real(d, &d.t_dg, tt.dg, st))) return r;
    if ((r = upload_real(d, &d.t_gam, tt.gam, st))) return r;
  } else {
    d.q_pitch = (d.nQ + 63) / 64 * 64;
    d.t_pitch = (d.nT + 63) / 64 * 64;
    // the split-weight rows of upload_packed serve the scalar kernel; both Euler kernels
    // (component-wise and characteristic) read the point-pair tables
    const bool rows = d.nv != 4;
    if ((r = upload_packed(d, tq, d.q_pitch, p.theta, &d.q_gop, &d.q_dg, &d.q_gam, &d.q_gam1, st, rows))) return r;
    if ((r = upload_packed(d, tt, d.t_pitch, p.theta, &d.t_gop, &d.t_dg, &d.t_gam, &d.t_gam1, st, rows))) return r;
    if (d.nv == 4) {
      if ((r = upload_pairs(d, tq, d.q_pitch, p.theta, &d.q_pgam, &d.q_pdg, st))) return r;
      if ((r = upload_pairs(d, tt, d.t_pitch, p.theta, &d.t_pgam, &d.t_pdg, st))) return r;
    }
  }
  {
    std::vector<double> inv(d.N);
    for (int64_t c = 0; c < d.N; ++c) inv[c] = 1.0 / m.area[c];
    if ((r = upload_real(d, &d.area, m.area, st))) return r;
    if ((r = upload_real(d, &d.inv_area, inv, st))) return r;
    // FP32C: the rounding remainder of 1/|Omega| (double-float reciprocal)
    std::vector<double> inv_lo(d.N, 0.0);
    if (!d.fp64)
      for (int64_t c = 0; c < d.N; ++c) inv_lo[c] = inv[c] - (double)(float)inv[c];
    if ((r = upload_real(d, &d.inv_area_lo, inv_lo, st))) return r;
    if ((r = upload(d, &d.area64, m.area, st))) return r;
    CK(cudaStreamSynchronize(st));
  }
  {
    // cell -> face lists with orientation (f: cell is L, ~f: cell is R)
    std::vector<int32_t> cq((size_t)4 * d.nQ), ct((size_t)3 * d.nT);
    for (int64_t c = 0; c < d.N; ++c) {
      const int nf = m.nvert[c];
      for (int k = 0; k < nf; ++k) {
        const int32_t f = m.cell_face[c * 4 + k];
        const bool left = m.fL[f] == (int32_t)c && m.fkL[f] == k;
        const int32_t e = left ? f : ~f;
        if (c < d.nQ) cq[(size_t)k * d.nQ + c] = e;
        else ct[(size_t)k * d.nT + (c - d.nQ)] = e;
      }
    }
    if ((r = upload(d, &d.q_cf, cq, st))) return r;
    if ((r = upload(d, &d.t_cf, ct, st))) return r;
    std::vector<int32_t> gl(d.nF), gr(d.nF);
    auto gbase = [&](int64_t c) -> int64_t { return c < d.nQ ? 8 * c : 8 * d.nQ + 6 * (c - d.nQ); };
    for (int64_t f = 0; f < d.nF; ++f) {
      gl[f] = (int32_t)(gbase(m.fL[f]) + 2 * m.fkL[f]);
      gr[f] = m.fR[f] >= 0 ? (int32_t)(gbase(m.fR[f]) + 2 * m.fkR[f]) : (m.fwall[f] >= 0 ? -2 : -1);
    }
    // inflow faces: gr = -3 - q, and n . x_G - c0 of their two Gauss points (edge k of the
    // L cell: point 0 near node k, point 1 near node k + 1, Eq. 5)
    std::vector<double> xi;
    const double ga = (3.0 + std::sqrt(3.0)) / 6.0, gb = (3.0 - std::sqrt(3.0)) / 6.0;
    const double* ln = p.inflow_line;
    for (int64_t f = 0; f < d.nF; ++f) {
      if (!m.fin[f]) continue;
      gr[f] = (int32_t)(-3 - (int64_t)xi.size() / 2);
      const int64_t c = m.fL[f];
      const int k = m.fkL[f], k1 = (k + 1) % m.nvert[c];
      const double* v = &m.verts[(size_t)c * 8];
      for (int q = 0; q < 2; ++q) {
        const double wa = q == 0 ? ga : gb, wb = q == 0 ? gb : ga;
        const double x = wa * v[2 * k] + wb * v[2 * k1], y = wa * v[2 * k + 1] + wb * v[2 * k1 + 1];
        xi.push_back(ln[0] * x + ln[1] * y - ln[2]);
      }
    }
    if (d.n_in) {
      if ((r = upload(d, &d.in_xi, xi, st))) return r;
      auto cons = [&](const double* q, double* w) {
        w[0] = q[0];
        w[1] = q[0] * q[1];
        w[2] = q[0] * q[2];
        w[3] = q[3] / (p.gas_gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2]);
      };
      cons(p.inflow_a, d.in_wa);
      cons(p.inflow_b, d.in_wb);
    }
    if ((r = upload(d, &d.gl, gl, st))) return r;
    if ((r = upload(d, &d.gr, gr, st))) return r;
    if ((r = upload_real(d, &d.fnx, m.fnx, st))) return r;
    if ((r = upload_real(d, &d.fny, m.fny, st))) return r;
    if ((r = upload_real(d, &d.flen, m.flen, st))) return r;
    if ((r = upload(d, &d.fnx64, m.fnx, st))) return r;
    if ((r = upload(d, &d.fny64, m.fny, st))) return r;
    if ((r = upload(d, &d.flen64, m.flen, st))) return r;
    // instance ranges (quads, triangles) and per-cell instance ids
    std::vector<int64_t> ranges((size_t)4 * d.n_inst, 0);
    for (int i = 0; i < d.n_inst; ++i) { ranges[4 * i] = ranges[4 * i + 1] = -1; ranges[4 * i + 2] = ranges[4 * i + 3] = -1; }
    for (int64_t c = 0; c < d.N; ++c) {
      const int i = m.inst[c];
      const int part = c < d.nQ ? 0 : 2;
      if (ranges[4 * i + part] < 0) ranges[4 * i + part] = c;
      ranges[4 * i + part + 1] = c + 1;
    }
    for (auto& x : ranges) if (x < 0) x = 0;
    // fixed partition of each instance's quad and triangle ranges into chunks (deterministic reductions)
    constexpr int64_t kChunk = 8192;
    std::vector<int64_t> chunks, chunk_off(1, 0);
    for (int i = 0; i < d.n_inst; ++i) {
      for (int part = 0; part < 2; ++part)
        for (int64_t c = ranges[4 * i + 2 * part]; c < ranges[4 * i + 2 * part + 1]; c += kChunk) {
          chunks.push_back(c);
          chunks.push_back(std::min(c + kChunk, ranges[4 * i + 2 * part + 1]));
        }
      chunk_off.push_back((int64_t)chunks.size() / 2);
    }
    d.n_chunks = (int64_t)chunks.size() / 2;
    if ((r = upload(d, &d.chunks, chunks, st))) return r;
    if ((r = upload(d, &d.chunk_off, chunk_off, st))) return r;
    if ((r = d.alloc(&d.partial, sizeof(double) * std::max<int64_t>(1, d.n_chunks) * d.nv))) return r;
    if (d.n_inst > 1) {
      if ((r = upload(d, &d.inst, m.inst, st))) return r;
    }
    CK(cudaStreamSynchronize(st));
  }
  // scratch
  const int64_t ngauss = 8 * d.nQ + 6 * d.nT;
  if ((r = d.alloc(&d.Wg, (size_t)ngauss * d.nv * d.esz))) return r;
  if ((r = d.alloc(&d.F, (size_t)d.nF * d.nv * d.esz))) return r;
  if ((r = d.alloc(&d.Ws, (size_t)d.N * d.nv * d.esz))) return r;
  if (!d.fp64 && (r = d.alloc(&d.Wslo, (size_t)d.N * d.nv * d.esz))) return r;
  if ((r = d.alloc(&d.dt_dev, sizeof(double) * d.n_inst))) return r;
  if ((r = d.alloc(&d.t_dev, sizeof(double) * d.n_inst))) return r;
  CK(cudaMemsetAsync(d.t_dev, 0, sizeof(double) * d.n_inst, st));
  CK(cudaMemsetAsync(d.dt_dev, 0, sizeof(double) * d.n_inst, st));
  if ((r = d.alloc(&d.red, sizeof(double) * d.n_inst * d.nv))) return r;
  if ((r = d.alloc(&d.cell_dt, sizeof(double) * d.N))) return r;
  if ((r = d.alloc(&d.flag, sizeof(int) * d.n_inst))) return r;
  CK(cudaMemsetAsync(d.flag, 0, sizeof(int) * d.n_inst, st));
  if ((r = d.alloc(&d.err, sizeof(int)))) return r;
  CK(cudaMemsetAsync(d.err, 0, sizeof(int), st));
  if (redo_bytes(d) && (r = d.alloc(&d.fix_marks, (size_t)redo_bytes(d)))) return r;
  if (!d.fp64 && d.nv == 4 && (r = setup_tma(d))) return r;
  CK(cudaStreamCreateWithFlags(&d.cap, cudaStreamNonBlocking));
  CK(cudaStreamSynchronize(st));
  *out = s.release();
  return WENO_OK;
}

int weno_solver_get_info(weno_solver_t s, weno_mesh_info* info) {
  if (!s || !info) return fail(WENO_EINVAL, "null argument");
  info->n_cells = s->N;
  info->n_quads = s->nQ;
  info->n_tris = s->nT;
  info->n_faces = s->nF;
  info->n_boundary = s->n_boundary;
  info->n_instances = s->n_inst;
  info->n_inflow = (int32_t)s->n_in;
  return WENO_OK;
}

int weno_residual(weno_solver_t s, const void* U, const void* U_lo, void* R, void* cuda_stream) {
  if (!s || !U || !R || (!s->fp64 && !U_lo)) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  WENO_DISPATCH(*s, launch_reconstruct, *s, U, U_lo, st);
  WENO_DISPATCH(*s, launch_face, *s, st);
  WENO_DISPATCH(*s, launch_gather, *s, 0, const_cast<void*>(U), const_cast<void*>(U_lo), R, st);
  return check_launch();
}

int weno_pass(weno_solver_t s, int32_t pass, const void* U, const void* U_lo, void* cuda_stream) {
  if (!s || (pass == 1 && (!U || (!s->fp64 && !U_lo)))) return fail(WENO_EINVAL, "null argument");
  if (pass < 1 || pass > 3) return fail(WENO_EINVAL, "pass must be 1, 2 or 3");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (pass == 1) WENO_DISPATCH(*s, launch_reconstruct, *s, U, U_lo, st);
  else if (pass == 2) WENO_DISPATCH(*s, launch_face, *s, st);
  else WENO_DISPATCH(*s, launch_gather, *s, 0, nullptr, nullptr, s->Ws, st);
  return check_launch();
}

int weno_step_instances(weno_solver_t s, void* U, void* U_lo, const double* dt_dev, void* cuda_stream) {
  if (!s || !U || !dt_dev || (!s->fp64 && !U_lo)) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (dt_dev != s->dt_dev)
    CK(cudaMemcpyAsync(s->dt_dev, dt_dev, sizeof(double) * s->n_inst, cudaMemcpyDeviceToDevice, st));
  cudaGraphExec_t exec = nullptr;
  for (auto& x : s->graphs)
    if (x.U == U && x.Ulo == U_lo) exec = x.exec;
  if (!exec) {
    int r = capture_step(*s, U, U_lo);
    if (r) return r;
    exec = s->graphs.back().exec;
  }
  CK(cudaGraphLaunch(exec, st));
  return WENO_OK;
}

int weno_set_time(weno_solver_t s, double t, void* cuda_stream) {
  if (!s || !std::isfinite(t)) return fail(WENO_EINVAL, "null solver or non-finite time");
  DeviceGuard g(s->dev);
  weno::dev::k_fill<<<(s->n_inst + 127) / 128, 128, 0, (cudaStream_t)cuda_stream>>>(s->t_dev, t, s->n_inst);
  CK(cudaGetLastError());
  return WENO_OK;
}

int weno_get_time(weno_solver_t s, double* t_out, void* cuda_stream) {
  if (!s || !t_out) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(cudaMemcpyAsync(t_out, s->t_dev, sizeof(double) * s->n_inst, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return WENO_OK;
}

int weno_step(weno_solver_t s, void* U, void* U_lo, double dt, void* cuda_stream) {
  if (!s || !U || (!s->fp64 && !U_lo)) return fail(WENO_EINVAL, "null argument");
  if (!(dt >= 0)) return fail(WENO_EINVAL, "dt must be >= 0");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  weno::dev::k_fill<<<(s->n_inst + 127) / 128, 128, 0, st>>>(s->dt_dev, dt, s->n_inst);
  int r = check_launch();
  if (r) return r;
  return weno_step_instances(s, U, U_lo, s->dt_dev, cuda_stream);
}

int weno_max_dt(weno_solver_t s, const void* U, const void* U_lo, double cfl, double* dt_out, void* cuda_stream) {
  if (!s || !U || !dt_out || (!s->fp64 && !U_lo)) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  WENO_DISPATCH(*s, launch_cell_dt, *s, U, U_lo, st);
  WENO_DISPATCH(*s, launch_reduce, *s, U, U_lo, 0, st);
  int r = check_launch();
  if (r) return r;
  std::vector<double> h(s->n_inst);
  CK(cudaMemcpyAsync(h.data(), s->red, sizeof(double) * s->n_inst, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < s->n_inst; ++i) dt_out[i] = cfl * h[i];
  return WENO_OK;
}

int weno_conservation(weno_solver_t s, const void* U, const void* U_lo, double* sums, void* cuda_stream) {
  if (!s || !U || !sums || (!s->fp64 && !U_lo)) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  WENO_DISPATCH(*s, launch_reduce, *s, U, U_lo, 1, st);
  int r = check_launch();
  if (r) return r;
  CK(cudaMemcpyAsync(sums, s->red, sizeof(double) * s->n_inst * s->nv, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return WENO_OK;
}

int weno_check(weno_solver_t s, void* cuda_stream) {
  if (!s) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<int> h(s->n_inst, 0);
  int t = 0;
  CK(cudaMemcpyAsync(h.data(), s->flag, sizeof(int) * s->n_inst, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&t, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemsetAsync(s->flag, 0, sizeof(int) * s->n_inst, st));
  CK(cudaMemsetAsync(s->err, 0, sizeof(int), st));
  CK(cudaStreamSynchronize(st));
  if (t) return fail(WENO_ETIMEOUT, "a bounded wait for a tensor-memory copy gave up; results of that launch are invalid");
  int bad = 0;
  for (int i = 0; i < s->n_inst; ++i) bad += h[i] != 0;
  if (bad)
    return fail(WENO_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or non-finite) at a Gauss point in " +
                                   std::to_string(bad) + " of " + std::to_string(s->n_inst) + " instance(s)");
  return WENO_OK;
}

int weno_check_instances(weno_solver_t s, int32_t* flags, void* cuda_stream) {
  if (!s || !flags) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int t = 0;
  CK(cudaMemcpyAsync(flags, s->flag, sizeof(int) * s->n_inst, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&t, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemsetAsync(s->flag, 0, sizeof(int) * s->n_inst, st));
  CK(cudaMemsetAsync(s->err, 0, sizeof(int), st));
  CK(cudaStreamSynchronize(st));
  if (t) return fail(WENO_ETIMEOUT, "a bounded wait for a tensor-memory copy gave up; results of that launch are invalid");
  return WENO_OK;
}

int weno_solver_launch_config(weno_solver_t s, int32_t* cfg) {
  if (!s || !cfg) return fail(WENO_EINVAL, "null argument");
  cfg[0] = s->k1q.block; cfg[1] = s->k1q.grid;
  cfg[2] = s->k2.block;  cfg[3] = s->k2.grid;
  cfg[4] = s->k3q.block; cfg[5] = s->k3q.grid;
  return WENO_OK;
}

int weno_solver_debug_stall(weno_solver_t s, int32_t on) {
  if (!s) return fail(WENO_EINVAL, "null argument");
  if (!s->tma) return fail(WENO_EINVAL, "this solver's kernels have no bounded waits (FP32C Euler only)");
  s->debug_stall = on != 0;
  s->drop_graphs();
  return WENO_OK;
}

int weno_autotune(weno_solver_t s, const void* U, const void* U_lo, void* cuda_stream) {
  if (!s || !U || (!s->fp64 && !U_lo)) return fail(WENO_EINVAL, "null argument");
  DeviceGuard g(s->dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int blocks[3] = {64, 128, 256};
  // grid candidates: one item per thread, or 1, 2, 4 resident waves of a persistent grid
  const int waves[4] = {0, 1, 2, 4};
  std::vector<Launch> generic, tma;
  for (int b : blocks)
    for (int w : waves) generic.push_back(Launch{b, w == 0 ? 0 : w * s->nsm * std::max(1, 2048 / b)});
  // TMA reconstruction: TILE x 4 threads; 1-4 blocks of 256 threads per SM (persistent), or one block per tile
  for (int w : {0, 1, 2, 3, 4}) tma.push_back(Launch{weno::dev::PairTile<12, 8>::THREADS, w * s->nsm * (64 / kTile)});
  auto tune = [&](Launch& L, auto run, const std::vector<Launch>& cands) -> int {
    float best = 1e30f;
    Launch bestL = L;
    for (const Launch& c : cands) {
      {
        L = c;
        run();
        float tmin = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, st);
          run();
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          tmin = std::min(tmin, ms);
        }
        if (cudaGetLastError() != cudaSuccess) continue;  // configuration not launchable
        if (tmin < best) { best = tmin; bestL = c; }
      }
    }
    L = bestL;
    return WENO_OK;
  };
  S& d = *s;
  void* u = const_cast<void*>(U);
  void* ul = const_cast<void*>(U_lo);
  const std::vector<Launch>& k1c = d.tma ? tma : generic;
  if (d.nQ) tune(d.k1q, [&] { WENO_DISPATCH(d, launch_reconstruct, d, U, U_lo, st, 1); }, k1c);
  if (d.nT) tune(d.k1t, [&] { WENO_DISPATCH(d, launch_reconstruct, d, U, U_lo, st, 2); }, k1c);
  tune(d.k2, [&] { WENO_DISPATCH(d, launch_face, d, st); }, generic);
  if (d.nQ) tune(d.k3q, [&] { WENO_DISPATCH(d, launch_gather, d, 0, u, ul, d.Ws, st, 1); }, generic);
  if (d.nT) tune(d.k3t, [&] { WENO_DISPATCH(d, launch_gather, d, 0, u, ul, d.Ws, st, 2); }, generic);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  d.drop_graphs();
  return WENO_OK;
}

void weno_solver_destroy(weno_solver_t s) { delete s; }

}  // extern "C"

namespace {

int capture_step(S& s, void* U, void* Ulo) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(s.cap, cudaStreamCaptureModeThreadLocal));
  WENO_DISPATCH(s, launch_step_body, s, U, Ulo, s.cap);
  cudaError_t le = cudaGetLastError();
  cudaError_t ce = cudaStreamEndCapture(s.cap, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(WENO_ECUDA, std::string("kernel launch in capture: ") + cudaGetErrorString(le));
  }
  if (ce != cudaSuccess) return fail(WENO_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(WENO_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
  if (s.graphs.size() >= 8) {
    cudaGraphExecDestroy(s.graphs.front().exec);
    s.graphs.erase(s.graphs.begin());
  }
  s.graphs.push_back({U, Ulo, exec});
  return WENO_OK;
}

}  // namespace

// ===========================================================================
// Residual whose scratch lives in a fixed array compiled into the library.
//
// For callers that may not allocate device memory once they are running:
// code that works inside a fixed device-memory budget handed out at start-up
// (for example when another component's memory pool owns the rest of the
// GPU), or whose per-step loop is not allowed to make allocation calls.
// weno_residual keeps its Gauss-point values and face fluxes in buffers the
// solver allocated; weno_residual_static puts them in g_static_scratch
// instead and allocates nothing.
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB, held by every GPU that loads the library
constexpr int kMaxStaticDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_base[kMaxStaticDevices] = {};

// Device address of g_static_scratch on the current device (looked up once
// per device; the host-side symbol itself is not a device address).
int static_scratch_base(int dev, void** base) {
  if (dev < 0 || dev >= kMaxStaticDevices) return fail(WENO_EINVAL, "device index out of range for the static scratch");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(WENO_ECUDA, std::string("cudaGetSymbolAddress(g_static_scratch): ") + cudaGetErrorString(e));
    g_static_base[dev] = p;
  }
  *base = g_static_base[dev];
  return WENO_OK;
}

template <typename T, int NV, bool COMP>
void launch_residual_static(S& s, const void* U, const void* Ulo, void* R, void* wg, void* fl, uint8_t* redo,
                            cudaStream_t st) {
  launch_reconstruct_into<T, NV, COMP>(s, U, Ulo, wg, st, 3, redo);
  launch_face_into<T, NV>(s, wg, fl, 0.0, st);
  if (s.nQ)
    weno::dev::k_gather<T, NV, 4, COMP, 0><<<grid_of(s.k3q, s.nQ), s.k3q.block, 0, st>>>(
        (const T*)fl, s.q_cf, (const T*)s.inv_area, (const T*)s.inv_area_lo, s.nQ, 0, nullptr, nullptr, nullptr,
        nullptr, (T*)R, s.dt_dev, s.inst);
  if (s.nT)
    weno::dev::k_gather<T, NV, 3, COMP, 0><<<grid_of(s.k3t, s.nT), s.k3t.block, 0, st>>>(
        (const T*)fl, s.t_cf, (const T*)s.inv_area, (const T*)s.inv_area_lo, s.nT, s.nQ, nullptr, nullptr, nullptr,
        nullptr, (T*)R, s.dt_dev, s.inst);
}

}  // namespace

extern "C" int weno_residual_static(weno_solver_t s, const void* U, const void* U_lo, void* R, void* cuda_stream) {
  if (!s || !U || !R || (!s->fp64 && !U_lo)) return fail(WENO_EINVAL, "null argument");
  // Gauss-point values first, face fluxes after them on a 256-byte boundary, then (FP32C Euler
  // solvers) the reconstruction's fix-up marks, a byte per tile and a bit per cell
  const size_t wg_bytes = (size_t)(8 * s->nQ + 6 * s->nT) * s->nv * s->esz;
  const size_t f_off = (wg_bytes + 255) / 256 * 256;
  const size_t r_off = (f_off + (size_t)s->nF * s->nv * s->esz + 255) / 256 * 256;
  const size_t need = r_off + (size_t)redo_bytes(*s);
  if (need > kStaticScratchBytes)
    return fail(WENO_EINVAL, "mesh too large for weno_residual_static: needs " + std::to_string(need) +
                                 " bytes of scratch, the fixed array holds " + std::to_string(kStaticScratchBytes));
  DeviceGuard g(s->dev);
  void* base = nullptr;
  int r = static_scratch_base(s->dev, &base);
  if (r) return r;
  unsigned char* b = static_cast<unsigned char*>(base);
  WENO_DISPATCH(*s, launch_residual_static, *s, U, U_lo, R, b, b + f_off, b + r_off, (cudaStream_t)cuda_stream);
  return check_launch();
}
