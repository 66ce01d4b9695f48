/*
 * weno3.h - C ABI of the GB300 library for the third-order WENO finite-volume
 * residual on unstructured quadrilateral / triangular / mixed meshes
 * (Zhao, Pan, Wang: "Weighted essentially non-oscillatory scheme on
 * unstructured quadrilateral and triangular meshes for hyperbolic
 * conservation laws", arXiv 1712.08317).
 *
 * The calls follow the paper's statement of the problem:
 *   u_t + div F(u) = 0 on a polygon mesh (Section 2, Eq. 1 for Euler; scalar
 *   linear advection as the scalar case), semi-discrete FV form
 *   dW_i/dt = L(W) (Eq. 4), edge integrals by 2-point Gauss quadrature (Eq. 5),
 *   third-order TVD Runge-Kutta in time (Section 4).
 *
 *   weno_mesh_create   nodes + cells -> faces, stencils (Sections 3.1, 3.2)
 *   weno_solver_create mesh + params -> least-squares reconstruction tables
 *                      and optimised linear weights (Sections 3.1-3.3), FP64,
 *                      uploaded to the GPU in the solver's precision
 *   weno_residual      R = L(U) (Eq. 4 with the WENO values of Section 3.4)
 *   weno_step          one SSP-RK3 step in place (Section 4)
 *
 * Conventions shared by every call:
 *  - Every call returns a weno_status (0 = WENO_OK); nothing aborts or traps.
 *    weno_last_error() gives a thread-local message for the last failure.
 *  - Host arrays passed in are read during the call and never retained.
 *  - The library owns its meshes, solvers, device tables and scratch memory;
 *    the caller owns the state arrays U / U_lo / R (device memory).
 *  - State layout: cell-major, U[cell * n_v + v] for the internal cell order
 *    (weno_mesh_cell_permutation maps internal -> input ids). n_v = 1 for
 *    scalar advection, 4 for Euler with W = (rho, rho u, rho v, rho E).
 *    FP64 solvers take double arrays.  FP32C solvers take float U (the
 *    rounded state) plus float U_lo (its compensation; U + U_lo is the
 *    state), and produce a float residual.
 *  - cuda_stream arguments are cudaStream_t values passed as void*
 *    (NULL = legacy default stream).  Calls are stream-ordered and
 *    asynchronous unless documented as synchronising.
 */
#ifndef WENO3_H
#define WENO3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct weno_mesh_s* weno_mesh_t;
typedef struct weno_solver_s* weno_solver_t;

typedef enum {
  WENO_OK = 0,
  WENO_EINVAL = -1,    /* bad argument (null pointer, out-of-range value)           */
  WENO_EMESH = -2,     /* cell with != 3/4 nodes, zero-area, non-convex, non-manifold */
  WENO_EPERIODIC = -3, /* a periodic boundary face without a translated partner     */
  WENO_ENOMEM = -4,    /* host or device allocation failed                          */
  WENO_ECUDA = -5,     /* a CUDA runtime call failed (message in weno_last_error)   */
  WENO_ENONPHYS = -6,  /* rho <= 0, p <= 0 or a non-finite value seen at a Gauss point */
  WENO_ETIMEOUT = -7   /* a bounded device wait (FP32C Euler reconstruction: the copy of
                          a tile's weight tables into shared memory) gave up; results of
                          the launches since the last check are invalid                */
} weno_status;

typedef enum { WENO_BC_PERIODIC = 0, WENO_BC_OUTFLOW = 1 } weno_bc_kind;
typedef enum { WENO_EQN_SCALAR = 0, WENO_EQN_EULER = 1 } weno_eqn_kind;
typedef enum { WENO_FP64 = 0, WENO_FP32C = 1 } weno_precision;

/* Boundary description of one mesh instance.  A zero-initialised struct is a
 * periodic box with no walls and no inflow sides; set bc, origin and extent. */
typedef struct {
  int32_t bc;        /* weno_bc_kind: periodic in x and y, or outflow on every boundary face */
  double origin[2];  /* box origin: periodic box, or the sides named by `walls`              */
  double extent[2];  /* box size: the periods, or the sides named by `walls`                 */
  int32_t walls;     /* outflow meshes, Euler: bit s set = box side s is a reflective wall
                        (0: x = origin[0], 1: x = origin[0] + extent[0], 2: y = origin[1],
                        3: y = origin[1] + extent[1]); a boundary face with both ends on such
                        a side sees, outside, the inner state with its normal momentum
                        reversed, and the mirror images across it in the stencils (Sections
                        3.1, 3.2) carry the mirrored cell's average with that momentum
                        component reversed.  0 = every boundary face is outflow.            */
  double wall_from[4]; /* per side s: the wall covers only the faces whose midpoint lies at
                        least wall_from[s] along the side from the origin corner (y - origin[1]
                        on sides 0, 1; x - origin[0] on sides 2, 3); 0 = the whole side.  The
                        double Mach reflection's wall starts at x = 1/6 (Section 4).         */
  int32_t inflow;    /* outflow meshes, Euler: bit s set = the faces of box side s that are not
                        walls see a prescribed outer state in the flux (weno_params.inflow_*);
                        the stencil images across them are the outflow ones.  0 = none.      */
} weno_mesh_opts;

/* Scheme parameters (defaults: weno_params_default). */
typedef struct {
  int32_t eqn;        /* weno_eqn_kind                                                     */
  int32_t precision;  /* weno_precision                                                    */
  double gas_gamma;   /* specific heat ratio of Eq. 1 (Euler)                              */
  double adv[2];      /* advection velocity (scalar)                                       */
  double eps;         /* epsilon of the nonlinear weights, Section 3.4, whose value the paper
                         does not state; default 1e-3, with which the scheme reproduces the
                         paper's Table 3 (density wave on regular quads) to about 1 %.  FP32C
                         solvers need eps >= 1e-15 (WENO_EINVAL otherwise), which keeps the
                         FP32 weights alpha <= 1 / eps^2 in range                           */
  double theta;       /* splitting parameter of Section 3.4 (3); must exceed 1, which keeps
                         sigma- > 0 (weno_solver_create returns WENO_EINVAL otherwise)      */
  double rcond;       /* relative singular-value cut of the minimum-norm least squares that
                         stand for the zeta-regularised solves of Eqs. 12 and 15 (1e-12)   */
  int32_t optimize;   /* 1: optimised linear weights of Section 3.3 (default), 0: raw      */
  int32_t linear;     /* 1: linear scheme R = sum gamma_j P^1_j (Eq. 14), 0: WENO          */
  int32_t n_threads;  /* host threads for the precompute (0 = all hardware threads)        */
  int32_t characteristic; /* Euler: 1 = reconstruct characteristic variables per face (Section 4:
                         normal flux Jacobian at the Roe average of the two cells), 0 =
                         component-wise (default)                                          */
  /* Prescribed outer state of inflow faces (weno_mesh_opts.inflow), Euler only: primitive
   * (rho, u, v, p) inflow_a at the Gauss points x of those faces with
   * n_x x + n_y y < c0 + s t, inflow_b elsewhere, inflow_line = (n_x, n_y, c0, s), t the
   * solver's time (weno_set_time, advanced by every step; the RK3 stages of Section 4 sit
   * at t, t + dt, t + dt/2).  A constant state: inflow_a = inflow_b.  The double Mach
   * reflection (Section 4) takes the post-shock state behind the moving Mach 10 shock and
   * the ambient state ahead of it.  Both states need rho > 0 and p > 0 when the mesh has
   * inflow faces; unused otherwise.  The comparison is made in FP64 in both precisions.   */
  double inflow_a[4];
  double inflow_b[4];
  double inflow_line[4];
} weno_params;

typedef struct {
  int64_t n_cells;      /* all cells (internal order: quads first, then triangles)   */
  int64_t n_quads;      /* internal ids [0, n_quads) are quads                        */
  int64_t n_tris;       /* internal ids [n_quads, n_cells) are triangles              */
  int64_t n_faces;      /* faces (periodic pairs counted once; outflow faces once)    */
  int64_t n_boundary;   /* outflow boundary faces                                     */
  int32_t n_instances;  /* 1, or the number of meshes joined by weno_mesh_concat      */
  int32_t n_inflow;     /* inflow faces (weno_mesh_opts.inflow)                       */
} weno_mesh_info;

/* Fills *p with the defaults: Euler, FP64, gamma 1.4, adv (1,1), eps 1e-3,
 * theta 3, rcond 1e-12, optimize 1, linear 0, n_threads 0, characteristic 0,
 * inflow states and line all 0 (meshes with inflow faces must set them). */
void weno_params_default(weno_params* p);

/* Builds a mesh (Section 2; stencils of Sections 3.1 and 3.2).
 * node_xy   [n_nodes][2] coordinates.
 * cell_ptr  [n_cells + 1] offsets into cell_nodes; cells have 3 or 4 nodes,
 *           either orientation (clockwise cells are reversed).
 * cell_nodes node ids.
 * opts      boundary description.
 * Cells are renumbered: quads first, then triangles, each in Morton order
 * of their centroids.  Errors: WENO_EINVAL, WENO_EMESH, WENO_EPERIODIC,
 * WENO_ENOMEM.  Synchronous, host only (no CUDA calls). */
int weno_mesh_create(const double* node_xy, int64_t n_nodes, const int64_t* cell_ptr,
                     const int64_t* cell_nodes, int64_t n_cells, const weno_mesh_opts* opts,
                     weno_mesh_t* out);

/* Joins independent meshes into one batched mesh: a flattened cell / face
 * index space with per-instance offsets.  Instance k keeps its own
 * boundary conditions; its input ids are offset by the input cell counts of
 * instances 0..k-1.  The inputs stay valid and owned by the caller. */
int weno_mesh_concat(const weno_mesh_t* meshes, int32_t n, weno_mesh_t* out);

int weno_mesh_get_info(weno_mesh_t mesh, weno_mesh_info* info);

/* perm[internal id] = input id, n_cells entries. */
int weno_mesh_cell_permutation(weno_mesh_t mesh, int64_t* perm);

/* instance[internal id] = instance index, n_cells entries (int32). */
int weno_mesh_cell_instance(weno_mesh_t mesh, int32_t* instance);

/* Diagnostics of the linear weights (Section 3.3, Tables 1 and 2): for every
 * cell the maximum |gamma| over its Gauss points and candidates before
 * (raw) and after (opt) the optimisation.  Both [n_cells] in internal order.
 * Runs the FP64 precompute on the host; synchronous. */
int weno_mesh_weight_stats(weno_mesh_t mesh, const weno_params* params, double* max_raw, double* max_opt);

/* Run-time tables of one cell (internal id) from the host FP64 precompute
 * (Sections 3.1-3.3), for inspection and tests:
 *   mg[2]            = {M, G}: 12, 8 for a quad; 9, 6 for a triangle
 *   slot_cells[M]    internal id of the cell read for stencil slots 1..M
 *                    (replacements resolved; a ghost reads the cell itself)
 *   grad_op[M][4]    candidate j's gradient g_j = [o0 o1; o2 o3] (dW_a, dW_b)
 *                    for its sub-stencil {i0, a, b}
 *   gauss_offset[G][2] x_G - c0 of the cell's Gauss points (2 per edge,
 *                    edge k holds points 2k (near node k) and 2k+1)
 *   gamma[G][M]      linear weights used at run time (optimised if requested)
 * Arrays are sized for a quad (12, 48, 16, 96 entries).  The precompute is
 * cached on the mesh.  Synchronous, host only. */
int weno_mesh_cell_tables(weno_mesh_t mesh, const weno_params* params, int64_t cell, int32_t* slot_cells,
                          double* grad_op, double* gauss_offset, double* gamma, int32_t* mg);

void weno_mesh_destroy(weno_mesh_t mesh);

/* Creates a solver on the current CUDA device: runs the FP64 precompute
 * (least squares, candidates, linear weights and their optimisation) on the
 * host and uploads the run-time tables in the solver's precision.  The mesh
 * may be destroyed afterwards.  Synchronous. */
int weno_solver_create(weno_mesh_t mesh, const weno_params* params, void* cuda_stream, weno_solver_t* out);

int weno_solver_get_info(weno_solver_t s, weno_mesh_info* info);

/* R = L(U) (Eq. 4) at the solver's time.  U, U_lo, R: device arrays
 * [n_cells * n_v] (U_lo only for FP32C, else NULL).  Stream-ordered. */
int weno_residual(weno_solver_t s, const void* U, const void* U_lo, void* R, void* cuda_stream);

/* R = L(U) exactly like weno_residual, but without touching any memory the
 * solver allocated for scratch: the Gauss-point values and face fluxes go to
 * a fixed 16 MiB array compiled into the library (every GPU that loads the
 * library holds it until the process exits).  The paper has no counterpart;
 * this call exists for callers that may not allocate device memory once
 * they are running (a device-memory budget fixed at start-up, or a loop that
 * may not make allocation calls), and it allocates nothing itself.
 *  - Limit: (8 n_quads + 6 n_tris) * n_v + 256-byte padding + n_faces * n_v
 *    elements of 8 (FP64) or 4 (FP32C) bytes, plus for FP32C Euler solvers
 *    about 3 bytes per 16 cells of marks (cells whose weights left the FP32
 *    range), must fit in 16 MiB, i.e. about 50k cells for FP64 Euler
 *    and 100k for FP32C; larger meshes get WENO_EINVAL with the sizes in
 *    weno_last_error().
 *  - The first call on each device looks up the array's device address on
 *    that device; make that first call before any stream capture.
 *  - All calls share the one array, which keeps the last call's contents;
 *    every element a call reads is written earlier in the same call, so
 *    nothing needs clearing.  Calls whose work overlaps on the GPU (other
 *    streams, other solvers, other host threads) race on the array: order
 *    them on one stream.
 * Stream-ordered. */
int weno_residual_static(weno_solver_t s, const void* U, const void* U_lo, void* R, void* cuda_stream);

/* Sets the solver's time (every instance) to t; it starts at 0.  The time
 * enters only through inflow faces and advances by dt with every step.
 * Stream-ordered. */
int weno_set_time(weno_solver_t s, double t, void* cuda_stream);

/* Copies the time of every instance to t_out [n_instances] (host);
 * synchronises the stream. */
int weno_get_time(weno_solver_t s, double* t_out, void* cuda_stream);

/* One SSP-RK3 step (Section 4) of size dt in place on U (and U_lo). Uses a
 * CUDA graph of the three stages, built on first use for these pointers.
 * The stages evaluate L at the times t, t + dt and t + dt/2; then t += dt.
 * Stream-ordered. */
int weno_step(weno_solver_t s, void* U, void* U_lo, double dt, void* cuda_stream);

/* Same with one dt per instance: dt_dev is a device array [n_instances] of
 * double, read when the step runs. */
int weno_step_instances(weno_solver_t s, void* U, void* U_lo, const double* dt_dev, void* cuda_stream);

/* Largest stable dt (reading of the CFL rule: dt = cfl * min_i 2|Omega_i| /
 * sum_p (|v_i . n_p| + c_i) |l_p|, c = 0 for scalar advection), per
 * instance: dt_out[n_instances] on the host.  Synchronising. */
int weno_max_dt(weno_solver_t s, const void* U, const void* U_lo, double cfl, double* dt_out, void* cuda_stream);

/* sum_i |Omega_i| (U + U_lo)_i in FP64 per instance and variable:
 * sums[n_instances * n_v] on the host.  Deterministic order. Synchronising. */
int weno_conservation(weno_solver_t s, const void* U, const void* U_lo, double* sums, void* cuda_stream);

/* Reads and clears the device flags raised by residual / step launches since
 * the last check: WENO_ETIMEOUT if a bounded device wait gave up, else
 * WENO_ENONPHYS if any Gauss point had rho <= 0, p <= 0 or a non-finite value
 * (weno_last_error names how many instances), else WENO_OK.  The scheme has
 * no positivity limiter (Section 3.4 gives none), so a state can leave the
 * physical set; the flag reports it and the launches keep running.
 * Synchronising. */
int weno_check(weno_solver_t s, void* cuda_stream);

/* Per-instance form of weno_check: flags[n_instances] (host) receives 1 for every
 * instance that had a non-physical Gauss-point state since the last check, 0
 * otherwise; the flags are cleared.  Returns WENO_OK (or WENO_ETIMEOUT, as
 * weno_check).  Synchronising. */
int weno_check_instances(weno_solver_t s, int32_t* flags, void* cuda_stream);

/* Launches one pass of the residual on its own (profiling aid; the kernels
 * are the ones weno_residual and weno_step run):
 *   pass 1: cell reconstruction of U (U_lo) into the solver's Gauss-point scratch
 *           (Sections 3.1-3.4);
 *   pass 2: face fluxes from that scratch into the solver's flux scratch (Eqs. 5-6);
 *   pass 3: signed gather of the face fluxes into the solver's stage buffer (Eq. 4).
 * U / U_lo are used by pass 1 only.  Stream-ordered. */
int weno_pass(weno_solver_t s, int32_t pass, const void* U, const void* U_lo, void* cuda_stream);

/* Times each kernel over a set of block sizes and grid sizes (cells per
 * thread) on this mesh and keeps the fastest; rebuilds the step graphs.
 * Does not modify U / U_lo.  Synchronising. */
int weno_autotune(weno_solver_t s, const void* U, const void* U_lo, void* cuda_stream);

/* Current launch configuration: cfg[6] = {cell block, cell grid, face block,
 * face grid, gather block, gather grid}. */
int weno_solver_launch_config(weno_solver_t s, int32_t* cfg);

/* Testing aid for the bounded device waits (the paper has no counterpart).
 * With on != 0, the FP32C Euler reconstruction initialises its table-copy
 * barriers for one arrival more than any thread makes, so every block's wait
 * runs out after its 1 s limit, the block records the timeout and exits, and
 * the next weno_check returns WENO_ETIMEOUT; results of those launches are
 * invalid.  on = 0 restores normal operation.  Step graphs are rebuilt.
 * WENO_EINVAL for solvers without such waits (FP64, scalar). */
int weno_solver_debug_stall(weno_solver_t s, int32_t on);

/* Measures the throughput of one SM pipe on the current device, as the peak
 * against which the reconstruction kernels' arithmetic is placed (the paper
 * has no counterpart; this is a measurement aid).  kind: 0 FP32 fused
 * multiply-add (scalar instructions), 1 FP32 fused multiply-add (paired f32x2
 * instructions), 2 FP64 fused multiply-add, 3 FP32 approximate reciprocal (the
 * special-function pipe).  Launches 4 blocks of 256 threads per SM, each
 * thread running 8 independent chains of `iters` dependent instructions, once
 * to warm up and three times timed with CUDA events on cuda_stream; writes the
 * operations of one launch to *ops (an FMA counts as one, a paired FMA as two)
 * and the fastest launch's milliseconds to *ms.  Allocates and frees a small
 * output buffer.  Errors: WENO_EINVAL (kind outside 0..3, iters <= 0, null
 * outputs), WENO_ENOMEM, WENO_ECUDA.  Synchronising. */
int weno_probe_peak(int32_t kind, int32_t iters, void* cuda_stream, double* ops, float* ms);

void weno_solver_destroy(weno_solver_t s);

const char* weno_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WENO3_H */
