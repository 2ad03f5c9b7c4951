/*
 * hweno.h -- C ABI of the B300 library for the compact simple HWENO scheme
 * with ADER time discretization on triangular meshes (Luo, Zhao, Qiu, Chen).
 *
 * One time step (Section 2) does, over every triangle and every edge:
 *   1. one HWENO reconstruction per cell from the cell averages of W, W_x, W_y
 *      on the compact stencil {K0, K1, K2, K3} (Section 2.2, Steps 1-6,
 *      Eqs. aver, pxy, smoo1, nonlinearweight, recon);
 *   2. the Lax-Wendroff procedure at the two Gauss points of every edge and the
 *      time Taylor expansion on each side (Section 2.1, Eqs. tay, tayext),
 *      followed by the local Lax-Friedrichs flux at the Gauss-Lobatto time nodes
 *      (Eqs. fx, flux);
 *   3. the finite-volume update of the cell averages (Eq. flx) and the
 *      Green-Gauss update of the derivative averages from the central edge
 *      values at t_{n+1} (Eqs. derave2d1, derave2d2, timeflux, taylor2dtime).
 *
 * Conventions shared by every entry point
 *   - Host state arrays are double, structure-of-arrays, in the caller's cell
 *     numbering: Wbar[c*ntri + i] is the average of component c of W over
 *     triangle i, Vbar / Ybar the averages of W_x / W_y (Eq. aver).
 *     Components: 1 for advection and Burgers, 4 (rho, rho u, rho v, E) for Euler.
 *   - The library renumbers cells internally along a Hilbert curve.  Host
 *     arrays never see it; the device-side state buffers and row calls below
 *     use the internal numbering (hw_mesh_permutation maps it to the caller's).
 *   - Device memory is owned by the caller: hw_state_init receives a workspace
 *     pointer of at least hw_workspace_bytes() bytes (for instance a torch
 *     uint8 CUDA tensor) and the library never frees it.  The library allocates
 *     no device memory of its own; it owns only the opaque host handles.
 *   - All device work is enqueued on the caller's CUDA stream.
 *   - Every function returns an hw_status; nothing else crosses the ABI on
 *     failure.  hw_last_error() gives a message for the calling thread.
 *     Device-side conditions (non-finite values, non-positive density or
 *     pressure, a spin limit reached) are latched in a device flag and
 *     reported by the next synchronising call (hw_run_to, hw_get_state,
 *     hw_status_flags).
 */
#ifndef HWENO_H_
#define HWENO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HW_OK = 0,
  HW_EINVAL = 1,      /* bad argument */
  HW_ENOMEM = 2,      /* workspace too small / host allocation failed */
  HW_ECUDA = 3,       /* a CUDA runtime call failed */
  HW_EMESH = 4,       /* non-manifold, inverted or degenerate mesh, ill-conditioned stencil */
  HW_ENONFINITE = 5,  /* NaN/Inf in the state, or rho <= 0 / p <= 0 (Euler) */
  HW_ETIMEOUT = 6,    /* a bounded device spin gave up */
  HW_ESTATE = 7       /* call not valid in the object's current state */
} hw_status;

typedef enum { HW_ADVECTION = 0, HW_BURGERS = 1, HW_EULER = 2 } hw_equation;
typedef enum { HW_FP64 = 0, HW_FP32 = 1 } hw_precision;
/* Boundary conditions.  HW_BC_PERIODIC and HW_BC_TRANSMISSIVE are mesh-wide
 * (hw_mesh_create); HW_BC_REFLECTIVE and HW_BC_INFLOW are set per boundary
 * edge with hw_mesh_set_boundary (the walls and the inflow/outflow ends of the
 * shock tubes of Section 3).  Every boundary edge has a ghost cell, the mirror
 * image of its triangle, that joins the stencil (Section 2.2) and gives the
 * exterior value of the flux:
 *   transmissive (outflow): the triangle's own data; W^ext = W^int;
 *   reflective (a wall; Euler, the scalar equations treat it as transmissive):
 *     the mirrored solution, momentum reflected across the edge and the
 *     derivative averages transformed accordingly; W^ext = the mirrored W^int;
 *   inflow: the state hw_options.inflow with zero derivative averages;
 *     W^ext = that state at every time node. */
typedef enum { HW_BC_PERIODIC = 0, HW_BC_TRANSMISSIVE = 1, HW_BC_REFLECTIVE = 2, HW_BC_INFLOW = 3 } hw_bc;

/* Solver options.  Defaults (hw_options_default): the paper's constants --
 * linear weights 0.94, 0.02, 0.02, 0.02 (Section 2.2, Step 3), epsilon 1e-8
 * (Step 5), CFL 0.5 (Section 3), gamma 1.4 (Example 3.2). */
typedef struct {
  int32_t eq;           /* hw_equation */
  int32_t positivity;   /* Euler only: 1 = apply the scale limiter of Zhang and Shu
                           (Section 3 uses it "in some extreme cases"): the
                           reconstruction and its space-time Taylor data are
                           pulled toward the cell average so that density and
                           pressure stay >= min(1e-13, rho_bar, p_bar) at the six
                           edge Gauss points and the three time nodes; 0 = off */
  int32_t time_rule;    /* time quadrature of the edge flux (Eq. flux): 0 = three-node
                           Gauss-Lobatto (Simpson) whose t_{n+1} node also gives the
                           Green-Gauss central values (Section 2.3, default); 1 = two-node
                           Gauss-Legendre, with the central values from a separate Taylor
                           evaluation at t_{n+1}.  1 is for the single-solve step only: it
                           is refused with the scale limiter, by the batched form and by
                           the adjoint step (HW_EINVAL) */
  int32_t step_kernels; /* kernels of a single-solve step: 0 = default (3 in HW_FP64,
                           1 in HW_FP32); 1 = a reconstruction kernel then a flux kernel
                           with the edge-point data in the workspace, each cell evaluating
                           the fluxes of its own edges; 2 = one fused reconstruct-and-flux
                           kernel that keeps the edge-point data in shared memory and
                           reconstructs each tile's halo itself (hw_state_init fails with
                           HW_EINVAL if a tile of the mesh has more halo cells than the
                           kernel holds); 3 = the reconstruction kernel, then the flux
                           phase with each edge evaluated once (by its left cell) into a
                           per-point flux buffer of the workspace, then the update kernel
                           (half the flux arithmetic; meshes below 2^29 cells).  Results
                           agree bit for bit between 1 and 3, to rounding with 2. */
  double ax, ay;        /* advection velocity (HW_ADVECTION) */
  double gamma_gas;     /* ratio of specific heats (HW_EULER) */
  double cfl;           /* dt = cfl * min_K inradius_K / lambda_K */
  double gamma_lin[4];  /* linear weights gamma_1..gamma_4: each > 0 and sum 1 within
                           1e-12 (Section 2.2, Step 3); HW_EINVAL otherwise */
  double eps;           /* epsilon in the nonlinear weights, > 0 */
  double inflow[4];     /* conservative state imposed at HW_BC_INFLOW edges (first m
                           components used); default rho = 1, zero momentum, E = 2.5 */
} hw_options;

typedef struct hw_mesh hw_mesh;
typedef struct hw_solver hw_solver;

void hw_options_default(hw_options* opt);

/* Build the mesh and its FP64 precompute (connectivity, stencils, per-cell
 * reconstruction operators for Steps 1-2 of Section 2.2, edge normals and
 * Gauss points) on the host.
 *   xy   : [nvert*2] vertex coordinates (x, y), host, read only
 *   tri  : [ntri*3] vertex indices, counter-clockwise, host, read only
 *   Lx,Ly: period in x / y (0 = not periodic); a periodic mesh lists each
 *          vertex once and triangles refer to vertices modulo the period
 *   bc   : hw_bc; HW_BC_PERIODIC requires every edge to have two triangles
 * Sizes: 1 <= ntri <= 2^30 - 1; in practice the device workspace bounds it
 * (hw_workspace_bytes: about 745 bytes per triangle for FP32 Euler).
 * Errors: HW_EINVAL (null pointers, an empty mesh, ntri beyond 2^30 - 1,
 * indices out of range, a periodic mesh without positive periods), HW_EMESH
 * (degenerate or clockwise triangle, an edge shared by more than two
 * triangles, an open edge on a periodic mesh, a mesh too coarse for its
 * period, an ill-conditioned stencil; hw_last_error names which). */
hw_status hw_mesh_create(const double* xy, int64_t nvert, const int32_t* tri, int64_t ntri, double Lx, double Ly,
                         int32_t bc, hw_mesh** out);
hw_status hw_mesh_destroy(hw_mesh* mesh);
/* Number of triangles. */
int64_t hw_mesh_ntri(const hw_mesh* mesh);
/* Boundary condition of every boundary edge: edge_bc[3*i + j] for local edge
 * j of triangle i (caller's numbering), read only where that edge is on the
 * boundary: HW_BC_TRANSMISSIVE, HW_BC_REFLECTIVE or HW_BC_INFLOW (see hw_bc).
 * Host array.  Call before hw_state_init / hw_batch_create; a mesh starts
 * with every boundary edge transmissive.  Errors: HW_EINVAL (null pointer, an
 * invalid type on a boundary edge; the mesh is then unchanged). */
hw_status hw_mesh_set_boundary(hw_mesh* mesh, const int32_t* edge_bc);
/* Neighbour across local edge j (from vertex j to vertex j+1) of triangle i,
 * caller's numbering, -1 on a boundary: nbr[3*i + j].  nbe (optional, may be
 * NULL) receives the neighbour's local index of the same edge. Host arrays. */
hw_status hw_mesh_neighbors(const hw_mesh* mesh, int32_t* nbr, int32_t* nbe);
/* Internal (Hilbert) order: perm[k] = caller's index of the k-th cell. */
hw_status hw_mesh_permutation(const hw_mesh* mesh, int32_t* perm);

/* Bytes of device workspace hw_state_init needs for this mesh / options /
 * precision (geometry, two state buffers, edge-point buffer, staging; in
 * HW_FP32 also one compensation word per cell and component: the FP32 form
 * adds each step's update to the cell averages by compensated summation, so
 * that their FP32 rounding does not accumulate over the steps; the
 * reconstruction and the fluxes use the FP32 averages). */
hw_status hw_workspace_bytes(const hw_mesh* mesh, const hw_options* opt, int32_t precision, size_t* bytes);

/* Upload geometry and the initial state (host arrays as described above) into
 * the caller's workspace and compute the first CFL time step.  The workspace
 * must stay valid until hw_solver_destroy.  cuda_stream: cudaStream_t (NULL =
 * legacy default stream).  Synchronises the stream before returning.  The
 * first call on a device also commits the library's static scratch array of
 * hw_step_static_scratch there (64 MiB, held until the process exits). */
hw_status hw_state_init(const hw_mesh* mesh, const hw_options* opt, int32_t precision, const double* Wbar,
                        const double* Vbar, const double* Ybar, void* workspace, size_t workspace_bytes,
                        void* cuda_stream, hw_solver** out);
/* Replace the state (host arrays) and set the time to t; recomputes the CFL
 * step.  The copy is enqueued on the stream; the host arrays must stay valid
 * until the stream reaches it (pinned memory gives a true asynchronous copy). */
hw_status hw_set_state(hw_solver* s, const double* Wbar, const double* Vbar, const double* Ybar, double t);
/* One time step, asynchronous on the stream.  dt > 0: that step size; dt <= 0:
 * the CFL step held on the device (a target time of hw_run_to holds only
 * inside that call). */
hw_status hw_step(hw_solver* s, double dt);
/* Advance to time T with CFL steps (last one clipped to hit T) through a
 * captured CUDA graph of several steps; synchronises.  nsteps (may be NULL)
 * receives the number of steps taken.  Returns HW_ENONFINITE if the state went
 * non-finite / non-physical.  On return the target is cleared: later hw_step
 * calls advance the state again. */
hw_status hw_run_to(hw_solver* s, double T, int64_t* nsteps);
/* Copy the state back to host arrays in the caller's numbering and report the
 * time; synchronises.  Any pointer may be NULL to skip it.  HW_FP32: Wbar is
 * the FP32 cell average plus its compensation, summed in double. */
hw_status hw_get_state(hw_solver* s, double* Wbar, double* Vbar, double* Ybar, double* t);
/* Sum over cells of |K| * Wbar_K per component, accumulated in FP64 on the
 * device in a fixed order (deterministic); sums[c], synchronises. */
hw_status hw_conservation(hw_solver* s, double* sums);
/* Device flags latched since the last call (bit 0: non-finite / non-physical
 * state, bit 1: spin limit reached, bit 2: a row index of
 * hw_state_rows_export / hw_state_rows_import outside [0, ntri), skipped);
 * clears them; synchronises. */
hw_status hw_status_flags(hw_solver* s, uint32_t* flags);
/* Current time, current device time step and steps taken; synchronises. */
hw_status hw_time(hw_solver* s, double* t, double* dt, int64_t* nsteps);
/* Per-kernel timing of the next hw_step calls (up to 4096 steps) with CUDA
 * events on the solver's stream, for measurement; enable = 0 stops it.
 * Enabling resets the accumulators. */
hw_status hw_profile(hw_solver* s, int32_t enable);
/* Synchronises on the recorded events; ms[0] = total reconstruction-kernel
 * time (the fused kernel's, when steps run it), ms[1] = total flux/update-kernel
 * time (both kernels of the edge-once phase; 0 with the fused kernel),
 * milliseconds over nsteps profiled steps. */
hw_status hw_profile_read(hw_solver* s, double* ms, int64_t* nsteps);
/* Kernels the solver's steps run: *path = 1 (separate), 2 (fused) or 3
 * (separate, each edge's flux once). */
hw_status hw_step_kernels(const hw_solver* s, int32_t* path);
hw_status hw_solver_destroy(hw_solver* s);

/* Same as hw_step, but the scratch of the step (the edge-point buffer between
 * the reconstruction and the flux kernels) is a static device array inside the
 * library instead of part of the workspace (the per-point flux buffer of the
 * edge-once flux phase, step_kernels 3 and the FP64 default, stays in the
 * workspace; the fused kernel of step_kernels 2 is not used here, the step
 * runs the separate kernels).  The paper has no counterpart: it
 * is for callers that cannot call cudaMalloc (hosts that own the device memory
 * pool, plug-ins handed fixed buffers, runtimes that must not allocate while
 * running); they still pass the state and geometry through the solver's
 * workspace, but need no memory for temporaries.
 *   - Limit: 18 * m * ld * (8 for FP64, 4 for FP32) bytes must fit in the
 *     64 MiB array, where ld is ntri rounded up to a multiple of 32 (FP32
 *     Euler: at most 232,992 triangles; FP64 Euler: at most 116,480); larger
 *     meshes get HW_EINVAL with a message naming both sizes.
 *   - The array's 64 MiB are committed on a device by the first hw_state_init
 *     on that device (which also looks up the array's device address there)
 *     and stay reserved until the process exits; hw_step_static_scratch itself
 *     makes no allocation of any kind.
 *   - All calls share the one array and it keeps the last call's contents
 *     (every slot a step reads is written earlier in the same step, so nothing
 *     needs clearing); calls whose work overlaps on the GPU (other streams,
 *     other solvers) race on it and must be serialised by the caller.
 *   - Allocates nothing (no cudaMalloc, cudaFree or allocating library call). */
hw_status hw_step_static_scratch(hw_solver* s, double dt);

/* ---------------------------------------------------------------------------
 * Device-side state buffers and the adjoint of a step.
 * An internal state buffer holds the state of every cell in the library's
 * internal order and precision: the records [ld][3m] (ld = ntri rounded up to
 * a multiple of 32; per cell Wbar, Vbar, Ybar, m values each), then, in
 * HW_FP32, the compensation words [ld][m] of the averages (the rounding error
 * the compensated update carries into the next step).  hw_state_bytes()
 * bytes, caller-allocated device memory, 16-byte aligned. */
hw_status hw_state_bytes(const hw_solver* s, size_t* bytes);
/* Copy the current state to / from an internal buffer (device to device,
 * asynchronous on the stream), compensation words included, so that an
 * export / import round trip continues the run bit for bit.  Import also sets
 * the time to t and recomputes the CFL step. */
hw_status hw_state_export(hw_solver* s, void* dst);
hw_status hw_state_import(hw_solver* s, const void* src, double t);
/* Rows of the current state, for a halo exchange that moves only the cells
 * another part of a partitioned mesh holds.  A row is a cell's record (3m
 * values) followed, in HW_FP32, by its m compensation words, in the solver's
 * precision: hw_state_row_words() values.  rows: n internal cell indices
 * (device memory, int32; hw_mesh_permutation maps them to the caller's
 * numbering); buf: n rows, packed (device memory).  Asynchronous on the
 * stream.  An index outside [0, ntri) is skipped and raises bit 2 of
 * hw_status_flags.  Import with refresh != 0 then recomputes the CFL step of
 * the state (call it with the last batch of rows of a step). */
hw_status hw_state_row_words(const hw_solver* s, int32_t* words);
hw_status hw_state_rows_export(hw_solver* s, const int32_t* rows, int64_t n, void* buf);
hw_status hw_state_rows_import(hw_solver* s, const int32_t* rows, int64_t n, const void* buf, int32_t refresh);
/* Convert host arrays (caller numbering, double, as for hw_get_state) to an
 * internal buffer and back; pure permutation and precision conversion (used
 * for cotangents); synchronise.  To a buffer: its compensation words are set to
 * zero.  From a buffer: the records alone (as for a cotangent). */
hw_status hw_host_to_internal(hw_solver* s, const double* Wbar, const double* Vbar, const double* Ybar, void* dst);
hw_status hw_internal_to_host(hw_solver* s, const void* src, double* Wbar, double* Vbar, double* Ybar);
/* Edge-point buffer: the time-Taylor data (W, W_t, W_tt) of every cell at
 * its six edge Gauss points, as a step computes them from the pre-step state
 * (Section 2.1); hw_pb_bytes() bytes of device memory, 16-byte aligned.
 * hw_step_keep is hw_step(s, dt) that leaves this data of the pre-step state
 * in pb_out (written there in place of the solver's own buffer), so that the
 * adjoint of the same step need not recompute it.  Not a step of the paper's
 * method: the reverse pass of a checkpointed rollout uses it.  Errors:
 * HW_EINVAL (null pointer, pb_out not 16-byte aligned). */
hw_status hw_pb_bytes(const hw_solver* s, size_t* bytes);
hw_status hw_step_keep(hw_solver* s, double dt, void* pb_out);
/* Adjoint (vector-Jacobian product) of one step of size dt held fixed:
 * Ubar_n = (dU^{n+1}/dU^n)^T Ubar_next, for the Euler equations without the
 * scale limiter.  U_n, Ubar_next, Ubar_n: internal buffers (device).  Pb_n:
 * the edge-point buffer hw_step_keep(s, dt, Pb_n) filled from U_n, or NULL to
 * recompute it here.  Non-smooth points (|.| in the
 * nonlinear weights and the viscosity, max in the viscosity) follow the
 * branch of the forward evaluation.  scratch: device memory of
 * hw_adjoint_scratch_bytes(), 256-byte aligned.  Asynchronous on the stream.
 * Errors: HW_EINVAL (null pointer, a state or edge-point buffer not
 * 16-byte aligned, scratch not 256-byte aligned, dt <= 0, not the Euler
 * equations, scale limiter on, walls or inflow edges on the mesh), HW_ENOMEM
 * (scratch_bytes too small). */
hw_status hw_adjoint_scratch_bytes(const hw_solver* s, size_t* bytes);
hw_status hw_step_adjoint(hw_solver* s, double dt, const void* U_n, const void* Pb_n, const void* Ubar_next,
                          void* Ubar_n, void* scratch, size_t scratch_bytes);

/* ---------------------------------------------------------------------------
 * Batched runs: many independent solves (same options, meshes of any sizes)
 * advanced together.  All time steps of all solves run inside one persistent
 * cooperative kernel launch (captured in a CUDA graph): per step a
 * reconstruction phase over the tiles of the solves still running, a grid
 * barrier, the flux/update phase, a barrier, the per-solve time step update
 * (each solve keeps its own CFL step and time, Section 3), a barrier.  Grid
 * barriers spin a bounded number of times; on time-out the launch stops and
 * the next call returns HW_ETIMEOUT.  A solve whose state becomes non-finite
 * or non-physical is stopped alone (reported by hw_batch_get_state) while the
 * others continue. */
typedef struct hw_batch hw_batch;
typedef struct {
  int32_t blocks_per_sm;     /* blocks of the persistent launch per SM; 0 = as many as fit */
  int32_t tile_order;        /* 0 solve by solve, 1 largest solves first, 2 round robin over solves */
  int32_t steps_per_launch;  /* time steps per launch (graph replay) at most */
  int32_t withhold_block;    /* testing only: this block withholds its first barrier arrival (-1: none) */
  int64_t spin_limit;        /* polls of a barrier wait before giving up; 0 = default (about 2 s) */
  int32_t launch_mode;       /* 0: each chunk of steps in one persistent cooperative launch with grid
                                barriers (blocks_per_sm applies); 1: every step as three launches
                                (reconstruction, flux/update, per-solve finish) captured in one graph,
                                each kernel at its own occupancy.  Same results bit for bit. */
} hw_batch_schedule;

void hw_batch_schedule_default(hw_batch_schedule* s);
/* Workspace bytes of a batch of n meshes (same options / precision as hw_state_init). */
hw_status hw_batch_workspace_bytes(const hw_mesh* const* meshes, int32_t n, const hw_options* opt, int32_t precision,
                                   size_t* bytes);
/* Upload the n meshes' geometry and initial states (host arrays per solve, as
 * for hw_state_init) into the caller's workspace; t = 0 for every solve.
 * The meshes may be destroyed afterwards.  Synchronises. */
hw_status hw_batch_create(const hw_mesh* const* meshes, int32_t n, const hw_options* opt, int32_t precision,
                          const double* const* Wbar, const double* const* Vbar, const double* const* Ybar,
                          void* workspace, size_t workspace_bytes, void* cuda_stream, hw_batch** out);
hw_status hw_batch_set_schedule(hw_batch* b, const hw_batch_schedule* s);
/* Current schedule and the grid it launches (blocks). */
hw_status hw_batch_get_schedule(const hw_batch* b, hw_batch_schedule* s, int32_t* grid_blocks);
/* Time every candidate schedule (launch mode 0 with each tile order and each
 * number of blocks per SM, launch mode 1 with each tile order) on trial_steps
 * steps from the initial state, keep the fastest, restore the initial state.
 * best / best_ms may be NULL. */
hw_status hw_batch_autotune(hw_batch* b, int32_t trial_steps, hw_batch_schedule* best, double* best_ms);
/* Advance every solve to time T (each with its own CFL steps, the last one
 * clipped to T); synchronises.  cell_steps (may be NULL): sum over solves of
 * triangles x steps taken.  HW_ENONFINITE if a solve failed (the others are
 * still advanced), HW_ETIMEOUT if a barrier wait gave up. */
hw_status hw_batch_run_to(hw_batch* b, double T, int64_t* cell_steps);
/* Exactly `steps` steps of every running solve in one launch (no target
 * time), timed with CUDA events (ms may be NULL); synchronises. */
hw_status hw_batch_steps(hw_batch* b, int32_t steps, double* ms);
/* Back to the initial states and t = 0. */
hw_status hw_batch_reset(hw_batch* b);
/* State of one solve in its caller numbering (as hw_get_state), its time, steps
 * and failure flag; any output may be NULL.  Synchronises. */
hw_status hw_batch_get_state(hw_batch* b, int32_t solve, double* Wbar, double* Vbar, double* Ybar, double* t,
                             int64_t* nsteps, int32_t* failed);
hw_status hw_batch_destroy(hw_batch* b);

/* Message of the last failing call on this thread. */
const char* hw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HWENO_H_ */
