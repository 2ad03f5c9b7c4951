// Host-side launch interface of the step kernels (internal).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "device.cuh"

namespace hw {

constexpr int kConsvBlocks = 296;                  // 2 x 148 SMs, fixed so the summation order is fixed
constexpr int kCells = 32;                         // cells per tile; plane strides are multiples of it
constexpr int kThreads = 6 * kCells;               // 6 threads per cell (k_edge, batched kernel, scale limiter)
constexpr int kLeanThreads = 2 * kCells;           // single-solve reconstruction: 2 threads per cell, so
                                                   // that the (cell, component) and (cell, point) task sets
                                                   // of a tile fill whole passes (2 and 3 for the Euler system)
constexpr int kReconPlanes = G_IH + 1;             // geometry planes 0 .. G_IH feed the reconstruction
constexpr int kEdgePlanes = G_INR + 1 - G_NRM;     // planes G_NRM .. G_INR feed the flux kernel
constexpr int kLimPlanes = NRGEO - G_PK;           // planes G_PK .. G_PN+2: flux blending (scale limiter)

inline int64_t padded_cells(int64_t n) { return (n + kCells - 1) / kCells * kCells; }

// Tiles of kCells cells; table == nullptr: tile k = cells [k*kCells, ...) of
// one mesh; otherwise table[k] = (first cell, cell count) with the first cell
// a multiple of kCells (several meshes side by side).
struct TileSet {
  const int2* table;
  int ntiles;
};

// Fused step: tiles of kFusedTile32 (FP32) or kFusedTile64 (FP64) cells, each
// with at most as many halo cells as its halo capacity; per cell the packed
// slots of its three neighbours in the tile's shared-memory records
// (kSlotBits bits each: below the tile size a tile cell, above it a halo cell,
// kSlotNone on a boundary).
constexpr int kFusedTile32 = 128, kFusedHalo32 = 64;
constexpr int kFusedTile64 = 64, kFusedHalo64 = 48;
constexpr int kSlotBits = 10, kSlotNone = (1 << kSlotBits) - 1;
struct FusedTiles {
  const int32_t* slot;       // [ld] packed neighbour slots
  const int32_t* halo_off;   // [ntiles + 1] offsets into halo
  const int32_t* halo;       // halo cells of each tile, ascending internal index
  int ntiles;
};

// TMA descriptors of one solver's geometry planes (2-D: cells x planes).
struct TensorMaps {
  CUtensorMap geo;      // reconstruction geometry, box kCells x kReconPlanes
  CUtensorMap egeo;     // flux geometry, box kCells x kEdgePlanes
  CUtensorMap idx;      // neighbour planes + packed edge indices, box kCells x 4
  CUtensorMap lgeo;     // flux-blending geometry (scale limiter), box kCells x kLimPlanes
};

// Per-solve device state of a batch.
struct BatchSolve {
  double t;                          // time
  double dt;                         // next step
  double T;                          // target time
  unsigned long long lam_min_bits;   // CFL minimum of the running step (bits of a positive double)
  long long nsteps;                  // steps taken (its parity selects the state buffer)
  int done;                          // target reached or failed
  int failed;                        // state became non-finite / non-physical
};

// Control block of a batched launch (grid barrier, running-solve counts, flags).
struct BatchCtl {
  unsigned bar_count;
  unsigned bar_gen;
  unsigned active[2];
  unsigned flags;                    // bit 0: non-physical state, bit 1: a bounded wait gave up
  int steps_run;
};

struct StepArgs {
  const void* rgeo;        // [NRGEO][ld] in the solver precision
  const int32_t* igeo;     // [NIGEO][ld]
  int N;                   // cells
  int ld;                  // plane stride
  int from;                // index (0/1) of the input state buffer
  const void* U;           // state in  [ld][3m] (record per cell)
  void* Un;                // state out [ld][3m]
  void* Pb;                // edge-point buffer [ld][6][3][m]
  void* C;                 // FP32 form: compensation of the cell averages [ld][m] (compensated
                           // summation of the updates), updated in place; nullptr: none
  const TensorMaps* maps;
  TileSet tiles;
  DevScalars* sc;
  double dt_fixed;         // > 0: use this step instead of the device CFL step
  EqParams P;
  FusedTiles fused;        // tables of the fused step (ntiles = 0: not available)
  // edge-once flux phase (EP non-null): oedges lists the n_oedges edges by
  // their left (owning) cell, i * 4 + j in internal order; EP [ld][6][2m]
  // receives the owner's time-integrated flux and central value per Gauss
  // point, which both cells of the edge then read
  const int32_t* oedges;
  int n_oedges;
  void* EP;
};

// Arguments of the batched persistent kernel.
struct BatchArgs {
  const void* rgeo;
  const int32_t* igeo;
  int N;                    // cells of all solves (with padding between solves)
  int ld;
  void* U0;                 // state buffer 0 [ld][3m]
  void* U1;                 // state buffer 1
  void* Pb;                 // edge-point buffer [ld][6][3][m]
  void* C;                  // FP32: compensation words of the cell averages [ld][m]; nullptr: none
  const TensorMaps* maps;
  const int4* tiles;        // (first cell, count, solve, 0)
  int ntiles;
  BatchSolve* bs;
  BatchCtl* ctl;
  int nsolves;
  double cfl;
  int max_steps;            // steps per launch
  unsigned long long spin_limit;
  int withhold_block;       // tests: this block skips its first barrier arrival (-1: none)
  int grid;
  EqParams P;
};

// Arguments of the adjoint step (Euler; all state-like buffers are per-cell
// records of the solver's internal layout).
struct AdjointArgs {
  const void* rgeo;
  const int32_t* igeo;
  int N;
  int ld;
  const void* U;           // state U^n
  const void* Pb;          // forward edge-point data of U^n
  const void* Ubar_next;   // cotangent of U^{n+1}
  void* Cb;                // scratch: stencil contributions [ld][4][3m]
  void* Ubar;              // result: cotangent of U^n [ld][3m]
  EqParams P;
  double dt;
};
void launch_adjoint(int prec, const AdjointArgs& a, cudaStream_t st);

// Resident blocks per SM of the batched kernel (cooperative launch limit).
int batch_blocks_per_sm(int prec, int eq, bool lim);
cudaError_t launch_batch(int prec, int eq, const BatchArgs& a, cudaStream_t st);
// One batched step as three launches (reconstruction, flux/update, per-solve
// finish); slot: the step's parity for the running-solve counts.
cudaError_t launch_batch_step(int prec, int eq, const BatchArgs& a, int slot, cudaStream_t st);
void launch_batch_cfl(int prec, int eq, const BatchArgs& a, cudaStream_t st);
void launch_batch_dt(BatchSolve* bs, int n, double cfl, double T, int has_T, cudaStream_t st);
void launch_batch_reset_ctl(BatchCtl* ctl, cudaStream_t st);

// Sets the kernels' shared-memory limits and caches their resident-block
// counts; call once per (precision, equation) before any stream capture.
void prepare_step_kernels(int prec, int eq);
void prepare_edge_once_kernels(int prec, int eq);
void launch_recon(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_edge(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_step(int prec, int eq, const StepArgs& a, cudaStream_t st);
// The fused reconstruct-and-flux kernel (a.fused must be set).
void launch_fused(int prec, int eq, const StepArgs& a, cudaStream_t st);
void prepare_fused_kernel(int prec, int eq);
void launch_cfl(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_reset(DevScalars* sc, double t, double cfl, cudaStream_t st);
void launch_set_target(DevScalars* sc, double T, int has_T, cudaStream_t st);
void launch_consv(int prec, const void* U, const void* C, const double* area, int N, int ld, int m, double* partial,
                  double* out, cudaStream_t st);
void launch_scatter(int prec, const double* host_order, const int32_t* perm, int N, int ld, int planes, void* U,
                    cudaStream_t st);
void launch_gather(int prec, const void* U, const void* C, int m, const int32_t* perm, int N, int ld, int planes,
                   double* host_order, cudaStream_t st);

}  // namespace hw

#include "../../include/hweno.h"
// TMA descriptors of the geometry and index planes of a workspace.
hw_status hw_encode_plane_maps(hw::TensorMaps* maps, int precision, char* rgeo, char* igeo, int64_t N, int64_t ld);
