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
constexpr int kThreads = 6 * kCells;               // 6 threads per cell
constexpr int kReconPlanes = G_IH + 1;             // geometry planes 0 .. G_IH feed the reconstruction
constexpr int kEdgePlanes = NRGEO - G_NRM;         // planes G_NRM .. G_INR feed the flux kernel

inline int64_t padded_cells(int64_t n) { return (n + kCells - 1) / kCells * kCells; }

// Tiles of kCells cells; table == nullptr: tile k = cells [k*kCells, ...) of
// one mesh; otherwise table[k] = (first cell, cell count) with the first cell
// a multiple of kCells (several meshes side by side).
struct TileSet {
  const int2* table;
  int ntiles;
};

// TMA descriptors of one solver's geometry planes (2-D: cells x planes).
struct TensorMaps {
  CUtensorMap geo;      // reconstruction geometry, box kCells x kReconPlanes
  CUtensorMap egeo;     // flux geometry, box kCells x kEdgePlanes
  CUtensorMap idx;      // neighbour planes + packed edge indices, box kCells x 4
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
  const TensorMaps* maps;
  TileSet tiles;
  DevScalars* sc;
  double dt_fixed;         // > 0: use this step instead of the device CFL step
  EqParams P;
};

// Sets the kernels' shared-memory limits and caches their resident-block
// counts; call once per (precision, equation) before any stream capture.
void prepare_step_kernels(int prec, int eq);
void launch_recon(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_edge(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_step(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_cfl(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_reset(DevScalars* sc, double t, double cfl, cudaStream_t st);
void launch_set_target(DevScalars* sc, double T, int has_T, cudaStream_t st);
void launch_consv(int prec, const void* U, const double* area, int N, int ld, int m, double* partial, double* out,
                  cudaStream_t st);
void launch_scatter(int prec, const double* host_order, const int32_t* perm, int N, int ld, int planes, void* U,
                    cudaStream_t st);
void launch_gather(int prec, const void* U, const int32_t* perm, int N, int ld, int planes, double* host_order,
                   cudaStream_t st);

}  // namespace hw
