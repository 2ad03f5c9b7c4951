// Host-side launch interface of the step kernels (internal).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace hw {

constexpr int kConsvBlocks = 296;  // 2 x 148 SMs, fixed so the summation order is fixed

struct StepArgs {
  const void* rgeo;        // [NRGEO][N] in the solver precision
  const int32_t* igeo;     // [NIGEO][N]
  int N;
  const void* U;           // state in  [3m][N]
  void* Un;                // state out [3m][N]
  void* Pb;                // edge-point buffer [6*3*m][N]
  DevScalars* sc;
  double dt_fixed;         // > 0: use this step instead of the device CFL step
  EqParams P;
};

void launch_recon(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_edge(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_step(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_cfl(int prec, int eq, const StepArgs& a, cudaStream_t st);
void launch_reset(DevScalars* sc, double t, double cfl, cudaStream_t st);
void launch_set_target(DevScalars* sc, double T, int has_T, cudaStream_t st);
void launch_consv(int prec, const void* U, const double* area, int N, int m, double* partial, double* out,
                  cudaStream_t st);
void launch_scatter(int prec, const double* host_order, const int32_t* perm, int N, int planes, void* U,
                    cudaStream_t st);
void launch_gather(int prec, const void* U, const int32_t* perm, int N, int planes, double* host_order,
                   cudaStream_t st);
void launch_round_geo(const double* src, float* dst, size_t n, cudaStream_t st);

}  // namespace hw
