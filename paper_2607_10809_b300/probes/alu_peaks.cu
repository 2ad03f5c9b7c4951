// FP32 / FP64 FMA throughput probe: eight independent FMA chains per thread,
// 8 resident blocks of 256 threads per SM, best of 5 timed launches.  Gives the
// CUDA-core peaks used as the ALU roofline of the FP64 form.
//   build: python paper_2607_10809_b300/build.py  (also builds this probe)
//   run:   paper_2607_10809_b300/_lib/alu_peaks
#include <cstdio>
#include <cuda_runtime.h>
template <typename T, int ILP>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) x[i] = (T)(threadIdx.x + i);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < ILP; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < ILP; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <typename T, int ILP>
double run(int blocks, int threads, int iters) {
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  fma_loop<T, ILP><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    fma_loop<T, ILP><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
  }
  cudaFree(out);
  double flops = 2.0 * ILP * (double)iters * blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  printf("device %s SMs %d cc %d.%d l2 %d MB smem/block optin %zu\n", p.name, p.multiProcessorCount, p.major, p.minor, p.l2CacheSize >> 20, p.sharedMemPerBlockOptin);
  int sms = p.multiProcessorCount;
  printf("fp32 TFLOP/s: %.2f\n", run<float, 8>(sms * 8, 256, 20000));
  printf("fp64 TFLOP/s: %.3f\n", run<double, 8>(sms * 8, 256, 2000));
  printf("fp64 TFLOP/s (4 blk/SM): %.3f\n", run<double, 4>(sms * 4, 256, 2000));
  return 0;
}
