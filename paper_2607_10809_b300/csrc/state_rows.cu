// Rows of the internal state buffer gathered to / scattered from a packed
// array: the halo exchange of a partitioned mesh moves only the cells another
// part holds, not the whole state.  A row is the cell's record (Wbar, Vbar,
// Ybar: 3m values) and, in FP32, its m compensation words.  A row index
// outside [0, N) is skipped and raises bit 2 (value 4) of the flags word.
#include <cuda_runtime.h>

#include <cstdint>

#include "state_rows.h"

namespace hw {

namespace {
// thread per (row, word); rows[k] is an internal cell index
template <typename R>
__global__ void k_rows_gather(const R* __restrict__ U, const R* __restrict__ C, int m, int N,
                              const int32_t* __restrict__ rows, int64_t n, R* __restrict__ out, unsigned* flags) {
  const int w = C ? 4 * m : 3 * m;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n * w) return;
  const int64_t r = k / w;
  const int o = (int)(k % w);
  const int64_t i = rows[r];
  if (i < 0 || i >= N) {
    if (o == 0) atomicOr(flags, 4u);
    return;
  }
  out[k] = o < 3 * m ? U[i * 3 * m + o] : C[i * m + (o - 3 * m)];
}

template <typename R>
__global__ void k_rows_scatter(R* __restrict__ U, R* __restrict__ C, int m, int N, const int32_t* __restrict__ rows,
                               int64_t n, const R* __restrict__ in, unsigned* flags) {
  const int w = C ? 4 * m : 3 * m;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n * w) return;
  const int64_t r = k / w;
  const int o = (int)(k % w);
  const int64_t i = rows[r];
  if (i < 0 || i >= N) {
    if (o == 0) atomicOr(flags, 4u);
    return;
  }
  if (o < 3 * m) U[i * 3 * m + o] = in[k];
  else C[i * m + (o - 3 * m)] = in[k];
}
}  // namespace

void launch_rows_gather(int prec, const void* U, const void* C, int m, int N, const int32_t* rows, int64_t n, void* out,
                        unsigned* flags, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t total = n * (C ? 4 * m : 3 * m);
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (prec == 0)
    k_rows_gather<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(U), static_cast<const double*>(C), m,
                                                  N, rows, n, static_cast<double*>(out), flags);
  else
    k_rows_gather<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(U), static_cast<const float*>(C), m, N,
                                                 rows, n, static_cast<float*>(out), flags);
}

void launch_rows_scatter(int prec, void* U, void* C, int m, int N, const int32_t* rows, int64_t n, const void* in,
                         unsigned* flags, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t total = n * (C ? 4 * m : 3 * m);
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (prec == 0)
    k_rows_scatter<double><<<blocks, 256, 0, st>>>(static_cast<double*>(U), static_cast<double*>(C), m, N, rows,
                                                   n, static_cast<const double*>(in), flags);
  else
    k_rows_scatter<float><<<blocks, 256, 0, st>>>(static_cast<float*>(U), static_cast<float*>(C), m, N, rows, n,
                                                  static_cast<const float*>(in), flags);
}

}  // namespace hw
