// Launchers of the row gather / scatter of the internal state (state_rows.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hw {
// prec 0: double, 1: float.  C: the compensation words [ld][m] (FP32) or
// nullptr; a row then has 4m words, else 3m.  rows: n internal cell indices
// (device memory); an index outside [0, N) is skipped and sets bit 2 (value 4) of
// *flags (device memory).
void launch_rows_gather(int prec, const void* U, const void* C, int m, int N, const int32_t* rows, int64_t n, void* out,
                        unsigned* flags, cudaStream_t st);
void launch_rows_scatter(int prec, void* U, void* C, int m, int N, const int32_t* rows, int64_t n, const void* in,
                         unsigned* flags, cudaStream_t st);
}  // namespace hw
