// Host helpers of the tensor-core path.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sra {

// 2-D TMA descriptor over a row-major bf16 matrix [rows][cols] (cols
// contiguous, 16-byte aligned rows) with a box of box_rows x box_cols and the
// 128-byte swizzle (box_cols * 2 == 128). Returns 0 on success.
int make_bf16_tile_map(CUtensorMap *map, const void *base, int rows, int cols, int box_rows, int box_cols);

int tc_gemm_selftest(const void *W, const void *X, float *D, int *status, cudaStream_t st);

}  // namespace sra
