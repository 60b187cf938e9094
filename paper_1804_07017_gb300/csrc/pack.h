// Operand packing (FP32 -> K-major bf16/fp16) for the tensor-core trailing update.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define LU_PACK_BF16 0
#define LU_PACK_FP16 1

// out[r][kk] = round(A[r + kk*lda]), r < rows, kk < k (row stride k).
int lu_launch_pack_rows(cudaStream_t st, int fmt, const float* A, int64_t lda, int64_t rows, int k, void* out);
// out[c][kk] = round(B[kk + c*ldb]), c < cols, kk < k (row stride k).
int lu_launch_pack_cols(cudaStream_t st, int fmt, const float* B, int64_t ldb, int64_t cols, int k, void* out);
