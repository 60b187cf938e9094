// Operand packing (FP32 -> K-major bf16/fp16) for the tensor-core trailing update.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define LU_PACK_BF16 0
#define LU_PACK_FP16 1
#define LU_PACK_BF16X3 2  // split bf16: K tripled, [hi|hi|lo] for A rows, [hi|lo|hi] for B columns
#define LU_PACK_BF16X6 3  // three-part split bf16, six products, K six times longer

static inline int lu_pack_segments(int fmt) { return fmt == LU_PACK_BF16X3 ? 3 : (fmt == LU_PACK_BF16X6 ? 6 : 1); }

// out[r][s*k + kk] = segment s of round(A[r + kk*lda]), r < rows, kk < k (row stride segments*k).
int lu_launch_pack_rows(cudaStream_t st, int fmt, const float* A, int64_t lda, int64_t rows, int k, void* out);
// out[c][s*k + kk] = segment s of round(B[kk + c*ldb]), c < cols, kk < k (row stride segments*k).
int lu_launch_pack_cols(cudaStream_t st, int fmt, const float* B, int64_t ldb, int64_t cols, int k, void* out);

// e4m3 with power-of-two block scales (one per row of A / per column of B):
// rscale[r] = 2^e, out[r][kk] = e4m3(A[r + kk*lda] / 2^e) (row stride k bytes).
int lu_launch_pack_rows_e4m3(cudaStream_t st, const float* A, int64_t lda, int64_t rows, int k, float* rscale,
                             void* out);
// cscale[c] = 2^e, out[c][kk] = e4m3(B[kk + c*ldb] / 2^e) (row stride k bytes).
int lu_launch_pack_cols_e4m3(cudaStream_t st, const float* B, int64_t ldb, int64_t cols, int k, float* cscale,
                             void* out);
