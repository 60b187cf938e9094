// FP64 iterative-refinement kernels (see ir.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

int64_t lu_ir_nchunks(int64_t n);
// R = B - A X (FP64); partial must hold lu_ir_nchunks(n) * min(nrhs, 16) * n doubles.
int lu_launch_residual(cudaStream_t st, int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X,
                       int64_t ldx, const double* B, int64_t ldb, double* R, int64_t ldr, double* partial);
// out[0] = ||A||_inf; partial must hold lu_ir_nchunks(n) * n doubles.
int lu_launch_norm_inf(cudaStream_t st, int64_t n, const double* A, int64_t lda, double* partial, double* out);
// out_eta[0] = max_c ||R_c|| / (anorm ||X_c|| + ||B_c||); done must be 0 on entry (left 0).
int lu_launch_eta(cudaStream_t st, int64_t n, int64_t nrhs, const double* R, int64_t ldr, const double* X, int64_t ldx,
                  const double* B, int64_t ldb, const double* anorm, double* eta_cols, double* out_eta,
                  unsigned int* done);
// out = (Tout) in, elementwise over rows x cols
template <typename Tin, typename Tout>
int lu_launch_cast(cudaStream_t st, int64_t rows, int64_t cols, const Tin* in, int64_t ldi, Tout* out, int64_t ldo);
// x += (double) d, elementwise over rows x cols
template <typename Tin>
int lu_launch_add_to_f64(cudaStream_t st, int64_t rows, int64_t cols, const Tin* d, int64_t ldd, double* x,
                         int64_t ldx);
