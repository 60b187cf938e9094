// Throughput probe of the CUDA cores' fused multiply-add, FP64 (DFMA) and FP32
// (FFMA): the denominator for the kernels that run on the CUDA cores (the FP64
// trailing update and residual, the batched factorization, the triangular
// solves).  It is a measurement utility, not a step of the factorization.
//
// Every thread runs kChains independent multiply-add chains a := a*b + c, so
// the issue rate, not the FMA latency, bounds it; the chains' results are
// written out so that none of the work can be dropped.  The caller times the
// launch with CUDA events; the work is 2 * kChains * iters flops per thread.
#include "internal.h"

namespace {

constexpr int kChains = 16;

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int64_t iters, T b, T c, T* sink) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = T(t % 97) * T(1e-3) + T(i);
    // per-thread register operands (the products stay the same to rounding), so
    // the FMAs read no constant-bank operand
    const T bb = b + T(threadIdx.x & 1) * T(1e-30), cc = c + T(threadIdx.x & 2) * T(1e-30);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], bb, cc);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    sink[t] = s;
}

}  // namespace

extern "C" int lu_peak_fma(lu_dtype dtype, int blocks, int threads, int64_t iters, void* sink, void* stream) {
    if (dtype != LU_F64 && dtype != LU_F32) return -1;
    if (blocks < 1) return -2;
    if (threads < 32 || threads > 256 || threads % 32) return -3;
    if (iters < 1) return -4;
    if (!sink) return -5;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // b just below 1 and c small keep every chain finite for any iteration count
    if (dtype == LU_F64)
        fma_peak_kernel<double><<<blocks, threads, 0, st>>>(iters, 0.9999999, 1e-7, static_cast<double*>(sink));
    else
        fma_peak_kernel<float><<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(sink));
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

extern "C" int lu_peak_fma_chains(void) { return kChains; }
