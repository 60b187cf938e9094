// FP64 iterative-refinement kernels of the mixed-precision solver (not part of
// the paper, whose experiments are FP64 only): the residual R = B - A X with
// the original FP64 matrix, the infinity norms and the normwise backward error
// eta = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf) (per right-hand side,
// maximum over them), and the precision conversions around the FP32 solves.
//
// Sums are formed in a fixed order (column chunks in increasing order, then
// the chunk partials in increasing order), so results are deterministic.
#include "internal.h"
#include "profile.h"
#include "ir.h"

namespace {

constexpr int kRows = 256;      // rows per CTA (one per thread)
constexpr int kChunk = 256;     // columns per CTA
constexpr int kMaxRhs = 16;

// partial[(chunk * nrhs + c) * n + i] = sum_{j in chunk} A(i, j) X(j, c)   (or |A(i,j)| when ABS)
template <bool ABS>
__global__ void __launch_bounds__(kRows) gemv_partial_kernel(int64_t n, int nrhs, const double* __restrict__ A,
                                                             int64_t lda, const double* __restrict__ X, int64_t ldx,
                                                             double* __restrict__ partial) {
    __shared__ double sx[kMaxRhs][kChunk];
    const int64_t i = (int64_t)blockIdx.x * kRows + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * kChunk;
    const int cw = (int)min((int64_t)kChunk, n - j0);
    if (!ABS) {
        for (int c = 0; c < nrhs; ++c)
            for (int j = threadIdx.x; j < cw; j += kRows) sx[c][j] = X[(j0 + j) + c * ldx];
        __syncthreads();
    }
    if (i >= n) return;
    double acc[kMaxRhs];
#pragma unroll
    for (int c = 0; c < kMaxRhs; ++c) acc[c] = 0.0;
    const double* a = A + i + j0 * lda;
    if (ABS) {
#pragma unroll 8
        for (int j = 0; j < cw; ++j) acc[0] += fabs(__ldcs(a + (int64_t)j * lda));
        partial[(int64_t)blockIdx.y * n + i] = acc[0];
        return;
    }
    if (nrhs == 1) {
#pragma unroll 8
        for (int j = 0; j < cw; ++j) acc[0] = fma(__ldcs(a + (int64_t)j * lda), sx[0][j], acc[0]);
    } else {
        for (int j = 0; j < cw; ++j) {
            const double v = __ldcs(a + (int64_t)j * lda);
#pragma unroll
            for (int c = 0; c < kMaxRhs; ++c)
                if (c < nrhs) acc[c] = fma(v, sx[c][j], acc[c]);
        }
    }
    for (int c = 0; c < nrhs; ++c) partial[((int64_t)blockIdx.y * nrhs + c) * n + i] = acc[c];
}

// R(i, c) = B(i, c) - sum_chunk partial   (in chunk order)
__global__ void residual_finish_kernel(int64_t n, int nrhs, int nchunks, const double* __restrict__ partial,
                                       const double* __restrict__ B, int64_t ldb, double* __restrict__ R, int64_t ldr) {
    const int64_t total = n * nrhs;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n;
        const int c = (int)(e / n);
        double s = 0.0;
        for (int q = 0; q < nchunks; ++q) s += partial[((int64_t)q * nrhs + c) * n + i];
        R[i + c * ldr] = B[i + c * ldb] - s;
    }
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;  // valid in thread 0
}

// out = max_i sum_q partial[q * n + i]   (||A||_inf from row-sum partials), as the
// bits of a non-negative double (whose integer order is its numeric order): each CTA
// sums its rows' partials in chunk order and takes the maximum, then an atomic max.
// *out_bits must be zero before the launch.
__global__ void __launch_bounds__(256) norm_finish_kernel(int64_t n, int nchunks, const double* __restrict__ partial,
                                                          unsigned long long* __restrict__ out_bits) {
    __shared__ double sh[32];
    double best = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nchunks; ++q) s += partial[(int64_t)q * n + i];
        best = (s > best || s != s) ? s : best;
    }
    best = block_max(best, sh);
    if (threadIdx.x == 0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(best));
}

// eta per rhs column (one CTA per column), then out_eta[0] = max over columns.
__global__ void __launch_bounds__(1024) eta_kernel(int64_t n, int nrhs, const double* __restrict__ R, int64_t ldr,
                                                   const double* __restrict__ X, int64_t ldx,
                                                   const double* __restrict__ B, int64_t ldb,
                                                   const double* __restrict__ anorm, double* __restrict__ eta_cols,
                                                   double* __restrict__ out_eta, unsigned int* __restrict__ done) {
    __shared__ double sh[32];
    const int c = blockIdx.x;
    double rm = 0.0, xm = 0.0, bm = 0.0;
    bool nan = false;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = R[i + c * ldr], x = X[i + c * ldx], b = B[i + c * ldb];
        nan |= (r != r) || (x != x);
        rm = fmax(rm, fabs(r));
        xm = fmax(xm, fabs(x));
        bm = fmax(bm, fabs(b));
    }
    __shared__ int s_nan;
    if (threadIdx.x == 0) s_nan = 0;
    __syncthreads();
    if (nan) s_nan = 1;
    rm = block_max(rm, sh);
    __syncthreads();
    xm = block_max(xm, sh);
    __syncthreads();
    bm = block_max(bm, sh);
    if (threadIdx.x == 0) {
        const double den = anorm[0] * xm + bm;
        double e = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
        if (s_nan) e = NAN;
        eta_cols[c] = e;
        __threadfence();
        const unsigned prev = atomicAdd(done, 1u);
        if (prev == (unsigned)nrhs - 1) {
            __threadfence();
            double m = 0.0;
            for (int q = 0; q < nrhs; ++q) {
                const double v = ((volatile double*)eta_cols)[q];
                m = (v > m || v != v) ? v : m;
            }
            out_eta[0] = m;
            *done = 0;
        }
    }
}

template <typename Tin, typename Tout>
__global__ void cast_kernel(int64_t rows, int64_t cols, const Tin* __restrict__ in, int64_t ldi, Tout* __restrict__ out,
                            int64_t ldo) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows, j = e / rows;
        out[i + j * ldo] = (Tout)in[i + j * ldi];
    }
}

template <typename Tin>
__global__ void add_to_f64_kernel(int64_t rows, int64_t cols, const Tin* __restrict__ d, int64_t ldd,
                                  double* __restrict__ x, int64_t ldx) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows, j = e / rows;
        x[i + j * ldx] += (double)d[i + j * ldd];
    }
}

unsigned grid_for(int64_t total) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(lu_cdiv(total, 256), 152 * 16)); }

}  // namespace

int64_t lu_ir_nchunks(int64_t n) { return lu_cdiv(std::max<int64_t>(n, 1), kChunk); }

int lu_launch_residual(cudaStream_t st, int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* X,
                       int64_t ldx, const double* B, int64_t ldb, double* R, int64_t ldr, double* partial) {
    if (n <= 0 || nrhs <= 0) return LU_SUCCESS;
    const int nch = (int)lu_ir_nchunks(n);
    for (int64_t c0 = 0; c0 < nrhs; c0 += kMaxRhs) {
        const int nr = (int)std::min<int64_t>(kMaxRhs, nrhs - c0);
        dim3 grid((unsigned)lu_cdiv(n, kRows), (unsigned)nch);
        {
            LuProfScope prof(st, LU_K_RESIDUAL, 8.0 * n * n + 8.0 * nch * nr * n, 2.0 * n * n * nr);
            gemv_partial_kernel<false><<<grid, kRows, 0, st>>>(n, nr, A, lda, X + c0 * ldx, ldx, partial);
        }
        LU_CHECK_LAUNCH();
        LuProfScope prof(st, LU_K_RESIDUAL, 8.0 * nch * nr * n + 24.0 * n * nr, 0.0);
        residual_finish_kernel<<<grid_for(n * nr), 256, 0, st>>>(n, nr, nch, partial, B + c0 * ldb, ldb, R + c0 * ldr,
                                                                 ldr);
        LU_CHECK_LAUNCH();
    }
    return LU_SUCCESS;
}

int lu_launch_norm_inf(cudaStream_t st, int64_t n, const double* A, int64_t lda, double* partial, double* out) {
    if (n <= 0) return LU_SUCCESS;
    const int nch = (int)lu_ir_nchunks(n);
    dim3 grid((unsigned)lu_cdiv(n, kRows), (unsigned)nch);
    {
        LuProfScope prof(st, LU_K_RESIDUAL, 8.0 * n * n, 1.0 * n * n);
        gemv_partial_kernel<true><<<grid, kRows, 0, st>>>(n, 1, A, lda, nullptr, 0, partial);
    }
    LU_CHECK_LAUNCH();
    LuProfScope prof(st, LU_K_RESIDUAL, 8.0 * nch * n, 0.0);
    LU_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
    norm_finish_kernel<<<(unsigned)std::min<int64_t>(lu_cdiv(n, 256), 1024), 256, 0, st>>>(
        n, nch, partial, reinterpret_cast<unsigned long long*>(out));
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

int lu_launch_eta(cudaStream_t st, int64_t n, int64_t nrhs, const double* R, int64_t ldr, const double* X, int64_t ldx,
                  const double* B, int64_t ldb, const double* anorm, double* eta_cols, double* out_eta,
                  unsigned int* done) {
    if (nrhs <= 0) return LU_SUCCESS;
    LuProfScope prof(st, LU_K_RESIDUAL, 24.0 * n * nrhs, 0.0);
    eta_kernel<<<(unsigned)nrhs, 1024, 0, st>>>(n, (int)nrhs, R, ldr, X, ldx, B, ldb, anorm, eta_cols, out_eta, done);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename Tin, typename Tout>
int lu_launch_cast(cudaStream_t st, int64_t rows, int64_t cols, const Tin* in, int64_t ldi, Tout* out, int64_t ldo) {
    if (rows <= 0 || cols <= 0) return LU_SUCCESS;
    LuProfScope prof(st, LU_K_RESIDUAL, (double)(sizeof(Tin) + sizeof(Tout)) * rows * cols, 0.0);
    cast_kernel<Tin, Tout><<<grid_for(rows * cols), 256, 0, st>>>(rows, cols, in, ldi, out, ldo);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename Tin>
int lu_launch_add_to_f64(cudaStream_t st, int64_t rows, int64_t cols, const Tin* d, int64_t ldd, double* x,
                         int64_t ldx) {
    if (rows <= 0 || cols <= 0) return LU_SUCCESS;
    LuProfScope prof(st, LU_K_RESIDUAL, (double)(sizeof(Tin) + 16) * rows * cols, 0.0);
    add_to_f64_kernel<Tin><<<grid_for(rows * cols), 256, 0, st>>>(rows, cols, d, ldd, x, ldx);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template int lu_launch_cast<double, float>(cudaStream_t, int64_t, int64_t, const double*, int64_t, float*, int64_t);
template int lu_launch_cast<float, double>(cudaStream_t, int64_t, int64_t, const float*, int64_t, double*, int64_t);
template int lu_launch_cast<double, double>(cudaStream_t, int64_t, int64_t, const double*, int64_t, double*, int64_t);
template int lu_launch_add_to_f64<float>(cudaStream_t, int64_t, int64_t, const float*, int64_t, double*, int64_t);
template int lu_launch_add_to_f64<double>(cudaStream_t, int64_t, int64_t, const double*, int64_t, double*, int64_t);
