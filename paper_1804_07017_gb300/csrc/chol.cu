// Cholesky factorization A = L L^T of a symmetric positive definite matrix on
// the blocked right-looking skeleton with depth-1 look-ahead of Sec. 3-4 (the
// paper names Cholesky among the factorizations that fit it).
//
// For symmetric positive definite A, Gaussian elimination without interchanges
// is stable and gives A = L~ U with L~ unit lower and U = D L~^T, D = diag(U) > 0;
// the Cholesky factor is L = L~ D^{1/2}.  The factorization therefore runs the
// LU driver (lu_factor_blocked) with the pivot search switched off -- panels
// below, no interchange plans or row exchanges -- and finishes with one scaling
// pass over the lower triangle.  A is stored with both triangles, but only the
// lower block triangle is kept current: the Schur complement of a symmetric
// matrix stays symmetric, so U12 = D1 L~21^T is formed from the block column
// below the panel (no RL2 on the upper part), and the trailing update
// A22 -= L~21 U12 skips the tiles above the diagonal panel blocks -- n^3/3
// flops, the symmetric rank-k update's count.
#include <cmath>

#include "internal.h"
#include "profile.h"

namespace {

constexpr int kLeafW = 32;  // widest panel leaf: one warp, one row per lane

// Elimination without interchanges of the w x w diagonal block (w <= 32) at A:
// lane r owns row r; at step j the rows below j take multipliers a_rj / a_jj and
// the rank-1 update of their remaining entries.  The first step whose pivot is
// not positive (or NaN) is recorded in sync->info as j_abs + j + 1.
template <typename T>
__global__ void __launch_bounds__(32) np_diag_kernel(T* __restrict__ A, int64_t lda, int w, int64_t j_abs,
                                                     LuSync* __restrict__ sync) {
    __shared__ T s[kLeafW][kLeafW + 1];
    const int lane = threadIdx.x;
    for (int c = 0; c < w; ++c)
        if (lane < w) s[lane][c] = A[lane + (int64_t)c * lda];
    __syncwarp();
    int bad = 0;
    for (int j = 0; j < w; ++j) {
        const T piv = s[j][j];
        if (!(piv > T(0)) && bad == 0) bad = j + 1;
        if (lane > j && lane < w) {
            const T l = s[lane][j] / piv;
            s[lane][j] = l;
            for (int c = j + 1; c < w; ++c) s[lane][c] = fma(-l, s[j][c], s[lane][c]);
        }
        __syncwarp();
    }
    for (int c = 0; c < w; ++c)
        if (lane < w) A[lane + (int64_t)c * lda] = s[lane][c];
    if (lane == 0 && bad != 0) atomicCAS(&sync->info, 0, (int)(j_abs + bad));
}

// Rows below the diagonal block: L21 := A21 U11^{-1}, one thread per row with the
// row's w <= 32 entries in registers; U11 (upper triangle of the factored
// diagonal block at A) staged in shared memory by every CTA.
template <typename T>
__global__ void __launch_bounds__(256) np_rows_kernel(T* __restrict__ A, int64_t lda, int64_t nrows, int w) {
    __shared__ T u[kLeafW][kLeafW + 1];
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        const int r = e % w, c = e / w;
        u[r][c] = A[r + (int64_t)c * lda];
    }
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    T* row = A + w + i;  // element (w + i, c) at row[c * lda]
    T x[kLeafW];
#pragma unroll
    for (int c = 0; c < kLeafW; ++c) x[c] = c < w ? row[(int64_t)c * lda] : T(0);
#pragma unroll
    for (int j = 0; j < kLeafW; ++j) {
        if (j < w) {
            x[j] = x[j] / u[j][j];
#pragma unroll
            for (int c = j + 1; c < kLeafW; ++c)
                if (c < w) x[c] = fma(-x[j], u[j][c], x[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < kLeafW; ++c)
        if (c < w) row[(int64_t)c * lda] = x[c];
}

// U12(p, c) = u_pp L~(c, k0 + p) for p < kb, c in [cb, ce): the block row of U
// from the block column of L~ (U = D L~^T for a symmetric matrix), written over
// A12 through a 32 x 32 shared-memory tile so both sides are read and written
// along columns.
template <typename T>
__global__ void __launch_bounds__(256) sym_u12_kernel(T* __restrict__ A, int64_t lda, int64_t k0, int kb,
                                                      int64_t cb, int64_t ncols) {
    __shared__ T tile[32][33];
    const int p0 = blockIdx.x * 32;
    const int64_t c0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int q = ty; q < 32; q += 8) {  // read L~(c0 + tx, k0 + p0 + q)
        const int p = p0 + q;
        const int64_t c = c0 + tx;
        tile[q][tx] = (p < kb && c < ncols) ? A[(cb + c) + (k0 + p) * lda] : T(0);
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {  // write U12(p0 + tx, c0 + q)
        const int p = p0 + tx;
        const int64_t c = c0 + q;
        if (p < kb && c < ncols) A[(k0 + p) + (cb + c) * lda] = A[(k0 + p) + (k0 + p) * lda] * tile[tx][q];
    }
}

// Strict lower triangle: l_ij = l~_ij sqrt(u_jj) (the diagonal is still u_jj here).
template <typename T>
__global__ void __launch_bounds__(256) chol_scale_lower_kernel(T* __restrict__ A, int64_t lda, int64_t n) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const T d = sqrt(A[j + j * lda]);
        for (int64_t i = j + 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            A[i + j * lda] *= d;
    }
}

// Diagonal: l_jj = sqrt(u_jj), after every column's scaling has read u_jj.
template <typename T>
__global__ void __launch_bounds__(256) chol_scale_diag_kernel(T* __restrict__ A, int64_t lda, int64_t n) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        A[j + j * lda] = sqrt(A[j + j * lda]);
}

template <typename T>
int potrf_impl(lu_context* h, int64_t n, T* A, int64_t lda, const lu_opts& o, int32_t* info,
               const LuTuEngine* eng = nullptr) {
    // only the lower block triangle is updated when the panels sit on a fixed grid
    // (their diagonal blocks then never straddle a band boundary)
    h->sym_band = o.nsched == 0 ? o.nb : 0;
    const int r = lu_factor_blocked<T>(h, n, A, lda, nullptr, o, info, eng, false);
    h->sym_band = 0;
    LU_TRY(r);
    if (n == 0) return LU_SUCCESS;
    cudaStream_t st = h->user;
    LuProfScope prof(st, LU_K_OTHER, 2.0 * sizeof(T) * (double)n * (double)n / 2.0, (double)n * (double)n / 2.0);
    const dim3 grid((unsigned)std::min<int64_t>(lu_cdiv(n, 256), 64), (unsigned)std::min<int64_t>(n, 65535));
    chol_scale_lower_kernel<T><<<grid, 256, 0, st>>>(A, lda, n);
    LU_CHECK_LAUNCH();
    chol_scale_diag_kernel<T><<<(unsigned)std::min<int64_t>(lu_cdiv(n, 256), 1024), 256, 0, st>>>(A, lda, n);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

}  // namespace

int lu_chol_factor_f32(lu_context* h, int64_t n, float* A, int64_t lda, const lu_opts& o, int32_t* info,
                       const LuTuEngine* eng) {
    return potrf_impl<float>(h, n, A, lda, o, info, eng);
}

template <typename T>
int lu_panel_nopiv(cudaStream_t st, T* A, int64_t lda, int64_t M, int64_t j0, int64_t width, LuSync* sync) {
    if (width <= 0) return LU_SUCCESS;
    if (width <= kLeafW) {
        T* D = A + j0 + j0 * lda;
        const int64_t below = M - j0 - width;
        LuProfScope prof(st, LU_K_PANEL, 2.0 * sizeof(T) * (double)(M - j0) * (double)width,
                         (double)(M - j0) * (double)width * (double)width);
        np_diag_kernel<T><<<1, 32, 0, st>>>(D, lda, (int)width, j0, sync);
        LU_CHECK_LAUNCH();
        if (below > 0) {
            np_rows_kernel<T><<<(unsigned)lu_cdiv(below, 256), 256, 0, st>>>(D, lda, below, (int)width);
            LU_CHECK_LAUNCH();
        }
        return LU_SUCCESS;
    }
    int64_t w1 = ((width / 2 + 7) / 8) * 8;
    if (w1 >= width) w1 = width / 2;
    const int64_t w2 = width - w1;
    LU_TRY(lu_panel_nopiv<T>(st, A, lda, M, j0, w1, sync));
    LU_TRY(lu_launch_trsm_lunit<T>(st, w1, w2, A + j0 + j0 * lda, lda, A + j0 + (j0 + w1) * lda, lda));
    if (M - j0 - w1 > 0)
        LU_TRY(lu_launch_gemm_update<T>(st, M - j0 - w1, w2, w1, A + (j0 + w1) + j0 * lda, lda, A + j0 + (j0 + w1) * lda,
                                        lda, A + (j0 + w1) + (j0 + w1) * lda, lda));
    return lu_panel_nopiv<T>(st, A, lda, M, j0 + w1, w2, sync);
}

template <typename T>
int lu_launch_sym_u12(cudaStream_t st, T* A, int64_t lda, int64_t k0, int64_t kb, int64_t cb, int64_t ce) {
    const int64_t nc = ce - cb;
    if (nc <= 0 || kb <= 0) return LU_SUCCESS;
    LuProfScope prof(st, LU_K_TRSM, sizeof(T) * 2.0 * (double)kb * (double)nc, (double)kb * (double)nc);
    const dim3 grid((unsigned)lu_cdiv(kb, 32), (unsigned)lu_cdiv(nc, 32));
    sym_u12_kernel<T><<<grid, 256, 0, st>>>(A, lda, k0, (int)kb, cb, nc);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template int lu_launch_sym_u12<double>(cudaStream_t, double*, int64_t, int64_t, int64_t, int64_t, int64_t);
template int lu_launch_sym_u12<float>(cudaStream_t, float*, int64_t, int64_t, int64_t, int64_t, int64_t);
template int lu_panel_nopiv<double>(cudaStream_t, double*, int64_t, int64_t, int64_t, int64_t, LuSync*);
template int lu_panel_nopiv<float>(cudaStream_t, float*, int64_t, int64_t, int64_t, int64_t, LuSync*);

extern "C" int lu_potrf_ex(lu_handle h, lu_dtype dtype, int64_t n, void* A, int64_t lda, const lu_opts* opts,
                           int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (n < 0) return -3;
    if (n > 0 && !A) return -4;
    if (lda < std::max<int64_t>(1, n)) return -5;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -6;
    if (!info) return -7;
    if (n > INT32_MAX / 2) return LU_ERR_UNSUPPORTED;
    if (o.nb == 0 && o.nsched == 0) lu_auto_opts(dtype == LU_F64 ? LU_TUNE_F64 : LU_TUNE_F32, n, &o);
    std::lock_guard<std::mutex> lk(h->mu);
    if (dtype == LU_F64) return potrf_impl<double>(h, n, (double*)A, lda, o, info);
    return potrf_impl<float>(h, n, (float*)A, lda, o, info);
}
