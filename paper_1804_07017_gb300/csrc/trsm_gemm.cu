// RL2 and RL3 of LU_blk (Sec. 3) on the CUDA cores, in the storage precision.
//
//   trsm_lunit:   B := trilu(L)^{-1} B   (L m x m unit lower, m <= 1024)
//   gemm_update:  C := C - A B           (FP64/FP32 fused multiply-add)
//
// Every output element is computed in a fixed order that does not depend on
// where its tile starts, so splitting an update into column ranges (the
// static look-ahead's TU^L / TU^R split, Sec. 4) gives bit-identical results.
#include "internal.h"
#include "profile.h"

namespace {

constexpr int kTrsmThreads = 256;

// One CTA solves COLS right-hand-side columns held in shared memory, sweeping
// 32-row diagonal blocks: a warp-shuffle substitution inside the block, then a
// rank-32 update of the rows below it.
template <typename T, int COLS>
__global__ void __launch_bounds__(kTrsmThreads)
    trsm_lunit_kernel(int m, int64_t n, const T* __restrict__ L, int64_t ldl, T* __restrict__ B,
                      int64_t ldb) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int mp = (m + 31) & ~31;
    T* sB = reinterpret_cast<T*>(smraw);  // [COLS][mp]
    T* sL = sB + (size_t)COLS * mp;        // [32][33] diagonal block, sL[j*33 + i] = L(J+i, J+j)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t col0 = (int64_t)blockIdx.x * COLS;
    const int nc = (int)min((int64_t)COLS, n - col0);
    for (int c = 0; c < COLS; ++c)
        for (int r = tid; r < mp; r += kTrsmThreads)
            sB[c * mp + r] = (c < nc && r < m) ? B[r + (col0 + c) * ldb] : T(0);
    for (int J = 0; J < m; J += 32) {
        const int jb = min(32, m - J);
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += kTrsmThreads) {
            const int i = e & 31, j = e >> 5;
            sL[j * 33 + i] = (i < jb && j < jb) ? L[(int64_t)(J + i) + (int64_t)(J + j) * ldl] : T(0);
        }
        __syncthreads();
        for (int c = warp; c < COLS; c += kTrsmThreads / 32) {
            T v = sB[c * mp + J + lane];
            for (int j = 0; j < jb; ++j) {
                const T xj = __shfl_sync(0xffffffffu, v, j);
                if (lane > j) v = fma(-sL[j * 33 + lane], xj, v);
            }
            if (lane < jb) sB[c * mp + J + lane] = v;
        }
        __syncthreads();
        // rank-jb update of the rows below: the row's jb multipliers are loaded
        // together (all in flight at once), then applied to the COLS columns
        for (int r = J + jb + tid; r < m; r += kTrsmThreads) {
            T l[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) l[j] = (j < jb) ? __ldg(&L[(int64_t)r + (int64_t)(J + j) * ldl]) : T(0);
            T acc[COLS];
#pragma unroll
            for (int c = 0; c < COLS; ++c) acc[c] = T(0);
#pragma unroll
            for (int j = 0; j < 32; ++j)
#pragma unroll
                for (int c = 0; c < COLS; ++c) acc[c] = fma(l[j], sB[c * mp + J + j], acc[c]);
#pragma unroll
            for (int c = 0; c < COLS; ++c) sB[c * mp + r] -= acc[c];
        }
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c)
        for (int r = tid; r < m; r += kTrsmThreads) B[r + (col0 + c) * ldb] = sB[c * mp + r];
}

constexpr int kGemmThreads = 256;
constexpr int BK = 16;

// C := C - A B with a BM x BN tile per CTA and a 4x4 register tile per thread;
// thread (tx, ty) owns rows tx + TX i and columns ty + TY j so that shared
// memory reads and the epilogue's column-major accesses are both coalesced.
// The narrow shapes (BN = 16, 32) serve the panel's own thin updates.  Every
// element accumulates its k products in order, whatever the tile shape.
template <typename T, int BM, int BN>
__global__ void __launch_bounds__(kGemmThreads)
    gemm_update_kernel(int64_t m, int64_t n, int k, const T* __restrict__ A, int64_t lda,
                       const T* __restrict__ B, int64_t ldb, T* __restrict__ C, int64_t ldc) {
    constexpr int TX = BM / 4, TY = BN / 4;
    static_assert(TX * TY == kGemmThreads, "tile shape");
    constexpr int NA = BM * BK / kGemmThreads, NB = BK * BN / kGemmThreads;
    __shared__ T sA[2][BK][BM];
    __shared__ T sB[2][BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    T ra[NA], rb[NB];
    auto load_regs = [&](int p0) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int e = tid + q * kGemmThreads;
            const int i = e % BM, p = e / BM;  // A tile: BM rows x BK cols
            ra[q] = (i0 + i < m && p0 + p < k) ? A[(i0 + i) + (int64_t)(p0 + p) * lda] : T(0);
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = tid + q * kGemmThreads;
            const int pb = e % BK, jb = e / BK;  // B tile: BK rows x BN cols
            rb[q] = (p0 + pb < k && j0 + jb < n) ? B[(int64_t)(p0 + pb) + (j0 + jb) * ldb] : T(0);
        }
    };
    auto store_smem = [&](int s) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int e = tid + q * kGemmThreads;
            sA[s][e / BM][e % BM] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = tid + q * kGemmThreads;
            sB[s][e % BK][e / BK] = rb[q];
        }
    };
    load_regs(0);
    store_smem(0);
    __syncthreads();
    int s = 0;
    for (int p0 = 0; p0 < k; p0 += BK) {
        const bool more = p0 + BK < k;
        if (more) load_regs(p0 + BK);
#pragma unroll
        for (int p = 0; p < BK; ++p) {
            T a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = sA[s][p][tx + TX * q];
                b[q] = sB[s][p][ty + TY * q];
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        if (more) {
            store_smem(s ^ 1);
            __syncthreads();
            s ^= 1;
        }
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int64_t j = j0 + ty + TY * y;
        if (j >= n) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int64_t i = i0 + tx + TX * x;
            if (i < m) C[i + j * ldc] -= acc[x][y];
        }
    }
}


}  // namespace

template <typename T>
int lu_launch_trsm_lunit(cudaStream_t st, int64_t m, int64_t n, const T* L, int64_t ldl, T* B,
                         int64_t ldb) {
    if (m <= 0 || n <= 0) return LU_SUCCESS;
    if (m > LU_MAX_NB) return LU_ERR_UNSUPPORTED;
    const int mp = (int)((m + 31) & ~31);
    const size_t smem16 = sizeof(T) * ((size_t)16 * mp + 32 * 33);
    const size_t smem8 = sizeof(T) * ((size_t)8 * mp + 32 * 33);
    static bool attr[2] = {false, false};
    const int ti = sizeof(T) == 8 ? 0 : 1;
    if (!attr[ti]) {
        LU_CHECK_CUDA(cudaFuncSetAttribute(trsm_lunit_kernel<T, 16>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        LU_CHECK_CUDA(cudaFuncSetAttribute(trsm_lunit_kernel<T, 8>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr[ti] = true;
    }
    LuProfScope prof(st, LU_K_TRSM, sizeof(T) * (2.0 * m * n + 0.5 * m * m), (double)m * m * n);
    if (smem16 <= 64 * 1024) {
        trsm_lunit_kernel<T, 16><<<(unsigned)lu_cdiv(n, 16), kTrsmThreads, smem16, st>>>((int)m, n, L, ldl, B, ldb);
    } else {
        trsm_lunit_kernel<T, 8><<<(unsigned)lu_cdiv(n, 8), kTrsmThreads, smem8, st>>>((int)m, n, L, ldl, B, ldb);
    }
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int lu_launch_gemm_update(cudaStream_t st, int64_t m, int64_t n, int64_t k, const T* A, int64_t lda,
                          const T* B, int64_t ldb, T* C, int64_t ldc) {
    if (m <= 0 || n <= 0 || k <= 0) return LU_SUCCESS;
    LuProfScope prof(st, LU_K_GEMM, sizeof(T) * (2.0 * m * n + (double)m * k + (double)k * n), 2.0 * m * n * k);
    if constexpr (sizeof(T) == 4) {
        if (n <= 16) {
            gemm_update_kernel<T, 256, 16><<<dim3((unsigned)lu_cdiv(m, 256), (unsigned)lu_cdiv(n, 16)), kGemmThreads,
                                              0, st>>>(m, n, (int)k, A, lda, B, ldb, C, ldc);
            LU_CHECK_LAUNCH();
            return LU_SUCCESS;
        }
    }
    if (n <= 32) {
        gemm_update_kernel<T, 128, 32><<<dim3((unsigned)lu_cdiv(m, 128), (unsigned)lu_cdiv(n, 32)), kGemmThreads, 0,
                                          st>>>(m, n, (int)k, A, lda, B, ldb, C, ldc);
    } else {
        if (lu_cdiv(n, 64) > 65535) return LU_ERR_UNSUPPORTED;
        gemm_update_kernel<T, 64, 64><<<dim3((unsigned)lu_cdiv(m, 64), (unsigned)lu_cdiv(n, 64)), kGemmThreads, 0,
                                        st>>>(m, n, (int)k, A, lda, B, ldb, C, ldc);
    }
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template int lu_launch_trsm_lunit<double>(cudaStream_t, int64_t, int64_t, const double*, int64_t,
                                          double*, int64_t);
template int lu_launch_trsm_lunit<float>(cudaStream_t, int64_t, int64_t, const float*, int64_t,
                                         float*, int64_t);
template int lu_launch_gemm_update<double>(cudaStream_t, int64_t, int64_t, int64_t, const double*,
                                           int64_t, const double*, int64_t, double*, int64_t);
template int lu_launch_gemm_update<float>(cudaStream_t, int64_t, int64_t, int64_t, const float*,
                                          int64_t, const float*, int64_t, float*, int64_t);

