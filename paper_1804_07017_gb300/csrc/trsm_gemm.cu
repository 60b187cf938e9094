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
#include "ptx.cuh"

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
    const int64_t nblocks = (n + COLS - 1) / COLS;
    for (int64_t cb = blockIdx.x; cb < nblocks; cb += gridDim.x) {
    const int64_t col0 = cb * COLS;
    const int nc = (int)min((int64_t)COLS, n - col0);
    __syncthreads();
    for (int c = 0; c < COLS; ++c)
        for (int r = tid; r < mp; r += kTrsmThreads) {
            if (c < nc && r < m)
                cp_async_elem<T>(sB + c * mp + r, B + r + (col0 + c) * ldb);
            else
                sB[c * mp + r] = T(0);
        }
    for (int J = 0; J < m; J += 32) {
        const int jb = min(32, m - J);
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += kTrsmThreads) {
            const int i = e & 31, j = e >> 5;
            if (i < jb && j < jb)
                cp_async_elem<T>(sL + j * 33 + i, L + (int64_t)(J + i) + (int64_t)(J + j) * ldl);
            else
                sL[j * 33 + i] = T(0);
        }
        cp_async_wait_all();
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
}


// The same solve as trsm_lunit_kernel (identical operations in identical
// order, so identical results) with the strictly lower triangle of L staged in
// shared memory once, packed by rows (row i at i(i-1)/2), so the 32-row sweep
// makes no global accesses: the panel-width TRSM of the look-ahead step
// (m = nb <= 256) otherwise pays two dependent global round trips per block.
template <typename T, int COLS>
__global__ void __launch_bounds__(kTrsmThreads)
    trsm_lunit_staged_kernel(int m, int64_t n, const T* __restrict__ L, int64_t ldl, T* __restrict__ B,
                             int64_t ldb) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int mp = (m + 31) & ~31;
    T* sB = reinterpret_cast<T*>(smraw);       // [COLS][mp]
    T* sLp = sB + (size_t)COLS * mp;           // packed strictly lower triangle
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t col0 = (int64_t)blockIdx.x * COLS;
    const int nc = (int)min((int64_t)COLS, n - col0);
    // staging by asynchronous element copies, all in flight at once (a load-then-store
    // loop would wait one global round trip per iteration); lanes run down a column
    // of L, so the global reads are coalesced
    for (int j = warp; j < m - 1; j += kTrsmThreads / 32)
        for (int i = j + 1 + lane; i < m; i += 32) cp_async_elem<T>(sLp + i * (i - 1) / 2 + j, L + i + (int64_t)j * ldl);
    for (int c = 0; c < COLS; ++c)
        for (int r = tid; r < mp; r += kTrsmThreads) {
            if (c < nc && r < m)
                cp_async_elem<T>(sB + c * mp + r, B + r + (col0 + c) * ldb);
            else
                sB[c * mp + r] = T(0);
        }
    cp_async_wait_all();
    __syncthreads();
    for (int J = 0; J < m; J += 32) {
        const int jb = min(32, m - J);
        for (int c = warp; c < COLS; c += kTrsmThreads / 32) {
            T v = sB[c * mp + J + lane];
            const int i = J + lane;
            for (int j = 0; j < jb; ++j) {
                const T xj = __shfl_sync(0xffffffffu, v, j);
                if (lane > j && lane < jb) v = fma(-sLp[i * (i - 1) / 2 + J + j], xj, v);
            }
            if (lane < jb) sB[c * mp + J + lane] = v;
        }
        __syncthreads();
        for (int r = J + jb + tid; r < m; r += kTrsmThreads) {
            const T* lr = sLp + r * (r - 1) / 2 + J;
            T l[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) l[j] = (j < jb) ? lr[j] : T(0);
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
        __syncthreads();
    }
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
                       const T* __restrict__ B, int64_t ldb, T* __restrict__ C, int64_t ldc, int64_t r0,
                       int64_t c0, int band) {
    constexpr int TX = BM / 4, TY = BN / 4;
    static_assert(TX * TY == kGemmThreads, "tile shape");
    constexpr int NA = BM * BK / kGemmThreads, NB = BK * BN / kGemmThreads;
    __shared__ T sA[2][BK][BM];
    __shared__ T sB[2][BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    // band > 0 (symmetric updates): a tile whose rows all lie above the band-wide
    // diagonal block of its first column (absolute row r0 + i, column c0 + j) is
    // not needed and is skipped
    if (band > 0 && r0 + i0 + BM <= ((c0 + j0) / band) * band) return;
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



// The same update for a short inner dimension (k <= kStagedK, the recursive
// panel's own RL3): the CTA's whole A (BM x k) and B (k x BN) tiles are copied
// to shared memory asynchronously and its C tile read into registers, all
// issued at once, so the launch pays one global round trip instead of one per
// 16-deep step.  Same thread mapping and the same k-ordered accumulation as
// gemm_update_kernel, so the results are identical.
constexpr int kStagedK = 128;

template <typename T, int BM, int BN>
__global__ void __launch_bounds__(kGemmThreads)
    gemm_update_staged_kernel(int64_t m, int64_t n, int k, const T* __restrict__ A, int64_t lda,
                              const T* __restrict__ B, int64_t ldb, T* __restrict__ C, int64_t ldc) {
    constexpr int TX = BM / 4, TY = BN / 4;
    static_assert(TX * TY == kGemmThreads, "tile shape");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sA = reinterpret_cast<T*>(smraw);  // [k][BM]: sA[p * BM + i] = A(i0 + i, p)
    T* sB = sA + (size_t)k * BM;           // [k][BN + 1]: sB[p * (BN + 1) + j] = B(p, j0 + j)
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    for (int e = tid; e < BM * k; e += kGemmThreads) {
        const int i = e % BM, p = e / BM;
        if (i0 + i < m)
            cp_async_elem<T>(sA + p * BM + i, A + (i0 + i) + (int64_t)p * lda);
        else
            sA[p * BM + i] = T(0);
    }
    for (int e = tid; e < BN * k; e += kGemmThreads) {
        const int p = e % k, j = e / k;
        if (j0 + j < n)
            cp_async_elem<T>(sB + p * (BN + 1) + j, B + p + (j0 + j) * ldb);
        else
            sB[p * (BN + 1) + j] = T(0);
    }
    T cur[4][4];
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int64_t i = i0 + tx + TX * x, j = j0 + ty + TY * y;
            cur[x][y] = (i < m && j < n) ? C[i + j * ldc] : T(0);
        }
    cp_async_wait_all();
    __syncthreads();
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 4
    for (int p = 0; p < k; ++p) {
        T a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = sA[p * BM + tx + TX * q];
            b[q] = sB[p * (BN + 1) + ty + TY * q];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int64_t j = j0 + ty + TY * y;
        if (j >= n) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int64_t i = i0 + tx + TX * x;
            if (i < m) C[i + j * ldc] = cur[x][y] - acc[x][y];
        }
    }
}


// RL2 + RL3 of a narrow node of the recursive panel (w1 <= 32, w2 <= 32) in one
// launch:  U12 := trilu(L11)^{-1} A12,  A22 := A22 - A21 U12.
// Every CTA solves the w1 x w2 block U12 itself, in shared memory, with the
// same operations in the same order as trsm_lunit_kernel (a warp per column,
// lane = row, x_i := fma(-L(i, j), x_j, x_i) for j = 0, 1, ...), then applies
// its BM-row tile of the update with gemm_update_kernel's accumulation order,
// so the results are bit-identical to the two separate launches.  U12 is
// written back over A12 by the last CTA to have read A12 (an arrival counter
// that this CTA resets), so no CTA can read an already solved block.
// Latency: every global read of the CTA -- its A21 tile (asynchronous copies
// into shared memory), its A22 outputs (into registers), L11 and A12 -- is
// issued before the substitution, so the launch pays one round trip.
template <typename T, int BM, int BN>
__global__ void __launch_bounds__(kGemmThreads)
    trsm_gemm_narrow_kernel(int64_t m2, int w2, int w1, const T* __restrict__ L11, T* __restrict__ A12,
                            const T* __restrict__ A21, T* __restrict__ A22, int64_t lda, unsigned* __restrict__ arrivals) {
    constexpr int TX = BM / 4, TY = BN / 4;
    static_assert(TX * TY == kGemmThreads, "tile shape");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sA = reinterpret_cast<T*>(smraw);  // [32][BM]: sA[p * BM + i] = A21(i0 + i, p)
    __shared__ T sL[32 * 33];              // sL[j * 33 + i] = L(i, j)
    __shared__ T sU[32][BN + 1];           // U12, row p = k index
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * BM;
    const int tx = tid % TX, ty = tid / TX;
    // this CTA's A21 tile, all copies in flight
    if (i0 < m2)
        for (int e = tid; e < 32 * BM; e += kGemmThreads) {
            const int i = e % BM, p = e / BM;
            if (i0 + i < m2 && p < w1)
                cp_async_elem<T>(sA + p * BM + i, A21 + (i0 + i) + (int64_t)p * lda);
            else
                sA[p * BM + i] = T(0);
        }
    // its outputs' current values
    T cur[4][4];
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int j = ty + TY * y;
            const int64_t i = i0 + tx + TX * x;
            cur[x][y] = (j < w2 && i < m2) ? A22[i + (int64_t)j * lda] : T(0);
        }
    for (int e = tid; e < 32 * 32; e += kGemmThreads) {
        const int i = e & 31, j = e >> 5;
        sL[j * 33 + i] = (i < w1 && j < w1) ? L11[i + (int64_t)j * lda] : T(0);
    }
    for (int e = tid; e < 32 * BN; e += kGemmThreads) {
        const int i = e & 31, j = e >> 5;
        sU[i][j] = (i < w1 && j < w2) ? A12[i + (int64_t)j * lda] : T(0);
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned old = atomicAdd(arrivals, 1u);
        s_last = old == gridDim.x - 1;
        if (s_last) *arrivals = 0u;
    }
    for (int c = warp; c < BN; c += kGemmThreads / 32) {
        T v = sU[lane][c];
        for (int j = 0; j < w1; ++j) {
            const T xj = __shfl_sync(0xffffffffu, v, j);
            if (lane > j) v = fma(-sL[j * 33 + lane], xj, v);
        }
        if (lane < w1) sU[lane][c] = v;
    }
    cp_async_wait_all();
    __syncthreads();
    if (s_last)
        for (int e = tid; e < w1 * w2; e += kGemmThreads) {
            const int i = e % w1, j = e / w1;
            A12[i + (int64_t)j * lda] = sU[i][j];
        }
    if (i0 >= m2) return;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int p = 0; p < w1; ++p) {
        T a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = sA[p * BM + tx + TX * q];
            b[q] = sU[p][ty + TY * q];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int j = ty + TY * y;
        if (j >= w2) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int64_t i = i0 + tx + TX * x;
            if (i < m2) A22[i + (int64_t)j * lda] = cur[x][y] - acc[x][y];
        }
    }
}

}  // namespace

template <typename T>
int lu_launch_trsm_lunit(cudaStream_t st, int64_t m, int64_t n, const T* L, int64_t ldl, T* B,
                         int64_t ldb, int max_ctas) {
    if (m <= 0 || n <= 0) return LU_SUCCESS;
    if (m > LU_MAX_NB) return LU_ERR_UNSUPPORTED;
    const int mp = (int)((m + 31) & ~31);
    const size_t smem16 = sizeof(T) * ((size_t)16 * mp + 32 * 33);
    const size_t smem8 = sizeof(T) * ((size_t)8 * mp + 32 * 33);
    LU_TRY(lu_func_smem(trsm_lunit_kernel<T, 16>, 200 * 1024));
    LU_TRY(lu_func_smem(trsm_lunit_kernel<T, 8>, 200 * 1024));
    // max_ctas > 0 caps the grid (the CTAs then loop over column blocks), so a wide
    // solve on the low-priority stream leaves SMs to the panel path
    auto grid_of = [&](int64_t blocks) {
        return (unsigned)(max_ctas > 0 ? std::min<int64_t>(blocks, max_ctas) : blocks);
    };
    LuProfScope prof(st, LU_K_TRSM, sizeof(T) * (2.0 * m * n + 0.5 * m * m), (double)m * m * n);
    // stage L in shared memory when the packed triangle and a 16-column block fit and
    // few CTAs share it (the look-ahead and in-panel solves); a wide solve keeps the
    // per-block loads, which many CTAs share through L2
    const size_t staged = sizeof(T) * ((size_t)16 * mp + (size_t)m * (m - 1) / 2);
    if (m > 32 && n <= 512 && staged <= 160 * 1024) {
        LU_TRY(lu_func_smem(trsm_lunit_staged_kernel<T, 16>, 160 * 1024));
        trsm_lunit_staged_kernel<T, 16><<<(unsigned)lu_cdiv(n, 16), kTrsmThreads, staged, st>>>((int)m, n, L, ldl, B,
                                                                                              ldb);
    } else if (smem16 <= 64 * 1024) {
        trsm_lunit_kernel<T, 16><<<grid_of(lu_cdiv(n, 16)), kTrsmThreads, smem16, st>>>((int)m, n, L, ldl, B, ldb);
    } else {
        trsm_lunit_kernel<T, 8><<<grid_of(lu_cdiv(n, 8)), kTrsmThreads, smem8, st>>>((int)m, n, L, ldl, B, ldb);
    }
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int lu_launch_gemm_update(cudaStream_t st, int64_t m, int64_t n, int64_t k, const T* A, int64_t lda,
                          const T* B, int64_t ldb, T* C, int64_t ldc) {
    return lu_launch_gemm_update_band<T>(st, m, n, k, A, lda, B, ldb, C, ldc, 0, 0, 0);
}

template <typename T>
int lu_launch_gemm_update_band(cudaStream_t st, int64_t m, int64_t n, int64_t k, const T* A, int64_t lda,
                               const T* B, int64_t ldb, T* C, int64_t ldc, int64_t r0, int64_t c0, int band) {
    if (m <= 0 || n <= 0 || k <= 0) return LU_SUCCESS;
    LuProfScope prof(st, LU_K_GEMM, sizeof(T) * (2.0 * m * n + (double)m * k + (double)k * n), 2.0 * m * n * k);
    if constexpr (sizeof(T) == 4) {
        if (n <= 16) {
            gemm_update_kernel<T, 256, 16><<<dim3((unsigned)lu_cdiv(m, 256), (unsigned)lu_cdiv(n, 16)), kGemmThreads,
                                              0, st>>>(m, n, (int)k, A, lda, B, ldb, C, ldc, r0, c0, band);
            LU_CHECK_LAUNCH();
            return LU_SUCCESS;
        }
    }
    if constexpr (sizeof(T) == 4) {
        // a short inner dimension (the recursive panel's own updates): one round trip
        if (n > 32 && k <= kStagedK && band == 0 && lu_cdiv(n, 64) <= 65535) {
            const size_t smem = sizeof(T) * ((size_t)k * 64 + (size_t)k * 65);
            LU_TRY(lu_func_smem(gemm_update_staged_kernel<T, 64, 64>, (int)(sizeof(T) * kStagedK * 129)));
            gemm_update_staged_kernel<T, 64, 64><<<dim3((unsigned)lu_cdiv(m, 64), (unsigned)lu_cdiv(n, 64)),
                                                   kGemmThreads, smem, st>>>(m, n, (int)k, A, lda, B, ldb, C, ldc);
            LU_CHECK_LAUNCH();
            return LU_SUCCESS;
        }
    }
    if (n <= 32) {
        gemm_update_kernel<T, 128, 32><<<dim3((unsigned)lu_cdiv(m, 128), (unsigned)lu_cdiv(n, 32)), kGemmThreads, 0,
                                          st>>>(m, n, (int)k, A, lda, B, ldb, C, ldc, r0, c0, band);
    } else {
        if (lu_cdiv(n, 64) > 65535) return LU_ERR_UNSUPPORTED;
        gemm_update_kernel<T, 64, 64><<<dim3((unsigned)lu_cdiv(m, 64), (unsigned)lu_cdiv(n, 64)), kGemmThreads, 0,
                                        st>>>(m, n, (int)k, A, lda, B, ldb, C, ldc, r0, c0, band);
    }
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template int lu_launch_trsm_lunit<double>(cudaStream_t, int64_t, int64_t, const double*, int64_t,
                                          double*, int64_t, int);
template int lu_launch_trsm_lunit<float>(cudaStream_t, int64_t, int64_t, const float*, int64_t,
                                         float*, int64_t, int);
template int lu_launch_gemm_update<double>(cudaStream_t, int64_t, int64_t, int64_t, const double*,
                                           int64_t, const double*, int64_t, double*, int64_t);
template int lu_launch_gemm_update_band<double>(cudaStream_t, int64_t, int64_t, int64_t, const double*, int64_t,
                                                const double*, int64_t, double*, int64_t, int64_t, int64_t, int);
template int lu_launch_gemm_update_band<float>(cudaStream_t, int64_t, int64_t, int64_t, const float*, int64_t,
                                               const float*, int64_t, float*, int64_t, int64_t, int64_t, int);
template int lu_launch_gemm_update<float>(cudaStream_t, int64_t, int64_t, int64_t, const float*,
                                          int64_t, const float*, int64_t, float*, int64_t);


template <typename T, int BM, int BN>
static int launch_narrow(cudaStream_t st, int64_t m2, int64_t w2, int64_t w1, const T* L11, T* A12, const T* A21,
                         T* A22, int64_t lda, unsigned* arrivals) {
    const size_t smem = sizeof(T) * 32 * BM;
    LU_TRY(lu_func_smem(trsm_gemm_narrow_kernel<T, BM, BN>, (int)smem));
    const unsigned gx = (unsigned)std::max<int64_t>(1, lu_cdiv(m2, BM));
    trsm_gemm_narrow_kernel<T, BM, BN><<<gx, kGemmThreads, smem, st>>>(m2, (int)w2, (int)w1, L11, A12, A21, A22, lda,
                                                                      arrivals);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int lu_launch_trsm_gemm_narrow(cudaStream_t st, int64_t m2, int64_t w2, int64_t w1, const T* L11, T* A12,
                               const T* A21, T* A22, int64_t lda, unsigned* arrivals) {
    if (w2 <= 0 || w1 <= 0) return LU_SUCCESS;
    if (w1 > 32 || w2 > 32) return LU_ERR_UNSUPPORTED;
    LuProfScope prof(st, LU_K_TRSM, sizeof(T) * (2.0 * m2 * w2 + (double)m2 * w1 + 2.0 * w1 * w2),
                     (double)w1 * w1 * w2 + 2.0 * m2 * w2 * w1);
    if (w2 <= 16) return launch_narrow<T, 256, 16>(st, m2, w2, w1, L11, A12, A21, A22, lda, arrivals);
    return launch_narrow<T, 128, 32>(st, m2, w2, w1, L11, A12, A21, A22, lda, arrivals);
}

template int lu_launch_trsm_gemm_narrow<double>(cudaStream_t, int64_t, int64_t, int64_t, const double*, double*,
                                                const double*, double*, int64_t, unsigned*);
template int lu_launch_trsm_gemm_narrow<float>(cudaStream_t, int64_t, int64_t, int64_t, const float*, float*,
                                               const float*, float*, int64_t, unsigned*);
