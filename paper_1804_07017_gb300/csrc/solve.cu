// Solves with the getrf factors (the getrs that pairs with getrf; not part of
// the paper, whose experiments stop at the factorization).
//
//   perm_from_ipiv:  the row order of P A from the sequential interchanges
//   permute_rows:    X := P B (gather)
//   trsv_blocked:    X := L^{-1} X (unit lower) or X := U^{-1} X, for up to 16
//                    right-hand sides per launch.  Rows are cut into 128-row
//                    blocks; a CTA takes the next block in dependency order
//                    from an atomic ticket, accumulates the contributions of
//                    already-solved blocks as they are published (a monotone
//                    "done" counter read with acquire loads and a bounded
//                    wait), solves its diagonal block in shared memory and
//                    publishes.  Tickets make the wait graph acyclic whatever
//                    the CTA scheduling order.
#include "internal.h"
#include "profile.h"

namespace {

// The interchanges are sequential, so one lane applies them to the row order
// held in shared memory while the warp prefetches the next 32 pivots.
__global__ void perm_from_ipiv_smem_kernel(int n, const int32_t* __restrict__ ipiv, int32_t* __restrict__ perm) {
    extern __shared__ int32_t order[];  // [n]
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = i;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int pv = (k0 + lane < n) ? ipiv[k0 + lane] - 1 : 0;
            const int cnt = min(32, n - k0);
            for (int t = 0; t < cnt; ++t) {
                const int p = __shfl_sync(0xffffffffu, pv, t);
                if (lane == 0) {
                    const int a = order[k0 + t];
                    order[k0 + t] = order[p];
                    order[p] = a;
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = order[i];
}

__global__ void perm_from_ipiv_global_kernel(int64_t n, const int32_t* __restrict__ ipiv, int32_t* __restrict__ perm) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm[i] = (int32_t)i;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int64_t k = 0; k < n; ++k) {
            const int64_t p = ipiv[k] - 1;
            const int32_t a = perm[k];
            perm[k] = perm[p];
            perm[p] = a;
        }
    }
}

template <typename T>
__global__ void permute_rows_kernel(int64_t n, int64_t nrhs, const int32_t* __restrict__ perm,
                                    const T* __restrict__ B, int64_t ldb, T* __restrict__ X, int64_t ldx) {
    const int64_t total = n * nrhs;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, c = e / n;
        X[i + c * ldx] = B[(int64_t)perm[i] + c * ldb];
    }
}

constexpr int kBS = 128;       // rows per block
constexpr int kNR = 16;        // right-hand sides per launch
constexpr int kTrsvThreads = 256;

template <typename T, bool LOWER>
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_blocked_kernel(int64_t n, int nrhs, const T* __restrict__ LU, int64_t lda, T* __restrict__ X,
                        int64_t ldx, LuSync* __restrict__ sync) {
    __shared__ T sX[kNR][kBS];
    __shared__ T sPart[kNR][kBS];
    __shared__ int s_chain, s_ready, s_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = (int)((n + kBS - 1) / kBS);
    if (tid == 0) s_chain = (int)atomicAdd(&sync->ticket, 1u);
    __syncthreads();
    const int chain = s_chain;  // position in dependency order
    const int blk = LOWER ? chain : nblk - 1 - chain;
    const int64_t r0 = (int64_t)blk * kBS;
    const int rows = (int)min((int64_t)kBS, n - r0);
    const int r = tid % kBS, h = tid / kBS;  // two halves split the columns of each source block
    T acc[kNR];
#pragma unroll
    for (int c = 0; c < kNR; ++c) acc[c] = T(0);

    int processed = 0;
    bool ok = true;
    while (processed < chain) {
        if (tid == 0) {
            unsigned v;
            uint64_t t0 = 0;
            unsigned spins = 0;
            int flag = 1;
            while ((int)(v = lu_ld_acquire(&sync->arrive)) <= processed) {
                if (((++spins) & 255u) == 0) {
                    if (lu_ld_acquire_s32(&sync->error) != 0) { flag = 0; break; }
                    uint64_t t = lu_globaltimer();
                    if (t0 == 0) t0 = t;
                    else if (t - t0 > LU_WAIT_NS) {
                        atomicExch(&sync->error, LU_ERR_TIMEOUT);
                        flag = 0;
                        break;
                    }
                }
            }
            s_ready = (int)v;
            s_flag = flag;
        }
        __syncthreads();
        if (!s_flag) { ok = false; break; }
        const int ready = min(s_ready, chain);
        for (int q = processed; q < ready; ++q) {
            const int I = LOWER ? q : nblk - 1 - q;
            const int64_t c0 = (int64_t)I * kBS;
            const int cols = (int)min((int64_t)kBS, n - c0);
            if (r < rows) {
                for (int j = h; j < cols; j += 2) {
                    const T l = LU[(r0 + r) + (c0 + j) * lda];
#pragma unroll
                    for (int c = 0; c < kNR; ++c)
                        if (c < nrhs) acc[c] = fma(l, __ldcg(&X[(c0 + j) + c * ldx]), acc[c]);
                }
            }
        }
        processed = ready;
        __syncthreads();
    }
    if (!ok) return;
    // combine the two halves: sX = rhs - contributions
    if (h == 1) {
#pragma unroll
        for (int c = 0; c < kNR; ++c) sPart[c][r] = acc[c];
    }
    __syncthreads();
    if (h == 0) {
#pragma unroll
        for (int c = 0; c < kNR; ++c)
            sX[c][r] = (r < rows && c < nrhs) ? X[(r0 + r) + c * ldx] - (acc[c] + sPart[c][r]) : T(0);
    }
    __syncthreads();
    // diagonal block, in 32-row sub-blocks
    const int nsub = (rows + 31) / 32;
    for (int sidx = 0; sidx < nsub; ++sidx) {
        const int sb = LOWER ? sidx : nsub - 1 - sidx;
        const int j0 = sb * 32;
        const int jb = min(32, rows - j0);
        // warp-level substitution inside the 32x32 sub-block, one rhs per warp
        for (int c = warp; c < nrhs; c += kTrsvThreads / 32) {
            T v = (lane < jb) ? sX[c][j0 + lane] : T(0);
            if (LOWER) {
                for (int j = 0; j < jb; ++j) {
                    const T xj = __shfl_sync(0xffffffffu, v, j);
                    if (lane > j && lane < jb) v = fma(-LU[(r0 + j0 + lane) + (r0 + j0 + j) * lda], xj, v);
                }
            } else {
                for (int j = jb - 1; j >= 0; --j) {
                    if (lane == j) v = v / LU[(r0 + j0 + j) + (r0 + j0 + j) * lda];
                    const T xj = __shfl_sync(0xffffffffu, v, j);
                    if (lane < j) v = fma(-LU[(r0 + j0 + lane) + (r0 + j0 + j) * lda], xj, v);
                }
            }
            if (lane < jb) sX[c][j0 + lane] = v;
        }
        __syncthreads();
        // update the other rows of this block that come later in the sweep
        const int lo = LOWER ? j0 + jb : 0;
        const int hi = LOWER ? rows : j0;
        for (int e = tid; e < (hi - lo) * nrhs; e += kTrsvThreads) {
            const int rr = lo + e % (hi - lo), c = e / (hi - lo);
            T a = T(0);
            for (int j = 0; j < jb; ++j) a = fma(LU[(r0 + rr) + (r0 + j0 + j) * lda], sX[c][j0 + j], a);
            sX[c][rr] -= a;
        }
        __syncthreads();
    }
    for (int e = tid; e < rows * nrhs; e += kTrsvThreads) {
        const int rr = e % rows, c = e / rows;
        X[(r0 + rr) + c * ldx] = sX[c][rr];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) lu_st_release(&sync->arrive, (unsigned)(chain + 1));
}

__global__ void finish_info_kernel(const LuSync* __restrict__ s, int32_t* __restrict__ info) {
    const int e = s->error;
    info[0] = e != 0 ? e : s->info;
}

}  // namespace

template <typename T>
int lu_launch_perm_from_ipiv(cudaStream_t st, int64_t n, const int32_t* ipiv, int32_t* perm) {
    if (n <= 0) return LU_SUCCESS;
    const size_t smem = sizeof(int32_t) * (size_t)n;
    LuProfScope prof(st, LU_K_SOLVE, 8.0 * n, 0.0);
    if (smem <= 200 * 1024) {
        static bool attr = false;
        if (!attr) {
            LU_CHECK_CUDA(cudaFuncSetAttribute(perm_from_ipiv_smem_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
            attr = true;
        }
        perm_from_ipiv_smem_kernel<<<1, 256, smem, st>>>((int)n, ipiv, perm);
    } else {
        perm_from_ipiv_global_kernel<<<1, 256, 0, st>>>(n, ipiv, perm);
    }
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int lu_launch_permute_rows(cudaStream_t st, int64_t n, int64_t nrhs, const int32_t* perm, const T* B,
                           int64_t ldb, T* X, int64_t ldx) {
    if (n <= 0 || nrhs <= 0) return LU_SUCCESS;
    const int64_t total = n * nrhs;
    const unsigned blocks = (unsigned)std::min<int64_t>(lu_cdiv(total, 256), 4096);
    LuProfScope prof(st, LU_K_SOLVE, 2.0 * n * nrhs * sizeof(T) + 4.0 * n, 0.0);
    permute_rows_kernel<T><<<blocks, 256, 0, st>>>(n, nrhs, perm, B, ldb, X, ldx);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int lu_launch_trsv_blocked(lu_context* c, cudaStream_t st, bool lower_unit, int64_t n, int64_t nrhs,
                           const T* LU, int64_t lda, T* X, int64_t ldx) {
    if (n <= 0 || nrhs <= 0) return LU_SUCCESS;
    const int nblk = (int)lu_cdiv(n, kBS);
    for (int64_t c0 = 0; c0 < nrhs; c0 += kNR) {
        const int nr = (int)std::min<int64_t>(kNR, nrhs - c0);
        // reset the ticket and the done counter (the error word is kept: sticky)
        LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[1].arrive, 0, sizeof(unsigned) * 2, st));
        LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[1].ticket, 0, sizeof(unsigned), st));
        LuProfScope prof(st, LU_K_SOLVE, sizeof(T) * (0.5 * n * n + 2.0 * n * nr), (double)n * n * nr);
        if (lower_unit)
            trsv_blocked_kernel<T, true><<<nblk, kTrsvThreads, 0, st>>>(n, nr, LU, lda, X + c0 * ldx, ldx, &c->sync[1]);
        else
            trsv_blocked_kernel<T, false><<<nblk, kTrsvThreads, 0, st>>>(n, nr, LU, lda, X + c0 * ldx, ldx, &c->sync[1]);
        LU_CHECK_LAUNCH();
    }
    return LU_SUCCESS;
}

int lu_launch_finish_info(cudaStream_t st, const LuSync* s, int32_t* info) {
    LuProfScope prof(st, LU_K_OTHER, 16.0, 0.0);
    finish_info_kernel<<<1, 1, 0, st>>>(s, info);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template int lu_launch_perm_from_ipiv<double>(cudaStream_t, int64_t, const int32_t*, int32_t*);
template int lu_launch_perm_from_ipiv<float>(cudaStream_t, int64_t, const int32_t*, int32_t*);
template int lu_launch_permute_rows<double>(cudaStream_t, int64_t, int64_t, const int32_t*, const double*,
                                            int64_t, double*, int64_t);
template int lu_launch_permute_rows<float>(cudaStream_t, int64_t, int64_t, const int32_t*, const float*,
                                           int64_t, float*, int64_t);
template int lu_launch_trsv_blocked<double>(lu_context*, cudaStream_t, bool, int64_t, int64_t,
                                            const double*, int64_t, double*, int64_t);
template int lu_launch_trsv_blocked<float>(lu_context*, cudaStream_t, bool, int64_t, int64_t,
                                           const float*, int64_t, float*, int64_t);
