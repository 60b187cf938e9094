// Solves with the getrf factors (the getrs that pairs with getrf; not part of
// the paper, whose experiments stop at the factorization).
//
//   perm_from_ipiv:  the row order of P A from the sequential interchanges
//   permute_rows:    X := P B (gather)
//   trsv_blocked:    X := L^{-1} X (unit lower) or X := U^{-1} X, for up to 16
//                    right-hand sides per launch.  Rows are cut into 128-row
//                    (FP32) / 64-row (FP64) blocks; a CTA takes the next block in dependency order
//                    from an atomic ticket, accumulates the contributions of
//                    already-solved blocks as they are published (a monotone
//                    "done" counter read with acquire loads and a bounded
//                    wait), solves its diagonal block in shared memory and
//                    publishes.  Tickets make the wait graph acyclic whatever
//                    the CTA scheduling order.
#include <cudaTypedefs.h>

#include <atomic>

#include "internal.h"
#include "ptx.cuh"
#include "profile.h"

namespace {

// The row order held in shared memory, updated 32 interchanges at a time by one
// warp: after interchanges k0 .. k0+31 in order, position x holds the entry that
// sigma_k0(sigma_k0+1(...sigma_k0+31(x))) held (sigma_k swaps k and ipiv[k]), so
// lane i follows that chain for position k0+i and, when interchange k0+i is the
// first of the 32 to reach its target below them, for that target; the warp
// then gathers all those positions at once.  The result equals applying the
// interchanges one by one.
__global__ void perm_from_ipiv_smem_kernel(int n, const int32_t* __restrict__ ipiv, int32_t* __restrict__ perm) {
    extern __shared__ int32_t order[];  // [n]
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = i;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        // the pivots of the next two chunks are loaded ahead, so their latency overlaps
        // the current chunk's work
        int pa = (lane < n) ? ipiv[lane] - 1 : 0;
        int pb = (32 + lane < n) ? ipiv[32 + lane] - 1 : 0;
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int cnt = min(32, n - k0);
            const int pcur = pa;
            pa = pb;
            pb = (k0 + 64 + lane < n) ? ipiv[k0 + 64 + lane] - 1 : 0;
            // past the last pivot, interchange k0+i with itself (no move)
            const int pv = (lane < cnt) ? pcur : k0 + lane;
            const int xr = k0 + lane;
            const bool is_t = lane < cnt && pv >= k0 + cnt;
            const unsigned same = __match_any_sync(0xffffffffu, is_t ? pv : -1 - lane);
            const bool first = is_t && (__ffs(same) - 1 == lane);
            // both chains at once, all 32 steps unrolled (the pivots come by shuffles that
            // do not depend on the chains)
            int src_r = xr, src_t = first ? pv : xr;
#pragma unroll
            for (int q = 31; q >= 0; --q) {
                const int pq = __shfl_sync(0xffffffffu, pv, q);
                const int b = k0 + q;
                src_r = (src_r == b) ? pq : ((src_r == pq) ? b : src_r);
                src_t = (src_t == b) ? pq : ((src_t == pq) ? b : src_t);
            }
            const int v_r = (lane < cnt) ? order[src_r] : 0;
            const int v_t = first ? order[src_t] : 0;
            __syncwarp();
            if (lane < cnt) order[xr] = v_r;
            if (first) order[pv] = v_t;
            __syncwarp();
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

constexpr int kNR = 16;        // right-hand sides per launch
constexpr int kTrsvThreads = 256;

template <typename T>
struct TrsvCfg {
    static constexpr int BS = sizeof(T) == 4 ? 128 : 64;  // rows per block
    static constexpr int kSplit = kTrsvThreads / BS;      // threads sharing one row of a source block
    static constexpr int kTile = BS * BS;                 // elements of one staged tile
    // diagonal tile + two off-diagonal tiles (column-major, dense), rhs block, partial sums,
    // mbarriers and 1 KB of alignment slack
    static constexpr size_t smem = sizeof(T) * (3 * (size_t)kTile + 2 * (size_t)kNR * BS) + 64 + 1024;
};

template <typename T>
struct TrsvPlainCfg {
    static constexpr int BS = sizeof(T) == 4 ? 128 : 64;  // rows per block
    static constexpr int kSplit = kTrsvThreads / BS;      // threads sharing one row of a source block
    static constexpr size_t smem = sizeof(T) * ((size_t)BS * (BS + 1) + 2 * (size_t)kNR * BS);
};

// Fallback for factors whose leading dimension TMA cannot address (not a
// multiple of 16 bytes).  One CTA per BS-row block, taken in dependency order
// from an atomic ticket.  The diagonal block is staged in shared memory before the CTA waits for its
// predecessors, so the critical path per block is: observe the predecessor's
// "done" count, add that block's contribution, run the register-resident
// substitution of the diagonal block, publish.
template <typename T, bool LOWER>
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_plain_kernel(int64_t n, int nrhs, const T* __restrict__ LU, int64_t lda, T* __restrict__ X,
                        int64_t ldx, LuSync* __restrict__ sync) {
    using C = TrsvPlainCfg<T>;
    constexpr int BS = C::BS;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sD = reinterpret_cast<T*>(smraw);   // [BS][BS+1], sD[i*(BS+1) + j] = LU(r0+i, r0+j)
    T* sX = sD + BS * (BS + 1);            // [kNR][BS]
    T* sPart = sX + kNR * BS;              // [kNR][BS]
    __shared__ int s_chain, s_ready, s_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = (int)((n + BS - 1) / BS);
    if (tid == 0) s_chain = (int)atomicAdd(&sync->ticket, 1u);
    __syncthreads();
    const int chain = s_chain;  // position in dependency order
    const int blk = LOWER ? chain : nblk - 1 - chain;
    const int64_t r0 = (int64_t)blk * BS;
    const int rows = (int)min((int64_t)BS, n - r0);
    // stage the diagonal block (independent of every other block)
    for (int e = tid; e < BS * BS; e += kTrsvThreads) {
        const int i = e % BS, j = e / BS;
        sD[i * (BS + 1) + j] = (i < rows && j < rows) ? LU[(r0 + i) + (r0 + j) * lda] : T(0);
    }
    const int r = tid % BS, h = tid / BS;
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
            const int64_t c0 = (int64_t)I * BS;
            const int cols = (int)min((int64_t)BS, n - c0);
            if (r < rows) {
                const T* lrow = LU + (r0 + r) + c0 * lda;
                const T* xs = X + c0;
                if (nrhs == 1) {
#pragma unroll 4
                    for (int j = h; j < cols; j += C::kSplit) acc[0] = fma(lrow[j * lda], __ldcg(xs + j), acc[0]);
                } else {
                    for (int j = h; j < cols; j += C::kSplit) {
                        const T l = lrow[j * lda];
#pragma unroll
                        for (int c = 0; c < kNR; ++c)
                            if (c < nrhs) acc[c] = fma(l, __ldcg(xs + j + c * ldx), acc[c]);
                    }
                }
            }
        }
        processed = ready;
        __syncthreads();
    }
    if (!ok) return;
    // combine the kSplit partial sums: sX = rhs - contributions
    for (int hh = 1; hh < C::kSplit; ++hh) {
        if (h == hh) {
#pragma unroll
            for (int c = 0; c < kNR; ++c) sPart[c * BS + r] = (hh == 1 ? T(0) : sPart[c * BS + r]) + acc[c];
        }
        __syncthreads();
    }
    if (h == 0) {
#pragma unroll
        for (int c = 0; c < kNR; ++c)
            sX[c * BS + r] = (r < rows && c < nrhs)
                                 ? X[(r0 + r) + c * ldx] - (acc[c] + (C::kSplit > 1 ? sPart[c * BS + r] : T(0)))
                                 : T(0);
    }
    __syncthreads();
    // register-resident substitution of the diagonal block: lane holds rows lane + 32 q
    constexpr int RQ = BS / 32;
    for (int c = warp; c < nrhs; c += kTrsvThreads / 32) {
        T v[RQ];
#pragma unroll
        for (int q = 0; q < RQ; ++q) v[q] = sX[c * BS + lane + 32 * q];
        if (LOWER) {
#pragma unroll
            for (int q0 = 0; q0 < RQ; ++q0) {
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = q0 * 32 + jj;
                    const T xj = __shfl_sync(0xffffffffu, v[q0], jj);
#pragma unroll
                    for (int q = q0; q < RQ; ++q) {
                        const int i = lane + 32 * q;
                        if (i > j) v[q] = fma(-sD[i * (BS + 1) + j], xj, v[q]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int q0 = RQ - 1; q0 >= 0; --q0) {
                for (int jj = 31; jj >= 0; --jj) {
                    const int j = q0 * 32 + jj;
                    if (lane == jj && j < rows) v[q0] = v[q0] / sD[j * (BS + 1) + j];
                    const T xj = __shfl_sync(0xffffffffu, v[q0], jj);
#pragma unroll
                    for (int q = 0; q <= q0; ++q) {
                        const int i = lane + 32 * q;
                        if (i < j) v[q] = fma(-sD[i * (BS + 1) + j], xj, v[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RQ; ++q) sX[c * BS + lane + 32 * q] = v[q];
    }
    __syncthreads();
    for (int e = tid; e < rows * nrhs; e += kTrsvThreads) {
        const int rr = e % rows, c = e / rows;
        X[(r0 + rr) + c * ldx] = sX[c * BS + rr];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) lu_st_release(&sync->arrive, (unsigned)(chain + 1));
}

// One CTA per BS-row block, taken in dependency order from an atomic ticket.
// The diagonal tile and the off-diagonal tiles L(blk, I) are brought into
// shared memory by TMA (2-D tiled cp.async.bulk.tensor, double-buffered, one
// tile ahead of use), so the critical path per block is: observe the
// predecessor's "done" count, read its solution block (L2), add its
// contribution from shared memory, run the register-resident substitution of
// the diagonal block, publish.
//
// INV = true: the diagonal tile is the precomputed inverse of the diagonal
// block (trinv_diag_kernel), loaded from the tensor map tmD, and the block's
// solve is one dense product x_blk = inv(D) (b_blk - sum of contributions)
// instead of a BS-step substitution.
template <typename T, bool LOWER, bool INV>
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_tma_kernel(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmD, int64_t n,
                    int nrhs, T* __restrict__ X, int64_t ldx, LuSync* __restrict__ sync) {
    using C = TrsvCfg<T>;
    constexpr int BS = C::BS;
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    T* sD = reinterpret_cast<T*>(base);           // [BS cols][BS rows] diagonal tile
    T* sT = sD + C::kTile;                        // two off-diagonal tiles
    T* sX = sT + 2 * C::kTile;                    // [kNR][BS]
    T* sPart = sX + kNR * BS;                     // [kNR][BS]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sPart + kNR * BS);  // [0] diag, [1],[2] tiles
    __shared__ int s_chain, s_ready, s_flag;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nblk = (int)((n + BS - 1) / BS);
    const uint32_t tile_bytes = (uint32_t)(C::kTile * sizeof(T));
    if (tid == 0) {
        s_chain = (int)atomicAdd(&sync->ticket, 1u);
        s_abort = 0;
        for (int b = 0; b < 3; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int chain = s_chain;  // position in dependency order
    const int blk = LOWER ? chain : nblk - 1 - chain;
    const int64_t r0 = (int64_t)blk * BS;
    const int rows = (int)min((int64_t)BS, n - r0);
    auto src_block = [&](int q) { return LOWER ? q : nblk - 1 - q; };
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], tile_bytes);
        if (INV)
            tma_load_2d(sD, &tmD, &bars[0], 0, (LOWER ? blk : nblk + blk) * BS);
        else
            tma_load_2d(sD, &tmL, &bars[0], (int)r0, (int)r0);
        if (chain > 0) {
            mbar_arrive_expect_tx(&bars[1], tile_bytes);
            tma_load_2d(sT, &tmL, &bars[1], (int)r0, src_block(0) * BS);
        }
    }
    const int r = tid % BS, h = tid / BS;
    T acc[kNR];
#pragma unroll
    for (int c = 0; c < kNR; ++c) acc[c] = T(0);

    int processed = 0;
    int issued = chain > 0 ? 1 : 0;  // off-diagonal tiles requested so far (uniform across the CTA)
    int consumed = 0;                // tiles whose arrival was observed
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
            // prefetch the next tile into the other buffer (its previous tile was consumed)
            if (q + 1 < chain) issued = q + 2;
            if (tid == 0 && q + 1 < chain) {
                const int nb = (q + 1) & 1;
                mbar_arrive_expect_tx(&bars[1 + nb], tile_bytes);
                tma_load_2d(sT + nb * C::kTile, &tmL, &bars[1 + nb], (int)r0, src_block(q + 1) * BS);
            }
            const int I = src_block(q);
            const int64_t c0 = (int64_t)I * BS;
            const int cols = (int)min((int64_t)BS, n - c0);
            for (int e = tid; e < kNR * BS; e += kTrsvThreads) {
                const int c = e / BS, j = e % BS;
                sX[e] = (c < nrhs && j < cols) ? __ldcg(&X[(c0 + j) + c * ldx]) : T(0);
            }
            if (!mbar_wait(&bars[1 + (q & 1)], (q >> 1) & 1, &s_abort)) { ok = false; }
            __syncthreads();
            if (!ok || s_abort) { ok = false; break; }
            consumed = q + 1;
            const T* tile = sT + (q & 1) * C::kTile;
            if (nrhs == 1) {
#pragma unroll 8
                for (int j = h; j < BS; j += C::kSplit) acc[0] = fma(tile[j * BS + r], sX[j], acc[0]);
            } else {
                for (int j = h; j < BS; j += C::kSplit) {
                    const T l = tile[j * BS + r];
#pragma unroll
                    for (int c = 0; c < kNR; ++c)
                        if (c < nrhs) acc[c] = fma(l, sX[c * BS + j], acc[c]);
                }
            }
            __syncthreads();
        }
        if (!ok) break;
        processed = ready;
    }
    if (ok && !mbar_wait(&bars[0], 0, &s_abort)) ok = false;
    __syncthreads();
    if (!ok || s_abort) {
        if (tid == 0) {
            atomicExch(&sync->error, LU_ERR_TIMEOUT);
            // drain (bounded) the tile copies this CTA issued, so none lands after it exits
            for (int q = consumed; q < issued; ++q) {
                const uint64_t t0 = lu_globaltimer();
                while (!mbar_try_wait(&bars[1 + (q & 1)], (q >> 1) & 1))
                    if (lu_globaltimer() - t0 > LU_MBAR_WAIT_NS) break;
            }
            const uint64_t t0 = lu_globaltimer();
            while (!mbar_try_wait(&bars[0], 0))
                if (lu_globaltimer() - t0 > LU_MBAR_WAIT_NS) break;
        }
        return;
    }
    // combine the kSplit partial sums: sX = rhs - contributions
    for (int hh = 1; hh < C::kSplit; ++hh) {
        if (h == hh) {
#pragma unroll
            for (int c = 0; c < kNR; ++c) sPart[c * BS + r] = (hh == 1 ? T(0) : sPart[c * BS + r]) + acc[c];
        }
        __syncthreads();
    }
    if (h == 0) {
#pragma unroll
        for (int c = 0; c < kNR; ++c)
            sX[c * BS + r] = (r < rows && c < nrhs)
                                 ? X[(r0 + r) + c * ldx] - (acc[c] + (C::kSplit > 1 ? sPart[c * BS + r] : T(0)))
                                 : T(0);
    }
    __syncthreads();
    if (INV) {
        // x = inv(D) sX: thread (r, h) sums columns j = h, h + kSplit, ... of row r
#pragma unroll
        for (int c = 0; c < kNR; ++c) acc[c] = T(0);
        if (nrhs == 1) {
#pragma unroll 8
            for (int j = h; j < BS; j += C::kSplit) acc[0] = fma(sD[j * BS + r], sX[j], acc[0]);
        } else {
            for (int j = h; j < BS; j += C::kSplit) {
                const T d = sD[j * BS + r];
#pragma unroll
                for (int c = 0; c < kNR; ++c)
                    if (c < nrhs) acc[c] = fma(d, sX[c * BS + j], acc[c]);
            }
        }
        for (int hh = 1; hh < C::kSplit; ++hh) {
            if (h == hh) {
#pragma unroll
                for (int c = 0; c < kNR; ++c) sPart[c * BS + r] = (hh == 1 ? T(0) : sPart[c * BS + r]) + acc[c];
            }
            __syncthreads();
        }
        if (h == 0) {
#pragma unroll
            for (int c = 0; c < kNR; ++c)
                if (r < rows && c < nrhs) X[(r0 + r) + c * ldx] = acc[c] + (C::kSplit > 1 ? sPart[c * BS + r] : T(0));
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) lu_st_release(&sync->arrive, (unsigned)(chain + 1));
        return;
    }
    // register-resident substitution of the diagonal block: lane holds rows lane + 32 q
    constexpr int RQ = BS / 32;
    for (int c = warp; c < nrhs; c += kTrsvThreads / 32) {
        T v[RQ];
#pragma unroll
        for (int q = 0; q < RQ; ++q) v[q] = sX[c * BS + lane + 32 * q];
        if (LOWER) {
#pragma unroll
            for (int q0 = 0; q0 < RQ; ++q0) {
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = q0 * 32 + jj;
                    const T xj = __shfl_sync(0xffffffffu, v[q0], jj);
#pragma unroll
                    for (int q = q0; q < RQ; ++q) {
                        const int i = lane + 32 * q;
                        if (i > j) v[q] = fma(-sD[j * BS + i], xj, v[q]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int q0 = RQ - 1; q0 >= 0; --q0) {
                for (int jj = 31; jj >= 0; --jj) {
                    const int j = q0 * 32 + jj;
                    if (lane == jj && j < rows) v[q0] = v[q0] / sD[j * BS + j];
                    const T xj = __shfl_sync(0xffffffffu, v[q0], jj);
#pragma unroll
                    for (int q = 0; q <= q0; ++q) {
                        const int i = lane + 32 * q;
                        if (i < j) v[q] = fma(-sD[j * BS + i], xj, v[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RQ; ++q) sX[c * BS + lane + 32 * q] = v[q];
    }
    __syncthreads();
    for (int e = tid; e < rows * nrhs; e += kTrsvThreads) {
        const int rr = e % rows, c = e / rows;
        X[(r0 + rr) + c * ldx] = sX[c * BS + rr];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) lu_st_release(&sync->arrive, (unsigned)(chain + 1));
}


// FP32, one right-hand side, inverse diagonal blocks: the solved values travel
// as 64-bit words {tag << 32 | value bits} in a side buffer xt, written by the
// block's CTA once and polled element by element by its successors, so one
// global round trip carries both the "ready" signal and the data (no counter,
// no fence).  tag is unique per launch, so words of earlier launches never
// match.  Each CTA prefetches its own right-hand side before it waits.  Per
// predecessor: poll its BS words (a bounded spin per thread), add its tile's
// contribution (tiles staged by TMA one ahead), then x = inv(D) (b - sum).
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <bool LOWER>
__global__ void __launch_bounds__(kTrsvThreads)
    trsv_tag_kernel(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmD, int64_t n,
                    float* __restrict__ X, unsigned long long* __restrict__ xt, unsigned tag,
                    LuSync* __restrict__ sync) {
    using C = TrsvCfg<float>;
    constexpr int BS = C::BS;
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    float* sD = reinterpret_cast<float*>(base);   // [BS cols][BS rows] inverse of the diagonal block
    float* sT = sD + C::kTile;                    // two off-diagonal tiles
    float* sX = sT + 2 * C::kTile;                // [BS]
    float* sPart = sX + kNR * BS;                 // [BS]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sPart + kNR * BS);
    __shared__ int s_chain;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x;
    const int nblk = (int)((n + BS - 1) / BS);
    const uint32_t tile_bytes = (uint32_t)(C::kTile * sizeof(float));
    if (tid == 0) {
        s_chain = (int)atomicAdd(&sync->ticket, 1u);
        s_abort = 0;
        for (int b = 0; b < 3; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int chain = s_chain;
    const int blk = LOWER ? chain : nblk - 1 - chain;
    const int64_t r0 = (int64_t)blk * BS;
    const int rows = (int)min((int64_t)BS, n - r0);
    auto src_block = [&](int q) { return LOWER ? q : nblk - 1 - q; };
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], tile_bytes);
        tma_load_2d(sD, &tmD, &bars[0], 0, (LOWER ? blk : nblk + blk) * BS);
        if (chain > 0) {
            mbar_arrive_expect_tx(&bars[1], tile_bytes);
            tma_load_2d(sT, &tmL, &bars[1], (int)r0, src_block(0) * BS);
        }
    }
    const int r = tid % BS, h = tid / BS;
    const float b = (h == 0 && r < rows) ? X[r0 + r] : 0.f;
    float acc = 0.f;
    int issued = chain > 0 ? 1 : 0, consumed = 0;
    bool ok = true;
    for (int q = 0; q < chain && ok; ++q) {
        if (tid == 0 && q + 1 < chain) {
            const int nb = (q + 1) & 1;
            mbar_arrive_expect_tx(&bars[1 + nb], tile_bytes);
            tma_load_2d(sT + nb * C::kTile, &tmL, &bars[1 + nb], (int)r0, src_block(q + 1) * BS);
            issued = q + 2;
        }
        const int64_t c0 = (int64_t)src_block(q) * BS;
        const int cols = (int)min((int64_t)BS, n - c0);
        if (h == 0) {
            float v = 0.f;
            if (r < cols) {
                const unsigned long long* w = xt + c0 + r;
                unsigned long long x = ld_relaxed_u64(w);
                if ((unsigned)(x >> 32) != tag) {
                    const uint64_t t0 = lu_globaltimer();
                    unsigned spins = 0;
                    while ((unsigned)((x = ld_relaxed_u64(w)) >> 32) != tag) {
                        if ((++spins & 255u) == 0) {
                            if (s_abort) break;
                            if (lu_globaltimer() - t0 > LU_WAIT_NS) {
                                s_abort = 1;
                                break;
                            }
                        }
                    }
                }
                v = __uint_as_float((unsigned)x);
            }
            sX[r] = v;
        }
        if (!mbar_wait(&bars[1 + (q & 1)], (q >> 1) & 1, &s_abort)) ok = false;
        __syncthreads();
        if (!ok || s_abort) {
            ok = false;
            break;
        }
        consumed = q + 1;
        const float* tile = sT + (q & 1) * C::kTile;
#pragma unroll 8
        for (int j = h; j < BS; j += C::kSplit) acc = fmaf(tile[j * BS + r], sX[j], acc);
        __syncthreads();
    }
    if (ok && !mbar_wait(&bars[0], 0, &s_abort)) ok = false;
    __syncthreads();
    if (!ok || s_abort) {
        if (tid == 0) {
            atomicExch(&sync->error, LU_ERR_TIMEOUT);
            for (int q = consumed; q < issued; ++q) {
                const uint64_t t0 = lu_globaltimer();
                while (!mbar_try_wait(&bars[1 + (q & 1)], (q >> 1) & 1))
                    if (lu_globaltimer() - t0 > LU_MBAR_WAIT_NS) break;
            }
            const uint64_t t0 = lu_globaltimer();
            while (!mbar_try_wait(&bars[0], 0))
                if (lu_globaltimer() - t0 > LU_MBAR_WAIT_NS) break;
        }
        return;
    }
    // rhs - contributions, then x = inv(D) (rhs - contributions)
    if (h == 1) sPart[r] = acc;
    __syncthreads();
    if (h == 0) sX[r] = (r < rows) ? b - (acc + sPart[r]) : 0.f;
    __syncthreads();
    float y = 0.f;
#pragma unroll 8
    for (int j = h; j < BS; j += C::kSplit) y = fmaf(sD[j * BS + r], sX[j], y);
    if (h == 1) sPart[r] = y;
    __syncthreads();
    if (h == 0 && r < rows) {
        const float x = y + sPart[r];
        X[r0 + r] = x;
        const unsigned long long word = ((unsigned long long)tag << 32) | __float_as_uint(x);
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(xt + r0 + r), "l"(word) : "memory");
    }
}

// Inverses of the diagonal blocks of the factors: blockIdx.y = 0 gives
// inv(L_bb) (unit lower), 1 gives inv(U_bb), for block b = blockIdx.x, into
// tile (blockIdx.y * nblk + b) of D (BS x BS, column-major, ld BS; zero outside
// the block's rows x rows).  Thread j computes column j of the inverse by
// substitution against the unit vector e_j, in lock step with the other
// columns (terms with k < j vanish), so the block stays in shared memory and
// no thread waits for another.
template <typename T>
__global__ void __launch_bounds__(TrsvCfg<T>::BS)
    trinv_diag_kernel(int64_t n, const T* __restrict__ LU, int64_t lda, T* __restrict__ D) {
    constexpr int BS = TrsvCfg<T>::BS;
    extern __shared__ unsigned char smraw[];
    T* sL = reinterpret_cast<T*>(smraw);  // [BS][BS + 1] row-major block
    T* sX = sL + BS * (BS + 1);           // [BS][BS + 1] inverse, row-major
    const int nblk = (int)((n + BS - 1) / BS);
    const int b = blockIdx.x, upper = blockIdx.y, j = threadIdx.x;
    const int64_t r0 = (int64_t)b * BS;
    const int rows = (int)min((int64_t)BS, n - r0);
    for (int c = 0; c < rows; ++c)
        if (j < rows) sL[j * (BS + 1) + c] = LU[(r0 + j) + (r0 + c) * lda];
    __syncthreads();
    if (!upper) {
        for (int i = 0; i < rows; ++i) {
            T s = (i == j) ? T(1) : T(0);
            for (int k = 0; k < i; ++k) s = fma(-sL[i * (BS + 1) + k], sX[k * (BS + 1) + j], s);
            sX[i * (BS + 1) + j] = s;
        }
    } else {
        for (int i = rows - 1; i >= 0; --i) {
            T s = (i == j) ? T(1) : T(0);
            for (int k = i + 1; k < rows; ++k) s = fma(-sL[i * (BS + 1) + k], sX[k * (BS + 1) + j], s);
            sX[i * (BS + 1) + j] = s / sL[i * (BS + 1) + i];
        }
    }
    __syncthreads();
    T* tile = D + (int64_t)(upper * nblk + b) * BS * BS;
    for (int i = 0; i < BS; ++i) tile[(int64_t)j * BS + i] = (i < rows && j < rows) ? sX[i * (BS + 1) + j] : T(0);
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
        LU_TRY(lu_func_smem(perm_from_ipiv_smem_kernel, 200 * 1024));
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
static int trsv_plain(lu_context* c, cudaStream_t st, bool lower_unit, int64_t n, int64_t nrhs, const T* LU,
                      int64_t lda, T* X, int64_t ldx) {
    using C = TrsvPlainCfg<T>;
    const int nblk = (int)lu_cdiv(n, C::BS);
    LU_TRY(lu_func_smem(trsv_plain_kernel<T, true>, (int)C::smem));
    LU_TRY(lu_func_smem(trsv_plain_kernel<T, false>, (int)C::smem));
    for (int64_t c0 = 0; c0 < nrhs; c0 += kNR) {
        const int nr = (int)std::min<int64_t>(kNR, nrhs - c0);
        LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[1].arrive, 0, sizeof(unsigned) * 2, st));
        LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[1].ticket, 0, sizeof(unsigned), st));
        LuProfScope prof(st, LU_K_SOLVE, sizeof(T) * (0.5 * n * n + 2.0 * n * nr), (double)n * n * nr);
        if (lower_unit)
            trsv_plain_kernel<T, true><<<nblk, kTrsvThreads, C::smem, st>>>(n, nr, LU, lda, X + c0 * ldx, ldx,
                                                                            &c->sync[1]);
        else
            trsv_plain_kernel<T, false><<<nblk, kTrsvThreads, C::smem, st>>>(n, nr, LU, lda, X + c0 * ldx, ldx,
                                                                             &c->sync[1]);
        LU_CHECK_LAUNCH();
    }
    return LU_SUCCESS;
}

// 2-D tensor map over the n x n factor matrix (column-major: rows innermost),
// one box = one BS x BS tile.
template <typename T>
static int make_factor_map(CUtensorMap* map, const T* LU, int64_t n, int64_t lda) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        LU_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) return LU_ERR_CUDA;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    using C = TrsvCfg<T>;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(lda * sizeof(T))};
    cuuint32_t box[2] = {(cuuint32_t)C::BS, (cuuint32_t)C::BS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                     const_cast<T*>(LU), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        lu_set_error_string("cuTensorMapEncodeTiled failed (triangular solve)", __FILE__, __LINE__);
        return LU_ERR_CUDA;
    }
    return LU_SUCCESS;
}

// Tensor map over the 2 * nblk inverse tiles (a BS x (2 nblk BS) column-major matrix).
template <typename T>
static int make_inverse_map(CUtensorMap* map, const T* D, int64_t nblk) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        LU_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) return LU_ERR_CUDA;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    using C = TrsvCfg<T>;
    cuuint64_t dims[2] = {(cuuint64_t)C::BS, (cuuint64_t)(2 * nblk * C::BS)};
    cuuint64_t strides[1] = {(cuuint64_t)(C::BS * sizeof(T))};
    cuuint32_t box[2] = {(cuuint32_t)C::BS, (cuuint32_t)C::BS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                     const_cast<T*>(D), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        lu_set_error_string("cuTensorMapEncodeTiled failed (inverse diagonal blocks)", __FILE__, __LINE__);
        return LU_ERR_CUDA;
    }
    return LU_SUCCESS;
}

template <typename T>
size_t lu_trinv_bytes(int64_t n) {
    using C = TrsvCfg<T>;
    return (size_t)2 * lu_cdiv(n, C::BS) * C::BS * C::BS * sizeof(T);
}

template <typename T>
int lu_launch_trinv_diag(cudaStream_t st, int64_t n, const T* LU, int64_t lda, T* D) {
    if (n <= 0) return LU_SUCCESS;
    using C = TrsvCfg<T>;
    const size_t smem = sizeof(T) * 2 * (size_t)C::BS * (C::BS + 1);
    LU_TRY(lu_func_smem(trinv_diag_kernel<T>, (int)smem));
    const int nblk = (int)lu_cdiv(n, C::BS);
    LuProfScope prof(st, LU_K_SOLVE, sizeof(T) * (2.0 * n * C::BS + 2.0 * nblk * C::BS * C::BS),
                     (double)nblk * C::BS * C::BS * C::BS / 3.0);
    trinv_diag_kernel<T><<<dim3(nblk, 2), C::BS, smem, st>>>(n, LU, lda, D);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int lu_launch_trsv_blocked(lu_context* c, cudaStream_t st, bool lower_unit, int64_t n, int64_t nrhs, const T* LU,
                           int64_t lda, T* X, int64_t ldx, const T* Dinv, unsigned long long* xtag) {
    if (n <= 0 || nrhs <= 0) return LU_SUCCESS;
    using C = TrsvCfg<T>;
    const int nblk = (int)lu_cdiv(n, C::BS);
    // TMA needs a 16-byte aligned base and a leading dimension that is a multiple of 16 bytes
    if ((reinterpret_cast<uintptr_t>(LU) & 15) != 0 || (lda * sizeof(T)) % 16 != 0)
        return trsv_plain(c, st, lower_unit, n, nrhs, LU, lda, X, ldx);
    CUtensorMap map, dmap;
    LU_TRY(make_factor_map<T>(&map, LU, n, lda));
    const bool inv = Dinv != nullptr && (reinterpret_cast<uintptr_t>(Dinv) & 15) == 0;
    if (inv)
        LU_TRY(make_inverse_map<T>(&dmap, Dinv, nblk));
    else
        dmap = map;
    LU_TRY(lu_func_smem(trsv_tma_kernel<T, true, false>, (int)C::smem));
    LU_TRY(lu_func_smem(trsv_tma_kernel<T, false, false>, (int)C::smem));
    LU_TRY(lu_func_smem(trsv_tma_kernel<T, true, true>, (int)C::smem));
    LU_TRY(lu_func_smem(trsv_tma_kernel<T, false, true>, (int)C::smem));
    if constexpr (sizeof(T) == 4) {
        if (inv && xtag && nrhs == 1) {
            LU_TRY(lu_func_smem(trsv_tag_kernel<true>, (int)C::smem));
            LU_TRY(lu_func_smem(trsv_tag_kernel<false>, (int)C::smem));
            // tags are unique per launch within the process (0 is never used: the buffer starts zeroed)
            static std::atomic<unsigned> next_tag{1};
            unsigned tag = next_tag.fetch_add(1);
            if (tag == 0) tag = next_tag.fetch_add(1);
            LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[1].ticket, 0, sizeof(unsigned), st));
            LuProfScope prof(st, LU_K_SOLVE, sizeof(T) * (0.5 * n * n + 2.0 * n), (double)n * n);
            auto fn = lower_unit ? trsv_tag_kernel<true> : trsv_tag_kernel<false>;
            fn<<<nblk, kTrsvThreads, C::smem, st>>>(map, dmap, n, (float*)X, xtag, tag, &c->sync[1]);
            LU_CHECK_LAUNCH();
            return LU_SUCCESS;
        }
    }
    for (int64_t c0 = 0; c0 < nrhs; c0 += kNR) {
        const int nr = (int)std::min<int64_t>(kNR, nrhs - c0);
        // reset the ticket and the done counter (the error word is kept: sticky)
        LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[1].arrive, 0, sizeof(unsigned) * 2, st));
        LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[1].ticket, 0, sizeof(unsigned), st));
        LuProfScope prof(st, LU_K_SOLVE, sizeof(T) * (0.5 * n * n + 2.0 * n * nr), (double)n * n * nr);
        auto fn = lower_unit ? (inv ? trsv_tma_kernel<T, true, true> : trsv_tma_kernel<T, true, false>)
                             : (inv ? trsv_tma_kernel<T, false, true> : trsv_tma_kernel<T, false, false>);
        fn<<<nblk, kTrsvThreads, C::smem, st>>>(map, dmap, n, nr, X + c0 * ldx, ldx, &c->sync[1]);
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
template size_t lu_trinv_bytes<double>(int64_t);
template size_t lu_trinv_bytes<float>(int64_t);
template int lu_launch_trinv_diag<double>(cudaStream_t, int64_t, const double*, int64_t, double*);
template int lu_launch_trinv_diag<float>(cudaStream_t, int64_t, const float*, int64_t, float*);
template int lu_launch_trsv_blocked<double>(lu_context*, cudaStream_t, bool, int64_t, int64_t,
                                            const double*, int64_t, double*, int64_t, const double*,
                                            unsigned long long*);
template int lu_launch_trsv_blocked<float>(lu_context*, cudaStream_t, bool, int64_t, int64_t,
                                           const float*, int64_t, float*, int64_t, const float*,
                                           unsigned long long*);
