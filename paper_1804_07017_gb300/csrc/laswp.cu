// Row interchanges (the laswp of the getrf decomposition, Sec. 3.4).
//
// The K = k2 - k1 sequential interchanges of one panel are first turned into a
// "plan": the list of (destination row, source row) moves whose simultaneous
// application equals applying the interchanges in order.  The plan touches
// the K rows of the panel block plus at most K distinct rows below it.  The
// apply kernel then moves, column by column, every planned element through
// shared memory (all reads of a column before any write), so a column's K
// contiguous block rows are read and written with coalesced accesses.
//
// Plan layout (int32): [0] = count, [1 .. 1+2K) = destination rows,
// [1+2K .. 1+4K) = source rows.  Entries 0..K-1 are the panel block rows in
// order (identity moves included), entries K.. are the rows below the block.
#include "internal.h"
#include "profile.h"

namespace {

constexpr int kPlanThreads = 256;

// The source row of a tracked position x is found by running the K
// transpositions (k1 + q <-> t[q]) backwards from x: after the interchanges in
// order, position x holds the row that sigma_0(sigma_1(...sigma_{K-1}(x)))
// held before.  Every position's chain is independent, so one thread follows
// one position; the rows below the block that receive a different row (first
// occurrence of each target) are then compacted in order by one warp.
__global__ void __launch_bounds__(kPlanThreads)
    laswp_plan_kernel(const int32_t* __restrict__ ipiv, int64_t k1, int K, int32_t* __restrict__ plan) {
    extern __shared__ int32_t sm[];
    int32_t* t = sm;            // [K] target row (absolute, 0-based) of interchange i
    int32_t* g = t + K;         // [K] 1 if interchange i's target is a first occurrence below the block that moves
    int32_t* gsrc = g + K;      // [K] the row that target position ends up holding
    int32_t* rank = gsrc + K;   // [K] exclusive prefix of g
    __shared__ int s_total;
    const int tid = threadIdx.x;
    const int kb = (int)k1, ke = (int)(k1 + K);
    for (int i = tid; i < K; i += kPlanThreads) t[i] = ipiv[k1 + i] - 1;
    __syncthreads();
    auto chain = [&](int x) {
#pragma unroll 1
        for (int q = K - 1; q >= 0; --q) {
            const int p = t[q], b = kb + q;
            x = (x == b) ? p : ((x == p) ? b : x);
        }
        return x;
    };
    int32_t* dst = plan + 1;
    int32_t* src = plan + 1 + 2 * K;
    for (int i = tid; i < K; i += kPlanThreads) {
        dst[i] = kb + i;
        src[i] = chain(kb + i);
        int flag = 0, s = 0;
        const int ti = t[i];
        if (ti >= ke) {
            bool first = true;
            for (int q = 0; q < i; ++q)
                if (t[q] == ti) {
                    first = false;
                    break;
                }
            if (first) {
                s = chain(ti);
                flag = s != ti;
            }
        }
        g[i] = flag;
        gsrc[i] = s;
    }
    __syncthreads();
    if (tid < 32) {
        int run = 0;
        for (int base = 0; base < K; base += 32) {
            const int i = base + tid;
            const int f = (i < K) ? g[i] : 0;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (i < K) rank[i] = run + __popc(bal & ((1u << tid) - 1u));
            run += __popc(bal);
        }
        if (tid == 0) s_total = run;
    }
    __syncthreads();
    for (int i = tid; i < K; i += kPlanThreads)
        if (g[i]) {
            dst[K + rank[i]] = t[i];
            src[K + rank[i]] = gsrc[i];
        }
    if (tid == 0) plan[0] = K + s_total;
}

constexpr int kApplyThreads = 256;  // 8 warps, one column per warp at a time

template <typename T>
__global__ void __launch_bounds__(kApplyThreads)
    laswp_apply_kernel(T* __restrict__ A, int64_t lda, int64_t c1, int64_t n1, int64_t c2, int64_t n2,
                       const int32_t* __restrict__ plan, int K) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* buf = reinterpret_cast<T*>(smraw) + (size_t)warp * 2 * K;
    const int cnt = plan[0];
    const int32_t* dst = plan + 1;
    const int32_t* src = plan + 1 + 2 * K;
    const int64_t ncols = n1 + n2;
    for (int64_t q = (int64_t)blockIdx.x * (kApplyThreads / 32) + warp; q < ncols;
         q += (int64_t)gridDim.x * (kApplyThreads / 32)) {
        const int64_t col = (q < n1) ? c1 + q : c2 + (q - n1);
        T* a = A + col * lda;
        for (int e = lane; e < cnt; e += 32) buf[e] = a[src[e]];
        __syncwarp();
        for (int e = lane; e < cnt; e += 32) a[dst[e]] = buf[e];
        __syncwarp();
    }
}

}  // namespace

int lu_launch_laswp_plan(cudaStream_t st, const int32_t* ipiv, int64_t k1, int64_t k2, int32_t* plan) {
    const int K = (int)(k2 - k1);
    if (K <= 0) return LU_SUCCESS;
    size_t smem = sizeof(int32_t) * 4 * (size_t)K;
    LU_TRY(lu_func_smem(laswp_plan_kernel, sizeof(int32_t) * 4 * LU_MAX_NB));
    LuProfScope prof(st, LU_K_LASWP, 20.0 * K, 0.0);
    laswp_plan_kernel<<<1, kPlanThreads, smem, st>>>(ipiv, k1, K, plan);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int lu_launch_laswp_apply(cudaStream_t st, T* A, int64_t lda, int64_t c1, int64_t n1, int64_t c2,
                          int64_t n2, const int32_t* plan, int64_t K, int num_sms, int max_blocks) {
    if (K <= 0 || n1 + n2 <= 0) return LU_SUCCESS;
    const int warps = kApplyThreads / 32;
    size_t smem = sizeof(T) * 2 * (size_t)K * warps;
    LU_TRY(lu_func_smem(laswp_apply_kernel<T>, (int)(sizeof(T) * 2 * LU_MAX_NB * warps)));
    int64_t blocks = lu_cdiv(n1 + n2, warps);
    blocks = std::min<int64_t>(blocks, max_blocks > 0 ? (int64_t)max_blocks : (int64_t)std::max(num_sms, 1) * 8);
    LuProfScope prof(st, LU_K_LASWP, 2.0 * 2.0 * K * (double)(n1 + n2) * sizeof(T), 0.0);
    laswp_apply_kernel<T><<<(unsigned)blocks, kApplyThreads, smem, st>>>(A, lda, c1, n1, c2, n2, plan, (int)K);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template int lu_launch_laswp_apply<double>(cudaStream_t, double*, int64_t, int64_t, int64_t, int64_t,
                                           int64_t, const int32_t*, int64_t, int, int);
template int lu_launch_laswp_apply<float>(cudaStream_t, float*, int64_t, int64_t, int64_t, int64_t,
                                          int64_t, const int32_t*, int64_t, int, int);
