// Panel-factorization leaf on one thread-block cluster with pushed messages
// (RL1 of LU_blk, Sec. 3: the unblocked LU with partial pivoting of a w-column
// block of the panel).
//
// The leaf's m rows are split across the C <= 16 CTAs of one cluster (256 or
// 512 threads each, every thread holding RQ rows); each CTA keeps its R x w
// block in shared memory and the SB columns of the current sub-block in
// registers (SB = 8 for FP32).  Per column jj:
//   1. every CTA reduces its local pivot candidate (redux.sync first maximum:
//      largest |a|, then smallest row) and PUSHES a message -- the candidate's
//      whole leaf row, its ordering key and its row index -- into every CTA's
//      shared memory with st.async, the pushes shared by all its warps; the
//      owner of row jj pushes that row too.  Each st.async completes
//      transaction bytes on the receiving CTA's mbarrier, so a CTA learns that
//      all C candidates have arrived by a local (bounded) wait: no cluster
//      barrier and no remote loads per column;
//   2. every CTA picks the pivot (first maximum over the C keys) from its own
//      shared memory, swaps rows jj and p where it owns them, scales column jj
//      (by the reciprocal of the pivot where that is representable, else by
//      division) and applies the rank-1 update to the register columns,
//      fusing the next column's candidate search into the update.  The
//      eliminated column then goes back to shared memory and the register
//      columns shift down by one, so the column loop is not unrolled.
// After SB columns the block is right-looking at the sub-block level: the
// CTA holding rows c0..c0+SB-1 computes U12 = L11^-1 A12 for the remaining
// leaf columns and pushes it to all CTAs, which apply the rank-SB update
// A22 -= L21 U12 from shared memory.  Messages are double-buffered by column
// parity; a CTA can run at most one column ahead of any other, because column
// jj+1 needs every CTA's jj+1 candidate, so a buffer is never overwritten
// before it has been read.  After the last column the leaf's interchanges are
// applied to the other columns of the enclosing panel.
#include <cooperative_groups.h>

#include <climits>
#include <cstdio>
#include <cstdlib>
#include <limits>

#include "internal.h"
#include "profile.h"
#include "ptx.cuh"

namespace cg = cooperative_groups;

namespace {

// Threads per CTA: a template parameter NT (256 beside the tensor-core update, 512
// where the leaf may fill an SM).  Registers per thread: 256 x 72 beside a 320 x 144
// tensor-core update CTA fills one SM's 64 K.
#ifndef LU_PF_PUSH_MAXREG
#define LU_PF_PUSH_MAXREG 72
#endif
constexpr int kMaxC = LU_PF_MAX_CTAS_CLUSTER;  // message slots per buffer
constexpr int kMaxPrev = 32;                   // widest preceding sibling folded into a leaf's prologue

// Ordering key of a pivot candidate: |a| as an unsigned integer plus one (IEEE
// order of non-negative values is the integer order of their bits); NaN and
// "no candidate" are 0 and carry row INT_MAX, so a NaN is never chosen.
template <typename T>
struct PivKey;
template <>
struct PivKey<float> {
    typedef uint32_t K;
    static __device__ __forceinline__ K of(float a) {
        const float v = fabsf(a);
        return (v != v) ? 0u : __float_as_uint(v) + 1u;
    }
    // first maximum over the warp: largest key, then the smallest row holding it
    static __device__ __forceinline__ void warp_best(K& k, int& i) {
        const K km = __reduce_max_sync(0xffffffffu, k);
        const unsigned im = __reduce_min_sync(0xffffffffu, k == km ? (unsigned)i : 0x7fffffffu);
        k = km;
        i = (int)im;
    }
};
template <>
struct PivKey<double> {
    typedef unsigned long long K;
    static __device__ __forceinline__ K of(double a) {
        const double v = fabs(a);
        return (v != v) ? 0ull : (unsigned long long)__double_as_longlong(v) + 1ull;
    }
    static __device__ __forceinline__ void warp_best(K& k, int& i) {
        const unsigned hi = (unsigned)(k >> 32), lo = (unsigned)k;
        const unsigned hm = __reduce_max_sync(0xffffffffu, hi);
        const unsigned lm = __reduce_max_sync(0xffffffffu, hi == hm ? lo : 0u);
        const K km = ((K)hm << 32) | lm;
        const unsigned im = __reduce_min_sync(0xffffffffu, k == km ? (unsigned)i : 0x7fffffffu);
        k = km;
        i = (int)im;
    }
};

// Register sub-block width: at most 32 registers of row data per thread.
template <typename T, int RQ>
constexpr int sub_block() {
    return (int)(32 * 4 / (RQ * sizeof(T))) >= 8 ? 8 : (int)(32 * 4 / (RQ * sizeof(T)));
}

template <typename T, int W>
struct MsgLayout {
    typedef typename PivKey<T>::K K;
    static constexpr int row_bytes = W * (int)sizeof(T);
    static constexpr int key_off = row_bytes;
    static constexpr int idx_off = row_bytes + (int)sizeof(K);
    static constexpr int bytes = (idx_off + 4 + 15) / 16 * 16;
    static constexpr int chunks = bytes / 16;
    static constexpr int jchunks = row_bytes / 16;
};

// 32-bit word `w` of element data laid out as consecutive T values.
template <typename T>
__device__ __forceinline__ uint32_t elem_word(const T* p, int w);
template <>
__device__ __forceinline__ uint32_t elem_word<float>(const float* p, int w) {
    return __float_as_uint(p[w]);
}
template <>
__device__ __forceinline__ uint32_t elem_word<double>(const double* p, int w) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(p[w >> 1]);
    return (w & 1) ? (uint32_t)(b >> 32) : (uint32_t)b;
}

__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// 16 bytes into CTA `rank`'s shared memory at the address that `laddr` has in
// this CTA; completes 16 transaction bytes on that CTA's mbarrier `lbar`.
__device__ __forceinline__ void push16(uint32_t laddr, uint32_t lbar, int rank, uint32_t a, uint32_t b, uint32_t c,
                                       uint32_t d) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     mapa_u32(laddr, rank)),
                 "r"(a), "r"(b), "r"(c), "r"(d), "r"(mapa_u32(lbar, rank))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_cta(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for one phase; on expiry records LU_ERR_TIMEOUT and marks the
// thread failed, after which it no longer waits (it still sends every message
// so that no CTA leaves the protocol early).
__device__ __forceinline__ void leaf_wait(uint32_t bar, uint32_t parity, LuSync* sync, bool& failed) {
    if (failed || mbar_try_cluster(bar, parity)) return;
    const uint64_t t0 = lu_globaltimer();
    unsigned spins = 0;
    while (!mbar_try_cluster(bar, parity)) {
        if ((++spins & 63u) == 0 && lu_globaltimer() - t0 > LU_WAIT_NS) {
            atomicExch(&sync->error, LU_ERR_TIMEOUT);
            failed = true;
            return;
        }
    }
}

template <typename T, int W, int RQ, int NT>
struct PushSmem {
    static constexpr int SB = sub_block<T, RQ>();
    static constexpr size_t msg = 2ull * kMaxC * MsgLayout<T, W>::bytes;
    static constexpr size_t jrow = 2ull * W * sizeof(T);
    static constexpr size_t su = (size_t)SB * W * sizeof(T);
    static constexpr size_t block = (size_t)NT * RQ * (W + 1) * sizeof(T);
    static constexpr size_t total = msg + jrow + su + block + 16;
};


// Prologue of a leaf that follows a sibling leaf: the sibling's rank-kprev
// update of this leaf's rows, A(r, c) -= sum_k L(r, k) U12(k, c), with the
// multipliers L(r, k) in the kprev columns left of the leaf and U12 staged in
// sU (kprev x (W+1)); the same k-ordered FMA accumulation followed by one
// subtraction as the separate update kernel.  Kept out of line so that its
// registers do not add to the column loop's.
template <typename T, int W, int RQ, int NT>
__device__ __noinline__ void leaf_prologue(const T* __restrict__ A, int64_t lda, int row0, int nrows, int w,
                                           int kprev, T* __restrict__ sA, const T* __restrict__ sU) {
    constexpr int WP = W + 1;
    constexpr int KC = 8;  // multipliers per round; the next round's are loaded during this one
#pragma unroll 1
    for (int q = 0; q < RQ; ++q) {
        const int r = threadIdx.x + NT * q;
        if (r >= nrows) continue;
        const T* lrow = A + (int64_t)(row0 + r) - (int64_t)kprev * lda;  // L(r, 0)
        T acc[W];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = T(0);
        T lc[KC], ln[KC];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) lc[kk] = (kk < kprev) ? lrow[(int64_t)kk * lda] : T(0);
#pragma unroll 1
        for (int k0 = 0; k0 < kprev; k0 += KC) {
#pragma unroll
            for (int kk = 0; kk < KC; ++kk)
                ln[kk] = (k0 + KC + kk < kprev) ? lrow[(int64_t)(k0 + KC + kk) * lda] : T(0);
#pragma unroll
            for (int kk = 0; kk < KC; ++kk)
                if (k0 + kk < kprev)
#pragma unroll
                    for (int c = 0; c < W; ++c) acc[c] = fma(lc[kk], sU[(k0 + kk) * (W + 1) + c], acc[c]);
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) lc[kk] = ln[kk];
        }
#pragma unroll
        for (int c = 0; c < W; ++c)
            if (c < w) sA[r * WP + c] -= acc[c];
    }
}

template <typename T, int W, int RQ, int NT>
__global__ void __maxnreg__(LU_PF_PUSH_MAXREG)
    pf_leaf_push_kernel(T* __restrict__ A, int64_t lda, int m, int w, int left_cols, int right_cols,
                        int32_t* __restrict__ ipiv, int ipiv_add, LuSync* __restrict__ sync, int sib, int kprev) {
    typedef PivKey<T> PK;
    typedef typename PK::K K;
    typedef MsgLayout<T, W> ML;
    constexpr int SB = PushSmem<T, W, RQ, NT>::SB;
    constexpr int R = NT * RQ;
    constexpr int WP = W + 1;
    constexpr int UCH = (int)(SB * W * sizeof(T) / 16);
    static_assert(W % SB == 0 && W <= 32 && (W * sizeof(T)) % 16 == 0, "leaf shape");

    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* msg = smem_raw;                                                   // [2][kMaxC][ML::bytes]
    T* jrow = reinterpret_cast<T*>(smem_raw + PushSmem<T, W, RQ, NT>::msg);              // [2][W]
    T* su = jrow + 2 * W;                                                            // [SB][W]
    T* sA = su + SB * W;                                                             // [R][WP]
    __shared__ __align__(8) uint64_t bars[3];
    __shared__ K red_k[NT / 32];
    __shared__ int red_i[NT / 32];
    __shared__ int s_piv[W];
    __shared__ int s_info;
    __shared__ int s_dst[2 * W], s_src[2 * W], s_cnt;
    __shared__ T sU0[kMaxPrev][W + 1];  // U12 of the preceding sibling leaf (prologue)

    const int C = (int)cluster.num_blocks();
    const int g = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = g * R;
    const int nrows = max(0, min(R, m - row0));
    const uint32_t bar0 = smem_u32(&bars[0]);
    const uint32_t col_bytes = (uint32_t)(C * ML::bytes + ML::row_bytes);
    const uint32_t u_bytes = (uint32_t)(SB * W * sizeof(T));
    const int nsb = (w + SB - 1) / SB;
    bool failed = false;

    if (tid == 0) {
        for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_cta(bar0, col_bytes);
        if (w > 1) mbar_expect_cta(bar0 + 8, col_bytes);
        if (nsb > 1) mbar_expect_cta(bar0 + 16, u_bytes);
        s_info = 0;
    }
    // the block, column by column, by asynchronous 4/8-byte copies (all in flight at once)
#pragma unroll 1
    for (int c = 0; c < W; ++c)
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const int r = tid + NT * q;
            if (r < nrows) {
                if (c < w)
                    cp_async_elem<T>(sA + r * WP + c, A + (int64_t)(row0 + r) + (int64_t)c * lda);
                else
                    sA[r * WP + c] = T(0);
            }
        }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
    // U12 of the preceding sibling leaf: rows -kprev..-1 of this leaf's columns
    for (int e = tid; e < kprev * w; e += NT) {
        const int k = e % kprev, c = e / kprev;
        sU0[k][c] = A[(int64_t)(k - kprev) + (int64_t)c * lda];
    }
    // every CTA's barriers are initialised before anyone pushes
    cluster.sync();
    if (kprev > 0) {
        leaf_prologue<T, W, RQ, NT>(A, lda, row0, nrows, w, kprev, sA, &sU0[0][0]);
        __syncthreads();
    }

    T v[RQ][SB];

    // CTA reduction of (key, row) and the pushes of column jj's messages.
    auto publish = [&](int jj, int cr, int ce, K bk, int bi) {
        PK::warp_best(bk, bi);
        if (lane == 0) {
            red_k[warp] = bk;
            red_i[warp] = bi;
        }
        __syncthreads();
        K ck = (lane < NT / 32) ? red_k[lane] : K(0);
        int ci = (lane < NT / 32) ? red_i[lane] : INT_MAX;
        PK::warp_best(ck, ci);
        const int buf = jj & 1;
        const int lc = (ci != INT_MAX) ? ci - row0 : -1;
        const int lj = jj - row0;
        const bool own_j = jj >= row0 && jj < row0 + nrows;
        // the owners put their register columns (cr .. ce-1) into the shared-memory rows
        if (lc >= 0 && tid == lc % NT) {
            const int oq = lc / NT;
#pragma unroll
            for (int q = 0; q < RQ; ++q)
                if (q == oq)
#pragma unroll
                    for (int k = 0; k < SB; ++k)
                        if (cr + k < ce) sA[lc * WP + cr + k] = v[q][k];
        }
        if (own_j && tid == lj % NT) {
            const int oq = lj / NT;
#pragma unroll
            for (int q = 0; q < RQ; ++q)
                if (q == oq)
#pragma unroll
                    for (int k = 0; k < SB; ++k)
                        if (cr + k < ce) sA[lj * WP + cr + k] = v[q][k];
        }
        // the rows are complete in shared memory; every warp then takes a share of the
        // C x (chunks) pushes, so they leave in one or two rounds instead of one warp's five
        __syncthreads();
        {
            const T* rp = sA + (lc >= 0 ? lc : 0) * WP;
            const uint32_t base = smem_u32(msg) + (uint32_t)((buf * kMaxC + g) * ML::bytes);
            // row chunks carry 4 row words; the last chunk holds the key and the row index
            for (int t = tid; t < C * ML::chunks; t += NT) {
                const int dst = t / ML::chunks, ch = t % ML::chunks;
                uint32_t x0, x1, x2, x3;
                if (ch < ML::jchunks) {
                    x0 = elem_word<T>(rp, 4 * ch);
                    x1 = elem_word<T>(rp, 4 * ch + 1);
                    x2 = elem_word<T>(rp, 4 * ch + 2);
                    x3 = elem_word<T>(rp, 4 * ch + 3);
                } else if (sizeof(K) == 8) {
                    x0 = (uint32_t)ck;
                    x1 = (uint32_t)((unsigned long long)ck >> 32);
                    x2 = (uint32_t)ci;
                    x3 = 0u;
                } else {
                    x0 = (uint32_t)ck;
                    x1 = (uint32_t)ci;
                    x2 = x3 = 0u;
                }
                push16(base + 16 * ch, bar0 + 8 * buf, dst, x0, x1, x2, x3);
            }
        }
        if (own_j) {
            const T* rp = sA + lj * WP;
            const uint32_t base = smem_u32(jrow + buf * W);
            for (int t = tid; t < C * ML::jchunks; t += NT) {
                const int dst = t / ML::jchunks, ch = t % ML::jchunks;
                push16(base + 16 * ch, bar0 + 8 * buf, dst, elem_word<T>(rp, 4 * ch), elem_word<T>(rp, 4 * ch + 1),
                       elem_word<T>(rp, 4 * ch + 2), elem_word<T>(rp, 4 * ch + 3));
            }
        }
    };

    for (int sb = 0; sb < nsb; ++sb) {
        const int c0 = sb * SB;
        const int ce = c0 + SB;
        const int nk = min(SB, w - c0);
        K bk = 0;
        int bi = INT_MAX;
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const int r = tid + NT * q;
#pragma unroll
            for (int k = 0; k < SB; ++k) v[q][k] = (r < nrows) ? sA[r * WP + c0 + k] : T(0);
            if (r < nrows && row0 + r >= c0) {
                const K kk = PK::of(v[q][0]);
                if (kk > bk) {
                    bk = kk;
                    bi = row0 + r;
                }
            }
        }
        publish(c0, c0, ce, bk, bi);
        // The sub-block's columns one after another, in a loop that is not unrolled
        // (one copy of its code, which the instruction cache holds): the current
        // column is always v[.][0].  Once eliminated, a column is final in every row,
        // so it goes back to shared memory and the register columns shift down by one.
#pragma unroll 1
        for (int k = 0; k < nk; ++k) {
            const int jj = c0 + k;
            const int left = SB - k;  // register columns still live: jj .. ce-1
            const int buf = jj & 1;
            leaf_wait(bar0 + 8 * buf, (uint32_t)((jj >> 1) & 1), sync, failed);
            if (tid == 0 && jj + 2 < w) mbar_expect_cta(bar0 + 8 * buf, col_bytes);
            // ---- pivot: first maximum over the C pushed candidates ----
            K ck = 0;
            int ci = INT_MAX;
            if (lane < C) {
                const unsigned char* mp = msg + (buf * kMaxC + lane) * ML::bytes;
                ck = *reinterpret_cast<const K*>(mp + ML::key_off);
                ci = *reinterpret_cast<const int*>(mp + ML::idx_off);
                if (ck == 0) ci = INT_MAX;
            }
            PK::warp_best(ck, ci);
            const int p = (ci == INT_MAX) ? jj : ci;
            const T* jr = jrow + buf * W;
            const T* pr = (ci == INT_MAX) ? jr : reinterpret_cast<const T*>(msg + (buf * kMaxC + ci / R) * ML::bytes);
            if (tid == 0) s_piv[jj] = p;
            // ---- interchange rows jj and p where this CTA holds them ----
            if (p != jj) {
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int pos = side ? p : jj;
                    const T* src = side ? jr : pr;
                    if (pos >= row0 && pos < row0 + nrows) {
                        const int lr = pos - row0;
                        if (warp == (lr % NT) >> 5 && lane < w && (lane < jj || lane >= ce))
                            sA[lr * WP + lane] = src[lane];
                        if (tid == lr % NT) {
                            const int oq = lr / NT;
#pragma unroll
                            for (int q = 0; q < RQ; ++q)
                                if (q == oq)
#pragma unroll
                                    for (int kk = 0; kk < SB; ++kk)
                                        if (kk < left) v[q][kk] = src[jj + kk];
                        }
                    }
                }
            }
            const T piv = pr[jj];
            if (piv == T(0) && tid == 0 && s_info == 0) s_info = jj + 1;
            // multiply by the reciprocal when it is representable (as getf2), else divide
            const bool use_rcp = fabs(piv) >= std::numeric_limits<T>::min();
            const T rpiv = use_rcp ? T(1) / piv : T(0);
            T prv[SB];
#pragma unroll
            for (int kk = 1; kk < SB; ++kk) prv[kk] = (kk < left) ? pr[jj + kk] : T(0);
            // ---- scale column jj, rank-1 update of the register columns ----
            bk = 0;
            bi = INT_MAX;
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                const int r = tid + NT * q;
                const int gr = row0 + r;
                if (r < nrows) {
                    if (gr > jj && piv != T(0)) {
                        const T l = use_rcp ? v[q][0] * rpiv : v[q][0] / piv;
                        v[q][0] = l;
#pragma unroll
                        for (int kk = 1; kk < SB; ++kk)
                            if (kk < left) v[q][kk] = fma(-l, prv[kk], v[q][kk]);
                    }
                    // column jj is final in this row: back to shared memory, shift down
                    sA[r * WP + jj] = v[q][0];
#pragma unroll
                    for (int kk = 0; kk + 1 < SB; ++kk) v[q][kk] = v[q][kk + 1];
                    if (gr > jj && k + 1 < nk) {
                        const K kk = PK::of(v[q][0]);
                        if (kk > bk) {
                            bk = kk;
                            bi = gr;
                        }
                    }
                }
            }
            if (k + 1 < nk) publish(jj + 1, jj + 1, ce, bk, bi);
        }
        if (c0 + SB < w) {
            __syncthreads();
            // ---- U12 := L11^-1 A12 by the CTA holding rows c0..c0+SB-1, pushed to all ----
            const int ug = c0 / R;  // always 0 (R >= W)
            if (g == ug) {
                const int lr0 = c0 - row0;
                if (warp == 0 && lane >= c0 + SB && lane < w) {
                    for (int i = 1; i < SB; ++i) {
                        T acc = sA[(lr0 + i) * WP + lane];
                        for (int kk = 0; kk < i; ++kk)
                            acc = fma(-sA[(lr0 + i) * WP + c0 + kk], sA[(lr0 + kk) * WP + lane], acc);
                        sA[(lr0 + i) * WP + lane] = acc;
                    }
                }
                __syncthreads();
                const uint32_t base = smem_u32(su);
                for (int t = tid; t < C * UCH; t += NT) {
                    const int dst = t / UCH, ch = t % UCH;
                    uint32_t x[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int wd = 4 * ch + e;
                        const int el = (int)(wd * 4 / sizeof(T));
                        const T* rp = sA + (lr0 + el / W) * WP + (el % W);
                        x[e] = elem_word<T>(rp, (int)(wd % (sizeof(T) / 4)));
                    }
                    push16(base + 16 * ch, bar0 + 16, dst, x[0], x[1], x[2], x[3]);
                }
            }
            leaf_wait(bar0 + 16, (uint32_t)(sb & 1), sync, failed);
            if (tid == 0 && c0 + 2 * SB < w) mbar_expect_cta(bar0 + 16, u_bytes);
            // ---- rank-SB update of the remaining leaf columns: A22 -= L21 U12 ----
            // The multipliers L21 of this thread's rows, from shared memory (it wrote them).
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                const int r = tid + NT * q;
#pragma unroll
                for (int kk = 0; kk < SB; ++kk) v[q][kk] = (r < nrows) ? sA[r * WP + c0 + kk] : T(0);
            }
            // Four columns at a time, so that each thread has RQ x 4 independent
            // multiply-add chains in flight (two warps per scheduler cannot hide
            // the latency of one chain per row); every element still takes its SB
            // products in order.  W is a multiple of 4 and c starts at a multiple
            // of SB, so the four columns never pass W.
            for (int cb = c0 + SB; cb < w; cb += 4) {
                T a[RQ][4];
#pragma unroll
                for (int q = 0; q < RQ; ++q) {
                    const int r = tid + NT * q;
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) a[q][cc] = sA[r * WP + cb + cc];
                }
#pragma unroll
                for (int kk = 0; kk < SB; ++kk) {
                    T u[4];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) u[cc] = su[kk * W + cb + cc];
#pragma unroll
                    for (int q = 0; q < RQ; ++q)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) a[q][cc] = fma(-v[q][kk], u[cc], a[q][cc]);
                }
#pragma unroll
                for (int q = 0; q < RQ; ++q) {
                    const int r = tid + NT * q;
                    if (r < nrows && row0 + r >= c0 + SB)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
                            if (cb + cc < w) sA[r * WP + cb + cc] = a[q][cc];
                }
            }
            __syncthreads();
        }
    }
    // No CTA leaves while another may still push into its shared memory: every
    // CTA has received all of its messages once its last wait has passed, so the
    // arrival is signalled here and the wait is taken just before exit.
    asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
    for (int c = 0; c < w; ++c)
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const int r = tid + NT * q;
            if (r < nrows) A[(int64_t)(row0 + r) + (int64_t)c * lda] = sA[r * WP + c];
        }
    if (g == 0) {
        for (int j = tid; j < w; j += NT) ipiv[j] = s_piv[j] + 1 + ipiv_add;
        if (tid == 0 && s_info != 0) atomicCAS(&sync->info, 0, s_info + ipiv_add);
    }
    const int other = left_cols + right_cols;
    if (other > 0) {
        // ---- the leaf's interchanges on the other columns of the panel ----
        // Plan: positions 0..w-1 (leaf rows) and the distinct targets below them.  After
        // the leaf's interchanges in order, position x holds the row that
        // sigma_0(sigma_1(...sigma_{w-1}(x))) held (sigma_k swaps k and s_piv[k]), so
        // one warp follows every position's chain at once: lane i the leaf row i and,
        // if interchange i is the first to reach its target below the leaf, that
        // target.  The moves are listed leaf rows first, then targets in order of
        // first occurrence.
        if (warp == 0) {
            auto chain = [&](int x) {
                for (int q = w - 1; q >= 0; --q) {
                    const int pq = s_piv[q];
                    x = (x == q) ? pq : ((x == pq) ? q : x);
                }
                return x;
            };
            const int src_l = lane < w ? chain(lane) : lane;
            const int pk = lane < w ? s_piv[lane] : -1;
            const bool is_t = pk >= w;
            const unsigned same = __match_any_sync(0xffffffffu, is_t ? pk : -1 - lane);
            const bool first = is_t && (__ffs(same) - 1 == lane);
            const int src_t = first ? chain(pk) : pk;
            const bool mv_l = lane < w && src_l != lane;
            const bool mv_t = first && src_t != pk;
            const unsigned bl = __ballot_sync(0xffffffffu, mv_l);
            const unsigned bt = __ballot_sync(0xffffffffu, mv_t);
            const int nl = __popc(bl);
            const unsigned below = (1u << lane) - 1u;
            if (mv_l) {
                s_dst[__popc(bl & below)] = lane;
                s_src[__popc(bl & below)] = src_l;
            }
            if (mv_t) {
                s_dst[nl + __popc(bt & below)] = pk;
                s_src[nl + __popc(bt & below)] = src_t;
            }
            if (lane == 0) s_cnt = nl + __popc(bt);
        }
        __syncthreads();
        const int cnt = s_cnt;
        // The sibling's columns (the first sib right columns): CTA 0 applies the
        // interchanges and then solves their top w rows with this leaf's unit-lower
        // L11 (lane = row, x_i := fma(-L(i, j), x_j, x_i) for j = 0, 1, ...), which
        // makes them the sibling's U12; the sibling folds the matching update into
        // its prologue.
        if (g == 0) {
            for (int t = warp; t < sib; t += NT / 32) {
                T* a = A + (int64_t)(w + t) * lda;
                T vv[(2 * W + 31) / 32];
#pragma unroll
                for (int u = 0; u < (2 * W + 31) / 32; ++u)
                    if (lane + 32 * u < cnt) vv[u] = a[s_src[lane + 32 * u]];
                __syncwarp();
#pragma unroll
                for (int u = 0; u < (2 * W + 31) / 32; ++u)
                    if (lane + 32 * u < cnt) a[s_dst[lane + 32 * u]] = vv[u];
                __syncwarp();
                T x = (lane < w) ? a[lane] : T(0);
                for (int j = 0; j < w; ++j) {
                    const T xj = __shfl_sync(0xffffffffu, x, j);
                    if (lane > j && lane < w) x = fma(-sA[lane * WP + j], xj, x);
                }
                if (lane < w) a[lane] = x;
            }
        }
        // columns q = g, g + C, ... of the other columns; one warp per column
        for (int q = g * (NT / 32) + warp; cnt > 0 && q < other; q += C * (NT / 32)) {
            if (q >= left_cols && q < left_cols + sib) continue;
            const int64_t col = (q < left_cols) ? (int64_t)q - left_cols : (int64_t)w + (q - left_cols);
            T* a = A + col * lda;
            T vv[(2 * W + 31) / 32];
#pragma unroll
            for (int t = 0; t < (2 * W + 31) / 32; ++t)
                if (lane + 32 * t < cnt) vv[t] = a[s_src[lane + 32 * t]];
            __syncwarp();
#pragma unroll
            for (int t = 0; t < (2 * W + 31) / 32; ++t)
                if (lane + 32 * t < cnt) a[s_dst[lane + 32 * t]] = vv[t];
        }
    }
    asm volatile("barrier.cluster.wait;" ::: "memory");
}

template <typename T>
struct PushTable {
    typedef void (*Fn)(T*, int64_t, int, int, int, int, int32_t*, int, LuSync*, int, int);
    static Fn get(int w, int rq, int nt, size_t* smem) {
#define LU_PUSH_CASE(WW, RR, NN)                                    \
    if (w == WW && rq == RR && nt == NN) {                          \
        if (smem) *smem = PushSmem<T, WW, RR, NN>::total;           \
        return pf_leaf_push_kernel<T, WW, RR, NN>;                  \
    }
        LU_PUSH_CASE(8, 1, 256) LU_PUSH_CASE(8, 2, 256) LU_PUSH_CASE(8, 4, 256) LU_PUSH_CASE(8, 8, 256)
        LU_PUSH_CASE(16, 1, 256) LU_PUSH_CASE(16, 2, 256) LU_PUSH_CASE(16, 4, 256) LU_PUSH_CASE(16, 8, 256)
        LU_PUSH_CASE(32, 1, 256) LU_PUSH_CASE(32, 2, 256) LU_PUSH_CASE(32, 4, 256)
        // 512 threads (FP32, leaves on SMs of their own): half the rows per thread
        if constexpr (sizeof(T) == 4) {
            LU_PUSH_CASE(8, 1, 512) LU_PUSH_CASE(8, 2, 512) LU_PUSH_CASE(8, 4, 512)
            LU_PUSH_CASE(16, 1, 512) LU_PUSH_CASE(16, 2, 512) LU_PUSH_CASE(16, 4, 512)
            LU_PUSH_CASE(32, 1, 512) LU_PUSH_CASE(32, 2, 512)
        }
#undef LU_PUSH_CASE
        return nullptr;
    }
};

}  // namespace

// Dynamic shared memory of the pushed-message leaf (0 if the shape is not compiled).
size_t lu_pf_push_smem(int esize, int w, int rq, int nt) {
    size_t s = 0;
    if (esize == 8)
        PushTable<double>::get(w, rq, nt, &s);
    else
        PushTable<float>::get(w, rq, nt, &s);
    return s;
}

template <typename T>
int lu_launch_pf_leaf_push(cudaStream_t st, T* A, int64_t lda, int64_t m, int w, int wc, int C, int R,
                           int64_t left_cols, int64_t right_cols, int32_t* ipiv, int64_t ipiv_add, LuSync* sync,
                           int sib, int kprev, int nt) {
    size_t smem = 0;
    auto fn = (nt > 0 && R % nt == 0) ? PushTable<T>::get(wc, R / nt, nt, &smem) : nullptr;
    if (!fn || C > kMaxC || sib < 0 || sib > wc || sib > right_cols || kprev < 0 || kprev > kMaxPrev)
        return LU_ERR_UNSUPPORTED;
    LU_TRY(lu_func_smem(fn, (int)smem, true));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(nt, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LuProfScope prof(st, LU_K_PANEL, 2.0 * m * w * sizeof(T) + 4.0 * w * (left_cols + right_cols) * sizeof(T),
                     (double)m * w * w);
    if (getenv("LU_GB300_TRACE_LAUNCH"))
        fprintf(stderr, "[lu launch] push leaf esize %d m %lld w %d (compiled %d) C %d R %d threads %d smem %zu left %lld "
                "right %lld\n", (int)sizeof(T), (long long)m, w, wc, C, R, nt, smem, (long long)left_cols,
                (long long)right_cols);
    LU_CHECK_CUDA(cudaLaunchKernelEx(&cfg, fn, A, lda, (int)m, w, (int)left_cols, (int)right_cols, ipiv, (int)ipiv_add,
                                     sync, sib, kprev));
    lu_count_launch();
    return LU_SUCCESS;
}

template int lu_launch_pf_leaf_push<double>(cudaStream_t, double*, int64_t, int64_t, int, int, int, int, int64_t,
                                            int64_t, int32_t*, int64_t, LuSync*, int, int, int);
template int lu_launch_pf_leaf_push<float>(cudaStream_t, float*, int64_t, int64_t, int, int, int, int, int64_t,
                                           int64_t, int32_t*, int64_t, LuSync*, int, int, int);
