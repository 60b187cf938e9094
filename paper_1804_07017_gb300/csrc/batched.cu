// Batched LU with partial pivoting and solve: many independent small matrices
// (n <= 512) in one persistent launch (not part of the paper).
//
// A first single-CTA kernel orders the matrices by decreasing n (counting
// sort), so that the persistent CTAs, which take matrices from an atomic
// counter, start the largest ones first (longest-processing-time order).
// Each CTA factors its matrix with the blocked right-looking algorithm of
// LU_blk (Sec. 3) scaled down to one CTA:
//   PF   the 32-column panel is loaded into shared memory and eliminated
//        column by column (block argmax, first maximum, true division; two
//        barriers per column, the update of a column also finding the next
//        column's pivot candidates);
//   the panel's interchanges, composed into one gather plan, are applied to
//   the other columns a warp per column, then RL2
//   (unit-lower solve of the U12 row block, one column per thread) and RL3
//   (A22 -= L21 U12 with 4x4 register tiles, L21 from shared memory);
// and then, if right-hand sides are given, solves P A X = B for them by
// blocks of factor columns staged in shared memory.
#include <climits>

#include "internal.h"
#include "profile.h"

namespace {

constexpr int kBT = 256;     // threads per CTA
constexpr int kBNB = 32;     // panel width
constexpr int kNMAX = 512;   // largest order handled
constexpr int kMaxRhs = 8;   // right-hand sides handled together
constexpr int kUS = 68;      // row stride of the U12 tile (16-byte rows for vector loads)

template <typename T>
struct BatchSmem {
    // panel [kBNB][kNMAX] column-major, then a U12 tile [kBNB][kUS] (64 columns) for the update
    static constexpr size_t bytes = sizeof(T) * ((size_t)kBNB * kNMAX + (size_t)kBNB * kUS) + 64;
};

// Four consecutive values from 16-byte-aligned shared memory.
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    v[3] = q1.y;
}

// s[c * kNMAX + r] = g[r + c * ld] for r < rows (<= kNMAX), c < cols: eight columns
// and both row halves are loaded before any is stored, so a thread keeps up to 16
// global loads in flight instead of waiting on each.
template <typename T>
__device__ __forceinline__ void stage_cols(T* __restrict__ s, const T* __restrict__ g, int64_t ld, int rows, int cols) {
    static_assert(kNMAX <= 2 * kBT, "two row slots per thread cover a column");
    constexpr int kB = 8;
    const int r0 = threadIdx.x, r1 = threadIdx.x + kBT;
    for (int c0 = 0; c0 < cols; c0 += kB) {
        T v0[kB], v1[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const T* gc = g + (int64_t)min(c0 + u, cols - 1) * ld;
            v0[u] = (c0 + u < cols && r0 < rows) ? gc[r0] : T(0);
            v1[u] = (c0 + u < cols && r1 < rows) ? gc[r1] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (c0 + u < cols && r0 < rows) s[(c0 + u) * kNMAX + r0] = v0[u];
            if (c0 + u < cols && r1 < rows) s[(c0 + u) * kNMAX + r1] = v1[u];
        }
    }
}

// order[] = matrix indices by decreasing n; n > kNMAX or
// n < 0 are placed last and flagged by the main kernel.
__global__ void __launch_bounds__(1024) batch_order_kernel(int batch, const int32_t* __restrict__ nvec,
                                                           int32_t* __restrict__ order, int* __restrict__ counter) {
    __shared__ int cnt[kNMAX + 2];
    __shared__ int start[kNMAX + 2];
    for (int i = threadIdx.x; i < kNMAX + 2; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    auto key = [&](int i) {
        const int n = nvec[i];
        return (n < 0 || n > kNMAX) ? kNMAX + 1 : kNMAX - n;  // 0 = largest
    };
    for (int i = threadIdx.x; i < batch; i += blockDim.x) atomicAdd(&cnt[key(i)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int b = 0; b < kNMAX + 2; ++b) {
            start[b] = s;
            s += cnt[b];
        }
        *counter = 0;
    }
    __syncthreads();
    // scatter (the order among equal n is irrelevant to the results)
    for (int i = threadIdx.x; i < batch; i += blockDim.x) order[atomicAdd(&start[key(i)], 1)] = i;
}

// Row of the largest |value| over the CTA (first index among equal maxima;
// NaN never wins), with one barrier: every thread reduces the per-warp winners
// itself.  red_v/red_i hold kBT/32 slots; callers alternate two such buffers so
// that the next call's writes cannot overtake this call's reads.
template <typename T>
__device__ int block_argmax(T v, int i, T* red_v, int* red_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
    if (lane == 0) {
        red_v[warp] = v;
        red_i[warp] = i;
    }
    __syncthreads();
    v = red_v[0];
    i = red_i[0];
#pragma unroll
    for (int w = 1; w < kBT / 32; ++w) {
        const T ov = red_v[w];
        const int oi = red_i[w];
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
    return i;
}

// Factor one n x n matrix (column-major, lda) in place; ipiv 1-based; returns info.
// RL3 of one panel step, A22 -= L21 U12, in TM x TN output tiles: a thread owns
// rows i0 + tx + 16a (a < TM/16) and the TN/16 adjacent columns j0 + (TN/16) ty + b,
// so its U12 values are adjacent in shared memory; every entry accumulates its
// kBNB products in k order and is then subtracted once, whatever the tile shape.
// L21 rows past mr hold stale shared data (inside the allocation) whose products
// are never stored.
template <typename T, int TM, int TN>
__device__ __forceinline__ void rl3_tiles(T* __restrict__ A, int64_t lda, int k0, int kb, int mr, int nr,
                                          const T* __restrict__ sP, T* __restrict__ sU) {
    constexpr int MA = TM / 16, NB = TN / 16;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int j0 = 0; j0 < nr; j0 += TN) {
        // U12 columns j0 .. j0+TN-1 into shared memory
        {
            constexpr int kPer = kBNB * TN / kBT;
            T v[kPer];
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int e = tid + t * kBT, kk = e & (kBNB - 1), jj = e / kBNB;
                v[t] = (j0 + jj < nr) ? A[(int64_t)(k0 + kk) + (int64_t)(k0 + kb + j0 + jj) * lda] : T(0);
            }
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
                const int e = tid + t * kBT, kk = e & (kBNB - 1), jj = e / kBNB;
                sU[kk * kUS + jj] = v[t];
            }
        }
        __syncthreads();
        for (int i0 = 0; i0 < mr; i0 += TM) {
            // the output tile is read before the product so that its load latency
            // overlaps the kk loop
            T acc[MA][NB], cv[MA][NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int jc = j0 + NB * ty + b;
                const T* col = A + (int64_t)(k0 + kb + min(jc, nr - 1)) * lda + (k0 + kb);
#pragma unroll
                for (int a = 0; a < MA; ++a) {
                    const int r = i0 + tx + 16 * a;
                    cv[a][b] = (jc < nr && r < mr) ? col[r] : T(0);
                    acc[a][b] = T(0);
                }
            }
            const T* lp = sP + kb + i0 + tx;
            const T* up = sU + NB * ty;
#pragma unroll 8
            for (int kk = 0; kk < kBNB; ++kk) {
                T lv[MA], uv[NB];
#pragma unroll
                for (int a = 0; a < MA; ++a) lv[a] = lp[kk * kNMAX + 16 * a];
                if constexpr (NB == 4) {
                    T q[4];
                    load4(up + kk * kUS, q);
#pragma unroll
                    for (int b = 0; b < 4; ++b) uv[b] = q[b];
                } else {
#pragma unroll
                    for (int b = 0; b < NB; ++b) uv[b] = up[kk * kUS + b];
                }
#pragma unroll
                for (int a = 0; a < MA; ++a)
#pragma unroll
                    for (int b = 0; b < NB; ++b) acc[a][b] = fma(lv[a], uv[b], acc[a][b]);
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int jc = j0 + NB * ty + b;
                if (jc >= nr) continue;
                T* col = A + (int64_t)(k0 + kb + jc) * lda + (k0 + kb);
#pragma unroll
                for (int a = 0; a < MA; ++a) {
                    const int r = i0 + tx + 16 * a;
                    if (r < mr) col[r] = cv[a][b] - acc[a][b];
                }
            }
        }
        __syncthreads();
    }
}

template <typename T>
__device__ int factor_one(int n, T* __restrict__ A, int64_t lda, int32_t* __restrict__ ipiv, T* sP, T* sU,
                          T* red_v, int* red_i, int small_cut) {
    // interchange plan of the current panel (relative rows)
    __shared__ int s_pdst[2 * kBNB], s_psrc[2 * kBNB], s_pcur[2 * kBNB], s_ptgt[kBNB], s_pb[kBNB], s_pcnt;
    const int tid = threadIdx.x;
    int finfo = 0;
    for (int k0 = 0; k0 < n; k0 += kBNB) {
        const int kb = min(kBNB, n - k0);
        const int m = n - k0;
        // ---- PF: panel rows [k0, n) x columns [k0, k0+kb) in shared memory ----
        stage_cols(sP, A + (int64_t)k0 + (int64_t)k0 * lda, lda, m, kb);
        __syncthreads();
        // Two barriers per column: one in the argmax, one after the row interchange.
        // The update of column j also finds this thread's candidate for column j+1.
        T bv = T(-1);
        int bi = INT_MAX;
        for (int r = tid; r < m; r += kBT) {
            const T v = fabs(sP[r]);
            if (v > bv || (v == bv && r < bi)) {
                bv = v;
                bi = r;
            }
        }
        for (int j = 0; j < kb; ++j) {
            const int buf = (j & 1) * (kBT / 32);
            int p = block_argmax(bv, bi, red_v + buf, red_i + buf);
            if (p == INT_MAX) p = j;
            if (tid == 0) ipiv[k0 + j] = k0 + p + 1;
            if (p != j && tid < kb) {
                const T t = sP[tid * kNMAX + j];
                sP[tid * kNMAX + j] = sP[tid * kNMAX + p];
                sP[tid * kNMAX + p] = t;
            }
            __syncthreads();
            const T piv = sP[j * kNMAX + j];
            bv = T(-1);
            bi = INT_MAX;
            if (piv == T(0)) {
                if (finfo == 0) finfo = k0 + j + 1;
                if (j + 1 < kb)
                    for (int r = j + 1 + tid; r < m; r += kBT) {
                        const T v = fabs(sP[(j + 1) * kNMAX + r]);
                        if (v > bv || (v == bv && r < bi)) {
                            bv = v;
                            bi = r;
                        }
                    }
                continue;
            }
            for (int r = j + 1 + tid; r < m; r += kBT) {
                const T l = sP[j * kNMAX + r] / piv;
                sP[j * kNMAX + r] = l;
                if (j + 1 < kb) {
                    const T v1 = fma(-l, sP[(j + 1) * kNMAX + j], sP[(j + 1) * kNMAX + r]);
                    sP[(j + 1) * kNMAX + r] = v1;
                    const T a1 = fabs(v1);
                    if (a1 > bv || (a1 == bv && r < bi)) {
                        bv = a1;
                        bi = r;
                    }
                }
                for (int c = j + 2; c < kb; ++c) sP[c * kNMAX + r] = fma(-l, sP[c * kNMAX + j], sP[c * kNMAX + r]);
            }
        }
        __syncthreads();
        for (int c = 0; c < kb; ++c)
            for (int r = tid; r < m; r += kBT) A[(int64_t)(k0 + r) + (int64_t)(k0 + c) * lda] = sP[c * kNMAX + r];
        // ---- the panel's interchanges on the other columns ----
        // The kb sequential interchanges are composed once into a gather plan
        // dst <- src over the panel rows and the distinct rows below them that they
        // reach; a warp then moves a column's entries all at once (every value read
        // before any is written), so a column costs one memory round trip instead of
        // kb dependent ones.
        if (tid < 32) {
            const int lane = tid;
            const unsigned full = 0xffffffffu;
            const int pj = (lane < kb) ? ipiv[k0 + lane] - 1 - k0 : -1;
            const bool below = pj >= kb;
            const unsigned same = __match_any_sync(full, below ? pj : -1 - lane);
            const int lead = __ffs(same) - 1;
            const bool first = below && lead == lane;
            const unsigned firsts = __ballot_sync(full, first);
            const int f = __popc(firsts & ((1u << lead) - 1u));
            if (lane < kb) s_pb[lane] = below ? kb + f : pj;
            s_pcur[lane] = lane;
            if (first) {
                s_ptgt[f] = pj;
                s_pcur[kb + f] = pj;
            }
            __syncwarp();
            if (lane == 0)
                for (int j = 0; j < kb; ++j) {
                    const int bj = s_pb[j];
                    if (bj != j) {
                        const int x = s_pcur[j];
                        s_pcur[j] = s_pcur[bj];
                        s_pcur[bj] = x;
                    }
                }
            __syncwarp();
            const int nt = __popc(firsts);
            const bool e0 = lane < kb && s_pcur[lane] != lane;
            const bool e1 = lane < nt && s_pcur[kb + lane] != s_ptgt[lane];
            const unsigned m0 = __ballot_sync(full, e0), m1 = __ballot_sync(full, e1);
            const unsigned lt = (1u << lane) - 1u;
            if (e0) {
                const int i = __popc(m0 & lt);
                s_pdst[i] = lane;
                s_psrc[i] = s_pcur[lane];
            }
            if (e1) {
                const int i = __popc(m0) + __popc(m1 & lt);
                s_pdst[i] = s_ptgt[lane];
                s_psrc[i] = s_pcur[kb + lane];
            }
            if (lane == 0) s_pcnt = __popc(m0) + __popc(m1);
        }
        __syncthreads();
        {
            const int cnt = s_pcnt, lane = tid & 31;
            const bool h0 = lane < cnt, h1 = lane + 32 < cnt;
            const int s0 = h0 ? s_psrc[lane] : 0, d0 = h0 ? s_pdst[lane] : 0;
            const int s1 = h1 ? s_psrc[lane + 32] : 0, d1 = h1 ? s_pdst[lane + 32] : 0;
            constexpr int kU = 4;  // columns per warp per round
            const int others = n - kb;
            for (int q0 = (tid >> 5) * kU; q0 < others && cnt > 0; q0 += (kBT / 32) * kU) {
                T v0[kU], v1[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int q = q0 + u;
                    const T* a = A + (int64_t)((q < k0) ? q : q + kb) * lda + k0;
                    v0[u] = (h0 && q < others) ? a[s0] : T(0);
                    v1[u] = (h1 && q < others) ? a[s1] : T(0);
                }
                __syncwarp();
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int q = q0 + u;
                    T* a = A + (int64_t)((q < k0) ? q : q + kb) * lda + k0;
                    if (h0 && q < others) a[d0] = v0[u];
                    if (h1 && q < others) a[d1] = v1[u];
                }
            }
        }
        __syncthreads();
        const int nr = n - k0 - kb;  // trailing columns
        if (nr <= 0) continue;
        // ---- RL2: U12 := trilu(L11)^-1 A12, one column per thread ----
        for (int c = tid; c < nr; c += kBT) {
            T x[kBNB];
            T* a = A + (int64_t)(k0 + kb + c) * lda + k0;
#pragma unroll
            for (int i = 0; i < kBNB; ++i) x[i] = (i < kb) ? a[i] : T(0);
#pragma unroll
            for (int j = 0; j < kBNB; ++j)
#pragma unroll
                for (int i = j + 1; i < kBNB; ++i)
                    if (i < kb) x[i] = fma(-sP[j * kNMAX + i], x[j], x[i]);
#pragma unroll
            for (int i = 0; i < kBNB; ++i)
                if (i < kb) a[i] = x[i];
        }
        __syncthreads();
        // ---- RL3: A22 -= L21 U12 (kb == kBNB here: a trailing block exists only after
        // a full panel); small trailing blocks take 32 x 32 tiles, which waste fewer
        // padded products, larger ones 64 x 64 (same per-element order either way)
        if (nr < small_cut) rl3_tiles<T, 32, 32>(A, lda, k0, kb, m - kb, nr, sP, sU);
        else rl3_tiles<T, 64, 64>(A, lda, k0, kb, m - kb, nr, sP, sU);
    }
    return finfo;
}

// X := (P A)^-1 B with the factors in A; B n x nrhs (nrhs <= kMaxRhs), staged in
// shared memory with blocks of kSB factor columns beside it.  Per block, a warp
// per right-hand side solves the diagonal block (lane = row, shuffles carry the
// solved entries) and then every thread updates the remaining rows; each entry
// receives its fma updates in the same order as the column-by-column
// substitution, so the result does not depend on the block width.
template <typename T>
__device__ void solve_one(int n, const T* __restrict__ A, int64_t lda, const int32_t* __restrict__ ipiv, int nrhs,
                          T* __restrict__ B, int64_t ldb, T* sB) {
    constexpr int kSB = kBNB - kMaxRhs;  // factor columns staged per block
    T* sL = sB + kMaxRhs * kNMAX;
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int* s_ipiv = reinterpret_cast<int*>(sL);  // free until the first factor block is staged
    for (int k = tid; k < n; k += kBT) s_ipiv[k] = ipiv[k];
    stage_cols(sB, B, ldb, n, nrhs);
    __syncthreads();
    if (tid < nrhs) {
        for (int k = 0; k < n; ++k) {
            const int p = s_ipiv[k] - 1;
            if (p != k) {
                const T t = sB[tid * kNMAX + k];
                sB[tid * kNMAX + k] = sB[tid * kNMAX + p];
                sB[tid * kNMAX + p] = t;
            }
        }
    }
    __syncthreads();
    // unit lower, blocks forward; sL holds L[j0:n, j0:j0+jb] (rows relative to j0)
    for (int j0 = 0; j0 < n; j0 += kSB) {
        const int jb = min(kSB, n - j0), mr = n - j0;
        stage_cols(sL, A + (int64_t)j0 + (int64_t)j0 * lda, lda, mr, jb);
        __syncthreads();
        if (warp < nrhs) {
            T* x = sB + warp * kNMAX + j0;
            T xi = lane < jb ? x[lane] : T(0);
            for (int j = 0; j < jb; ++j) {
                const T xj = __shfl_sync(full, xi, j);
                if (lane > j && lane < jb) xi = fma(-sL[j * kNMAX + lane], xj, xi);
            }
            if (lane < jb) x[lane] = xi;
        }
        __syncthreads();
        const int rows = mr - jb;
        for (int e = tid; e < rows * nrhs; e += kBT) {
            const int i = jb + e % rows, c = e / rows;
            T* x = sB + c * kNMAX + j0;
            T xi = x[i];
            for (int j = 0; j < jb; ++j) xi = fma(-sL[j * kNMAX + i], x[j], xi);
            x[i] = xi;
        }
        __syncthreads();
    }
    // upper, blocks backward; sL holds U[0:j1, j0:j1]
    for (int j1 = n; j1 > 0; j1 -= kSB) {
        const int j0 = max(0, j1 - kSB), jb = j1 - j0;
        stage_cols(sL, A + (int64_t)j0 * lda, lda, j1, jb);
        __syncthreads();
        if (warp < nrhs) {
            T* x = sB + warp * kNMAX + j0;
            T xi = lane < jb ? x[lane] : T(0);
            for (int j = jb - 1; j >= 0; --j) {
                if (lane == j) xi = xi / sL[j * kNMAX + j0 + j];
                const T xj = __shfl_sync(full, xi, j);
                if (lane < j) xi = fma(-sL[j * kNMAX + j0 + lane], xj, xi);
            }
            if (lane < jb) x[lane] = xi;
        }
        __syncthreads();
        for (int e = tid; e < j0 * nrhs; e += kBT) {
            const int i = e % j0, c = e / j0;
            T* x = sB + c * kNMAX;
            T xi = x[i];
            for (int j = jb - 1; j >= 0; --j) xi = fma(-sL[j * kNMAX + i], x[j0 + j], xi);
            x[i] = xi;
        }
        __syncthreads();
    }
    for (int e = tid; e < n * nrhs; e += kBT) {
        const int i = e % n, c = e / n;
        B[i + (int64_t)c * ldb] = sB[c * kNMAX + i];
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kBT) batched_gesv_kernel(int batch, const int32_t* __restrict__ nvec,
                                                           T* const* __restrict__ Aptr, const int64_t* __restrict__ ldav,
                                                           int32_t* const* __restrict__ ipivp,
                                                           const int32_t* __restrict__ nrhsv, T* const* __restrict__ Bptr,
                                                           const int64_t* __restrict__ ldbv,
                                                           int32_t* __restrict__ info,
                                                           const int32_t* __restrict__ order, int* __restrict__ counter,
                                                           int do_factor, int small_cut) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sP = reinterpret_cast<T*>(smraw);
    T* sU = sP + (size_t)kBNB * kNMAX;
    __shared__ T red_v[2 * (kBT / 32)];
    __shared__ int red_i[2 * (kBT / 32)];
    __shared__ int s_idx;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= batch) break;
        const int mid = order[idx];
        const int n = nvec[mid];
        const int64_t lda = ldav[mid];
        if (n < 0 || n > kNMAX) {
            if (threadIdx.x == 0) info[mid] = LU_ERR_UNSUPPORTED;
            continue;
        }
        if (lda < max(1, n)) {
            if (threadIdx.x == 0) info[mid] = -4;
            continue;
        }
        int finfo = 0;
        if (n > 0 && do_factor)
            finfo = factor_one<T>(n, Aptr[mid], lda, ipivp[mid], sP, sU, red_v, red_i, small_cut);
        if (threadIdx.x == 0) info[mid] = finfo;
        if (Bptr && n > 0 && finfo == 0) {
            const int nrhs = nrhsv[mid];
            const int64_t ldb = ldbv[mid];
            if (nrhs < 0 || nrhs > kMaxRhs || ldb < max(1, n)) {
                if (threadIdx.x == 0) info[mid] = nrhs < 0 || nrhs > kMaxRhs ? LU_ERR_UNSUPPORTED : -9;
                continue;
            }
            if (nrhs > 0) solve_one<T>(n, Aptr[mid], lda, ipivp[mid], nrhs, Bptr[mid], ldb, sP);
        }
    }
}

}  // namespace

// Trailing orders below which a panel step's RL3 takes 32 x 32 tiles: the tuned
// value for this device and precision (lu_tune_batched), else the default.
static int batched_tile_cut(lu_dtype dtype) {
    const int kind = dtype == LU_F64 ? LU_TUNE_BATCHED_F64 : LU_TUNE_BATCHED_F32;
    const int v = lu_tuned_value(kind, kNMAX);
    return v > 0 ? v : (dtype == LU_F64 ? LU_BATCHED_CUT_F64 : LU_BATCHED_CUT_F32);
}

template <typename T>
static int gesv_batched_impl(lu_context* c, int batch, const int32_t* n, T* const* A, const int64_t* lda,
                             int32_t* const* ipiv, const int32_t* nrhs, T* const* B, const int64_t* ldb, int32_t* info,
                             int do_factor, int small_cut) {
    cudaStream_t st = c->user;
    const size_t need = sizeof(int32_t) * ((size_t)batch + 64);
    if (c->batch_ws_bytes < need) {
        if (c->batch_ws) {
            LU_CHECK_CUDA(cudaStreamSynchronize(st));
            cudaFree(c->batch_ws);
            c->batch_ws = nullptr;
            c->batch_ws_bytes = 0;
        }
        if (cudaMalloc(&c->batch_ws, need) != cudaSuccess) {
            cudaGetLastError();
            return LU_ERR_NOMEM;
        }
        c->batch_ws_bytes = need;
    }
    int* counter = reinterpret_cast<int*>(c->batch_ws);
    int32_t* order = reinterpret_cast<int32_t*>(c->batch_ws) + 64;
    {
        LuProfScope prof(st, LU_K_OTHER, 12.0 * batch, 0.0);
        batch_order_kernel<<<1, 1024, 0, st>>>(batch, n, order, counter);
    }
    LU_CHECK_LAUNCH();
    LU_TRY(lu_func_smem(batched_gesv_kernel<T>, (int)BatchSmem<T>::bytes));
    int per_sm = 0;
    LU_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_gesv_kernel<T>, kBT,
                                                                BatchSmem<T>::bytes));
    const int grid = std::max(1, std::min(batch, c->num_sms * std::max(per_sm, 1)));
    LuProfScope prof(st, LU_K_BATCHED, 0.0, 0.0);
    batched_gesv_kernel<T><<<grid, kBT, BatchSmem<T>::bytes, st>>>(batch, n, A, lda, ipiv, nrhs, B, ldb, info, order,
                                                                   counter, do_factor, small_cut);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

static int batched_entry(lu_handle h, lu_dtype dtype, int batch, const int32_t* n, void* const* A,
                         const int64_t* lda, int32_t* const* ipiv, const int32_t* nrhs, void* const* B,
                         const int64_t* ldb, int32_t* info, int do_factor) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (batch < 0) return -3;
    if (batch > 0 && (!n || !A || !lda || !ipiv)) return -4;
    if (B && (!nrhs || !ldb)) return -8;
    if (!do_factor && batch > 0 && !B) return -9;
    if (batch > 0 && !info) return -11;
    if (batch == 0) return LU_SUCCESS;
    const int cut = h->batched_cut_override > 0 ? h->batched_cut_override : batched_tile_cut(dtype);
    std::lock_guard<std::mutex> lk(h->mu);
    LU_TRY(lu_ctx_reserve(h, 1, 1));
    if (dtype == LU_F64)
        return gesv_batched_impl<double>(h, batch, n, (double* const*)A, lda, ipiv, nrhs, (double* const*)B, ldb, info,
                                         do_factor, cut);
    return gesv_batched_impl<float>(h, batch, n, (float* const*)A, lda, ipiv, nrhs, (float* const*)B, ldb, info,
                                    do_factor, cut);
}

extern "C" int lu_gesv_batched(lu_handle h, lu_dtype dtype, int batch, const int32_t* n, void* const* A,
                               const int64_t* lda, int32_t* const* ipiv, const int32_t* nrhs, void* const* B,
                               const int64_t* ldb, int32_t* info) {
    return batched_entry(h, dtype, batch, n, A, lda, ipiv, nrhs, B, ldb, info, 1);
}

extern "C" int lu_factor_batched(lu_handle h, lu_dtype dtype, int batch, const int32_t* n, void* const* A,
                                 const int64_t* lda, int32_t* const* ipiv, int32_t* info) {
    return batched_entry(h, dtype, batch, n, A, lda, ipiv, nullptr, nullptr, nullptr, info, 1);
}

extern "C" int lu_solve_batched(lu_handle h, lu_dtype dtype, int batch, const int32_t* n, void* const* LU,
                                const int64_t* lda, int32_t* const* ipiv, const int32_t* nrhs, void* const* B,
                                const int64_t* ldb, int32_t* info) {
    return batched_entry(h, dtype, batch, n, LU, lda, ipiv, nrhs, B, ldb, info, 0);
}

namespace {

// Seeded U[-1, 1) entries for the tuner's synthetic batch: splitmix64 (Steele,
// Lea and Flood, 2014) of the element index, top 53 bits as a fraction.
template <typename T>
__global__ void batch_fill_kernel(T* __restrict__ X, int64_t count, uint64_t seed) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        X[e] = (T)(2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0);
    }
}

template <typename T>
int tune_batched_impl(lu_handle h, lu_dtype dtype, int batch, const int32_t* n, const int32_t* nrhs, int reps,
                      const int* cuts, int count, int* best, float* ms) {
    std::vector<int64_t> aoff(batch), boff(batch), poff(batch);
    int64_t ta = 0, tb = 0, tp = 0;
    for (int i = 0; i < batch; ++i) {
        aoff[i] = ta;
        boff[i] = tb;
        poff[i] = tp;
        ta += (int64_t)n[i] * n[i];
        tb += (int64_t)n[i] * std::max(nrhs[i], 0);
        tp += std::max(n[i], 1);
    }
    T *A = nullptr, *A0 = nullptr, *B = nullptr, *B0 = nullptr;
    int32_t *piv = nullptr, *info = nullptr, *dn = nullptr, *dr = nullptr;
    int64_t *dlda = nullptr, *dldb = nullptr;
    void **dA = nullptr, **dB = nullptr, **dP = nullptr;
    auto cleanup = [&]() {
        void* ps[] = {A, A0, B, B0, piv, info, dn, dr, dlda, dldb, dA, dB, dP};
        for (void* q : ps)
            if (q) cudaFree(q);
    };
    const size_t ea = (size_t)std::max<int64_t>(ta, 1), eb = (size_t)std::max<int64_t>(tb, 1);
    if (cudaMalloc(&A, sizeof(T) * ea) != cudaSuccess || cudaMalloc(&A0, sizeof(T) * ea) != cudaSuccess ||
        cudaMalloc(&B, sizeof(T) * eb) != cudaSuccess || cudaMalloc(&B0, sizeof(T) * eb) != cudaSuccess ||
        cudaMalloc(&piv, sizeof(int32_t) * (size_t)std::max<int64_t>(tp, 1)) != cudaSuccess ||
        cudaMalloc(&info, sizeof(int32_t) * batch) != cudaSuccess || cudaMalloc(&dn, sizeof(int32_t) * batch) != cudaSuccess ||
        cudaMalloc(&dr, sizeof(int32_t) * batch) != cudaSuccess || cudaMalloc(&dlda, sizeof(int64_t) * batch) != cudaSuccess ||
        cudaMalloc(&dldb, sizeof(int64_t) * batch) != cudaSuccess || cudaMalloc(&dA, sizeof(void*) * batch) != cudaSuccess ||
        cudaMalloc(&dB, sizeof(void*) * batch) != cudaSuccess || cudaMalloc(&dP, sizeof(void*) * batch) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return LU_ERR_NOMEM;
    }
    std::vector<void*> ha(batch), hb(batch), hp(batch);
    std::vector<int64_t> hl(batch), hlb(batch);
    for (int i = 0; i < batch; ++i) {
        ha[i] = A + aoff[i];
        hb[i] = B + boff[i];
        hp[i] = piv + poff[i];
        hl[i] = std::max(n[i], 1);
        hlb[i] = std::max(n[i], 1);
    }
    cudaStream_t st;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        st = h->user;
    }
    int rc = LU_SUCCESS;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMemcpy(dn, n, sizeof(int32_t) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dr, nrhs, sizeof(int32_t) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dlda, hl.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dldb, hlb.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dA, ha.data(), sizeof(void*) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dB, hb.data(), sizeof(void*) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dP, hp.data(), sizeof(void*) * batch, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = LU_ERR_CUDA;
    if (rc == LU_SUCCESS) {
        batch_fill_kernel<T><<<4 * h->num_sms, 256, 0, st>>>(A0, (int64_t)ea, 0x5eedull);
        batch_fill_kernel<T><<<4 * h->num_sms, 256, 0, st>>>(B0, (int64_t)eb, 0xb0b0ull);
        if (cudaGetLastError() != cudaSuccess) rc = LU_ERR_CUDA;
    }
    float best_ms = -1.f;
    int best_cut = 0;
    for (int ci = 0; ci < count && rc == LU_SUCCESS; ++ci) {
        float t = -1.f;
        h->batched_cut_override = cuts[ci];
        for (int r = 0; r < reps && rc == LU_SUCCESS; ++r) {
            float el = 0.f;
            if (cudaMemcpyAsync(A, A0, sizeof(T) * ea, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(B, B0, sizeof(T) * eb, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaEventRecord(e0, st) != cudaSuccess) {
                rc = LU_ERR_CUDA;
                break;
            }
            const int r2 = lu_gesv_batched(h, dtype, batch, dn, dA, dlda, (int32_t* const*)dP, dr, dB, dldb, info);
            if (r2 != LU_SUCCESS) {
                rc = r2;
                break;
            }
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&el, e0, e1) != cudaSuccess) {
                rc = LU_ERR_CUDA;
                break;
            }
            if (t < 0.f || el < t) t = el;
        }
        if (ms) ms[ci] = t;
        if (rc == LU_SUCCESS && t >= 0.f && (best_ms < 0.f || t < best_ms)) {
            best_ms = t;
            best_cut = cuts[ci];
        }
    }
    h->batched_cut_override = 0;
    if (rc == LU_ERR_CUDA) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cleanup();
    if (rc != LU_SUCCESS) return rc;
    *best = best_cut;
    return lu_tune_set(nullptr, dtype == LU_F64 ? LU_TUNE_BATCHED_F64 : LU_TUNE_BATCHED_F32, kNMAX, best_cut, best_ms);
}

}  // namespace

extern "C" int lu_tune_batched(lu_handle h, lu_dtype dtype, int batch, const int32_t* n, const int32_t* nrhs, int reps,
                               const int* cuts, int count, int* best, float* ms) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (batch < 1) return -3;
    if (!n) return -4;
    if (!nrhs) return -5;
    for (int i = 0; i < batch; ++i) {
        if (n[i] < 0 || n[i] > kNMAX) return -4;
        if (nrhs[i] < 0 || nrhs[i] > kMaxRhs) return -5;
    }
    if (reps < 1) return -6;
    if (!cuts || count < 1) return -7;
    for (int i = 0; i < count; ++i)
        if (cuts[i] < 1 || cuts[i] > kNMAX + 1) return -7;
    if (!best) return -9;
    if (dtype == LU_F64) return tune_batched_impl<double>(h, dtype, batch, n, nrhs, reps, cuts, count, best, ms);
    return tune_batched_impl<float>(h, dtype, batch, n, nrhs, reps, cuts, count, best, ms);
}
