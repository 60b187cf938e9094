// Householder QR (geqrf) on the same look-ahead skeleton as the LU: the
// paper's second dense factorization (Sec. 6.3; 4n^3/3 flops for a square
// matrix), reorganised exactly as Sec. 4 reorganises LU_blk.
//
// Step k, panel k = columns [k0, k0+kb):
//   PF_k  A(k0:m, panel) = Q_k R_k with Q_k = H_k0 ... H_{k0+kb-1},
//         H_j = I - tau_j v_j v_j^T (LAPACK layout: R on and above the diagonal,
//         v_j below it with v_j(j) = 1 implied); then the compact-WY factor T_k
//         (Q_k = I - V_k T_k V_k^T, T_k upper triangular) and V_k made explicit.
//   TU_k  A(k0:m, c) := Q_k^T A(k0:m, c) = A - V_k (T_k^T (V_k^T A)) for the
//         columns c right of the panel: two products with V_k^T / T_k^T (a
//         transposed-operand GEMM, split along its long inner dimension with a
//         fixed-order reduction) and C -= V_k W (the LU's RL3 kernel).
// With look-ahead, TU_k on panel k+1 and PF_{k+1} run on the high-priority
// stream while TU_k on the remaining columns runs on the other stream.
//
// The panel leaf (up to 64 columns) keeps its rows in shared memory across a
// grid of co-resident CTAs; per column: every CTA sums the squares of its part
// of the column, one grid barrier, every CTA forms the reflector (norm, beta,
// tau, the scaling) from the same fixed-order sum, every CTA forms its part of
// w = v^T A for the columns to the right, a second barrier, the rank-1 update.
// Wider panels split in two halves with a block-reflector update between them.
#include <math.h>

#include <cstring>

#include "internal.h"
#include "pack.h"
#include "profile.h"
#include "ptx.cuh"
#include "tc.h"

namespace {

constexpr int kQrThreads = 256;
constexpr int kQrMaxLeaf = 64;

// Warp-wide sum whose result is the same in every lane: each lane adds partials
// lane, lane + 32, ... (in that order), then a butterfly over the lanes, whose
// additions are commutative pairwise, so every lane ends with the same bits.
template <typename T>
__device__ __forceinline__ T warp_sum_slots(const T* __restrict__ p, int count, int stride, int lane) {
    T s = T(0);
    for (int q = lane; q < count; q += 32) s += __ldcg(&p[(int64_t)q * stride]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

template <typename T>
__device__ __forceinline__ T warp_allsum(T s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Leaf: Householder QR of the m x w block at A (w <= kQrMaxLeaf), rows split
// across gridDim.x CTAs of R rows.  slots (global): [2][G] partial sums of
// squares, [2] alpha, [G][kQrMaxLeaf] partial dot products.
//
// Work is split by columns between the warps of a CTA: in the step of column
// jj, warp q owns the columns jj+1+q, jj+1+q+8, ... (its lanes run down the
// CTA's rows), so a column's dot product and its rank-1 update stay in one warp
// and need no CTA-wide reduction.  Warp 0 owns column jj+1; while updating it
// it also forms that column's sum of squares for the next step.  Per column:
// warp 0 publishes the CTA's sum of squares (and alpha), grid barrier, every
// warp forms the reflector from the same fixed-order sum, the CTA scales the
// column, every warp forms its columns' partial v^T A, grid barrier, every warp
// sums its columns' partials in a fixed order and updates them.
template <typename T>
__global__ void __launch_bounds__(kQrThreads) qr_leaf_kernel(T* __restrict__ A, int64_t lda, int m, int w, int R,
                                                             T* __restrict__ tau, LuSync* __restrict__ sync,
                                                             T* __restrict__ slots) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sA = reinterpret_cast<T*>(smem_raw);  // [w][R] this CTA's rows, column-major
    __shared__ int sh_flag;
    constexpr int NW = kQrThreads / 32;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int row0 = g * R;
    const int nrows = max(0, min(R, m - row0));
    // the sums of squares and alpha alternate between two buffers by column parity:
    // a column without a reflector passes only one barrier, so the next column's
    // writes must not land where a slower CTA may still be reading
    T* s_ss = slots;                 // [2][G]
    T* s_alpha = slots + 2 * G;      // [2]
    T* s_w = slots + 2 * G + 2;      // [G][kQrMaxLeaf]
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < nrows; r += kQrThreads)
            cp_async_elem<T>(sA + c * R + r, A + (int64_t)(row0 + r) + (int64_t)c * lda);
    cp_async_wait_all();
    __syncthreads();
    unsigned int target = 0;
    bool ok = true;
    const int kmax = min(m, w);
    // warp 0's sum of squares of column jj below the diagonal (valid when have_ss)
    T ss = T(0);
    bool have_ss = false;
    for (int jj = 0; jj < kmax && ok; ++jj) {
        const int lj = jj - row0;                        // local row of jj (owned if 0 <= lj < nrows)
        const bool own_j = lj >= 0 && lj < nrows;
        const int rs = max(0, lj + 1);                   // first local row below jj
        const int par = jj & 1;
        if (warp == 0) {
            __syncwarp();  // column jj's last update came from other lanes of this warp
            if (!have_ss) {
                T s = T(0);
                for (int r = rs + lane; r < nrows; r += 32) {
                    const T x = sA[jj * R + r];
                    s = fma(x, x, s);
                }
                ss = warp_allsum(s);
            }
            if (lane == 0) {
                s_ss[par * G + g] = ss;
                if (own_j) s_alpha[par] = sA[jj * R + lj];
            }
        }
        have_ss = false;
        target += G;
        if (!lu_grid_barrier(sync, target, &sh_flag)) {
            ok = false;
            break;
        }
        // the reflector, formed identically in every warp of every CTA
        const T sum = warp_sum_slots(s_ss + par * G, G, 1, lane);
        const T alpha = __ldcg(&s_alpha[par]);
        if (sum == T(0)) {
            // nothing below the diagonal: H_j = I (tau = 0), the column stays as it is
            if (g == 0 && tid == 0) tau[jj] = T(0);
            continue;
        }
        const T norm = sqrt(fma(alpha, alpha, sum));
        const T beta = alpha >= T(0) ? -norm : norm;
        const T t = (beta - alpha) / beta;
        const T scale = T(1) / (alpha - beta);
        if (g == 0 && tid == 0) tau[jj] = t;
        for (int r = rs + tid; r < nrows; r += kQrThreads) sA[jj * R + r] *= scale;
        if (own_j && tid == 0) sA[jj * R + lj] = beta;
        __syncthreads();
        // partial w_c = A(jj, c) + sum_{i > jj} v_i A(i, c) of this warp's columns
        for (int c = jj + 1 + warp; c < w; c += NW) {
            T acc = T(0);
            for (int r = rs + lane; r < nrows; r += 32) acc = fma(sA[jj * R + r], sA[c * R + r], acc);
            acc = warp_allsum(acc);
            if (own_j) acc += sA[c * R + lj];
            if (lane == 0) s_w[g * kQrMaxLeaf + c] = acc;
        }
        target += G;
        if (!lu_grid_barrier(sync, target, &sh_flag)) {
            ok = false;
            break;
        }
        // rank-1 update A(jj:, c) -= v (tau w_c) of this warp's columns, each w_c the
        // G partials summed in a fixed order; warp 0 also forms the next column's
        // sum of squares below its diagonal
        const int rs1 = max(0, lj + 2);
        for (int c = jj + 1 + warp; c < w; c += NW) {
            const T tw = t * warp_sum_slots(s_w + c, G, kQrMaxLeaf, lane);
            T s = T(0);
            for (int r = rs + lane; r < nrows; r += 32) {
                const T x = fma(-sA[jj * R + r], tw, sA[c * R + r]);
                sA[c * R + r] = x;
                if (r >= rs1) s = fma(x, x, s);
            }
            if (own_j && lane == 0) sA[c * R + lj] -= tw;
            if (c == jj + 1) {
                ss = warp_allsum(s);
                have_ss = true;
            }
        }
    }
    __syncthreads();
    if (ok)
        for (int c = 0; c < w; ++c)
            for (int r = tid; r < nrows; r += kQrThreads) A[(int64_t)(row0 + r) + (int64_t)c * lda] = sA[c * R + r];
    lu_grid_exit(sync);
}

// Transposed-operand product C(M x N) = A(K x M)^T B(K x N): 64 x 64 output
// tiles, 4 x 4 outputs per thread.  K is cut into fixed slices of kTnSlice rows;
// every slice's partial product is summed from zero and the partials are added
// in slice order, whether one CTA runs all slices (split = 0) or each slice has
// its own CTA (split = 1, blockIdx.z = slice, partials to P[s] (M x N, ld = M)
// for qr_splitk_reduce).  So the result does not depend on how a product is cut
// into launches.  The K rows stream through shared memory in chunks of kTnChunk
// rows by asynchronous element copies, two chunks in flight, so a chunk's global
// latency is paid once and overlaps the previous chunk's arithmetic.
constexpr int kTnBM = 64, kTnBN = 64, kTnSlice = 128, kTnChunk = 64, kTnPad = kTnBM + 1;

template <typename T>
constexpr size_t gemm_tn_smem() {
    return sizeof(T) * 2 * 2 * kTnChunk * kTnPad;
}

template <typename T>
__global__ void __launch_bounds__(256) gemm_tn_kernel(int M, int N, int64_t K, int split, const T* __restrict__ A,
                                                      int64_t lda, const T* __restrict__ B, int64_t ldb,
                                                      T* __restrict__ C, int64_t ldc) {
    static_assert(kTnSlice % kTnChunk == 0, "a slice is whole chunks");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // buf[b][0][k][i] = A(k0 + k, i0 + i), buf[b][1][k][j] = B(k0 + k, j0 + j)
    T* buf = reinterpret_cast<T*>(smem_raw);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * kTnBM, j0 = blockIdx.y * kTnBN;
    const int64_t nsl = (K + kTnSlice - 1) / kTnSlice;
    const int64_t s0 = split ? (int64_t)blockIdx.z : 0, s1 = split ? s0 + 1 : nsl;
    const int64_t kbeg = s0 * kTnSlice, kend = min(K, s1 * kTnSlice);
    const int64_t nch = (kend - kbeg + kTnChunk - 1) / kTnChunk;
    auto issue = [&](int64_t q) {
        T* sA = buf + (size_t)(q & 1) * 2 * kTnChunk * kTnPad;
        T* sB = sA + kTnChunk * kTnPad;
        const int64_t k0 = kbeg + q * kTnChunk;
        const int64_t ke = min(kend, k0 + kTnChunk);
        for (int e = tid; e < kTnChunk * kTnBM; e += 256) {
            const int kk = e & (kTnChunk - 1), ii = e / kTnChunk;
            const int64_t k = k0 + kk;
            if (k < ke && i0 + ii < M)
                cp_async_elem<T>(sA + kk * kTnPad + ii, A + k + (int64_t)(i0 + ii) * lda);
            else
                sA[kk * kTnPad + ii] = T(0);
            if (k < ke && j0 + ii < N)
                cp_async_elem<T>(sB + kk * kTnPad + ii, B + k + (int64_t)(j0 + ii) * ldb);
            else
                sB[kk * kTnPad + ii] = T(0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    T tot[4][4], acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) tot[x][y] = acc[x][y] = T(0);
    if (nch > 0) issue(0);
    if (nch > 1) issue(1);
    for (int64_t q = 0; q < nch; ++q) {
        if (q + 1 < nch)
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        else
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const T* sA = buf + (size_t)(q & 1) * 2 * kTnChunk * kTnPad;
        const T* sB = sA + kTnChunk * kTnPad;
#pragma unroll 8
        for (int kk = 0; kk < kTnChunk; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = sA[kk * kTnPad + tx + 16 * x];
#pragma unroll
            for (int y = 0; y < 4; ++y) b[y] = sB[kk * kTnPad + ty + 16 * y];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        // a slice ends: its partial product joins the total (slice order)
        const int64_t kq = kbeg + (q + 1) * kTnChunk;
        if (kq % kTnSlice == 0 || q + 1 == nch) {
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    tot[x][y] += acc[x][y];
                    acc[x][y] = T(0);
                }
        }
        __syncthreads();
        if (q + 2 < nch) issue(q + 2);
    }
    T* out = split ? C + (int64_t)blockIdx.z * M * N : C;
    const int64_t ldo = split ? (int64_t)M : ldc;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int i = i0 + tx + 16 * x, j = j0 + ty + 16 * y;
            if (i < M && j < N) out[i + (int64_t)j * ldo] = tot[x][y];
        }
}

// C(M x N) = sum over s = 0 .. S-1 of P[s], in that order (deterministic).
template <typename T>
__global__ void qr_splitk_reduce(int M, int N, int S, const T* __restrict__ P, T* __restrict__ C, int64_t ldc) {
    const int64_t total = (int64_t)M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int q = 0; q < S; ++q) s += P[(int64_t)q * total + e];
        const int64_t i = e % M, j = e / M;
        C[i + j * ldc] = s;
    }
}

// V (m x w, ld = ldv) := the unit lower trapezoidal reflector block stored
// below the diagonal of A(m x w): ones on the diagonal, zeros above it.
template <typename T>
__global__ void qr_extract_v(int64_t m, int w, const T* __restrict__ A, int64_t lda, T* __restrict__ V, int64_t ldv) {
    const int64_t total = m * w;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % m;
        const int j = (int)(e / m);
        V[i + (int64_t)j * ldv] = i > j ? A[i + (int64_t)j * lda] : (i == j ? T(1) : T(0));
    }
}

// Compact-WY factor (larft, forward, columnwise) from the Gram matrix
// Gm = V^T V (w x w) and tau: T(j, j) = tau_j and, for i < j,
// T(0:j, j) = -tau_j T(0:j, 0:j) Gm(0:j, j); the strict lower part is zeroed.
// One CTA; column j depends on the columns before it.
template <typename T>
__global__ void __launch_bounds__(256) qr_larft_kernel(int w, const T* __restrict__ Gm, int64_t ldg,
                                                       const T* __restrict__ tau, T* __restrict__ Tm, int64_t ldt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sT = reinterpret_cast<T*>(smem_raw);  // [w][w] column-major
    T* z = sT + (size_t)w * w;               // [w]
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) sT[e] = T(0);
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        const T tj = tau[j];
        for (int i = threadIdx.x; i < j; i += blockDim.x) z[i] = Gm[i + (int64_t)j * ldg];
        __syncthreads();
        // T(0:j, j) = -tau_j T(0:j, 0:j) z, T upper triangular: row i sums over l >= i
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            T s = T(0);
            for (int l = i; l < j; ++l) s = fma(sT[i + l * w], z[l], s);
            sT[i + j * w] = -tj * s;
        }
        if (threadIdx.x == 0) sT[j + j * w] = tj;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) Tm[(e % w) + (int64_t)(e / w) * ldt] = sT[e];
}

}  // namespace

namespace {

constexpr int64_t kQrPartCap = 8 << 20;  // elements of one split-K partial buffer

// Workspace of one QR factorization, carved from the handle's device buffer.
template <typename T>
struct QrWork {
    T* V[2];      // explicit reflector blocks of panels k (parity), m x nbmax
    T* Tm[2];     // their compact-WY factors, nbmax x nbmax
    T* Vp;        // left half of a split panel, m x kQrMaxLeaf
    T* Tp;        // its factor, kQrMaxLeaf^2
    T* Gm;        // Gram matrix V^T V, nbmax^2
    T* Whi[2];    // V^T C and T^T (V^T C) on the panel stream, nbmax x nbmax
    T* Wlo[2];    // the same on the update stream, nbmax x n
    T* part[2];   // split-K partials: [0] panel stream, [1] update stream
    int nbmax;
    // tensor-core update C -= V W2 (FP32 only): packed V per panel parity, packed W2 per stream
    int prec = -1;
    char* Vpk[2] = {nullptr, nullptr};
    char* Wpk[2] = {nullptr, nullptr};
    static size_t tc_bytes(int prec, int64_t m, int64_t n, int nbmax) {
        if (prec < 0) return 0;
        const size_t seg = 2 * (size_t)lu_pack_segments(lu_prec_pack_fmt(prec));
        return (2 * (size_t)m * nbmax + (size_t)nbmax * nbmax + (size_t)n * nbmax) * seg + 4 * 256;
    }
    static size_t bytes(int64_t m, int64_t n, int nbmax) {
        const size_t e = 2 * (size_t)m * nbmax + 2 * (size_t)nbmax * nbmax + (size_t)m * kQrMaxLeaf +
                         (size_t)kQrMaxLeaf * kQrMaxLeaf + (size_t)nbmax * nbmax + 2 * (size_t)nbmax * nbmax +
                         2 * (size_t)nbmax * n + 2 * (size_t)kQrPartCap + 16 * 8;
        return e * sizeof(T) + 16 * 256;
    }
    void carve(char* base, int64_t m, int64_t n, int nb) {
        nbmax = nb;
        size_t off = 0;
        auto take = [&](size_t elems) {
            T* p = reinterpret_cast<T*>(base + off);
            off += (elems * sizeof(T) + 255) / 256 * 256;
            return p;
        };
        for (int i = 0; i < 2; ++i) V[i] = take((size_t)m * nb);
        for (int i = 0; i < 2; ++i) Tm[i] = take((size_t)nb * nb);
        Vp = take((size_t)m * kQrMaxLeaf);
        Tp = take((size_t)kQrMaxLeaf * kQrMaxLeaf);
        Gm = take((size_t)nb * nb);
        for (int i = 0; i < 2; ++i) Whi[i] = take((size_t)nb * nb);
        for (int i = 0; i < 2; ++i) Wlo[i] = take((size_t)nb * n);
        for (int i = 0; i < 2; ++i) part[i] = take((size_t)kQrPartCap);
        if (prec >= 0) {
            const size_t seg = 2 * (size_t)lu_pack_segments(lu_prec_pack_fmt(prec));
            auto takeb = [&](size_t bytes) {
                char* p = base + off;
                off += (bytes + 255) / 256 * 256;
                return p;
            };
            for (int i = 0; i < 2; ++i) Vpk[i] = takeb((size_t)m * nb * seg);
            Wpk[0] = takeb((size_t)nb * nb * seg);
            Wpk[1] = takeb((size_t)n * nb * seg);
        }
    }
};

// C(M x N) = A^T B with A (K x M) and B (K x N), split along K when the output
// has too few tiles to fill the GPU.
template <typename T>
int qr_gemm_tn(lu_context* c, cudaStream_t st, int M, int N, int64_t K, const T* A, int64_t lda, const T* B,
               int64_t ldb, T* C, int64_t ldc, T* part) {
    if (M <= 0 || N <= 0) return LU_SUCCESS;
    const int64_t tiles = lu_cdiv(M, kTnBM) * lu_cdiv(N, kTnBN);
    const int64_t nsl = lu_cdiv(std::max<int64_t>(K, 1), kTnSlice);
    // one CTA per K slice when the output alone has too few tiles to fill the GPU
    // and the partials fit (the choice changes the speed, not the bits)
    const bool split = tiles < 2 * (int64_t)c->num_sms && nsl > 1 && nsl <= 65535 &&
                       nsl * (int64_t)M * N <= kQrPartCap;
    LuProfScope prof(st, LU_K_GEMM, sizeof(T) * ((double)K * (M + N) + (double)M * N), 2.0 * M * N * K);
    const dim3 grid((unsigned)lu_cdiv(M, kTnBM), (unsigned)lu_cdiv(N, kTnBN), split ? (unsigned)nsl : 1u);
    LU_TRY(lu_func_smem(gemm_tn_kernel<T>, (int)gemm_tn_smem<T>()));
    gemm_tn_kernel<T><<<grid, 256, gemm_tn_smem<T>(), st>>>(M, N, K, split ? 1 : 0, A, lda, B, ldb, split ? part : C,
                                                           ldc);
    LU_CHECK_LAUNCH();
    if (split) {
        const int64_t total = (int64_t)M * N;
        qr_splitk_reduce<T><<<(unsigned)std::min<int64_t>(lu_cdiv(total, 256), 4 * (int64_t)c->num_sms), 256, 0, st>>>(
            M, N, (int)nsl, part, C, ldc);
        LU_CHECK_LAUNCH();
    }
    return LU_SUCCESS;
}

// Q^T applied to columns [cb, ce) of rows [r0, m): C -= V (T^T (V^T C)),
// V (m - r0) x kb with ld ldv, T kb x kb with ld kb.
// Optional tensor-core form of the last product: V packed once per panel (vpk),
// W2 packed per call into wpk, the tcgen05 update on C with the given tile
// counter; prec < 0 or a width that is not a multiple of 64 keeps the CUDA cores.
struct QrTc {
    int prec = -1;
    const char* vpk = nullptr;
    char* wpk = nullptr;
    int* counter = nullptr;
};

template <typename T>
int qr_apply(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t m, int64_t r0, int kb, int64_t cb,
             int64_t ce, const T* V, int64_t ldv, const T* Tm, T* W, T* W2, int64_t wcap, T* part,
             const QrTc& tc = QrTc()) {
    const int64_t rows = m - r0, nc = ce - cb;
    if (nc <= 0 || rows <= 0 || kb <= 0) return LU_SUCCESS;
    if ((int64_t)kb * nc > wcap) return LU_ERR_UNSUPPORTED;  // W and W2 hold kb x nc each
    T* C = A + r0 + cb * lda;
    LU_TRY(qr_gemm_tn<T>(c, st, kb, (int)nc, rows, V, ldv, C, lda, W, kb, part));
    LU_TRY(qr_gemm_tn<T>(c, st, kb, (int)nc, kb, Tm, kb, W, kb, W2, kb, part));
    if constexpr (sizeof(T) == 4) {
        if (tc.prec >= 0 && tc.vpk && kb % 64 == 0) {
            const int fmt = lu_prec_pack_fmt(tc.prec);
            const int sg = lu_pack_segments(fmt);
            LU_TRY(lu_launch_pack_cols(st, fmt, (const float*)W2, kb, nc, kb, tc.wpk));
            LU_CHECK_CUDA(cudaMemsetAsync(tc.counter, 0, sizeof(int), st));
            return lu_launch_tc_update(st, LU_TC_KIND_F16, tc.prec == LU_TU_FP16 ? LU_TC_FMT_F16 : LU_TC_FMT_BF16,
                                       (float*)A, lda, r0, rows, cb, nc, (int64_t)kb * sg, tc.vpk, rows, tc.wpk, nc,
                                       1.0f, tc.counter, &c->sync[0].error, c->num_sms, 256);
        }
    }
    return lu_launch_gemm_update<T>(st, rows, nc, kb, V, ldv, W2, kb, C, lda);
}

// Explicit V (rows x w) and its factor T (w x w) for reflectors already in A(r0:m, j0:j0+w).
template <typename T>
int qr_form_vt(lu_context* c, cudaStream_t st, const T* A, int64_t lda, int64_t m, int64_t r0, int64_t j0, int w,
               const T* tau, T* V, T* Tm, T* Gm, T* part) {
    const int64_t rows = m - r0;
    {
        LuProfScope prof(st, LU_K_OTHER, 2.0 * sizeof(T) * rows * w, 0.0);
        qr_extract_v<T><<<(unsigned)std::min<int64_t>(lu_cdiv(rows * w, 256), 4 * (int64_t)c->num_sms), 256, 0, st>>>(
            rows, w, A + r0 + j0 * lda, lda, V, rows);
        LU_CHECK_LAUNCH();
    }
    LU_TRY(qr_gemm_tn<T>(c, st, w, w, rows, V, rows, V, rows, Gm, w, part));
    const size_t smem = sizeof(T) * ((size_t)w * w + w);
    LU_TRY(lu_func_smem(qr_larft_kernel<T>, (int)smem));
    LuProfScope prof(st, LU_K_OTHER, sizeof(T) * 2.0 * w * w, (double)w * w * w / 3.0);
    qr_larft_kernel<T><<<1, 256, smem, st>>>(w, Gm, w, tau + j0, Tm, w);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

template <typename T>
int qr_leaf(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t m, int64_t j0, int w, T* tau) {
    const int64_t rows = m - j0;
    if (rows <= 0 || w <= 0) return LU_SUCCESS;
    // as many rows per CTA as shared memory holds: fewer CTAs make the two grid
    // barriers and the cross-CTA sums of every column cheaper, and the per-column
    // work of a CTA stays small (R x w multiply-adds over 256 threads)
    const int64_t Rmax = std::max<int64_t>(32, (int64_t)(200 * 1024 / (sizeof(T) * (size_t)w)) / 32 * 32);
    const int64_t G0 = std::min<int64_t>({(int64_t)c->num_sms, (int64_t)LU_PF_MAX_CTAS, lu_cdiv(rows, Rmax)});
    const int64_t R = lu_cdiv(lu_cdiv(rows, G0), 32) * 32;
    const int64_t G = lu_cdiv(rows, R);
    const size_t smem = sizeof(T) * (size_t)R * w;
    if (smem > 200 * 1024 || G > LU_PF_MAX_CTAS) return LU_ERR_UNSUPPORTED;
    LU_TRY(lu_func_smem(qr_leaf_kernel<T>, (int)smem));
    LuProfScope prof(st, LU_K_PANEL, 2.0 * sizeof(T) * rows * w, 2.0 * rows * w * w);
    qr_leaf_kernel<T><<<(unsigned)G, kQrThreads, smem, st>>>(A + j0 + j0 * lda, lda, (int)rows, w, (int)R, tau + j0,
                                                             &c->sync[0], reinterpret_cast<T*>(c->pf_slots));
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

// PF: Householder QR of columns [j0, j0+w) over rows [j0, m); w <= 2 * kQrMaxLeaf.
template <typename T>
int qr_panel(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t m, int64_t j0, int w, T* tau, QrWork<T>& wk) {
    if (w <= kQrMaxLeaf) return qr_leaf<T>(c, st, A, lda, m, j0, w, tau);
    const int w1 = kQrMaxLeaf;
    LU_TRY(qr_leaf<T>(c, st, A, lda, m, j0, w1, tau));
    LU_TRY(qr_form_vt<T>(c, st, A, lda, m, j0, j0, w1, tau, wk.Vp, wk.Tp, wk.Gm, wk.part[0]));
    LU_TRY(qr_apply<T>(c, st, A, lda, m, j0, w1, j0 + w1, j0 + w, wk.Vp, m - j0, wk.Tp, wk.Whi[0], wk.Whi[1],
                       (int64_t)wk.nbmax * wk.nbmax, wk.part[0]));
    return qr_leaf<T>(c, st, A, lda, m, j0 + w1, w - w1, tau);
}

}  // namespace

template <typename T>
static int qr_factor(lu_context* c, int64_t m, int64_t n, T* A, int64_t lda, T* tau, const lu_opts& o,
                     int32_t* info, int prec = -1) {
    const int64_t kmax = std::min(m, n);
    std::vector<int64_t> s;
    int wmin = 1, wmax = 1;
    lu_panel_bounds(kmax, o, &s, &wmin, &wmax);
    if (wmax > 2 * kQrMaxLeaf) return LU_ERR_UNSUPPORTED;
    LU_TRY(lu_ctx_reserve(c, std::max(m, n), wmin));
    LU_TRY(lu_mx_reserve(c, QrWork<T>::bytes(m, n, wmax) + QrWork<T>::tc_bytes(prec, m, n, wmax)));
    QrWork<T> wk;
    wk.prec = prec;
    wk.carve((char*)c->mx, m, n, wmax);
    cudaStream_t user = c->user;
    LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[0], 0, sizeof(LuSync), user));
    if (kmax == 0) return lu_launch_finish_info(user, &c->sync[0], info);
    LU_CHECK_CUDA(cudaEventRecord(c->ev_fork, user));
    LU_CHECK_CUDA(cudaStreamWaitEvent(c->hi, c->ev_fork, 0));
    LU_CHECK_CUDA(cudaStreamWaitEvent(c->lo, c->ev_fork, 0));
    const int64_t nk = (int64_t)s.size() - 1;
    cudaStream_t hi = c->hi, lo = c->lo;
    auto width = [&](int64_t k) { return (int)(s[(size_t)k + 1] - s[(size_t)k]); };
    // PF_k, then V_k and T_k (parity k) for the updates of step k
    auto panel = [&](int64_t k) -> int {
        const int64_t k0 = s[(size_t)k];
        LU_TRY(qr_panel<T>(c, hi, A, lda, m, k0, width(k), tau, wk));
        if (k0 + width(k) < n) {
            LU_TRY(qr_form_vt<T>(c, hi, A, lda, m, k0, k0, width(k), tau, wk.V[k & 1], wk.Tm[k & 1], wk.Gm,
                                 wk.part[0]));
            if constexpr (sizeof(T) == 4)
                if (wk.prec >= 0 && width(k) % 64 == 0)
                    LU_TRY(lu_launch_pack_rows(hi, lu_prec_pack_fmt(wk.prec), (const float*)wk.V[k & 1], m - k0,
                                               m - k0, width(k), wk.Vpk[k & 1]));
        }
        return LU_SUCCESS;
    };
    // TU_k on columns [cb, ce) with the narrow buffers (which = 0: at most one panel
    // wide, the look-ahead's TU_k^L) or the wide ones (1: any width)
    auto tu = [&](cudaStream_t st, int64_t k, int64_t cb, int64_t ce, int which) -> int {
        const int64_t k0 = s[(size_t)k];
        T** W = which ? wk.Wlo : wk.Whi;
        const int64_t cap = which ? (int64_t)wk.nbmax * n : (int64_t)wk.nbmax * wk.nbmax;
        QrTc tc;
        if (wk.prec >= 0) {
            tc.prec = wk.prec;
            tc.vpk = wk.Vpk[k & 1];
            tc.wpk = wk.Wpk[which];
            tc.counter = (int*)&c->sync[4 + which].ticket;
        }
        return qr_apply<T>(c, st, A, lda, m, k0, width(k), cb, ce, wk.V[k & 1], m - k0, wk.Tm[k & 1], W[0], W[1],
                           cap, wk.part[which], tc);
    };
    LU_TRY(panel(0));
    for (int64_t k = 0; k < nk; ++k) {
        const int64_t c1 = s[(size_t)k + 1];                                // first column right of panel k
        const int64_t c2 = k + 1 < nk ? s[(size_t)k + 2] : c1;             // end of panel k+1
        if (o.lookahead) {
            // PU(k+1) = TU_k on panel k+1, then PF_{k+1}, beside TU_k on the rest
            if (k + 1 < nk) LU_TRY(tu(hi, k, c1, c2, 0));
            LU_CHECK_CUDA(cudaEventRecord(c->ev_pf, hi));
            LU_CHECK_CUDA(cudaStreamWaitEvent(lo, c->ev_pf, 0));
            LU_TRY(tu(lo, k, c2, n, 1));
            LU_CHECK_CUDA(cudaEventRecord(c->ev_tu, lo));
            if (k + 1 < nk) {
                LU_TRY(panel(k + 1));
                LU_CHECK_CUDA(cudaStreamWaitEvent(hi, c->ev_tu, 0));
            }
        } else {
            LU_TRY(tu(hi, k, c1, n, 1));  // every column right of the panel: the wide buffers
            if (k + 1 < nk) LU_TRY(panel(k + 1));
        }
    }
    LU_CHECK_CUDA(cudaEventRecord(c->ev_join_hi, hi));
    LU_CHECK_CUDA(cudaEventRecord(c->ev_join_lo, lo));
    LU_CHECK_CUDA(cudaStreamWaitEvent(user, c->ev_join_hi, 0));
    LU_CHECK_CUDA(cudaStreamWaitEvent(user, c->ev_join_lo, 0));
    return lu_launch_finish_info(user, &c->sync[0], info);
}

extern "C" int lu_geqrf_ex(lu_handle h, lu_dtype dtype, int64_t m, int64_t n, void* A, int64_t lda, void* tau,
                           const lu_opts* opts, int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (m > 0 && n > 0 && !A) return -5;
    if (lda < std::max<int64_t>(1, m)) return -6;
    if (std::min(m, n) > 0 && !tau) return -7;
    lu_opts o;
    lu_default_opts(&o);
    o.nb = 128;
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -8;
    if (!info) return -9;
    if (o.nb == 0) o.nb = 128;
    if (o.lookahead > 1 || o.rtm) return LU_ERR_UNSUPPORTED;
    if (m > INT32_MAX / 2 || n > INT32_MAX / 2) return LU_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(h->mu);
    if (dtype == LU_F64) return qr_factor<double>(h, m, n, (double*)A, lda, (double*)tau, o, info);
    return qr_factor<float>(h, m, n, (float*)A, lda, (float*)tau, o, info);
}

extern "C" int lu_geqrf_mixed_ex(lu_handle h, lu_prec prec, int64_t m, int64_t n, float* A, int64_t lda, float* tau,
                                 const lu_opts* opts, int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (prec == LU_TU_FP8 || (!lu_prec_is_tc(prec) && prec != LU_TU_F32)) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (m > 0 && n > 0 && !A) return -5;
    if (lda < std::max<int64_t>(1, m)) return -6;
    if (std::min(m, n) > 0 && !tau) return -7;
    lu_opts o;
    lu_default_opts(&o);
    o.nb = 128;
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -8;
    if (!info) return -9;
    if (o.nb == 0) o.nb = 128;
    if (o.lookahead > 1 || o.rtm) return LU_ERR_UNSUPPORTED;
    if (m > INT32_MAX / 2 || n > INT32_MAX / 2) return LU_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(h->mu);
    return qr_factor<float>(h, m, n, A, lda, tau, o, info, lu_prec_is_tc(prec) ? (int)prec : -1);
}
