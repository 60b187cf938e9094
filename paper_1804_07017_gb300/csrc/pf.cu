// Panel factorization PF (RL1 of LU_blk, Sec. 3): [A11; A21] := LU_unb([A11; A21]).
//
// A tall panel is factored recursively: the left half, then the interchanges
// applied to the right half, its TRSM (RL2) and GEMM (RL3) update inside the
// panel, the right half, and finally the right half's interchanges applied to
// the left half.  The recursion bottoms out in a leaf of at most
// LU_PF_MAX_LEAF columns factored column by column by one multi-CTA kernel:
//
//   * the leaf's rows are split across G CTAs, each holding its R x w block
//     in shared memory for the whole leaf;
//   * per column: every CTA finds its local pivot candidate (warp-shuffle
//     argmax, ties to the smallest row), publishes value, row index and the
//     candidate row; one grid barrier; every CTA then picks the global pivot
//     (first maximum), swaps rows, scales the column by a true division and
//     applies the rank-1 update to the remaining leaf columns, fusing the
//     next column's candidate search into that update.
//
// One grid barrier per column is the latency floor of partial pivoting: the
// pivot of column j depends on the fully updated column j.
#include <climits>

#include "internal.h"
#include "profile.h"

namespace {

template <typename T>
__device__ __forceinline__ void argmax_merge(T& v, int& i, T ov, int oi) {
    if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}

template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_merge(v, i, ov, oi);
    }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) pf_leaf_kernel(T* __restrict__ A, int64_t lda, int m, int w,
                                                     int R, int32_t* __restrict__ ipiv,
                                                     int ipiv_add, LuSync* __restrict__ sync,
                                                     T* __restrict__ slots,
                                                     int* __restrict__ slot_idx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sA = reinterpret_cast<T*>(smem_raw);  // [w][R], column-major block of this CTA's rows
    T* prow = sA + (size_t)w * R;             // pivot row (w values)
    T* jrowv = prow + w;                      // previous contents of row jj (w values)
    T* s_rows = jrowv + w;                    // [G][w] every CTA's candidate row
    T* s_cv = s_rows + (size_t)gridDim.x * w; // [G] candidate values
    int* s_ci = reinterpret_cast<int*>(s_cv + gridDim.x);  // [G] candidate rows
    __shared__ T red_v[NT / 32];
    __shared__ int red_i[NT / 32];
    __shared__ T sh_bv;
    __shared__ int sh_bi, sh_p, sh_gw, sh_flag;

    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int row0 = g * R;
    const int nrows = max(0, min(R, m - row0));

    T* cand_val = slots;                                   // [2][MAXC]
    T* cand_row = slots + 2 * LU_PF_MAX_CTAS;              // [2][MAXC][MAXW]
    T* jrow = cand_row + 2 * LU_PF_MAX_CTAS * LU_PF_MAX_LEAF;  // [2][MAXW]
    int* cand_idx = slot_idx;                              // [2][MAXC]

    for (int c = 0; c < w; ++c)
        for (int r = tid; r < nrows; r += NT) sA[c * R + r] = A[(int64_t)(row0 + r) + (int64_t)c * lda];
    __syncthreads();

    T bv = T(-1);
    int bi = INT_MAX;
    for (int r = tid; r < nrows; r += NT) argmax_merge(bv, bi, (T)fabs(sA[r]), row0 + r);

    for (int jj = 0; jj < w; ++jj) {
        const int buf = jj & 1;
        // ---- local candidate (block argmax) ----
        warp_argmax(bv, bi);
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        if (warp == 0) {
            T v = (lane < NT / 32) ? red_v[lane] : T(-1);
            int i = (lane < NT / 32) ? red_i[lane] : INT_MAX;
            warp_argmax(v, i);
            if (lane == 0) {
                sh_bv = v;
                sh_bi = i;
            }
        }
        __syncthreads();
        // ---- publish candidate (value, row, row contents) and row jj ----
        const int my_bi = sh_bi;
        if (tid == 0) {
            cand_val[buf * LU_PF_MAX_CTAS + g] = sh_bv;
            cand_idx[buf * LU_PF_MAX_CTAS + g] = my_bi;
        }
        if (tid < w && my_bi != INT_MAX)
            cand_row[(buf * LU_PF_MAX_CTAS + g) * LU_PF_MAX_LEAF + tid] = sA[tid * R + (my_bi - row0)];
        if (jj >= row0 && jj < row0 + nrows && tid < w)
            jrow[buf * LU_PF_MAX_LEAF + tid] = sA[tid * R + (jj - row0)];
        if (tid < w) __threadfence();
        if (!lu_grid_barrier(sync, (unsigned)(jj + 1) * (unsigned)G, &sh_flag)) break;
        // ---- one round trip: every candidate's value, index and row, plus row jj ----
        for (int q = tid; q < G; q += NT) {
            s_cv[q] = __ldcg(&cand_val[buf * LU_PF_MAX_CTAS + q]);
            s_ci[q] = __ldcg(&cand_idx[buf * LU_PF_MAX_CTAS + q]);
        }
        for (int e = tid; e < G * w; e += NT) {
            const int q = e / w, c = e - q * w;
            s_rows[e] = __ldcg(&cand_row[(buf * LU_PF_MAX_CTAS + q) * LU_PF_MAX_LEAF + c]);
        }
        if (tid < w) jrowv[tid] = __ldcg(&jrow[buf * LU_PF_MAX_LEAF + tid]);
        __syncthreads();
        // ---- global pivot: first maximum over all CTAs' candidates ----
        if (warp == 0) {
            T v = T(-1);
            int i = INT_MAX, q_best = -1;
            for (int q = lane; q < G; q += 32) {
                const T cv = s_cv[q];
                const int ci = s_ci[q];
                if (ci != INT_MAX && (cv > v || (cv == v && ci < i))) {
                    v = cv;
                    i = ci;
                    q_best = q;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                T ov = __shfl_xor_sync(0xffffffffu, v, o);
                int oi = __shfl_xor_sync(0xffffffffu, i, o);
                int oq = __shfl_xor_sync(0xffffffffu, q_best, o);
                if (ov > v || (ov == v && oi < i)) {
                    v = ov;
                    i = oi;
                    q_best = oq;
                }
            }
            if (lane == 0) {
                sh_p = (i == INT_MAX) ? jj : i;
                sh_gw = (i == INT_MAX) ? -1 : q_best;
            }
        }
        __syncthreads();
        const int p = sh_p, gw = sh_gw;
        if (tid < w) prow[tid] = (gw >= 0) ? s_rows[gw * w + tid] : jrowv[tid];
        if (g == 0 && tid == 0) ipiv[jj] = p + 1 + ipiv_add;
        __syncthreads();
        // ---- interchange rows jj and p (within this leaf's columns) ----
        if (p != jj && tid < w) {
            if (p >= row0 && p < row0 + nrows) sA[tid * R + (p - row0)] = jrowv[tid];
            if (jj >= row0 && jj < row0 + nrows) sA[tid * R + (jj - row0)] = prow[tid];
        }
        const T piv = prow[jj];
        if (piv == T(0) && g == 0 && tid == 0) atomicCAS(&sync->info, 0, jj + 1 + ipiv_add);
        __syncthreads();
        // ---- scale column jj, rank-1 update, next column's local candidate ----
        bv = T(-1);
        bi = INT_MAX;
        const bool has_next = jj + 1 < w;
        for (int r = tid; r < nrows; r += NT) {
            const int gr = row0 + r;
            if (gr <= jj) continue;
            if (piv != T(0)) {
                const T l = sA[jj * R + r] / piv;
                sA[jj * R + r] = l;
                for (int c = jj + 1; c < w; ++c) sA[c * R + r] = fma(-l, prow[c], sA[c * R + r]);
            }
            if (has_next) argmax_merge(bv, bi, (T)fabs(sA[(jj + 1) * R + r]), gr);
        }
    }
    __syncthreads();
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < nrows; r += NT) A[(int64_t)(row0 + r) + (int64_t)c * lda] = sA[c * R + r];
    lu_grid_exit(sync);
}

constexpr int kPfThreads = 256;

}  // namespace

// Leaf shape: as few CTAs as the shared-memory budget allows (fewer CTAs make the
// per-column grid barrier cheaper), rows per CTA a multiple of 32.
bool lu_pf_leaf_shape(int64_t m, int w, int esize, int max_ctas, int64_t* R_out, int64_t* G_out, size_t* smem_out) {
    auto smem_of = [&](int64_t R, int64_t G) {
        return (size_t)(R * w + 2 * w + G * w + G) * esize + (size_t)G * sizeof(int);
    };
    int64_t R = ((int64_t)LU_PF_SMEM_BUDGET / esize - 2 * w) / w;  // rows that fit with no exchange area
    R = R / 32 * 32;
    int64_t Rmin = std::max<int64_t>(32, lu_cdiv(lu_cdiv(m, max_ctas), 32) * 32);
    if (R > lu_cdiv(m, 32) * 32) R = lu_cdiv(m, 32) * 32;
    while (R >= Rmin) {
        const int64_t G = lu_cdiv(m, R);
        if (G <= max_ctas && smem_of(R, G) <= (size_t)LU_PF_SMEM_BUDGET) {
            *R_out = R;
            *G_out = G;
            *smem_out = smem_of(R, G);
            return true;
        }
        R -= 32;
    }
    return false;
}

template <typename T>
int lu_launch_pf_leaf(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t m, int w,
                      int32_t* ipiv, int64_t ipiv_add, int max_ctas) {
    if (w < 1 || w > LU_PF_MAX_LEAF || m < w) return LU_ERR_UNSUPPORTED;
    if (max_ctas <= 0 || max_ctas > LU_PF_MAX_CTAS) max_ctas = LU_PF_MAX_CTAS;
    int64_t R = 0, G = 0;
    size_t smem = 0;
    if (!lu_pf_leaf_shape(m, w, (int)sizeof(T), max_ctas, &R, &G, &smem)) return LU_ERR_UNSUPPORTED;
    LU_TRY(lu_func_smem(pf_leaf_kernel<T, kPfThreads>, LU_PF_SMEM_BUDGET));
    T* slots = reinterpret_cast<T*>(c->pf_slots);
    int* slot_idx = reinterpret_cast<int*>(reinterpret_cast<char*>(c->pf_slots) +
                                           sizeof(double) * (2 * LU_PF_MAX_CTAS * (LU_PF_MAX_LEAF + 1) +
                                                             2 * LU_PF_MAX_LEAF));
    LuProfScope prof(st, LU_K_PANEL, 2.0 * m * w * sizeof(T), (double)m * w * w);
    pf_leaf_kernel<T, kPfThreads><<<(unsigned)G, kPfThreads, smem, st>>>(A, lda, (int)m, w, (int)R, ipiv,
                                                                (int)ipiv_add, &c->sync[0], slots,
                                                                slot_idx);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

namespace {

// One level of the recursive panel: columns [j0, j0+width) over rows [j0, M);
// [pc0, pc0+pw) is the whole panel, whose other columns a cluster leaf updates
// with its own interchanges.
// Runs launch(stream) on the leaf partition's stream when one is active (entered
// and left through events on st, with its context current), else on st.
template <typename F>
int on_leaf_sms(lu_context* c, cudaStream_t st, F&& launch) {
    if (!c->green_active) return launch(st);
    cudaStream_t ls = nullptr;
    LU_TRY(lu_green_leaf_fork(c, st, &ls));
    const int r = launch(ls);
    const int r2 = lu_green_leaf_join(c, st);
    return r != LU_SUCCESS ? r : r2;
}

template <typename T>
int panel_rec(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t M, int64_t j0, int64_t width,
              int32_t* ipiv, const lu_opts& o, int leaf, bool cluster, int64_t pc0, int64_t pw) {
    if (width <= 0) return LU_SUCCESS;
    const int64_t rows = M - j0;
    const int nt_want = sizeof(T) == 4 ? c->pf_threads : 256;
    if (width <= leaf) {
        if (cluster) {
            int C = 0, R = 0, nt = 256;
            size_t smem = 0;
            if (lu_pf_cluster_shape<T>(rows, (int)width, c->pf_smem_budget, &C, &R, &smem, o.pf_ctas, nt_want, &nt))
                return on_leaf_sms(c, st, [&](cudaStream_t ls) {
                    return lu_launch_pf_leaf_cluster<T>(ls, A + j0 + j0 * lda, lda, rows, (int)width, C, R, smem,
                                                        j0 - pc0, pc0 + pw - (j0 + width), ipiv + j0, j0, &c->sync[0],
                                                        0, 0, nt);
                });
            return LU_ERR_UNSUPPORTED;
        }
        return lu_launch_pf_leaf<T>(c, st, A + j0 + j0 * lda, lda, rows, (int)width, ipiv + j0, j0, o.pf_ctas);
    }
    int64_t w1 = ((width / 2 + 7) / 8) * 8;
    if (w1 >= width) w1 = width / 2;
    if (w1 < 1) w1 = 1;
    const int64_t w2 = width - w1;
    // Two sibling leaves (16 columns, or 32 in FP32): the first also forms its sibling's
    // U12 and the second applies the matching rank-w1 update in its prologue (no
    // launch in between).
    const int64_t pair_max = sizeof(T) == 4 ? 32 : 16;
    if (cluster && w1 <= pair_max && w2 <= pair_max && w1 <= leaf && w2 <= leaf && lu_pf_leaf_pairs_supported()) {
        int Ca = 0, Ra = 0, Cb = 0, Rb = 0, nta = 256, ntb = 256;
        size_t sa = 0, sb = 0;
        if (lu_pf_cluster_shape<T>(rows, (int)w1, c->pf_smem_budget, &Ca, &Ra, &sa, o.pf_ctas, nt_want, &nta) &&
            lu_pf_cluster_shape<T>(rows - w1, (int)w2, c->pf_smem_budget, &Cb, &Rb, &sb, o.pf_ctas, nt_want, &ntb)) {
            const int64_t jb = j0 + w1;
            return on_leaf_sms(c, st, [&](cudaStream_t ls) {
                LU_TRY(lu_launch_pf_leaf_cluster<T>(ls, A + j0 + j0 * lda, lda, rows, (int)w1, Ca, Ra, sa, j0 - pc0,
                                                    pc0 + pw - (j0 + w1), ipiv + j0, j0, &c->sync[0], (int)w2, 0,
                                                    nta));
                return lu_launch_pf_leaf_cluster<T>(ls, A + jb + jb * lda, lda, rows - w1, (int)w2, Cb, Rb, sb,
                                                    jb - pc0, pc0 + pw - (jb + w2), ipiv + jb, jb, &c->sync[0], 0,
                                                    (int)w1, ntb);
            });
        }
    }
    LU_TRY(panel_rec<T>(c, st, A, lda, M, j0, w1, ipiv, o, leaf, cluster, pc0, pw));
    if (!cluster) {
        // interchanges of the left half applied to the right half's columns
        LU_TRY(lu_launch_laswp_plan(st, ipiv, j0, j0 + w1, c->plan_tmp));
        LU_TRY(lu_launch_laswp_apply<T>(st, A, lda, j0 + w1, w2, 0, 0, c->plan_tmp, w1, c->num_sms));
    }
    // RL2 and RL3 restricted to the panel; narrow nodes in one launch (the arrival
    // counter is the ticket word of the panel's sync block, unused by the leaves)
    if (w1 <= 32 && w2 <= 32) {
        LU_TRY(lu_launch_trsm_gemm_narrow<T>(st, M - j0 - w1, w2, w1, A + j0 + j0 * lda, A + j0 + (j0 + w1) * lda,
                                             A + (j0 + w1) + j0 * lda, A + (j0 + w1) + (j0 + w1) * lda, lda,
                                             &c->sync[0].ticket));
    } else {
        LU_TRY(lu_launch_trsm_lunit<T>(st, w1, w2, A + j0 + j0 * lda, lda, A + j0 + (j0 + w1) * lda, lda));
        if (M - j0 - w1 > 0)
            LU_TRY(lu_launch_gemm_update<T>(st, M - j0 - w1, w2, w1, A + (j0 + w1) + j0 * lda, lda,
                                            A + j0 + (j0 + w1) * lda, lda, A + (j0 + w1) + (j0 + w1) * lda, lda));
    }
    LU_TRY(panel_rec<T>(c, st, A, lda, M, j0 + w1, w2, ipiv, o, leaf, cluster, pc0, pw));
    if (!cluster) {
        // interchanges of the right half applied back to the left half's columns
        LU_TRY(lu_launch_laswp_plan(st, ipiv, j0 + w1, j0 + width, c->plan_tmp));
        LU_TRY(lu_launch_laswp_apply<T>(st, A, lda, j0, w1, 0, 0, c->plan_tmp, w2, c->num_sms));
    }
    return LU_SUCCESS;
}

}  // namespace

template <typename T>
int lu_panel_recursive(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t M, int64_t j0, int64_t width,
                       int32_t* ipiv, const lu_opts& o) {
    if (width <= 0) return LU_SUCCESS;
    const int64_t rows = M - j0;
    // Cluster leaves (distributed shared memory, hardware barrier) when the tallest
    // leaf fits one cluster; otherwise grid-barrier leaves.
    const int nt_want = sizeof(T) == 4 ? c->pf_threads : 256;
    int leaf = o.leaf > 0 ? std::min(o.leaf, LU_PF_MAX_LEAF) : 32;
    while (leaf > 8) {
        int C, R;
        size_t smem;
        if (lu_pf_cluster_shape<T>(rows, std::min<int>(leaf, (int)width), c->pf_smem_budget, &C, &R, &smem,
                                   o.pf_ctas, nt_want))
            break;
        leaf >>= 1;
    }
    {
        int C, R;
        size_t smem;
        if (lu_pf_cluster_shape<T>(rows, std::min<int>(leaf, (int)width), c->pf_smem_budget, &C, &R, &smem,
                                   o.pf_ctas, nt_want))
            return panel_rec<T>(c, st, A, lda, M, j0, width, ipiv, o, leaf, true, j0, width);
    }
    leaf = o.leaf > 0 ? std::min(o.leaf, LU_PF_MAX_LEAF) : 32;
    const int max_ctas = o.pf_ctas > 0 ? o.pf_ctas : LU_PF_MAX_CTAS;
    while (leaf > 1) {
        int64_t R, G;
        size_t smem;
        if (lu_pf_leaf_shape(rows, leaf, (int)sizeof(T), max_ctas, &R, &G, &smem)) break;
        leaf >>= 1;
    }
    return panel_rec<T>(c, st, A, lda, M, j0, width, ipiv, o, leaf, false, j0, width);
}

template int lu_launch_pf_leaf<double>(lu_context*, cudaStream_t, double*, int64_t, int64_t, int,
                                       int32_t*, int64_t, int);
template int lu_launch_pf_leaf<float>(lu_context*, cudaStream_t, float*, int64_t, int64_t, int,
                                      int32_t*, int64_t, int);
template int lu_panel_recursive<double>(lu_context*, cudaStream_t, double*, int64_t, int64_t,
                                        int64_t, int64_t, int32_t*, const lu_opts&);
template int lu_panel_recursive<float>(lu_context*, cudaStream_t, float*, int64_t, int64_t,
                                       int64_t, int64_t, int32_t*, const lu_opts&);
