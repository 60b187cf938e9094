// Panel-factorization leaf on one thread-block cluster (RL1 of LU_blk, Sec. 3).
//
// The leaf's m rows are split across the C CTAs of one cluster (C <= 16), each
// keeping its R x w block in shared memory.  Per column the CTAs exchange their
// pivot candidates through distributed shared memory and cross one hardware
// cluster barrier (barrier.cluster arrive.release / wait.acquire) instead of a
// grid barrier in global memory:
//   1. each CTA reduces its local candidate (warp shuffles), writes value, row
//      index and the candidate's w values into its own shared-memory slot (the
//      owner of row jj also writes row jj);
//   2. cluster barrier;
//   3. every CTA reads all C candidates and row jj from the other CTAs' slots
//      (ld through map_shared_rank), picks the first maximum, swaps rows jj and
//      p inside its block, divides the column by the pivot and applies the
//      rank-1 update, fusing the next column's candidate search into it.
// Slots are double-buffered by column parity, so one barrier per column
// suffices.  After the last column the leaf's interchanges are applied to the
// other columns of the enclosing panel (so the recursion above needs no
// separate row-interchange launches) and the block is written back.
#include <cooperative_groups.h>

#include <climits>

#include "internal.h"
#include "profile.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kNT = 256;

template <typename T>
__device__ __forceinline__ void cmerge(T& v, int& i, T ov, int oi) {
    if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}

template <typename T>
struct Slot {
    T val[2];
    int idx[2];
    T row[2][LU_PF_MAX_LEAF];
    T jrow[2][LU_PF_MAX_LEAF];
};

template <typename T>
__global__ void __launch_bounds__(kNT) pf_leaf_cluster_kernel(T* __restrict__ A, int64_t lda, int m, int w, int R,
                                                              int left_cols, int right_cols,
                                                              int32_t* __restrict__ ipiv, int ipiv_add,
                                                              int* __restrict__ info) {
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sA = reinterpret_cast<T*>(smem_raw);                        // [w][R]
    Slot<T>* slot = reinterpret_cast<Slot<T>*>(sA + (size_t)w * R);  // this CTA's exchange slot
    T* cand_rows = reinterpret_cast<T*>(slot + 1);                  // [C][w] candidates read back
    T* prow = cand_rows + (size_t)LU_PF_MAX_CTAS_CLUSTER * w;        // pivot row
    T* jrowv = prow + w;                                            // row jj before the swap
    __shared__ T red_v[kNT / 32];
    __shared__ int red_i[kNT / 32];
    __shared__ T s_cv[LU_PF_MAX_CTAS_CLUSTER];
    __shared__ int s_ci[LU_PF_MAX_CTAS_CLUSTER];
    __shared__ int sh_bi, sh_p, sh_gw;
    __shared__ T sh_bv;
    __shared__ int s_piv[LU_PF_MAX_LEAF];
    // interchange plan for the other panel columns
    __shared__ int s_dst[2 * LU_PF_MAX_LEAF], s_src[2 * LU_PF_MAX_LEAF], s_cnt;

    const int C = (int)cluster.num_blocks();
    const int g = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = g * R;
    const int nrows = max(0, min(R, m - row0));

    for (int c = 0; c < w; ++c)
        for (int r = tid; r < nrows; r += kNT) sA[c * R + r] = A[(int64_t)(row0 + r) + (int64_t)c * lda];
    __syncthreads();

    T bv = T(-1);
    int bi = INT_MAX;
    for (int r = tid; r < nrows; r += kNT) cmerge(bv, bi, (T)fabs(sA[r]), row0 + r);

    for (int jj = 0; jj < w; ++jj) {
        const int buf = jj & 1;
        // ---- local candidate ----
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            cmerge(bv, bi, ov, oi);
        }
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        if (warp == 0) {
            T v = (lane < kNT / 32) ? red_v[lane] : T(-1);
            int i = (lane < kNT / 32) ? red_i[lane] : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                T ov = __shfl_xor_sync(0xffffffffu, v, o);
                int oi = __shfl_xor_sync(0xffffffffu, i, o);
                cmerge(v, i, ov, oi);
            }
            if (lane == 0) {
                sh_bv = v;
                sh_bi = i;
            }
        }
        __syncthreads();
        // ---- publish into this CTA's slot ----
        const int my_bi = sh_bi;
        if (tid == 0) {
            slot->val[buf] = sh_bv;
            slot->idx[buf] = my_bi;
        }
        if (tid < w) {
            if (my_bi != INT_MAX) slot->row[buf][tid] = sA[tid * R + (my_bi - row0)];
            if (jj >= row0 && jj < row0 + nrows) slot->jrow[buf][tid] = sA[tid * R + (jj - row0)];
        }
        cluster.sync();
        // ---- read every CTA's candidate and row jj ----
        for (int q = tid; q < C; q += kNT) {
            const Slot<T>* rs = cluster.map_shared_rank(slot, q);
            s_cv[q] = rs->val[buf];
            s_ci[q] = rs->idx[buf];
        }
        for (int e = tid; e < C * w; e += kNT) {
            const int q = e / w, c = e - q * w;
            const Slot<T>* rs = cluster.map_shared_rank(slot, q);
            cand_rows[e] = rs->row[buf][c];
        }
        if (tid < w) {
            const int owner = jj / R;
            const Slot<T>* rs = cluster.map_shared_rank(slot, owner);
            jrowv[tid] = rs->jrow[buf][tid];
        }
        __syncthreads();
        if (warp == 0) {
            T v = T(-1);
            int i = INT_MAX, qb = -1;
            for (int q = lane; q < C; q += 32) {
                if (s_ci[q] != INT_MAX && (s_cv[q] > v || (s_cv[q] == v && s_ci[q] < i))) {
                    v = s_cv[q];
                    i = s_ci[q];
                    qb = q;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                T ov = __shfl_xor_sync(0xffffffffu, v, o);
                int oi = __shfl_xor_sync(0xffffffffu, i, o);
                int oq = __shfl_xor_sync(0xffffffffu, qb, o);
                if (ov > v || (ov == v && oi < i)) {
                    v = ov;
                    i = oi;
                    qb = oq;
                }
            }
            if (lane == 0) {
                sh_p = (i == INT_MAX) ? jj : i;
                sh_gw = (i == INT_MAX) ? -1 : qb;
            }
        }
        __syncthreads();
        const int p = sh_p, gw = sh_gw;
        if (tid < w) prow[tid] = (gw >= 0) ? cand_rows[gw * w + tid] : jrowv[tid];
        if (tid == 0) {
            s_piv[jj] = p;
            if (g == 0) ipiv[jj] = p + 1 + ipiv_add;
        }
        __syncthreads();
        if (p != jj && tid < w) {
            if (p >= row0 && p < row0 + nrows) sA[tid * R + (p - row0)] = jrowv[tid];
            if (jj >= row0 && jj < row0 + nrows) sA[tid * R + (jj - row0)] = prow[tid];
        }
        const T piv = prow[jj];
        if (piv == T(0) && g == 0 && tid == 0) atomicCAS(info, 0, jj + 1 + ipiv_add);
        __syncthreads();
        bv = T(-1);
        bi = INT_MAX;
        const bool has_next = jj + 1 < w;
        for (int r = tid; r < nrows; r += kNT) {
            const int gr = row0 + r;
            if (gr <= jj) continue;
            if (piv != T(0)) {
                const T l = sA[jj * R + r] / piv;
                sA[jj * R + r] = l;
                for (int c = jj + 1; c < w; ++c) sA[c * R + r] = fma(-l, prow[c], sA[c * R + r]);
            }
            if (has_next) cmerge(bv, bi, (T)fabs(sA[(jj + 1) * R + r]), gr);
        }
    }
    // every CTA is done reading the other CTAs' slots before any CTA may exit
    cluster.sync();
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < nrows; r += kNT) A[(int64_t)(row0 + r) + (int64_t)c * lda] = sA[c * R + r];
    const int other = left_cols + right_cols;
    if (other <= 0) return;
    // ---- the leaf's interchanges on the other columns of the panel ----
    // Plan: positions 0..w-1 (leaf rows) and the distinct targets below them.
    if (tid == 0) {
        int tgt[LU_PF_MAX_LEAF], cur[2 * LU_PF_MAX_LEAF];
        int nt = 0;
        for (int i = 0; i < w; ++i) cur[i] = i;
        for (int k = 0; k < w; ++k) {
            const int pk = s_piv[k];
            if (pk == k) continue;
            int b;
            if (pk < w) {
                b = pk;
            } else {
                int f = -1;
                for (int t = 0; t < nt; ++t)
                    if (tgt[t] == pk) f = t;
                if (f < 0) {
                    f = nt++;
                    tgt[f] = pk;
                    cur[w + f] = pk;
                }
                b = w + f;
            }
            const int x = cur[k];
            cur[k] = cur[b];
            cur[b] = x;
        }
        int cnt = 0;
        for (int i = 0; i < w; ++i)
            if (cur[i] != i) {
                s_dst[cnt] = i;
                s_src[cnt] = cur[i];
                ++cnt;
            }
        for (int t = 0; t < nt; ++t)
            if (cur[w + t] != tgt[t]) {
                s_dst[cnt] = tgt[t];
                s_src[cnt] = cur[w + t];
                ++cnt;
            }
        s_cnt = cnt;
    }
    __syncthreads();
    const int cnt = s_cnt;
    if (cnt == 0) return;
    // columns q = g, g + C, ... of the other columns; one warp per column
    for (int q = g * (kNT / 32) + warp; q < other; q += C * (kNT / 32)) {
        const int64_t col = (q < left_cols) ? (int64_t)q - left_cols : (int64_t)w + (q - left_cols);
        T* a = A + col * lda;
        T v[(2 * LU_PF_MAX_LEAF) / 32];
#pragma unroll
        for (int t = 0; t < (2 * LU_PF_MAX_LEAF) / 32; ++t)
            if (lane + 32 * t < cnt) v[t] = a[s_src[lane + 32 * t]];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < (2 * LU_PF_MAX_LEAF) / 32; ++t)
            if (lane + 32 * t < cnt) a[s_dst[lane + 32 * t]] = v[t];
    }
}

size_t cluster_smem(int w, int R, int esize) {
    const size_t slot = esize == 8 ? sizeof(Slot<double>) : sizeof(Slot<float>);
    return (size_t)w * R * esize + slot + (size_t)LU_PF_MAX_CTAS_CLUSTER * w * esize + 2 * (size_t)w * esize + 16;
}

template <typename T>
int max_clusters_for(int C, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kNT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, pf_leaf_cluster_kernel<T>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return num;
}

}  // namespace

// Largest cluster size usable for the leaf (0 if clusters are unavailable); cached per type.
template <typename T>
static int cluster_limit() {
    static int lim[2] = {-1, -1};
    const int ti = sizeof(T) == 8 ? 0 : 1;
    if (lim[ti] >= 0) return lim[ti];
    int best = 0;
    if (cudaFuncSetAttribute(pf_leaf_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess)
        cudaGetLastError();
    if (cudaFuncSetAttribute(pf_leaf_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess)
        cudaGetLastError();
    for (int C = LU_PF_MAX_CTAS_CLUSTER; C >= 1; C >>= 1) {
        if (max_clusters_for<T>(C, 64 * 1024) > 0) {
            best = C;
            break;
        }
    }
    lim[ti] = best;
    return best;
}

// Shape of a cluster leaf: C CTAs of R rows (a multiple of 32) within the budget.
template <typename T>
bool lu_pf_cluster_shape(int64_t m, int w, size_t budget, int* C_out, int* R_out, size_t* smem_out) {
    const int cmax = cluster_limit<T>();
    if (cmax <= 0 || w > LU_PF_MAX_LEAF) return false;
    for (int C = 1; C <= cmax; C <<= 1) {
        const int64_t R = std::max<int64_t>(32, lu_cdiv(lu_cdiv(m, C), 32) * 32);
        const size_t smem = cluster_smem(w, (int)R, (int)sizeof(T));
        // prefer few CTAs, but not so few that one CTA's update work dominates the barrier
        if (smem <= budget && (R <= 1024 || C == cmax)) {
            *C_out = C;
            *R_out = (int)R;
            *smem_out = smem;
            return true;
        }
    }
    return false;
}

template <typename T>
int lu_launch_pf_leaf_cluster(cudaStream_t st, T* A, int64_t lda, int64_t m, int w, int C, int R, size_t smem,
                              int64_t left_cols, int64_t right_cols, int32_t* ipiv, int64_t ipiv_add, int* info) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kNT, 1, 1);
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
    LU_CHECK_CUDA(cudaLaunchKernelEx(&cfg, pf_leaf_cluster_kernel<T>, A, lda, (int)m, w, R, (int)left_cols,
                                     (int)right_cols, ipiv, (int)ipiv_add, info));
    lu_count_launch();
    return LU_SUCCESS;
}

template bool lu_pf_cluster_shape<double>(int64_t, int, size_t, int*, int*, size_t*);
template bool lu_pf_cluster_shape<float>(int64_t, int, size_t, int*, int*, size_t*);
template int lu_launch_pf_leaf_cluster<double>(cudaStream_t, double*, int64_t, int64_t, int, int, int, size_t, int64_t,
                                               int64_t, int32_t*, int64_t, int*);
template int lu_launch_pf_leaf_cluster<float>(cudaStream_t, float*, int64_t, int64_t, int, int, int, size_t, int64_t,
                                              int64_t, int32_t*, int64_t, int*);
