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
#include <cstdio>
#include <cstdlib>

#include <map>
#include <mutex>

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

// Warp-wide first-maximum reduction of (value, row, source) triples.
template <typename T>
__device__ __forceinline__ void warp_best(T& v, int& i, int& q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        const int oq = __shfl_xor_sync(0xffffffffu, q, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
            q = oq;
        }
    }
}

// W: compiled leaf width (so every per-row update is straight-line code); the
// leaf factors its first w <= W columns.  RQ: rows per thread (thread t owns
// rows t + kNT*q of its CTA's block).
// The block is row-major in shared memory with a padded stride W+1.
// HW = true: the cluster's hardware barrier (barrier.cluster arrive / wait, split
// so that a CTA arrives as soon as it has published and waits only when it
// needs the other candidates); HW = false: the bounded grid barrier on sync.
template <typename T, int W, int RQ, bool HW>
__global__ void __launch_bounds__(kNT) pf_leaf_cluster_kernel(T* __restrict__ A, int64_t lda, int m, int w,
                                                              int left_cols, int right_cols, int32_t* __restrict__ ipiv,
                                                              int ipiv_add, LuSync* __restrict__ sync) {
    int* info = &sync->info;
    constexpr int R = kNT * RQ;
    constexpr int WP = W + 1;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sA = reinterpret_cast<T*>(smem_raw);                       // [R][WP]
    Slot<T>* slot = reinterpret_cast<Slot<T>*>(sA + (size_t)R * WP);
    __shared__ T red_v[kNT / 32];
    __shared__ int red_i[kNT / 32];
    __shared__ int s_piv[W];
    __shared__ int s_dst[2 * W], s_src[2 * W], s_cnt;
    __shared__ int s_ok;

    const int C = (int)cluster.num_blocks();
    const int g = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = g * R;
    const int nrows = max(0, min(R, m - row0));
    // the cluster's CTAs synchronise through the bounded grid barrier on sync
    unsigned int phase = 0;

    for (int c = 0; c < W; ++c)
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const int r = tid + kNT * q;
            if (r < nrows) sA[r * WP + c] = (c < w) ? A[(int64_t)(row0 + r) + (int64_t)c * lda] : T(0);
        }
    __syncthreads();

    // local candidate of column 0
    T bv = T(-1);
    int bi = INT_MAX;
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
        const int r = tid + kNT * q;
        if (r < nrows) cmerge(bv, bi, (T)fabs(sA[r * WP]), row0 + r);
    }

    // block reduction + publish of column jj's candidate into slot[jj & 1]
    auto publish = [&](int jj) {
        int dummy = 0;
        warp_best(bv, bi, dummy);
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        T v = (lane < kNT / 32) ? red_v[lane] : T(-1);
        int i = (lane < kNT / 32) ? red_i[lane] : INT_MAX;
        warp_best(v, i, dummy);
        const int buf = jj & 1;
        if (tid == 0) {
            slot->val[buf] = v;
            slot->idx[buf] = i;
        }
        // the candidate row and row jj are copied by the warp that owns them
        if (i != INT_MAX) {
            const int lr = i - row0;
            if (warp == (lr % kNT) >> 5)
                for (int c = lane; c < W; c += 32) slot->row[buf][c] = sA[lr * WP + c];
        }
        if (jj >= row0 && jj < row0 + nrows) {
            const int lr = jj - row0;
            if (warp == (lr % kNT) >> 5)
                for (int c = lane; c < W; c += 32) slot->jrow[buf][c] = sA[lr * WP + c];
        }
        if (HW) {
            cluster.barrier_arrive();
            return true;
        }
        return lu_grid_barrier(sync, (++phase) * (unsigned)C, &s_ok);
    };

    bool ok = publish(0);
    for (int jj = 0; jj < w && ok; ++jj) {
        const int buf = jj & 1;
        if (HW) cluster.barrier_wait();
        // ---- every warp selects the pivot from the C published candidates ----
        T cv = T(-1);
        int ci = INT_MAX, cq = -1;
        if (lane < C) {
            const Slot<T>* rs = cluster.map_shared_rank(slot, lane);
            cv = rs->val[buf];
            ci = rs->idx[buf];
            cq = (ci == INT_MAX) ? -1 : lane;
            if (ci == INT_MAX) cv = T(-1);
        }
        warp_best(cv, ci, cq);
        const int p = (ci == INT_MAX) ? jj : ci;
        // lane c holds element c of the pivot row and of row jj (W <= 32 lanes)
        T pr = T(0), jr = T(0);
        if (lane < W) {
            const Slot<T>* ro = cluster.map_shared_rank(slot, jj / R);
            jr = ro->jrow[buf][lane];
            pr = (cq >= 0) ? cluster.map_shared_rank(slot, cq)->row[buf][lane] : jr;
        }
        if (tid == 0) {
            s_piv[jj] = p;
            if (g == 0) ipiv[jj] = p + 1 + ipiv_add;
        }
        // ---- interchange rows jj and p inside this CTA's block ----
        if (p != jj) {
            if (p >= row0 && p < row0 + nrows) {
                const int lr = p - row0;
                if (warp == (lr % kNT) >> 5 && lane < W) sA[lr * WP + lane] = jr;
            }
            if (jj >= row0 && jj < row0 + nrows) {
                const int lr = jj - row0;
                if (warp == (lr % kNT) >> 5 && lane < W) sA[lr * WP + lane] = pr;
            }
        }
        __syncwarp();
        T prv[W];
#pragma unroll
        for (int c = 0; c < W; ++c) prv[c] = __shfl_sync(0xffffffffu, pr, c);
        const T piv = __shfl_sync(0xffffffffu, pr, jj);
        if (piv == T(0) && g == 0 && tid == 0) atomicCAS(info, 0, jj + 1 + ipiv_add);
        // ---- scale column jj, rank-1 update, next column's local candidate ----
        bv = T(-1);
        bi = INT_MAX;
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const int r = tid + kNT * q;
            const int gr = row0 + r;
            if (r < nrows && gr > jj) {
                T* rowp = sA + r * WP;
                if (piv != T(0)) {
                    const T l = rowp[jj] / piv;
                    rowp[jj] = l;
#pragma unroll
                    for (int c = 0; c < W; ++c)
                        if (c > jj) rowp[c] = fma(-l, prv[c], rowp[c]);
                }
                if (jj + 1 < w) cmerge(bv, bi, (T)fabs(rowp[jj + 1]), gr);
            }
        }
        if (jj + 1 < w) ok = publish(jj + 1);
    }
    // no CTA leaves while another may still read its slot
    if (HW) {
        cluster.sync();
    } else {
        if (ok) ok = lu_grid_barrier(sync, (++phase) * (unsigned)C, &s_ok);
        lu_grid_exit(sync);
        if (!ok) return;
    }
    for (int c = 0; c < w; ++c)
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
            const int r = tid + kNT * q;
            if (r < nrows) A[(int64_t)(row0 + r) + (int64_t)c * lda] = sA[r * WP + c];
        }
    const int other = left_cols + right_cols;
    if (other <= 0) return;
    // ---- the leaf's interchanges on the other columns of the panel ----
    // Plan: positions 0..W-1 (leaf rows) and the distinct targets below them.
    if (tid == 0) {
        int tgt[W], cur[2 * W];
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
        T v[(2 * W + 31) / 32];
#pragma unroll
        for (int t = 0; t < (2 * W + 31) / 32; ++t)
            if (lane + 32 * t < cnt) v[t] = a[s_src[lane + 32 * t]];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < (2 * W + 31) / 32; ++t)
            if (lane + 32 * t < cnt) a[s_dst[lane + 32 * t]] = v[t];
    }
}

template <typename T>
size_t cluster_smem(int w, int rq) {
    return (size_t)kNT * rq * (w + 1) * sizeof(T) + sizeof(Slot<T>) + 16;
}


template <typename T>
struct LeafTable {
    typedef void (*Fn)(T*, int64_t, int, int, int, int, int32_t*, int, LuSync*);
    static Fn get(int w, int rq, bool hw) {
#define LU_LEAF_CASE(WW, RR) \
    if (w == WW && rq == RR) return hw ? pf_leaf_cluster_kernel<T, WW, RR, true> : pf_leaf_cluster_kernel<T, WW, RR, false>;
        LU_LEAF_CASE(8, 1) LU_LEAF_CASE(8, 2) LU_LEAF_CASE(8, 4) LU_LEAF_CASE(8, 8)
        LU_LEAF_CASE(16, 1) LU_LEAF_CASE(16, 2) LU_LEAF_CASE(16, 4) LU_LEAF_CASE(16, 8)
        LU_LEAF_CASE(32, 1) LU_LEAF_CASE(32, 2) LU_LEAF_CASE(32, 4)
#undef LU_LEAF_CASE
        return nullptr;
    }
};

template <typename T>
int max_clusters_for(typename LeafTable<T>::Fn fn, int C, size_t smem) {
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
    if (cudaOccupancyMaxActiveClusters(&num, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return num;
}

}  // namespace

// Largest cluster size usable for the leaf (0 if clusters are unavailable); cached per
// (device, type), since kernel attributes and cluster occupancy belong to a device.
template <typename T>
static int cluster_limit() {
    static std::mutex mu;
    static std::map<int, int> lim;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    auto it = lim.find(dev);
    if (it != lim.end()) return it->second;
    const int ws[3] = {8, 16, 32}, rqs[4] = {1, 2, 4, 8};
    for (int hw = 0; hw < 2; ++hw)
        for (int w : ws)
            for (int rq : rqs) {
                auto fn = LeafTable<T>::get(w, rq, hw != 0);
                if (!fn) continue;
                if (lu_func_smem(fn, 220 * 1024, true) != LU_SUCCESS) cudaGetLastError();
            }
    int best = 0;
    auto fn = LeafTable<T>::get(16, 1, false);
    for (int C = LU_PF_MAX_CTAS_CLUSTER; C >= 1; C >>= 1) {
        if (max_clusters_for<T>(fn, C, cluster_smem<T>(16, 1)) > 0) {
            best = C;
            break;
        }
    }
    lim[dev] = best;
    return best;
}

// Shape of a cluster leaf: C CTAs of kNT*rq rows within the shared-memory budget,
// w one of the compiled widths (8, 16, 32).
static int compiled_width(int w) { return w <= 8 ? 8 : (w <= 16 ? 16 : (w <= 32 ? 32 : 0)); }

static int leaf_mode();

template <typename T>
bool lu_pf_cluster_shape(int64_t m, int w, size_t budget, int* C_out, int* R_out, size_t* smem_out, int max_c,
                         int nt, int* nt_out) {
    if (m < w) return false;
    w = compiled_width(w);
    if (w == 0) return false;
    int cmax = cluster_limit<T>();
    if (max_c > 0) cmax = std::min(cmax, max_c);
    if (cmax <= 0) return false;
    // the 512-thread leaf exists only as the pushed-message kernel (FP32)
    if (nt != kNT && (leaf_mode() != 2 || lu_pf_push_smem((int)sizeof(T), w, 1, nt) == 0)) nt = kNT;
    const int rqs[4] = {1, 2, 4, 8};
    for (int rq : rqs) {
        const size_t push = lu_pf_push_smem((int)sizeof(T), w, rq, nt);
        if (nt == kNT ? !LeafTable<T>::get(w, rq, false) : push == 0) continue;
        const int64_t R = (int64_t)nt * rq;
        const int64_t C = lu_cdiv(m, R);
        if (C > cmax) continue;
        const size_t smem = nt == kNT ? std::max(cluster_smem<T>(w, rq), push) : push;
        if (smem > budget) return false;
        int Cp = 1;
        while (Cp < C) Cp <<= 1;  // power-of-two cluster sizes
        if (Cp > cmax) continue;
        *C_out = Cp;
        *R_out = (int)R;
        *smem_out = smem;
        if (nt_out) *nt_out = nt;
        return true;
    }
    return false;
}

// Default: pushed messages with mbarrier completion (pf_push.cu).
// LU_GB300_PF_BARRIER=cluster selects candidates read through distributed
// shared memory after a hardware cluster barrier; =global the same with the
// bounded global-memory barrier.
static int leaf_mode() {
    static int mode = -1;
    if (mode < 0) {
        const char* e = getenv("LU_GB300_PF_BARRIER");
        mode = (e && e[0] == 'g') ? 0 : ((e && e[0] == 'c') ? 1 : 2);
    }
    return mode;
}

bool lu_pf_leaf_pairs_supported() { return leaf_mode() == 2; }

template <typename T>
int lu_launch_pf_leaf_cluster(cudaStream_t st, T* A, int64_t lda, int64_t m, int w, int C, int R, size_t smem,
                              int64_t left_cols, int64_t right_cols, int32_t* ipiv, int64_t ipiv_add, LuSync* sync,
                              int sib, int kprev, int nt) {
    const int mode = leaf_mode();
    if (mode == 2)
        return lu_launch_pf_leaf_push<T>(st, A, lda, m, w, compiled_width(w), C, R, left_cols, right_cols, ipiv,
                                         ipiv_add, sync, sib, kprev, nt);
    if (sib != 0 || kprev != 0 || nt != kNT) return LU_ERR_UNSUPPORTED;
    const int hw = mode;
    auto fn = LeafTable<T>::get(compiled_width(w), R / kNT, hw != 0);
    if (!fn) return LU_ERR_UNSUPPORTED;
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
    if (getenv("LU_GB300_TRACE_LAUNCH"))
        fprintf(stderr, "[lu launch] cluster leaf esize %d m %lld w %d C %d R %d smem %zu left %lld right %lld\n",
                (int)sizeof(T), (long long)m, w, C, R, smem, (long long)left_cols, (long long)right_cols);
    LU_CHECK_CUDA(cudaLaunchKernelEx(&cfg, fn, A, lda, (int)m, w, (int)left_cols, (int)right_cols, ipiv,
                                     (int)ipiv_add, sync));
    lu_count_launch();
    return LU_SUCCESS;
}

template bool lu_pf_cluster_shape<double>(int64_t, int, size_t, int*, int*, size_t*, int, int, int*);
template bool lu_pf_cluster_shape<float>(int64_t, int, size_t, int*, int*, size_t*, int, int, int*);
template int lu_launch_pf_leaf_cluster<double>(cudaStream_t, double*, int64_t, int64_t, int, int, int, size_t, int64_t,
                                               int64_t, int32_t*, int64_t, LuSync*, int, int, int);
template int lu_launch_pf_leaf_cluster<float>(cudaStream_t, float*, int64_t, int64_t, int, int, int, size_t, int64_t,
                                              int64_t, int32_t*, int64_t, LuSync*, int, int, int);
