// Trailing update TU (RL3 of LU_blk, Sec. 3), C := C - A B, on the 5th-generation
// tensor cores (tcgen05) for the mixed-precision factorization.
//
//   C      FP32, column-major (the FP32 working copy of the matrix)
//   A      L21 of the current panel, bf16/fp16 (or e4m3), stored row-major
//          ("K-major": the panel's nb values of one row are contiguous)
//   B      U12 of the current panel, same type, stored one output column per
//          row (K-major as well)
//
// Structure (one CTA per SM, persistent, 320 threads):
//   warp 0      tile scheduler + TMA producer: takes tile indices from a global
//               atomic counter (so CTAs of a later launch on another stream can
//               join the same update and take the remaining tiles -- the GPU
//               counterpart of the malleable BLAS of Sec. 4.2), then streams
//               64-wide K chunks of the A and B tiles into a 3-stage ring of
//               128B-swizzled shared-memory buffers with cp.async.bulk.tensor;
//   warp 1      allocates 2 x BN TMEM columns (two accumulators) and issues
//               tcgen05.mma (M = 128, N = BN, K = 16 per instruction) from one
//               thread, committing each stage back to the producer and each
//               finished accumulator to the epilogue;
//   warps 2-9   epilogue: tcgen05.ld of the accumulator (lane = row), coalesced
//               loads of C, C - acc, coalesced stores.  Two warps per TMEM lane
//               quadrant split the tile's columns; with two accumulators the
//               epilogue of tile t overlaps the MMAs of tile t+1.
// Every wait is bounded (%globaltimer); on expiry the kernel records
// LU_ERR_TIMEOUT, drains its own copies/MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.h"
#include "ptx.cuh"
#include "profile.h"
#include "tc.h"

namespace {

constexpr int kTM = 128;         // rows per tile (UMMA M)
constexpr int kTK = 64;          // K elements per stage for 16-bit types (128 bytes)
constexpr int kStages = 3;
constexpr int kRing = 4;         // tile-index ring depth
constexpr int kThreads = 320;    // 10 warps
constexpr int kEpiWarps = 8;
constexpr uint64_t kWaitNs = 2000000000ull;

// Shared-memory matrix descriptor for a K-major operand tile written by TMA with
// 128-byte swizzling: 8-row x 128-byte swizzle atoms stacked at 1024-byte
// stride (SBO), version 1, layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_issue(int kind, uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    if (kind == LU_TC_KIND_F16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 bits, 32 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
struct TcLayout {
    static constexpr int kABytes = kTM * 128;  // 128 rows x 128 bytes per stage
    static constexpr int kBBytes = BN * 128;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kBarOffset = kStages * kStageBytes;
    // barriers: full[S], empty[S], tfull[2], tempty[2], ring_full[R], ring_empty[R], drain
    static constexpr int kNumBars = 2 * kStages + 4 + 2 * kRing + 1;
    static constexpr int kMiscOffset = kBarOffset + kNumBars * 8;
    static constexpr int kSmemBytes = kMiscOffset + 64 + 1024;  // + alignment slack
};

// 144 registers x 320 threads leaves room on the SM for a panel-factorization CTA
// (256 threads x <= 64 registers) next to this one.
template <int BN>
__global__ void __maxnreg__(144)
    tc_update_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcUpdateParams p) {
    using L = TcLayout<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOffset);
    uint64_t* full = bars;
    uint64_t* empty = bars + kStages;
    uint64_t* tfull = bars + 2 * kStages;
    uint64_t* tempty = tfull + 2;
    uint64_t* rfull = tempty + 2;
    uint64_t* rempty = rfull + kRing;
    uint64_t* drain = rempty + kRing;
    int* misc = reinterpret_cast<int*>(smem + L::kMiscOffset);
    volatile int* ring = misc;                 // [kRing] tile indices
    volatile int* abort_flag = misc + kRing;   // CTA-wide abort
    volatile int* consumed = misc + kRing + 1; // K chunks consumed by the MMA warp
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(misc + kRing + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kchunks = p.k / p.kchunk;
    const uint32_t stage_tx = (uint32_t)((kTM + BN) * 128);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps);
        }
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&rfull[r], 1);
            mbar_init(&rempty[r], 1 + kEpiWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- scheduler + TMA producer ----------------
            uint32_t stage = 0, phase = 0;
            int issued = 0;
            for (int t = 0;; ++t) {
                int tile = atomicAdd(p.counter, 1);
                // a symmetric update takes only the tiles on or below the band's diagonal blocks
                while (p.band > 0 && tile < p.tiles &&
                       p.row0 + (tile % p.tiles_m) * kTM + kTM <= ((p.col0 + (tile / p.tiles_m) * BN) / p.band) * p.band)
                    tile = atomicAdd(p.counter, 1);
                if (tile >= p.tiles) tile = -1;
                const int slot = t % kRing;
                if (!mbar_wait(&rempty[slot], ((t / kRing) & 1) ^ 1, abort_flag)) break;
                ring[slot] = tile;
                mbar_arrive(&rfull[slot]);
                if (tile < 0) break;
                const int tm = tile % p.tiles_m, tn = tile / p.tiles_m;
                const int ya = tm * kTM;  // operand buffers start at the update's first row / column
                const int yb = tn * BN;
                bool ok = true;
                for (int kc = 0; kc < kchunks; ++kc) {
                    if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) { ok = false; break; }
                    uint8_t* sa = smem + stage * L::kStageBytes;
                    uint8_t* sb = sa + L::kABytes;
                    mbar_arrive_expect_tx(&full[stage], stage_tx);
                    tma_load_2d(sa, &tmA, &full[stage], kc * 128 / p.elem_bytes, ya);
                    tma_load_2d(sb, &tmB, &full[stage], kc * 128 / p.elem_bytes, yb);
                    ++issued;
                    if (++stage == kStages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
            }
            if (*abort_flag) {
                // drain: wait (bounded) for every copy issued but not consumed
                for (int q = *consumed; q < issued; ++q) {
                    const uint64_t t0 = lu_globaltimer();
                    while (!mbar_try_wait(&full[q % kStages], (q / kStages) & 1))
                        if (lu_globaltimer() - t0 > kWaitNs) break;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            uint32_t stage = 0, phase = 0;
            int used = 0;
            for (int t = 0;; ++t) {
                const int slot = t % kRing;
                if (!mbar_wait(&rfull[slot], (t / kRing) & 1, abort_flag)) break;
                const int tile = ring[slot];
                mbar_arrive(&rempty[slot]);
                if (tile < 0) break;
                const int ab = t & 1;
                if (!mbar_wait(&tempty[ab], ((t >> 1) & 1) ^ 1, abort_flag)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(ab * BN);
                bool ok = true;
                for (int kc = 0; kc < kchunks; ++kc) {
                    if (!mbar_wait(&full[stage], phase, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + stage * L::kStageBytes);
                    const uint32_t sb = sa + L::kABytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_issue(p.kind, d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), p.idesc,
                                  (kc > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&empty[stage]);
                    *consumed = ++used;
                    if (++stage == kStages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                mma_commit(&tfull[ab]);
            }
            // make sure no MMA is still writing TMEM before it is freed
            mma_commit(drain);
            const uint64_t t0 = lu_globaltimer();
            while (!mbar_try_wait(drain, 0))
                if (lu_globaltimer() - t0 > kWaitNs) break;
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3;            // TMEM lane quadrant this warp may access
        const int h = (warp - 2) >> 2;     // which half of the tile's columns
        for (int t = 0;; ++t) {
            const int slot = t % kRing;
            if (!mbar_wait(&rfull[slot], (t / kRing) & 1, abort_flag)) break;
            const int tile = ring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&rempty[slot]);
            if (tile < 0) break;
            const int ab = t & 1;
            if (!mbar_wait(&tfull[ab], (t >> 1) & 1, abort_flag)) break;
            tc_fence_after();
            const int tm = tile % p.tiles_m, tn = tile / p.tiles_m;
            const int r_local = tm * kTM + q * 32 + lane;
            const bool row_ok = r_local < p.m;
            const int64_t row = (int64_t)p.row0 + r_local;
#pragma unroll 1
            for (int cb = 0; cb < BN / 2; cb += 32) {
                const int ct = h * (BN / 2) + cb;  // column within the tile
                const int c_local = tn * BN + ct;
                float cv[32], acc[32];
                float* cp = p.C + row + (int64_t)(p.col0 + c_local) * p.ldc;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    cv[j] = (row_ok && c_local + j < p.ncols) ? __ldcs(cp + (int64_t)j * p.ldc) : 0.f;
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * BN + ct), acc);
                if (p.rscale) {
                    // power-of-two block scales: exact rescaling of the FP32 accumulator
                    const float rs = row_ok ? p.rscale[r_local] * p.scale : 0.f;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (row_ok && c_local + j < p.ncols)
                            __stcs(cp + (int64_t)j * p.ldc, cv[j] - acc[j] * (rs * p.cscale[c_local + j]));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (row_ok && c_local + j < p.ncols)
                            __stcs(cp + (int64_t)j * p.ldc, cv[j] - acc[j] * p.scale);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[ab]);
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(p.error, LU_ERR_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * BN) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encoder() {
    if (g_encode) return LU_SUCCESS;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    LU_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) {
        lu_set_error_string("cuTensorMapEncodeTiled unavailable", __FILE__, __LINE__);
        return LU_ERR_CUDA;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return LU_SUCCESS;
}

// 2-D map over a row-major [rows][kdim] operand buffer, box = 128 bytes of K x box_rows.
int make_operand_map(CUtensorMap* map, const void* base, int elem_bytes, int64_t kdim, int64_t rows, int box_rows) {
    LU_TRY(get_encoder());
    const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(kdim * elem_bytes)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        lu_set_error_string("cuTensorMapEncodeTiled failed", __FILE__, __LINE__);
        return LU_ERR_CUDA;
    }
    return LU_SUCCESS;
}

template <int BN>
int launch_bn(cudaStream_t st, const CUtensorMap& ma, const CUtensorMap& mb, const TcUpdateParams& p, int grid) {
    using L = TcLayout<BN>;
    LU_TRY(lu_func_smem(tc_update_kernel<BN>, L::kSmemBytes));
    LuProfScope prof(st, LU_K_TC_UPDATE, 8.0 * p.m * p.ncols + (double)p.elem_bytes * p.k * (p.m + p.ncols),
                     2.0 * p.m * p.ncols * p.k);
    tc_update_kernel<BN><<<grid, kThreads, L::kSmemBytes, st>>>(ma, mb, p);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

}  // namespace

int lu_tc_smem_bytes(int bn) { return bn == 256 ? TcLayout<256>::kSmemBytes : TcLayout<128>::kSmemBytes; }

// C[row0 .. row0+m) x [col0 .. col0+ncols) -= A[0..m, 0..k) * B[0..ncols, 0..k)^T with A, B the
// K-major low-precision operand buffers (a_rows / b_rows rows of k elements each, a_rows >= m,
// b_rows >= ncols).
int lu_launch_tc_update(cudaStream_t st, int kind, int fmt, float* C, int64_t ldc, int64_t row0, int64_t m,
                        int64_t col0, int64_t ncols, int64_t k, const void* Abuf, int64_t a_rows, const void* Bbuf,
                        int64_t b_rows, float scale, int* counter, int* error, int grid, int bn,
                        const float* rscale, const float* cscale, int band) {
    if (m <= 0 || ncols <= 0) return LU_SUCCESS;
    const int elem = (kind == LU_TC_KIND_F16) ? 2 : 1;
    const int kchunk = 128 / elem;
    if (k <= 0 || k % kchunk != 0) return LU_ERR_UNSUPPORTED;
    if (bn != 128 && bn != 256) return LU_ERR_UNSUPPORTED;
    if (row0 + m > INT32_MAX || col0 + ncols > INT32_MAX) return LU_ERR_UNSUPPORTED;
    CUtensorMap ma, mb;
    LU_TRY(make_operand_map(&ma, Abuf, elem, k, a_rows, kTM));
    LU_TRY(make_operand_map(&mb, Bbuf, elem, k, b_rows, bn));
    TcUpdateParams p;
    p.C = C;
    p.ldc = ldc;
    p.row0 = (int)row0;
    p.m = (int)m;
    p.col0 = (int)col0;
    p.ncols = (int)ncols;
    p.k = (int)k;
    p.kchunk = kchunk;
    p.elem_bytes = elem;
    p.tiles_m = (int)lu_cdiv(m, kTM);
    p.tiles_n = (int)lu_cdiv(ncols, bn);
    p.tiles = p.tiles_m * p.tiles_n;
    p.counter = counter;
    p.error = error;
    p.kind = kind;
    p.scale = scale;
    p.rscale = rscale;
    p.cscale = cscale;
    p.band = band;
    // instruction descriptor: D = F32, A/B format, both K-major, N >> 3, M >> 4
    uint32_t idesc = (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(bn >> 3) << 17) |
                     ((uint32_t)(kTM >> 4) << 24);
    p.idesc = idesc;
    grid = std::max(1, std::min(grid, p.tiles));
    if (bn == 256) return launch_bn<256>(st, ma, mb, p, grid);
    return launch_bn<128>(st, ma, mb, p, grid);
}
