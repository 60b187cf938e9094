// Operand packing for the tensor-core trailing update: FP32 panel blocks are
// rounded (ties to even) to bf16 / fp16 and laid out K-major, i.e. the nb
// values that one output row (of L21) or one output column (of U12) contracts
// over become contiguous -- the layout the TMA boxes and the tcgen05 shared
// memory descriptors of gemm_tc.cu expect.
//
// Split-bf16 mode (LU_PACK_BF16X3): each FP32 value x is written as
// hi = bf16(x) and lo = bf16(x - hi), and the K dimension is tripled so that
// one plain bf16 GEMM computes hi_A hi_B + hi_A lo_B + lo_A hi_B:
//     A row:    [ hi(0..k) | hi(0..k) | lo(0..k) ]
//     B column: [ hi(0..k) | lo(0..k) | hi(0..k) ]
// The dropped lo_A lo_B term is ~2^-16 relative, so the product carries about
// 16 significant bits instead of 8, at three times the tensor work but the same
// FP32 traffic of the updated matrix.  LU_PACK_BF16X6 splits into three parts
// and keeps the six products whose weight is at least 2^-16, which carries the
// full 24-bit FP32 significand.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "internal.h"
#include "profile.h"
#include "pack.h"

namespace {

template <int FMT>
__device__ __forceinline__ uint16_t to16(float x) {
    if (FMT == LU_PACK_FP16) return __half_as_ushort(__float2half_rn(x));
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// part 0 = bf16(x), part 1 = bf16(x - part0), part 2 = bf16(x - part0 - part1); the
// differences are exact in FP32 because each part removes the leading bits.
__device__ __forceinline__ uint16_t bf16_part(float x, int part) {
    const float p0 = __bfloat162float(__float2bfloat16_rn(x));
    if (part == 0) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    const float r1 = x - p0;
    const float p1 = __bfloat162float(__float2bfloat16_rn(r1));
    if (part == 1) return __bfloat16_as_ushort(__float2bfloat16_rn(r1));
    return __bfloat16_as_ushort(__float2bfloat16_rn(r1 - p1));
}

// Which part each K segment holds, for A rows and for B columns:
//   x3: A [0,0,1]  B [0,1,0]              -> p0p0 + p0p1 + p1p0
//   x6: A [0,0,1,0,1,2]  B [0,1,0,2,1,0]  -> p0p0 + p0p1 + p1p0 + p0p2 + p1p1 + p2p0
__device__ __forceinline__ int seg_part(int fmt, bool is_a, int seg) {
    if (fmt == LU_PACK_BF16X3) return is_a ? (seg == 2 ? 1 : 0) : (seg == 1 ? 1 : 0);
    const int a[6] = {0, 0, 1, 0, 1, 2}, b[6] = {0, 1, 0, 2, 1, 0};
    return is_a ? a[seg] : b[seg];
}

// value of segment `seg` of the split operand for A (rows) or B (columns)
template <int FMT, bool IS_A>
__device__ __forceinline__ uint16_t seg_val(float x, int seg) {
    if (FMT != LU_PACK_BF16X3 && FMT != LU_PACK_BF16X6) return to16<FMT>(x);
    return bf16_part(x, seg_part(FMT, IS_A, seg));
}

// Apack[r][kk] = round(A[r + kk*lda]) for r in [0, rows), kk in [0, k); out row stride = k.
// A 32-row x 64-column tile goes through shared memory so that both the
// column-major reads and the row-major writes are coalesced.
template <int FMT>
__global__ void __launch_bounds__(256) pack_rows_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int k,
                                                        uint16_t* __restrict__ out_base) {
    __shared__ uint16_t tile[32][64 + 2];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 64;
    const int seg = blockIdx.z;  // segment of the split operand (0 for single-term formats)
    const int nseg = gridDim.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int kk = ty; kk < 64; kk += 8) {
        const int64_t r = r0 + tx;
        const int kc = k0 + kk;
        tile[tx][kk] = (r < rows && kc < k) ? seg_val<FMT, true>(A[r + (int64_t)kc * lda], seg) : (uint16_t)0;
    }
    __syncthreads();
    // row stride of the packed buffer is nseg * k; this segment starts at seg * k
    uint16_t* out = out_base + (int64_t)seg * k;
    const int64_t stride = (int64_t)nseg * k;
    // write: each warp writes rows; lane covers 2 consecutive k values (32-bit stores)
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t r = r0 + rr;
        const int kc = k0 + 2 * tx;
        if (r < rows && kc < k) {
            if (kc + 1 < k && (k & 1) == 0) {
                const uint32_t v = (uint32_t)tile[rr][2 * tx] | ((uint32_t)tile[rr][2 * tx + 1] << 16);
                *reinterpret_cast<uint32_t*>(out + r * stride + kc) = v;
            } else {
                out[r * stride + kc] = tile[rr][2 * tx];
                if (kc + 1 < k) out[r * stride + kc + 1] = tile[rr][2 * tx + 1];
            }
        }
    }
}

// Bpack[c][seg*k + kk] = segment seg of B[kk + c*ldb], c in [0, cols): B's columns are
// already K-contiguous.
template <int FMT>
__global__ void __launch_bounds__(256) pack_cols_kernel(const float* __restrict__ B, int64_t ldb, int64_t cols, int k,
                                                        int nseg, uint16_t* __restrict__ out) {
    const int64_t kt = (int64_t)k * nseg;
    const int64_t total = cols * kt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / kt;
        const int q = (int)(e - c * kt);
        const int seg = q / k, kk = q - seg * k;
        out[e] = seg_val<FMT, false>(B[kk + c * ldb], seg);
    }
}

// ---------------------------------------------------------------------------
// e4m3 operands with power-of-two block scales (one scale per row of L21, one
// per column of U12).  The exponent is the smallest e with amax / 2^e <= 448:
// with amax = f 2^x, f in [0.5, 1) and 448 = 0.875 2^9, e = x - 9 + (f > 0.875).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int e4m3_block_exponent(float amax) {
    if (!(amax > 0.f)) return 0;
    int x;
    const float f = frexpf(amax, &x);
    return x - 9 + (f > 0.875f ? 1 : 0);
}

__device__ __forceinline__ uint8_t to_e4m3(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// rscale[r] = 2^e of row r (one thread per row; column-major reads are coalesced across threads)
__global__ void __launch_bounds__(256) row_scale_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int k,
                                                        float* __restrict__ rscale) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float amax = 0.f;
    for (int kk = 0; kk < k; ++kk) amax = fmaxf(amax, fabsf(A[r + (int64_t)kk * lda]));
    rscale[r] = ldexpf(1.f, e4m3_block_exponent(amax));
}

// out[r][kk] = e4m3(A[r + kk*lda] / rscale[r]), 32-row x 64-column tiles through shared memory
__global__ void __launch_bounds__(256) pack_rows_e4m3_kernel(const float* __restrict__ A, int64_t lda, int64_t rows,
                                                             int k, const float* __restrict__ rscale,
                                                             uint8_t* __restrict__ out) {
    __shared__ uint8_t tile[32][64 + 4];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r = r0 + tx;
    const int sexp = (r < rows) ? -ilogbf(rscale[r]) : 0;
    for (int kk = ty; kk < 64; kk += 8) {
        const int kc = k0 + kk;
        tile[tx][kk] = (r < rows && kc < k) ? to_e4m3(ldexpf(A[r + (int64_t)kc * lda], sexp)) : (uint8_t)0;
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t ro = r0 + rr;
        const int kc = k0 + 2 * tx;
        if (ro < rows && kc < k) {
            out[ro * k + kc] = tile[rr][2 * tx];
            if (kc + 1 < k) out[ro * k + kc + 1] = tile[rr][2 * tx + 1];
        }
    }
}

// one warp per column of B (K-contiguous): block maximum, scale, e4m3 bytes
__global__ void __launch_bounds__(256) pack_cols_e4m3_kernel(const float* __restrict__ B, int64_t ldb, int64_t cols,
                                                             int k, float* __restrict__ cscale,
                                                             uint8_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= cols) return;
    const float* b = B + c * ldb;
    float amax = 0.f;
    for (int kk = lane; kk < k; kk += 32) amax = fmaxf(amax, fabsf(b[kk]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const int e = e4m3_block_exponent(amax);
    if (lane == 0) cscale[c] = ldexpf(1.f, e);
    for (int kk = lane; kk < k; kk += 32) out[c * k + kk] = to_e4m3(ldexpf(b[kk], -e));
}

}  // namespace

int lu_launch_pack_rows_e4m3(cudaStream_t st, const float* A, int64_t lda, int64_t rows, int k, float* rscale,
                             void* out) {
    if (rows <= 0 || k <= 0) return LU_SUCCESS;
    {
        LuProfScope prof(st, LU_K_PACK, 4.0 * rows * k, 0.0);
        row_scale_kernel<<<(unsigned)lu_cdiv(rows, 256), 256, 0, st>>>(A, lda, rows, k, rscale);
    }
    LU_CHECK_LAUNCH();
    dim3 grid((unsigned)lu_cdiv(rows, 32), (unsigned)lu_cdiv(k, 64));
    LuProfScope prof(st, LU_K_PACK, 5.0 * rows * k, 0.0);
    pack_rows_e4m3_kernel<<<grid, 256, 0, st>>>(A, lda, rows, k, rscale, (uint8_t*)out);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

int lu_launch_pack_cols_e4m3(cudaStream_t st, const float* B, int64_t ldb, int64_t cols, int k, float* cscale,
                             void* out) {
    if (cols <= 0 || k <= 0) return LU_SUCCESS;
    LuProfScope prof(st, LU_K_PACK, 5.0 * cols * k, 0.0);
    pack_cols_e4m3_kernel<<<(unsigned)lu_cdiv(cols, 8), 256, 0, st>>>(B, ldb, cols, k, cscale, (uint8_t*)out);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

int lu_launch_pack_rows(cudaStream_t st, int fmt, const float* A, int64_t lda, int64_t rows, int k, void* out) {
    if (rows <= 0 || k <= 0) return LU_SUCCESS;
    if (lu_cdiv(k, 64) > 65535) return LU_ERR_UNSUPPORTED;
    const int nseg = lu_pack_segments(fmt);
    dim3 grid((unsigned)lu_cdiv(rows, 32), (unsigned)lu_cdiv(k, 64), (unsigned)nseg);
    LuProfScope prof(st, LU_K_PACK, (4.0 + 2.0 * nseg) * rows * k, 0.0);
    if (fmt == LU_PACK_BF16)
        pack_rows_kernel<LU_PACK_BF16><<<grid, 256, 0, st>>>(A, lda, rows, k, (uint16_t*)out);
    else if (fmt == LU_PACK_FP16)
        pack_rows_kernel<LU_PACK_FP16><<<grid, 256, 0, st>>>(A, lda, rows, k, (uint16_t*)out);
    else if (fmt == LU_PACK_BF16X3)
        pack_rows_kernel<LU_PACK_BF16X3><<<grid, 256, 0, st>>>(A, lda, rows, k, (uint16_t*)out);
    else
        pack_rows_kernel<LU_PACK_BF16X6><<<grid, 256, 0, st>>>(A, lda, rows, k, (uint16_t*)out);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

int lu_launch_pack_cols(cudaStream_t st, int fmt, const float* B, int64_t ldb, int64_t cols, int k, void* out) {
    if (cols <= 0 || k <= 0) return LU_SUCCESS;
    const int nseg = lu_pack_segments(fmt);
    const int64_t total = cols * (int64_t)k * nseg;
    const unsigned blocks = (unsigned)std::min<int64_t>(lu_cdiv(total, 256), 8192);
    LuProfScope prof(st, LU_K_PACK, (4.0 / nseg + 2.0) * total, 0.0);
    if (fmt == LU_PACK_BF16)
        pack_cols_kernel<LU_PACK_BF16><<<blocks, 256, 0, st>>>(B, ldb, cols, k, 1, (uint16_t*)out);
    else if (fmt == LU_PACK_FP16)
        pack_cols_kernel<LU_PACK_FP16><<<blocks, 256, 0, st>>>(B, ldb, cols, k, 1, (uint16_t*)out);
    else if (fmt == LU_PACK_BF16X3)
        pack_cols_kernel<LU_PACK_BF16X3><<<blocks, 256, 0, st>>>(B, ldb, cols, k, 3, (uint16_t*)out);
    else
        pack_cols_kernel<LU_PACK_BF16X6><<<blocks, 256, 0, st>>>(B, ldb, cols, k, 6, (uint16_t*)out);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}
