// Operand packing for the tensor-core trailing update: FP32 panel blocks are
// rounded (ties to even) to bf16 / fp16 and laid out K-major, i.e. the nb
// values that one output row (of L21) or one output column (of U12) contracts
// over become contiguous -- the layout the TMA boxes and the tcgen05 shared
// memory descriptors of gemm_tc.cu expect.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "pack.h"

namespace {

template <int FMT>
__device__ __forceinline__ uint16_t to16(float x) {
    if (FMT == LU_PACK_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}

// Apack[r][kk] = round(A[r + kk*lda]) for r in [0, rows), kk in [0, k); out row stride = k.
// A 32-row x 64-column tile goes through shared memory so that both the
// column-major reads and the row-major writes are coalesced.
template <int FMT>
__global__ void __launch_bounds__(256) pack_rows_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int k,
                                                        uint16_t* __restrict__ out) {
    __shared__ uint16_t tile[32][64 + 2];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int kk = ty; kk < 64; kk += 8) {
        const int64_t r = r0 + tx;
        const int kc = k0 + kk;
        tile[tx][kk] = (r < rows && kc < k) ? to16<FMT>(A[r + (int64_t)kc * lda]) : (uint16_t)0;
    }
    __syncthreads();
    // write: each warp writes rows; lane covers 2 consecutive k values (32-bit stores)
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t r = r0 + rr;
        const int kc = k0 + 2 * tx;
        if (r < rows && kc < k) {
            if (kc + 1 < k && (k & 1) == 0) {
                const uint32_t v = (uint32_t)tile[rr][2 * tx] | ((uint32_t)tile[rr][2 * tx + 1] << 16);
                *reinterpret_cast<uint32_t*>(out + r * k + kc) = v;
            } else {
                out[r * k + kc] = tile[rr][2 * tx];
                if (kc + 1 < k) out[r * k + kc + 1] = tile[rr][2 * tx + 1];
            }
        }
    }
}

// Bpack[c][kk] = round(B[kk + c*ldb]) for c in [0, cols): B's columns are already K-contiguous.
template <int FMT>
__global__ void __launch_bounds__(256) pack_cols_kernel(const float* __restrict__ B, int64_t ldb, int64_t cols, int k,
                                                        uint16_t* __restrict__ out) {
    const int64_t total = cols * (int64_t)k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / k;
        const int kk = (int)(e - c * k);
        out[e] = to16<FMT>(B[kk + c * ldb]);
    }
}

}  // namespace

int lu_launch_pack_rows(cudaStream_t st, int fmt, const float* A, int64_t lda, int64_t rows, int k, void* out) {
    if (rows <= 0 || k <= 0) return LU_SUCCESS;
    if (lu_cdiv(k, 64) > 65535) return LU_ERR_UNSUPPORTED;
    dim3 grid((unsigned)lu_cdiv(rows, 32), (unsigned)lu_cdiv(k, 64));
    if (fmt == LU_PACK_BF16)
        pack_rows_kernel<LU_PACK_BF16><<<grid, 256, 0, st>>>(A, lda, rows, k, (uint16_t*)out);
    else
        pack_rows_kernel<LU_PACK_FP16><<<grid, 256, 0, st>>>(A, lda, rows, k, (uint16_t*)out);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}

int lu_launch_pack_cols(cudaStream_t st, int fmt, const float* B, int64_t ldb, int64_t cols, int k, void* out) {
    if (cols <= 0 || k <= 0) return LU_SUCCESS;
    const int64_t total = cols * (int64_t)k;
    const unsigned blocks = (unsigned)std::min<int64_t>(lu_cdiv(total, 256), 8192);
    if (fmt == LU_PACK_BF16)
        pack_cols_kernel<LU_PACK_BF16><<<blocks, 256, 0, st>>>(B, ldb, cols, k, (uint16_t*)out);
    else
        pack_cols_kernel<LU_PACK_FP16><<<blocks, 256, 0, st>>>(B, ldb, cols, k, (uint16_t*)out);
    LU_CHECK_LAUNCH();
    return LU_SUCCESS;
}
