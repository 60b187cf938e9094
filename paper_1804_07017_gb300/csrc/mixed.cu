// Mixed-precision path: FP32 panels and factors, trailing update on the tensor
// cores with bf16/fp16 operands and FP32 accumulation.
#include "internal.h"
#include "pack.h"
#include "tc.h"

// Grow the handle's mixed-precision workspace to at least `bytes`.
int lu_mx_reserve(lu_context* c, size_t bytes) {
    if (c->mx && c->mx_bytes >= bytes) return LU_SUCCESS;
    if (c->mx) {
        LU_CHECK_CUDA(cudaDeviceSynchronize());
        cudaFree(c->mx);
        c->mx = nullptr;
        c->mx_bytes = 0;
    }
    if (cudaMalloc(&c->mx, bytes) != cudaSuccess) {
        cudaGetLastError();
        return LU_ERR_NOMEM;
    }
    c->mx_bytes = bytes;
    return LU_SUCCESS;
}

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

extern "C" int lu_gemm_update_tc_ex(lu_handle h, lu_prec prec, int64_t m, int64_t n, int64_t k, const float* A,
                                    int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (prec != LU_TU_BF16 && prec != LU_TU_FP16) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0 || k % 64 != 0) return -5;
    if (m > 0 && k > 0 && !A) return -6;
    if (lda < std::max<int64_t>(1, m)) return -7;
    if (k > 0 && n > 0 && !B) return -8;
    if (ldb < std::max<int64_t>(1, k)) return -9;
    if (m > 0 && n > 0 && !C) return -10;
    if (ldc < std::max<int64_t>(1, m)) return -11;
    if (!info) return -12;
    std::lock_guard<std::mutex> lk(h->mu);
    LU_TRY(lu_ctx_reserve(h, 1, 1));
    cudaStream_t st = h->user;
    LU_CHECK_CUDA(cudaMemsetAsync(&h->sync[2], 0, sizeof(LuSync), st));
    if (m > 0 && n > 0 && k > 0) {
        const size_t abytes = al256((size_t)m * k * 2), bbytes = al256((size_t)n * k * 2);
        LU_TRY(lu_mx_reserve(h, abytes + bbytes));
        char* a = (char*)h->mx;
        char* b = a + abytes;
        const int fmt = prec == LU_TU_BF16 ? LU_PACK_BF16 : LU_PACK_FP16;
        LU_TRY(lu_launch_pack_rows(st, fmt, A, lda, m, (int)k, a));
        LU_TRY(lu_launch_pack_cols(st, fmt, B, ldb, n, (int)k, b));
        LU_TRY(lu_launch_tc_update(st, LU_TC_KIND_F16, prec == LU_TU_BF16 ? LU_TC_FMT_BF16 : LU_TC_FMT_F16, C, ldc, 0, m,
                                   0, n, k, a, m, b, n, 1.0f, (int*)&h->sync[2].ticket, &h->sync[2].error, h->num_sms,
                                   256));
    }
    return lu_launch_finish_info(st, &h->sync[2], info);
}
