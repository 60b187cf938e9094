// Declarations for the tensor-core trailing update and the mixed-precision path.
#pragma once
#include <stdint.h>

#define LU_TC_KIND_F16 0  // tcgen05.mma kind::f16 (bf16 or fp16 operands)
#define LU_TC_KIND_F8 1   // tcgen05.mma kind::f8f6f4 (e4m3 operands)
#define LU_TC_FMT_F16 0   // instruction-descriptor operand format codes (kind::f16)
#define LU_TC_FMT_BF16 1
#define LU_TC_FMT_E4M3 0  // (kind::f8f6f4)

struct TcUpdateParams {
    float* C;
    int64_t ldc;
    int row0, m;       // first absolute row of the update and its row count
    int col0, ncols;   // first absolute column and the column count
    int k, kchunk, elem_bytes;
    int tiles_m, tiles_n, tiles;
    int* counter;      // dynamic tile counter (zeroed before the first CTA of an update starts)
    int* error;        // receives LU_ERR_TIMEOUT if a bounded wait expires
    int kind;
    uint32_t idesc;
    float scale;       // acc is multiplied by this before the subtraction
    const float* rscale;  // optional per-row factor of acc (power-of-two block scales), m entries
    const float* cscale;  // optional per-column factor of acc, ncols entries
    int band;          // > 0: symmetric update; tiles whose rows all lie above the band-wide
                       // diagonal block of their first column are skipped
};

int lu_tc_smem_bytes(int bn);
int lu_launch_tc_update(cudaStream_t st, int kind, int fmt, float* C, int64_t ldc, int64_t row0, int64_t m,
                        int64_t col0, int64_t ncols, int64_t k, const void* Abuf, int64_t a_rows, const void* Bbuf,
                        int64_t b_rows, float scale, int* counter, int* error, int grid, int bn,
                        const float* rscale = nullptr, const float* cscale = nullptr, int band = 0);
