// Shared device/host helpers for the GB300 LU library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/lu_gb300.h"

#define LU_CHECK_CUDA(call)                                                        \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            lu_set_error_string(cudaGetErrorString(_e), __FILE__, __LINE__);       \
            return LU_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

#define LU_CHECK_LAUNCH()                                                          \
    do {                                                                           \
        lu_count_launch();                                                         \
        cudaError_t _e = cudaGetLastError();                                       \
        if (_e != cudaSuccess) {                                                   \
            lu_set_error_string(cudaGetErrorString(_e), __FILE__, __LINE__);       \
            return LU_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

#define LU_TRY(call)                                                               \
    do {                                                                           \
        int _r = (call);                                                           \
        if (_r != LU_SUCCESS) return _r;                                           \
    } while (0)

void lu_set_error_string(const char* what, const char* file, int line);
void lu_count_launch();

// Kernel attributes belong to a device's context, so they are set once per
// (current device, kernel): the dynamic shared-memory limit `smem_bytes` and,
// with `nonportable_cluster`, permission for clusters above 8 CTAs.  Thread
// safe; a failed set is not remembered, so the next call tries again.
int lu_func_attrs(const void* fn, int smem_bytes, bool nonportable_cluster);
template <typename F>
inline int lu_func_smem(F* fn, int smem_bytes, bool nonportable_cluster = false) {
    return lu_func_attrs(reinterpret_cast<const void*>(fn), smem_bytes, nonportable_cluster);
}

// Bounded-wait budget for every device-side spin (nanoseconds of %globaltimer).
#define LU_WAIT_NS (4000000000ull)

// Device-side status words shared by kernels that synchronise CTAs.
struct LuSync {
    unsigned int arrive;  // grid-barrier arrivals (monotone within one launch)
    unsigned int exit;    // CTAs that left the launch; the last one resets both
    int error;            // 0, or LU_ERR_TIMEOUT when a bounded wait gave up
    int info;             // first exactly-zero pivot (1-based), 0 if none
    unsigned int ticket;  // dynamic block-index ticket (triangular solves)
    unsigned int pad[3];
};

__device__ __forceinline__ uint64_t lu_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int lu_ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int lu_ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void lu_st_release(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int lu_atom_add_release(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Grid-wide barrier for a launch whose CTAs are all resident.  Thread 0 of each
// CTA arrives and spins (bounded); returns false if the wait timed out or
// another CTA reported an error, in which case the caller must leave.
__device__ __forceinline__ bool lu_grid_barrier(LuSync* s, unsigned int target, int* sh_flag,
                                                uint64_t limit_ns = LU_WAIT_NS) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        lu_atom_add_release(&s->arrive, 1u);
        uint64_t t0 = 0;
        unsigned int spins = 0;
        while (lu_ld_acquire(&s->arrive) < target) {
            if (((++spins) & 255u) == 0) {
                if (lu_ld_acquire_s32(&s->error) != 0) { ok = 0; break; }
                uint64_t t = lu_globaltimer();
                if (t0 == 0) t0 = t;
                else if (t - t0 > limit_ns) {
                    atomicExch(&s->error, LU_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        *sh_flag = ok;
    }
    __syncthreads();
    return *sh_flag != 0;
}

// Called once per CTA at the very end of a grid-synchronised launch: the last
// CTA out resets the counters so the next launch starts from zero.
__device__ __forceinline__ void lu_grid_exit(LuSync* s) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int old = atomicAdd(&s->exit, 1u);
        if (old == gridDim.x * gridDim.y * gridDim.z - 1) {
            s->arrive = 0;
            s->exit = 0;
            __threadfence();
        }
    }
}

template <typename T>
struct LuTypeName;
template <>
struct LuTypeName<double> { static constexpr const char* name = "f64"; };
template <>
struct LuTypeName<float> { static constexpr const char* name = "f32"; };

static inline int64_t lu_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
