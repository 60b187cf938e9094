// Exercise of the bounded-wait path shared by every grid-synchronised kernel:
// a grid barrier whose target can never be reached (one more arrival than
// there are CTAs) waits for the given limit, records LU_ERR_TIMEOUT in the
// sync block, and every CTA returns.  The GPU is never hung: each wait gives up
// after limit_ns of %globaltimer time.
#include "internal.h"
#include "profile.h"

namespace {

__global__ void timeout_probe_kernel(LuSync* s, uint64_t limit_ns) {
    __shared__ int flag;
    lu_grid_barrier(s, gridDim.x + 1u, &flag, limit_ns);
    lu_grid_exit(s);
}

}  // namespace

extern "C" int lu_selftest_wait_timeout(lu_handle h, int64_t limit_ns, int32_t* status) {
    if (!h) return LU_ERR_HANDLE;
    if (limit_ns <= 0 || limit_ns > 2000000000LL) return -2;
    if (!status) return -3;
    std::lock_guard<std::mutex> lk(h->mu);
    LU_TRY(lu_ctx_reserve(h, 1, 1));
    cudaStream_t st = h->user;
    LuSync* s = &h->sync[6];
    LU_CHECK_CUDA(cudaMemsetAsync(s, 0, sizeof(LuSync), st));
    {
        LuProfScope prof(st, LU_K_OTHER, 0.0, 0.0);
        timeout_probe_kernel<<<2, 32, 0, st>>>(s, (uint64_t)limit_ns);
    }
    LU_CHECK_LAUNCH();
    return lu_launch_finish_info(st, s, status);
}
