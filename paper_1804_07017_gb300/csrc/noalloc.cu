// lu_panel_factor_noalloc: the panel factorization (RL1) for callers that must
// not allocate device memory -- code running where cudaMalloc is unavailable or
// forbidden: inside a host callback, a custom allocator's own path, a real-time
// loop that has preallocated everything, or a process whose memory pool is
// owned by someone else.  The scratch the panel kernels need (grid-barrier
// counters, the leaf's candidate-exchange slots and the interchange plan of
// the recursion) lives in the file-scope array below instead of in a handle's
// cudaMalloc'd workspace.  The caller still owns and passes A, ipiv and info.
//
// The array is a module-scope __device__ variable: every GPU that loads this
// library holds kNoallocBytes of it until the process exits.  Host code cannot
// use the symbol itself (in host code it names a host-side stand-in, not device
// memory), so the first call on each device, with that device current, looks up
// the array's device address with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture.  Every call on a device shares the one
// array: calls whose executions overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "internal.h"

namespace {

// Layout: [0, 256) LuSync; then the leaf exchange slots; then one interchange plan.
constexpr size_t kSyncBytes = 256;
constexpr size_t kSlotBytes = sizeof(double) * (2 * LU_PF_MAX_CTAS * (LU_PF_MAX_LEAF + 1) + 2 * LU_PF_MAX_LEAF) +
                              sizeof(int) * 2 * LU_PF_MAX_CTAS;
constexpr size_t kSlotBytesAligned = (kSlotBytes + 255) / 256 * 256;
constexpr size_t kPlanBytes = sizeof(int32_t) * (1 + 4 * (size_t)LU_MAX_NB);
constexpr size_t kNoallocBytes = kSyncBytes + kSlotBytesAligned + (kPlanBytes + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

int scratch_address(int dev, char** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            lu_set_error_string(cudaGetErrorString(e), __FILE__, __LINE__);
            return LU_ERR_CUDA;
        }
        g_ptr[dev] = p;
    }
    *out = static_cast<char*>(g_ptr[dev]);
    return LU_SUCCESS;
}

}  // namespace

extern "C" size_t lu_noalloc_scratch_bytes(void) { return kNoallocBytes; }

extern "C" int lu_panel_factor_noalloc(lu_dtype dtype, int64_t m, int64_t w, void* A, int64_t lda, int32_t* ipiv,
                                       const lu_opts* opts, int32_t* info, void* stream) {
    if (dtype != LU_F64 && dtype != LU_F32) return -1;
    if (m < 0) return -2;
    if (w < 0 || w > m) return -3;
    if (m > 0 && w > 0 && !A) return -4;
    if (lda < std::max<int64_t>(1, m)) return -5;
    if (w > 0 && !ipiv) return -6;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -7;
    if (!info) return -8;
    // the one interchange plan in the array covers at most LU_MAX_NB interchanges
    if (w > LU_MAX_NB || m > INT32_MAX / 2) return LU_ERR_UNSUPPORTED;
    int dev = 0;
    LU_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LU_ERR_UNSUPPORTED;
    char* base = nullptr;
    LU_TRY(scratch_address(dev, &base));
    // A handle-less context whose workspace pointers all point into the array.
    lu_context c;
    c.device = dev;
    LU_CHECK_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev));
    c.sync = reinterpret_cast<LuSync*>(base);
    c.pf_slots = base + kSyncBytes;
    c.plan_tmp = reinterpret_cast<int32_t*>(base + kSyncBytes + kSlotBytesAligned);
    c.plans = nullptr;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: the counters, error and info words start at zero
    LU_CHECK_CUDA(cudaMemsetAsync(c.sync, 0, sizeof(LuSync), st));
    if (w > 0 && m > 0) {
        if (dtype == LU_F64)
            LU_TRY(lu_panel_recursive<double>(&c, st, (double*)A, lda, m, 0, w, ipiv, o));
        else
            LU_TRY(lu_panel_recursive<float>(&c, st, (float*)A, lda, m, 0, w, ipiv, o));
    }
    return lu_launch_finish_info(st, c.sync, info);
}
