// SM partition for the panel leaves (lu_opts.pf_sms): the panel-factorization
// leaf of PF_{k+1} is the critical path of the mixed-precision factorization,
// and beside the trailing update its CTAs share SMs with the update's.  With a
// partition, two green contexts split the SMs: the leaves run on a small
// partition (a stream of its own, entered and left through events from the
// panel stream), the right trailing update TU_right(k) on the rest, so neither
// ever occupies the other's SMs.  The rest of the panel path (TU_k^L, RL2, the
// in-panel products) stays on the full device.  Green contexts share the
// primary context's memory; the driver entry points are looked up through the
// runtime, so the library does not link the driver library.
#include <cuda.h>

#include <map>
#include <mutex>

#include "internal.h"

namespace {

struct DriverApi {
    bool ok = false;
    decltype(&cuDeviceGetDevResource) getRes = nullptr;
    decltype(&cuDevSmResourceSplitByCount) split = nullptr;
    decltype(&cuDevResourceGenerateDesc) desc = nullptr;
    decltype(&cuGreenCtxCreate) create = nullptr;
    decltype(&cuGreenCtxDestroy) destroy = nullptr;
    decltype(&cuGreenCtxStreamCreate) stream = nullptr;
    decltype(&cuCtxFromGreenCtx) fromGreen = nullptr;
    decltype(&cuCtxPushCurrent) push = nullptr;
    decltype(&cuCtxPopCurrent) pop = nullptr;
    decltype(&cuCtxGetCurrent) current = nullptr;
};

template <typename F>
bool entry(const char* name, F** fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion(name, &p, 13000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        cudaGetLastError();
        return false;
    }
    *fn = reinterpret_cast<F*>(p);
    return true;
}

const DriverApi& api() {
    static DriverApi a;
    static std::once_flag once;
    std::call_once(once, [] {
        a.ok = entry("cuDeviceGetDevResource", &a.getRes) && entry("cuDevSmResourceSplitByCount", &a.split) &&
               entry("cuDevResourceGenerateDesc", &a.desc) && entry("cuGreenCtxCreate", &a.create) &&
               entry("cuGreenCtxDestroy", &a.destroy) && entry("cuGreenCtxStreamCreate", &a.stream) &&
               entry("cuCtxFromGreenCtx", &a.fromGreen) && entry("cuCtxPushCurrent", &a.push) &&
               entry("cuCtxPopCurrent", &a.pop) && entry("cuCtxGetCurrent", &a.current);
    });
    return a;
}

// Occupancy probe only (never launched): a kernel with the panel leaf's largest
// cluster and shared-memory footprint.
__global__ void green_cluster_fit_kernel(int* p) {
    if (p) p[0] = 0;
}

}  // namespace

struct LuGreen {
    int requested = 0;       // the partition size asked for
    int part_sms = 0;        // SMs of the leaf partition
    int rest_sms = 0;        // SMs of the rest
    CUgreenCtx g_leaf = nullptr, g_rest = nullptr;
    CUcontext c_leaf = nullptr, c_rest = nullptr;
    cudaStream_t s_leaf = nullptr, s_rest = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

void* lu_current_ctx() {
    const DriverApi& a = api();
    CUcontext ctx = nullptr;
    if (a.ok && a.current(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    return ctx;
}

int lu_green_setup(lu_context* c, int part_sms) {
    if (part_sms <= 0) return LU_ERR_UNSUPPORTED;
    if (c->green && c->green->requested == part_sms) return LU_SUCCESS;
    if (c->green) lu_green_release(c);
    const DriverApi& a = api();
    if (!a.ok) return LU_ERR_UNSUPPORTED;
    CUdevResource all, part, rest;
    unsigned groups = 1;
    if (a.getRes((CUdevice)c->device, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return LU_ERR_UNSUPPORTED;
    if (a.split(&part, &groups, &all, &rest, CU_DEV_SM_RESOURCE_SPLIT_MAX_POTENTIAL_CLUSTER_SIZE,
                (unsigned)part_sms) != CUDA_SUCCESS || groups < 1)
        return LU_ERR_UNSUPPORTED;
    CUdevResourceDesc d_part, d_rest;
    if (a.desc(&d_part, &part, 1) != CUDA_SUCCESS || a.desc(&d_rest, &rest, 1) != CUDA_SUCCESS)
        return LU_ERR_UNSUPPORTED;
    LuGreen* g = new LuGreen();
    g->requested = part_sms;
    g->part_sms = (int)part.sm.smCount;
    g->rest_sms = (int)rest.sm.smCount;
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    CUstream sl = nullptr, sr = nullptr;
    bool ok = a.create(&g->g_leaf, d_part, (CUdevice)c->device, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
              a.create(&g->g_rest, d_rest, (CUdevice)c->device, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
              a.fromGreen(&g->c_leaf, g->g_leaf) == CUDA_SUCCESS && a.fromGreen(&g->c_rest, g->g_rest) == CUDA_SUCCESS &&
              a.stream(&sl, g->g_leaf, CU_STREAM_NON_BLOCKING, hi_prio) == CUDA_SUCCESS &&
              a.stream(&sr, g->g_rest, CU_STREAM_NON_BLOCKING, lo_prio) == CUDA_SUCCESS;
    g->s_leaf = reinterpret_cast<cudaStream_t>(sl);
    g->s_rest = reinterpret_cast<cudaStream_t>(sr);
    ok = ok && cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming) == cudaSuccess;
    c->green = g;
    // the leaf partition must hold the widest cluster a leaf launches (16 CTAs of 512
    // threads and up to 160 KB of shared memory); otherwise the partition is not used
    if (ok && a.push(g->c_leaf) == CUDA_SUCCESS) {
        int fits = 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(LU_PF_MAX_CTAS_CLUSTER, 1, 1);
        cfg.blockDim = dim3(512, 1, 1);
        cfg.dynamicSmemBytes = LU_PF_SMEM_PART;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = LU_PF_MAX_CTAS_CLUSTER;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ok = cudaFuncSetAttribute(green_cluster_fit_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(green_cluster_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  LU_PF_SMEM_PART) == cudaSuccess &&
             cudaOccupancyMaxActiveClusters(&fits, green_cluster_fit_kernel, &cfg) == cudaSuccess && fits >= 1;
        CUcontext dummy = nullptr;
        a.pop(&dummy);
    } else {
        ok = false;
    }
    if (!ok) {
        cudaGetLastError();
        lu_green_release(c);
        return LU_ERR_UNSUPPORTED;
    }
    return LU_SUCCESS;
}

void lu_green_release(lu_context* c) {
    LuGreen* g = c->green;
    if (!g) return;
    const DriverApi& a = api();
    cudaDeviceSynchronize();
    if (g->s_leaf) cudaStreamDestroy(g->s_leaf);
    if (g->s_rest) cudaStreamDestroy(g->s_rest);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    if (a.ok) {
        if (g->g_leaf) a.destroy(g->g_leaf);
        if (g->g_rest) a.destroy(g->g_rest);
    }
    delete g;
    c->green = nullptr;
    c->green_active = false;
}

cudaStream_t lu_green_rest_stream(lu_context* c) { return c->green ? c->green->s_rest : nullptr; }
int lu_green_rest_sms(lu_context* c) { return c->green ? c->green->rest_sms : c->num_sms; }

int lu_green_enter(lu_context* c, bool leaf) {
    const DriverApi& a = api();
    if (!c->green || !a.ok) return LU_ERR_UNSUPPORTED;
    if (a.push(leaf ? c->green->c_leaf : c->green->c_rest) != CUDA_SUCCESS) return LU_ERR_CUDA;
    return LU_SUCCESS;
}

void lu_green_leave() {
    const DriverApi& a = api();
    CUcontext dummy = nullptr;
    if (a.ok) a.pop(&dummy);
}

int lu_green_leaf_fork(lu_context* c, cudaStream_t st, cudaStream_t* leaf_st) {
    LU_CHECK_CUDA(cudaEventRecord(c->green->ev_in, st));
    LU_CHECK_CUDA(cudaStreamWaitEvent(c->green->s_leaf, c->green->ev_in, 0));
    *leaf_st = c->green->s_leaf;
    return lu_green_enter(c, true);
}

int lu_green_leaf_join(lu_context* c, cudaStream_t st) {
    lu_green_leave();
    LU_CHECK_CUDA(cudaEventRecord(c->green->ev_out, c->green->s_leaf));
    LU_CHECK_CUDA(cudaStreamWaitEvent(st, c->green->ev_out, 0));
    return LU_SUCCESS;
}
