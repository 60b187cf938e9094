// Runtime-task schedule of the blocked LU (the comparison schedule of Sec. 3.3,
// Listing 4, where a task runtime orders PF and per-panel updates by their data
// dependencies instead of the static look-ahead of Sec. 4).
//
// Tasks of step k (panel k = columns [s_k, s_{k+1})):
//   PF(k)      the panel factorization and its interchange plan;
//   TU(k, j)   for every later block column j: panel k's interchanges on that
//              column block, RL2 on its block row and RL3 below it;
//   LS(k)      panel k's interchanges on the columns left of the panel.
// Dependencies: TU(k, j) needs PF(k) and TU(k-1, j); PF(k+1) needs TU(k, k+1);
// LS(k) needs PF(k) (which follows every update of the columns it moves) and
// every TU(k-1, j): those read the L21 blocks of the earlier panels, whose rows
// LS(k) exchanges.
//
// On the GPU the runtime is the CUDA graph executor: the DAG is captured once
// across one stream per block-column class (tasks of one column stay ordered
// on its stream), PF(k) and TU(k, k+1) -- the critical chain -- on the
// high-priority stream, LS on a stream of its own, and instantiated with node
// priorities.  Each replay starts every task as soon as its inputs are ready,
// so the look-ahead depth is whatever the dependencies allow.  Every element
// sees the same operations in the same order as in the static schedules, so
// the factors are bit-identical to theirs.
#include <cstring>

#include "internal.h"

namespace {

constexpr int kMaxColStreams = 64;

int rtm_resources(lu_context* c, int64_t nk) {
    int lo_prio = 0, hi_prio = 0;
    LU_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    const int64_t ncol = std::min<int64_t>(nk, kMaxColStreams);
    while ((int64_t)c->rtm_cols.size() < ncol) {
        cudaStream_t st = nullptr;
        LU_CHECK_CUDA(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo_prio));
        c->rtm_cols.push_back(st);
    }
    if (!c->rtm_left) LU_CHECK_CUDA(cudaStreamCreateWithPriority(&c->rtm_left, cudaStreamNonBlocking, lo_prio));
    if (!c->rtm_origin) LU_CHECK_CUDA(cudaStreamCreateWithFlags(&c->rtm_origin, cudaStreamNonBlocking));
    while ((int64_t)c->rtm_sev.size() < ncol) {
        cudaEvent_t e = nullptr;
        LU_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->rtm_sev.push_back(e);
    }
    for (auto* v : {&c->rtm_pf, &c->rtm_col})
        while ((int64_t)v->size() < nk + 1) {
            cudaEvent_t e = nullptr;
            LU_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            v->push_back(e);
        }
    if (!c->rtm_ev) LU_CHECK_CUDA(cudaEventCreateWithFlags(&c->rtm_ev, cudaEventDisableTiming));
    if (!c->rtm_ev2) LU_CHECK_CUDA(cudaEventCreateWithFlags(&c->rtm_ev2, cudaEventDisableTiming));
    return LU_SUCCESS;
}

// Issue the whole DAG, forked from and joined back into `origin`.
template <typename T>
int issue(lu_context* c, cudaStream_t origin, const std::vector<int64_t>& s, int64_t n, T* A, int64_t lda,
          int32_t* ipiv, const lu_opts& o, bool pivot) {
    const int64_t nk = (int64_t)s.size() - 1;
    const int64_t ncol = std::min<int64_t>(nk, kMaxColStreams);
    cudaStream_t hi = c->hi, left = c->rtm_left;
    auto col = [&](int64_t j) { return c->rtm_cols[(size_t)(j % ncol)]; };
    LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[0], 0, sizeof(LuSync), origin));
    LU_CHECK_CUDA(cudaEventRecord(c->rtm_ev, origin));
    LU_CHECK_CUDA(cudaStreamWaitEvent(hi, c->rtm_ev, 0));
    LU_CHECK_CUDA(cudaStreamWaitEvent(left, c->rtm_ev, 0));
    for (int64_t q = 0; q < ncol; ++q) LU_CHECK_CUDA(cudaStreamWaitEvent(c->rtm_cols[(size_t)q], c->rtm_ev, 0));
    auto width = [&](int64_t k) { return s[(size_t)k + 1] - s[(size_t)k]; };
    LU_TRY(lu_step_pf<T>(c, hi, A, lda, n, 0, 0, width(0), ipiv, o, pivot));
    LU_CHECK_CUDA(cudaEventRecord(c->rtm_pf[0], hi));
    std::vector<char> used((size_t)ncol, 0);
    for (int64_t k = 0; k < nk; ++k) {
        const int64_t k0 = s[(size_t)k], kb = width(k);
        // LS(k): panel k's interchanges on the columns left of it, once PF(k) is
        // done and every update of step k-1 (the last task on each column stream)
        // has stopped reading the rows it moves
        if (pivot && k0 > 0) {
            LU_CHECK_CUDA(cudaStreamWaitEvent(left, c->rtm_pf[(size_t)k], 0));
            for (int64_t q = 0; q < ncol; ++q)
                if (used[(size_t)q]) LU_CHECK_CUDA(cudaStreamWaitEvent(left, c->rtm_sev[(size_t)q], 0));
            LU_TRY(lu_step_tu<T>(c, left, n, A, lda, k, k0, kb, n, n, k0, pivot));
        }
        // the critical chain: TU(k, k+1) after TU(k-1, k+1), then PF(k+1)
        if (k + 1 < nk) {
            if (k >= 1) LU_CHECK_CUDA(cudaStreamWaitEvent(hi, c->rtm_col[(size_t)k + 1], 0));
            LU_TRY(lu_step_tu<T>(c, hi, n, A, lda, k, k0, kb, s[(size_t)k + 1], s[(size_t)k + 2], 0, pivot));
            LU_TRY(lu_step_pf<T>(c, hi, A, lda, n, k + 1, s[(size_t)k + 1], width(k + 1), ipiv, o, pivot));
            LU_CHECK_CUDA(cudaEventRecord(c->rtm_pf[(size_t)k + 1], hi));
        }
        // TU(k, j) for the other block columns, each on its column's stream
        for (int64_t j = k + 2; j < nk; ++j) {
            cudaStream_t st = col(j);
            LU_CHECK_CUDA(cudaStreamWaitEvent(st, c->rtm_pf[(size_t)k], 0));
            LU_TRY(lu_step_tu<T>(c, st, n, A, lda, k, k0, kb, s[(size_t)j], s[(size_t)j + 1], 0, pivot));
            LU_CHECK_CUDA(cudaEventRecord(c->rtm_col[(size_t)j], st));
            const int64_t q = j % ncol;
            LU_CHECK_CUDA(cudaEventRecord(c->rtm_sev[(size_t)q], st));
            used[(size_t)q] = 1;
        }
    }
    // join every forked stream back into the origin
    cudaStream_t forked[2] = {hi, left};
    for (cudaStream_t st : forked) {
        LU_CHECK_CUDA(cudaEventRecord(c->rtm_ev2, st));
        LU_CHECK_CUDA(cudaStreamWaitEvent(origin, c->rtm_ev2, 0));
    }
    for (int64_t q = 0; q < ncol; ++q) {
        LU_CHECK_CUDA(cudaEventRecord(c->rtm_ev2, c->rtm_cols[(size_t)q]));
        LU_CHECK_CUDA(cudaStreamWaitEvent(origin, c->rtm_ev2, 0));
    }
    return LU_SUCCESS;
}

}  // namespace

template <typename T>
int lu_factor_rtm(lu_context* c, int64_t n, T* A, int64_t lda, int32_t* ipiv, const lu_opts& o, int32_t* info,
                  bool pivot) {
    std::vector<int64_t> s;
    int wmin = 1, wmax = 1;
    lu_panel_bounds(n, o, &s, &wmin, &wmax);
    LU_TRY(lu_ctx_reserve(c, n, wmin));
    cudaStream_t user = c->user;
    c->trace_steps = 0;
    if (n == 0) {
        LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[0], 0, sizeof(LuSync), user));
        return lu_launch_finish_info(user, &c->sync[0], info);
    }
    const int64_t nk = (int64_t)s.size() - 1;
    LU_TRY(rtm_resources(c, nk));
    c->tu_reserve = 0;
    cudaStream_t origin = c->rtm_origin;
    LU_CHECK_CUDA(cudaEventRecord(c->ev_fork, user));
    LU_CHECK_CUDA(cudaStreamWaitEvent(origin, c->ev_fork, 0));
    if (lu_profile_active()) {
        // per-launch profiling events cannot live in a graph: issue the DAG eagerly
        LU_TRY(issue<T>(c, origin, s, n, A, lda, ipiv, o, pivot));
    } else {
        uint64_t h = 1469598103934665603ull;  // FNV-1a over the panel bounds
        for (int64_t b : s) h = (h ^ (uint64_t)b) * 1099511628211ull;
        const uint64_t key[12] = {(uint64_t)(uintptr_t)A, (uint64_t)lda, (uint64_t)n, (uint64_t)(uintptr_t)ipiv,
                                  (uint64_t)sizeof(T), (uint64_t)pivot, h, (uint64_t)o.leaf,
                                  (uint64_t)o.pf_ctas, (uint64_t)(uintptr_t)c->ws, (uint64_t)nk, 1};
        if (!c->rtm_exec || memcmp(key, c->rtm_key, sizeof(key)) != 0) {
            if (c->rtm_exec) cudaGraphExecDestroy(c->rtm_exec);
            c->rtm_exec = nullptr;
            memset(c->rtm_key, 0, sizeof(c->rtm_key));
            const long long before = lu_launches_so_far();
            cudaGraph_t g = nullptr;
            LU_CHECK_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
            const int rc = issue<T>(c, origin, s, n, A, lda, ipiv, o, pivot);
            const cudaError_t ee = cudaStreamEndCapture(origin, &g);
            c->rtm_launches = lu_launches_so_far() - before;
            lu_count_launches(-c->rtm_launches);  // nothing ran yet
            if (rc != LU_SUCCESS || ee != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                if (rc != LU_SUCCESS) return rc;
                lu_set_error_string(cudaGetErrorString(ee), __FILE__, __LINE__);
                return LU_ERR_CUDA;
            }
            const cudaError_t ie = cudaGraphInstantiateWithFlags(&c->rtm_exec, g, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                c->rtm_exec = nullptr;
                lu_set_error_string(cudaGetErrorString(ie), __FILE__, __LINE__);
                return LU_ERR_CUDA;
            }
            memcpy(c->rtm_key, key, sizeof(key));
        }
        LU_CHECK_CUDA(cudaGraphLaunch(c->rtm_exec, origin));
        lu_count_launches(c->rtm_launches);
    }
    LU_CHECK_CUDA(cudaEventRecord(c->ev_join_hi, origin));
    LU_CHECK_CUDA(cudaStreamWaitEvent(user, c->ev_join_hi, 0));
    return lu_launch_finish_info(user, &c->sync[0], info);
}

template int lu_factor_rtm<double>(lu_context*, int64_t, double*, int64_t, int32_t*, const lu_opts&, int32_t*, bool);
template int lu_factor_rtm<float>(lu_context*, int64_t, float*, int64_t, int32_t*, const lu_opts&, int32_t*, bool);
