// Host side of the library: handles, workspace, the blocked factorization
// driver with depth-1 static look-ahead, and the solve driver.
//
// The factorization follows LU_blk (Sec. 3): for each panel k, PF_k (RL1,
// recursive, see pf.cu), then the interchanges, TRSM (RL2) and GEMM (RL3) on
// the trailing columns.  With look-ahead (Sec. 4, Listing 5) TU_k is split at
// the next panel's columns: the high-priority stream runs PU(k+1) = TU_k^L
// followed by PF_{k+1}, while the low-priority stream runs TU_right(k) over
// the remaining columns (plus the deferred interchanges on the columns left of
// panel k).  Stream priority makes the panel path's CTAs the first to be
// scheduled as trailing-update CTAs retire, and because the trailing update is
// a grid of independent tiles, the SMs that PU(k+1) releases are picked up by
// the rest of TU_right(k): the counterpart of the malleable BLAS of Sec. 4.2.
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "internal.h"

static std::atomic<long long> g_launches{0};
static char g_last_error[512] = "";
static std::mutex g_err_mu;

void lu_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void lu_count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long lu_launches_so_far() { return g_launches.load(); }

void lu_set_error_string(const char* what, const char* file, int line) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", what, file, line);
}

int lu_func_attrs(const void* fn, int smem_bytes, bool nonportable_cluster) {
    static std::mutex mu;
    // (device, context, kernel) -> shared-memory limit set; the context distinguishes
    // the primary context from the green contexts of an SM partition
    static std::map<std::tuple<int, void*, const void*>, int> done;
    int dev = 0;
    LU_CHECK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, lu_current_ctx(), fn);
    auto it = done.find(key);
    if (it != done.end() && it->second >= smem_bytes) return LU_SUCCESS;
    if (nonportable_cluster)
        LU_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    LU_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes));
    done[key] = smem_bytes;
    return LU_SUCCESS;
}

extern "C" int lu_step_trace(lu_handle h, int enable) {
    if (!h) return LU_ERR_HANDLE;
    std::lock_guard<std::mutex> lk(h->mu);
    h->trace_on = enable != 0;
    return LU_SUCCESS;
}

extern "C" int64_t lu_step_trace_read(lu_handle h, int cap, int64_t* k0, int32_t* kb, float* span_ms, float* pu_ms,
                                      float* tu_ms) {
    if (!h) return LU_ERR_HANDLE;
    if (cap < 0) return -2;
    std::lock_guard<std::mutex> lk(h->mu);
    const int64_t cnt = std::min<int64_t>(h->trace_steps, (int64_t)h->trace.size());
    for (int64_t i = 0; i < cnt && i < cap; ++i) {
        const auto& t = h->trace[(size_t)i];
        float pu = 0.f, tu = 0.f, tue = 0.f;
        if (t.has_pu) {
            LU_CHECK_CUDA(cudaEventSynchronize(t.pu1));
            LU_CHECK_CUDA(cudaEventElapsedTime(&pu, t.pu0, t.pu1));
        }
        if (t.has_tu) {
            LU_CHECK_CUDA(cudaEventSynchronize(t.tu1));
            LU_CHECK_CUDA(cudaEventElapsedTime(&tu, t.tu0, t.tu1));
            LU_CHECK_CUDA(cudaEventElapsedTime(&tue, t.pu0, t.tu1));
        }
        if (k0) k0[i] = t.k0;
        if (kb) kb[i] = (int32_t)t.kb;
        if (span_ms) span_ms[i] = std::max(pu, tue);
        if (pu_ms) pu_ms[i] = pu;
        if (tu_ms) tu_ms[i] = tu;
    }
    return cnt;
}

extern "C" int64_t lu_launch_count(void) { return (int64_t)g_launches.load(); }
extern "C" const char* lu_last_error(void) { return g_last_error; }

extern "C" void lu_default_opts(lu_opts* o) {
    if (!o) return;
    o->nb = 256;
    o->lookahead = 1;
    o->steal = 1;
    o->leaf = 0;
    o->pf_ctas = 0;
    o->tu_reserve = 0;
    o->nsched = 0;
    o->sched = nullptr;
    o->rtm = 0;
    o->pf_sms = 0;
}

int lu_ctx_init(lu_context* c) {
    LU_CHECK_CUDA(cudaGetDevice(&c->device));
    LU_CHECK_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    int lo_prio = 0, hi_prio = 0;
    LU_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    LU_CHECK_CUDA(cudaStreamCreateWithPriority(&c->hi, cudaStreamNonBlocking, hi_prio));
    LU_CHECK_CUDA(cudaStreamCreateWithPriority(&c->lo, cudaStreamNonBlocking, lo_prio));
    cudaEvent_t* evs[] = {&c->ev_fork, &c->ev_pf, &c->ev_tu, &c->ev_join_hi, &c->ev_join_lo, &c->ev_steal,
                          &c->ev_tu2};
    for (cudaEvent_t* e : evs) LU_CHECK_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return LU_SUCCESS;
}

int lu_ctx_release(lu_context* c) {
    lu_green_release(c);
    if (c->ws) cudaFree(c->ws);
    c->ws = nullptr;
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    if (c->mx) cudaFree(c->mx);
    c->mx = nullptr;
    if (c->host_eta) cudaFreeHost(c->host_eta);
    c->host_eta = nullptr;
    if (c->batch_ws) cudaFree(c->batch_ws);
    c->batch_ws = nullptr;
    if (c->fgraph_exec) cudaGraphExecDestroy(c->fgraph_exec);
    c->fgraph_exec = nullptr;
    if (c->ev_g0) cudaEventDestroy(c->ev_g0);
    if (c->ev_g1) cudaEventDestroy(c->ev_g1);
    if (c->gs) cudaStreamDestroy(c->gs);
    c->ev_g0 = c->ev_g1 = nullptr;
    c->gs = nullptr;
    cudaEvent_t evs[] = {c->ev_fork, c->ev_pf, c->ev_tu, c->ev_join_hi, c->ev_join_lo, c->ev_steal, c->ev_tu2};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (c->rtm_exec) cudaGraphExecDestroy(c->rtm_exec);
    c->rtm_exec = nullptr;
    for (cudaStream_t x : c->rtm_cols)
        if (x) cudaStreamDestroy(x);
    c->rtm_cols.clear();
    for (cudaStream_t x : {c->rtm_left, c->rtm_origin})
        if (x) cudaStreamDestroy(x);
    c->rtm_left = c->rtm_origin = nullptr;
    for (auto* v : {&c->rtm_pf, &c->rtm_col, &c->rtm_sev})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    c->rtm_pf.clear();
    c->rtm_col.clear();
    c->rtm_sev.clear();
    for (cudaEvent_t e : {c->rtm_ev, c->rtm_ev2})
        if (e) cudaEventDestroy(e);
    c->rtm_ev = c->rtm_ev2 = nullptr;
    for (auto& t : c->trace) {
        cudaEvent_t te[] = {t.pu0, t.pu1, t.tu0, t.tu1};
        for (cudaEvent_t e : te)
            if (e) cudaEventDestroy(e);
    }
    c->trace.clear();
    if (c->hi) cudaStreamDestroy(c->hi);
    if (c->lo) cudaStreamDestroy(c->lo);
    return LU_SUCCESS;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int lu_ctx_reserve(lu_context* c, int64_t n, int nb) {
    nb = std::max(1, std::min(nb, LU_MAX_NB));
    const size_t nk = (size_t)std::max<int64_t>(1, lu_cdiv(std::max<int64_t>(n, 1), nb));
    const size_t plan_stride = 1 + 4 * (size_t)LU_MAX_NB;
    const size_t need_sync = align_up(sizeof(LuSync) * 8, 256);
    const size_t need_slots = align_up(sizeof(double) * (2 * LU_PF_MAX_CTAS * (LU_PF_MAX_LEAF + 1) + 2 * LU_PF_MAX_LEAF) +
                                           sizeof(int) * 2 * LU_PF_MAX_CTAS, 256);
    const size_t plans_cap = std::max(nk, c->plans_cap);
    const size_t need_plans = align_up(sizeof(int32_t) * plan_stride * (plans_cap + 1), 256);
    const size_t perm_cap = std::max<size_t>((size_t)std::max<int64_t>(n, 1), c->perm_cap);
    const size_t need_perm = align_up(sizeof(int32_t) * perm_cap, 256);
    const size_t total = need_sync + need_slots + need_plans + need_perm;
    if (c->ws && total <= c->ws_bytes) return LU_SUCCESS;
    if (c->ws) {
        LU_CHECK_CUDA(cudaStreamSynchronize(c->user));
        LU_CHECK_CUDA(cudaDeviceSynchronize());
        cudaFree(c->ws);
        c->ws = nullptr;
    }
    if (cudaMalloc(&c->ws, total) != cudaSuccess) {
        cudaGetLastError();
        c->ws_bytes = 0;
        return LU_ERR_NOMEM;
    }
    c->ws_bytes = total;
    char* p = c->ws;
    c->sync = reinterpret_cast<LuSync*>(p);
    p += need_sync;
    c->pf_slots = p;
    p += need_slots;
    c->plan_stride = plan_stride;
    c->plans_cap = plans_cap;
    c->plan_tmp = reinterpret_cast<int32_t*>(p);
    c->plans = c->plan_tmp + plan_stride;
    p += need_plans;
    c->perm = reinterpret_cast<int32_t*>(p);
    c->perm_cap = perm_cap;
    LU_CHECK_CUDA(cudaMemset(c->ws, 0, total));
    return LU_SUCCESS;
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
extern "C" int lu_create(lu_handle* h) {
    if (!h) return -1;
    lu_context* c = new (std::nothrow) lu_context();
    if (!c) return LU_ERR_NOMEM;
    int r = lu_ctx_init(c);
    if (r != LU_SUCCESS) {
        lu_ctx_release(c);
        delete c;
        return r;
    }
    *h = c;
    return LU_SUCCESS;
}

extern "C" int lu_destroy(lu_handle h) {
    if (!h) return LU_ERR_HANDLE;
    cudaDeviceSynchronize();
    lu_ctx_release(h);
    delete h;
    return LU_SUCCESS;
}

extern "C" int lu_set_stream(lu_handle h, void* stream) {
    if (!h) return LU_ERR_HANDLE;
    h->user = reinterpret_cast<cudaStream_t>(stream);
    return LU_SUCCESS;
}

static lu_handle g_default = nullptr;
static std::mutex g_default_mu;

static lu_handle default_handle() {
    std::lock_guard<std::mutex> lk(g_default_mu);
    if (!g_default) {
        if (lu_create(&g_default) != LU_SUCCESS) g_default = nullptr;
    }
    return g_default;
}

// ---------------------------------------------------------------------------
// factorization driver
// ---------------------------------------------------------------------------
int lu_check_opts(const lu_opts& o) {
    if (o.nb < 0 || o.nb > LU_MAX_NB) return -1;  // 0: resolved by the factorization entry points
    if (o.lookahead < 0 || o.lookahead > 2) return -1;
    if (o.leaf < 0 || o.pf_ctas < 0 || o.pf_ctas > LU_PF_MAX_CTAS) return -1;
    if (o.tu_reserve < 0 || o.nsched < 0 || o.nsched > (1 << 20)) return -1;
    if (o.rtm < 0 || o.rtm > 1) return -1;
    if (o.pf_sms < 0 || o.pf_sms > 4096) return -1;
    if (o.nsched > 0) {
        if (!o.sched) return -1;
        for (int i = 0; i < o.nsched; ++i)
            if (o.sched[i] < 1 || o.sched[i] > LU_MAX_NB) return -1;
    }
    return 0;
}

void lu_panel_bounds(int64_t n, const lu_opts& o, std::vector<int64_t>* s, int* wmin, int* wmax) {
    s->clear();
    s->push_back(0);
    int lo = LU_MAX_NB, hi = 1;
    for (int64_t c = 0, k = 0; c < n; ++k) {
        const int b = o.nsched > 0 ? o.sched[std::min<int64_t>(k, o.nsched - 1)] : o.nb;
        lo = std::min(lo, b);
        hi = std::max(hi, b);
        c = std::min<int64_t>(n, c + b);
        s->push_back(c);
    }
    if (wmin) *wmin = std::min(lo, hi);
    if (wmax) *wmax = hi;
}

int lu_resolve_reserve(const lu_context* c, const lu_opts& o) {
    if (!o.lookahead) return 0;
    if (o.tu_reserve > 0) return std::min(o.tu_reserve, std::max(0, c->num_sms - 1));
    return std::max(4, c->num_sms / 6);
}

// TU restricted to columns [c_begin, c_end) for step k (panel columns [k0, k0+kb)):
// laswp with panel k's plan, TRSM of the U12 block row, GEMM of the rows below.
// With a tensor-core engine the GEMM is the tcgen05 update on packed operands.
template <typename T>
static int trailing_update(lu_context* c, cudaStream_t st, int64_t n, T* A, int64_t lda, int64_t k, int64_t k0,
                           int64_t kb, int64_t c_begin, int64_t c_end, int64_t left_cols, const int32_t* plan,
                           const LuTuEngine* eng, int which, bool pivot) {
    const int64_t ncols = c_end - c_begin;
    // the right update's interchanges and RL2 run on at most the right update's share
    // of the SMs (as its tensor-core part), leaving the rest to the panel path
    const int cap = which == 1 ? (c->green_active ? lu_green_rest_sms(c) : std::max(1, c->num_sms - c->tu_reserve)) : 0;
    if (pivot && (ncols > 0 || left_cols > 0))
        LU_TRY(lu_launch_laswp_apply<T>(st, A, lda, c_begin, std::max<int64_t>(ncols, 0), 0, left_cols,
                                        plan, kb, c->num_sms, cap));
    if (ncols <= 0) return LU_SUCCESS;
    T* A11 = A + k0 + k0 * lda;
    T* A12 = A + k0 + c_begin * lda;
    // symmetric elimination keeps only the lower block triangle current: U12 is
    // formed from L21 (U12 = D1 L21^T) instead of RL2 on the (stale) upper part
    const int band = pivot ? 0 : c->sym_band;
    if (band > 0) LU_TRY(lu_launch_sym_u12<T>(st, A, lda, k0, kb, c_begin, c_end));
    else LU_TRY(lu_launch_trsm_lunit<T>(st, kb, ncols, A11, lda, A12, lda, cap));
    const int64_t m2 = n - (k0 + kb);
    if (m2 <= 0) return LU_SUCCESS;
    if (eng && eng->uses_tc(kb)) {
        return eng->update(st, (float*)A, lda, k, k0, kb, c_begin, c_end, which);
    }
    return lu_launch_gemm_update_band<T>(st, m2, ncols, kb, A + (k0 + kb) + k0 * lda, lda, A12, lda,
                                         A + (k0 + kb) + c_begin * lda, lda, k0 + kb, c_begin, band);
}

template <typename T>
int lu_step_tu(lu_context* c, cudaStream_t st, int64_t n, T* A, int64_t lda, int64_t k, int64_t k0, int64_t kb,
               int64_t cb, int64_t ce, int64_t left, bool pivot) {
    return trailing_update<T>(c, st, n, A, lda, k, k0, kb, cb, ce, left, c->plans + (size_t)k * c->plan_stride,
                              nullptr, 0, pivot);
}

template <typename T>
int lu_step_pf(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t n, int64_t k, int64_t k0, int64_t kb,
               int32_t* ipiv, const lu_opts& o, bool pivot) {
    if (!pivot) return lu_panel_nopiv<T>(st, A, lda, n, k0, kb, &c->sync[0]);
    LU_TRY(lu_panel_recursive<T>(c, st, A, lda, n, k0, kb, ipiv, o));
    return lu_launch_laswp_plan(st, ipiv, k0, k0 + kb, c->plans + (size_t)k * c->plan_stride);
}

template int lu_step_tu<double>(lu_context*, cudaStream_t, int64_t, double*, int64_t, int64_t, int64_t, int64_t,
                                int64_t, int64_t, int64_t, bool);
template int lu_step_tu<float>(lu_context*, cudaStream_t, int64_t, float*, int64_t, int64_t, int64_t, int64_t,
                               int64_t, int64_t, int64_t, bool);
template int lu_step_pf<double>(lu_context*, cudaStream_t, double*, int64_t, int64_t, int64_t, int64_t, int64_t,
                                int32_t*, const lu_opts&, bool);
template int lu_step_pf<float>(lu_context*, cudaStream_t, float*, int64_t, int64_t, int64_t, int64_t, int64_t,
                               int32_t*, const lu_opts&, bool);

// Timing events of one traced step (created on first use, kept by the handle).
static int trace_slot(lu_context* c, int64_t k, lu_context::StepTrace** out) {
    if ((int64_t)c->trace.size() <= k) c->trace.resize((size_t)k + 1);
    lu_context::StepTrace& t = c->trace[(size_t)k];
    cudaEvent_t* evs[] = {&t.pu0, &t.pu1, &t.tu0, &t.tu1};
    for (cudaEvent_t* e : evs)
        if (!*e) LU_CHECK_CUDA(cudaEventCreate(e));
    *out = &t;
    return LU_SUCCESS;
}

template <typename T>
int lu_factor_blocked(lu_context* c, int64_t n, T* A, int64_t lda, int32_t* ipiv, const lu_opts& o, int32_t* info,
                      const LuTuEngine* eng, bool pivot) {
    if (o.nb < 1 && o.nsched < 1) return LU_ERR_UNSUPPORTED;  // nb = 0 is resolved before this point
    if (o.rtm) return eng ? LU_ERR_UNSUPPORTED : lu_factor_rtm<T>(c, n, A, lda, ipiv, o, info, pivot);
    std::vector<int64_t> s;
    int wmin = 1, wmax = 1;
    lu_panel_bounds(n, o, &s, &wmin, &wmax);
    LU_TRY(lu_ctx_reserve(c, n, wmin));
    cudaStream_t user = c->user;
    LU_CHECK_CUDA(cudaMemsetAsync(&c->sync[0], 0, sizeof(LuSync), user));
    c->trace_steps = 0;
    if (n == 0) return lu_launch_finish_info(user, &c->sync[0], info);
    c->tu_reserve = lu_resolve_reserve(c, o);
    // an SM partition for the panel leaves: the right update then runs on the other SMs
    c->green_active = o.pf_sms > 0 && o.lookahead >= 1 && lu_green_setup(c, o.pf_sms) == LU_SUCCESS;
    struct GreenOff {
        lu_context* c;
        size_t budget;
        int threads;
        ~GreenOff() {
            c->green_active = false;
            c->pf_smem_budget = budget;
            c->pf_threads = threads;
        }
    } green_off{c, c->pf_smem_budget, c->pf_threads};
    // on their own SMs the leaves need not leave room for update CTAs: wider leaves
    // (32 columns at up to 16384 rows) fit, and 512 threads per CTA halve the rows
    // each thread carries through the per-column chain
    if (c->green_active) {
        c->pf_smem_budget = std::max<size_t>(c->pf_smem_budget, LU_PF_SMEM_PART);
        c->pf_threads = 512;
    }
    cudaStream_t lo = c->green_active ? lu_green_rest_stream(c) : c->lo;
    LU_CHECK_CUDA(cudaEventRecord(c->ev_fork, user));
    LU_CHECK_CUDA(cudaStreamWaitEvent(c->hi, c->ev_fork, 0));
    LU_CHECK_CUDA(cudaStreamWaitEvent(lo, c->ev_fork, 0));
    const int64_t nk = (int64_t)s.size() - 1;
    auto start = [&](int64_t j) { return s[(size_t)std::min(j, nk)]; };  // first column of panel j (n past the end)
    auto plan_of = [&](int64_t k) { return c->plans + (size_t)k * c->plan_stride; };
    cudaStream_t hi = c->hi;
    const bool trace = c->trace_on;
    // PF(k) followed by its interchange plan (and, for the tensor-core engine, the packed L21)
    auto panel = [&](int64_t k) -> int {
        const int64_t k0 = s[k], kb = s[k + 1] - s[k];
        if (!pivot) {
            LU_TRY(lu_panel_nopiv<T>(hi, A, lda, n, k0, kb, &c->sync[0]));
        } else {
            LU_TRY(lu_panel_recursive<T>(c, hi, A, lda, n, k0, kb, ipiv, o));
            LU_TRY(lu_launch_laswp_plan(hi, ipiv, k0, k0 + kb, plan_of(k)));
        }
        if (eng && eng->uses_tc(kb) && k0 + kb < n) LU_TRY(eng->pack_panel(hi, (const float*)A, lda, k, k0, kb));
        return LU_SUCCESS;
    };
    // TU_k restricted to columns [cb, ce), plus panel k's interchanges on `left` leading columns
    auto tu = [&](cudaStream_t st, int64_t k, int64_t cb, int64_t ce, int64_t left, int which) -> int {
        return trailing_update<T>(c, st, n, A, lda, k, s[k], s[k + 1] - s[k], cb, ce, left, plan_of(k), eng, which,
                                  pivot);
    };
    LU_TRY(panel(0));
    const int depth = o.lookahead;
    cudaEvent_t ev_tu[2] = {c->ev_tu, c->ev_tu2};  // TU_right of even / odd steps
    for (int64_t k = 0; k < nk; ++k) {
        const int64_t k0 = s[k];
        lu_context::StepTrace* tr = nullptr;
        if (trace) {
            LU_TRY(trace_slot(c, k, &tr));
            tr->k0 = k0;
            tr->kb = s[k + 1] - k0;
            tr->has_pu = k + 1 < nk;
            tr->has_tu = true;
            LU_CHECK_CUDA(cudaEventRecord(tr->pu0, hi));
        }
        if (depth == 0) {
            // Listing 3: TU_k over every column right of panel k, then PF_{k+1}
            if (tr) LU_CHECK_CUDA(cudaEventRecord(tr->tu0, hi));
            LU_TRY(tu(hi, k, start(k + 1), n, k0, 0));
            if (tr) LU_CHECK_CUDA(cudaEventRecord(tr->tu1, hi));
            if (k + 1 < nk) LU_TRY(panel(k + 1));
            if (tr) LU_CHECK_CUDA(cudaEventRecord(tr->pu1, hi));
            continue;
        }
        // Depth d: the high-priority stream owns the next d panels.  PU(k+1) =
        // TU_k on panel k+1, then PF_{k+1}.  TU_k^L (a few narrow launches) is
        // issued before TU_right(k) is released, so that it does not wait behind
        // the right update's thousands of CTAs; PF_{k+1} then overlaps TU_right(k).
        if (k + 1 < nk) LU_TRY(tu(hi, k, start(k + 1), start(k + 2), 0, 0));
        LU_CHECK_CUDA(cudaEventRecord(c->ev_pf, hi));
        LU_CHECK_CUDA(cudaStreamWaitEvent(lo, c->ev_pf, 0));
        // TU_right(k): the columns past the panels the high-priority stream owns,
        // and panel k's deferred interchanges on the columns left of it
        if (tr) LU_CHECK_CUDA(cudaEventRecord(tr->tu0, lo));
        if (c->green_active) {
            // launched with the partition's context current, so the update's CTAs stay on its SMs
            LU_TRY(lu_green_enter(c, false));
            const int r = tu(lo, k, start(k + 1 + depth), n, k0, 1);
            lu_green_leave();
            LU_TRY(r);
        } else {
            LU_TRY(tu(lo, k, start(k + 1 + depth), n, k0, 1));
        }
        if (tr) LU_CHECK_CUDA(cudaEventRecord(tr->tu1, lo));
        LU_CHECK_CUDA(cudaEventRecord(ev_tu[k & 1], lo));
        if (k + 1 < nk) {
            LU_TRY(panel(k + 1));
            if (tr) LU_CHECK_CUDA(cudaEventRecord(tr->pu1, hi));
            if (eng && o.steal) LU_TRY(eng->steal(hi, k));
        }
        if (depth == 1) {
            // the next step's TU_k+1 on panel k+2 reads columns TU_right(k) writes
            if (k + 1 < nk) LU_CHECK_CUDA(cudaStreamWaitEvent(hi, ev_tu[k & 1], 0));
        } else if (k + 2 < nk) {
            // depth 2: panel k+2 was part of TU_right(k-1); once that is done the
            // high-priority stream applies TU_k to it, so PF_{k+2} in the next step
            // waits for nothing on the update stream
            if (k > 0) LU_CHECK_CUDA(cudaStreamWaitEvent(hi, ev_tu[(k - 1) & 1], 0));
            LU_TRY(tu(hi, k, start(k + 2), start(k + 3), 0, 0));
        }
    }
    if (trace) c->trace_steps = nk;
    LU_CHECK_CUDA(cudaEventRecord(c->ev_join_hi, hi));
    LU_CHECK_CUDA(cudaEventRecord(c->ev_join_lo, lo));
    LU_CHECK_CUDA(cudaStreamWaitEvent(user, c->ev_join_hi, 0));
    LU_CHECK_CUDA(cudaStreamWaitEvent(user, c->ev_join_lo, 0));
    return lu_launch_finish_info(user, &c->sync[0], info);
}

template int lu_factor_blocked<double>(lu_context*, int64_t, double*, int64_t, int32_t*, const lu_opts&, int32_t*,
                                       const LuTuEngine*, bool);
template int lu_factor_blocked<float>(lu_context*, int64_t, float*, int64_t, int32_t*, const lu_opts&, int32_t*,
                                      const LuTuEngine*, bool);

extern "C" int lu_factor_ex(lu_handle h, lu_dtype dtype, int64_t n, void* A, int64_t lda, int32_t* ipiv,
                            const lu_opts* opts, int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (n < 0) return -3;
    if (n > 0 && !A) return -4;
    if (lda < std::max<int64_t>(1, n)) return -5;
    if (n > 0 && !ipiv) return -6;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -7;
    if (!info) return -8;
    if (n > INT32_MAX / 2) return LU_ERR_UNSUPPORTED;
    if (o.nb == 0 && o.nsched == 0) lu_auto_opts(dtype == LU_F64 ? LU_TUNE_F64 : LU_TUNE_F32, n, &o);
    std::lock_guard<std::mutex> lk(h->mu);
    if (dtype == LU_F64) return lu_factor_blocked<double>(h, n, (double*)A, lda, ipiv, o, info, nullptr);
    return lu_factor_blocked<float>(h, n, (float*)A, lda, ipiv, o, info, nullptr);
}

extern "C" int lu_factor(int64_t n, double* A, int64_t lda, int32_t* ipiv, int nb) {
    if (n < 0) return -1;
    if (n > 0 && !A) return -2;
    if (lda < std::max<int64_t>(1, n)) return -3;
    if (n > 0 && !ipiv) return -4;
    if (nb < 0 || nb > LU_MAX_NB) return -5;
    lu_handle h = default_handle();
    if (!h) return LU_ERR_CUDA;
    lu_opts o;
    lu_default_opts(&o);
    o.nb = nb;
    int32_t* dinfo = nullptr;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        LU_TRY(lu_ctx_reserve(h, n, nb));
        dinfo = reinterpret_cast<int32_t*>(&h->sync[3].info);
    }
    cudaStream_t saved = h->user;
    h->user = nullptr;
    int r = lu_factor_ex(h, LU_F64, n, A, lda, ipiv, &o, dinfo);
    h->user = saved;
    if (r != LU_SUCCESS) return r;
    int32_t info = 0;
    LU_CHECK_CUDA(cudaMemcpy(&info, dinfo, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return info;
}

// ---------------------------------------------------------------------------
// solve driver
// ---------------------------------------------------------------------------
template <typename T>
static int solve_impl(lu_context* c, int64_t n, int64_t nrhs, const T* LU, int64_t lda, const int32_t* ipiv,
                      T* B, int64_t ldb, T* tmp) {
    cudaStream_t st = c->user;
    LU_TRY(lu_ctx_reserve(c, n, 1));
    LU_TRY(lu_launch_perm_from_ipiv<T>(st, n, ipiv, c->perm));
    LU_TRY(lu_launch_permute_rows<T>(st, n, nrhs, c->perm, B, ldb, tmp, n));
    LU_CHECK_CUDA(cudaMemcpy2DAsync(B, ldb * sizeof(T), tmp, n * sizeof(T), n * sizeof(T), nrhs,
                                    cudaMemcpyDeviceToDevice, st));
    LU_TRY(lu_launch_trsv_blocked<T>(c, st, true, n, nrhs, LU, lda, B, ldb));
    LU_TRY(lu_launch_trsv_blocked<T>(c, st, false, n, nrhs, LU, lda, B, ldb));
    return LU_SUCCESS;
}

// Scratch for the row gather of a solve (n x nrhs), owned by the handle.
static int solve_scratch(lu_context* c, size_t bytes, void** out) {
    if (c->scratch_bytes < bytes) {
        if (c->scratch) {
            LU_CHECK_CUDA(cudaDeviceSynchronize());
            cudaFree(c->scratch);
            c->scratch = nullptr;
            c->scratch_bytes = 0;
        }
        if (cudaMalloc(&c->scratch, bytes) != cudaSuccess) {
            cudaGetLastError();
            return LU_ERR_NOMEM;
        }
        c->scratch_bytes = bytes;
    }
    *out = c->scratch;
    return LU_SUCCESS;
}

extern "C" int lu_solve_ex(lu_handle h, lu_dtype dtype, int64_t n, int64_t nrhs, const void* LU, int64_t lda,
                           const int32_t* ipiv, void* B, int64_t ldb) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (n < 0) return -3;
    if (nrhs < 0) return -4;
    if (n > 0 && !LU) return -5;
    if (lda < std::max<int64_t>(1, n)) return -6;
    if (n > 0 && !ipiv) return -7;
    if (n > 0 && nrhs > 0 && !B) return -8;
    if (ldb < std::max<int64_t>(1, n)) return -9;
    if (n == 0 || nrhs == 0) return LU_SUCCESS;
    std::lock_guard<std::mutex> lk(h->mu);
    const size_t es = dtype == LU_F64 ? 8 : 4;
    void* tmp = nullptr;
    LU_TRY(solve_scratch(h, es * (size_t)n * (size_t)nrhs, &tmp));
    if (dtype == LU_F64)
        return solve_impl<double>(h, n, nrhs, (const double*)LU, lda, ipiv, (double*)B, ldb, (double*)tmp);
    return solve_impl<float>(h, n, nrhs, (const float*)LU, lda, ipiv, (float*)B, ldb, (float*)tmp);
}

extern "C" int lu_solve(int64_t n, int64_t nrhs, const double* LU, const int32_t* ipiv, double* B) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (n > 0 && !LU) return -3;
    if (n > 0 && !ipiv) return -4;
    if (n > 0 && nrhs > 0 && !B) return -5;
    lu_handle h = default_handle();
    if (!h) return LU_ERR_CUDA;
    cudaStream_t saved = h->user;
    h->user = nullptr;
    int r = lu_solve_ex(h, LU_F64, n, nrhs, LU, std::max<int64_t>(1, n), ipiv, B, std::max<int64_t>(1, n));
    h->user = saved;
    if (r != LU_SUCCESS) return r;
    LU_CHECK_CUDA(cudaStreamSynchronize(nullptr));
    int err = 0;
    if (h->sync) LU_CHECK_CUDA(cudaMemcpy(&err, &h->sync[1].error, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != 0) {
        cudaMemset(&h->sync[1].error, 0, sizeof(int));
        return err;
    }
    return LU_SUCCESS;
}

// ---------------------------------------------------------------------------
// individual steps
// ---------------------------------------------------------------------------
extern "C" int lu_panel_factor_ex(lu_handle h, lu_dtype dtype, int64_t m, int64_t w, void* A, int64_t lda,
                                  int32_t* ipiv, const lu_opts* opts, int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (m < 0) return -3;
    if (w < 0 || w > m || w > LU_MAX_NB) return -4;
    if (m > 0 && w > 0 && !A) return -5;
    if (lda < std::max<int64_t>(1, m)) return -6;
    if (w > 0 && !ipiv) return -7;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -8;
    if (!info) return -9;
    std::lock_guard<std::mutex> lk(h->mu);
    LU_TRY(lu_ctx_reserve(h, m, (int)std::max<int64_t>(w, 1)));
    LU_CHECK_CUDA(cudaMemsetAsync(&h->sync[0], 0, sizeof(LuSync), h->user));
    if (w > 0) {
        if (dtype == LU_F64)
            LU_TRY(lu_panel_recursive<double>(h, h->user, (double*)A, lda, m, 0, w, ipiv, o));
        else
            LU_TRY(lu_panel_recursive<float>(h, h->user, (float*)A, lda, m, 0, w, ipiv, o));
    }
    return lu_launch_finish_info(h->user, &h->sync[0], info);
}

extern "C" int lu_laswp_ex(lu_handle h, lu_dtype dtype, int64_t ncols, void* A, int64_t lda, int64_t k1,
                           int64_t k2, const int32_t* ipiv) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (ncols < 0) return -3;
    if (ncols > 0 && !A) return -4;
    if (lda < 1) return -5;
    if (k1 < 0) return -6;
    if (k2 < k1 || k2 - k1 > LU_MAX_NB) return -7;
    if (k2 > k1 && !ipiv) return -8;
    if (ncols == 0 || k2 == k1) return LU_SUCCESS;
    std::lock_guard<std::mutex> lk(h->mu);
    LU_TRY(lu_ctx_reserve(h, k2, (int)(k2 - k1)));
    LU_TRY(lu_launch_laswp_plan(h->user, ipiv, k1, k2, h->plan_tmp));
    if (dtype == LU_F64)
        return lu_launch_laswp_apply<double>(h->user, (double*)A, lda, 0, ncols, 0, 0, h->plan_tmp, k2 - k1,
                                             h->num_sms);
    return lu_launch_laswp_apply<float>(h->user, (float*)A, lda, 0, ncols, 0, 0, h->plan_tmp, k2 - k1,
                                        h->num_sms);
}

extern "C" int lu_trsm_ex(lu_handle h, lu_dtype dtype, int64_t m, int64_t n, const void* L, int64_t ldl, void* B,
                          int64_t ldb) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (m < 0 || m > LU_MAX_NB) return -3;
    if (n < 0) return -4;
    if (m > 0 && !L) return -5;
    if (ldl < std::max<int64_t>(1, m)) return -6;
    if (m > 0 && n > 0 && !B) return -7;
    if (ldb < std::max<int64_t>(1, m)) return -8;
    if (dtype == LU_F64)
        return lu_launch_trsm_lunit<double>(h->user, m, n, (const double*)L, ldl, (double*)B, ldb);
    return lu_launch_trsm_lunit<float>(h->user, m, n, (const float*)L, ldl, (float*)B, ldb);
}

extern "C" int lu_gemm_update_ex(lu_handle h, lu_dtype dtype, int64_t m, int64_t n, int64_t k, const void* A,
                                 int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc) {
    if (!h) return LU_ERR_HANDLE;
    if (dtype != LU_F64 && dtype != LU_F32) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0 || k > INT32_MAX) return -5;
    if (m > 0 && k > 0 && !A) return -6;
    if (lda < std::max<int64_t>(1, m)) return -7;
    if (k > 0 && n > 0 && !B) return -8;
    if (ldb < std::max<int64_t>(1, k)) return -9;
    if (m > 0 && n > 0 && !C) return -10;
    if (ldc < std::max<int64_t>(1, m)) return -11;
    if (dtype == LU_F64)
        return lu_launch_gemm_update<double>(h->user, m, n, k, (const double*)A, lda, (const double*)B, ldb,
                                             (double*)C, ldc);
    return lu_launch_gemm_update<float>(h->user, m, n, k, (const float*)A, lda, (const float*)B, ldb, (float*)C,
                                        ldc);
}
