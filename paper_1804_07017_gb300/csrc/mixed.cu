// Mixed-precision path: FP32 panels and factors, trailing update on the tensor
// cores with bf16/fp16 operands and FP32 accumulation.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cstring>

#include "internal.h"
#include "ir.h"
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
    if (!lu_prec_is_tc(prec)) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0 || k % (prec == LU_TU_FP8 ? 128 : 64) != 0) return -5;
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
    if (m > 0 && n > 0 && k > 0 && prec == LU_TU_FP8) {
        const size_t abytes = al256((size_t)m * k), bbytes = al256((size_t)n * k);
        const size_t rbytes = al256(sizeof(float) * m), cbytes = al256(sizeof(float) * n);
        LU_TRY(lu_mx_reserve(h, abytes + bbytes + rbytes + cbytes));
        char* a = (char*)h->mx;
        char* b = a + abytes;
        float* rs = (float*)(b + bbytes);
        float* cs = (float*)((char*)rs + rbytes);
        LU_TRY(lu_launch_pack_rows_e4m3(st, A, lda, m, (int)k, rs, a));
        LU_TRY(lu_launch_pack_cols_e4m3(st, B, ldb, n, (int)k, cs, b));
        LU_TRY(lu_launch_tc_update(st, LU_TC_KIND_F8, LU_TC_FMT_E4M3, C, ldc, 0, m, 0, n, k, a, m, b, n, 1.0f,
                                   (int*)&h->sync[2].ticket, &h->sync[2].error, h->num_sms, 256, rs, cs));
    } else if (m > 0 && n > 0 && k > 0) {
        const int fmt = lu_prec_pack_fmt(prec);
        const int sg = lu_pack_segments(fmt);
        const size_t abytes = al256((size_t)m * k * 2 * sg), bbytes = al256((size_t)n * k * 2 * sg);
        LU_TRY(lu_mx_reserve(h, abytes + bbytes));
        char* a = (char*)h->mx;
        char* b = a + abytes;
        LU_TRY(lu_launch_pack_rows(st, fmt, A, lda, m, (int)k, a));
        LU_TRY(lu_launch_pack_cols(st, fmt, B, ldb, n, (int)k, b));
        LU_TRY(lu_launch_tc_update(st, LU_TC_KIND_F16, prec == LU_TU_FP16 ? LU_TC_FMT_F16 : LU_TC_FMT_BF16, C, ldc, 0,
                                   m, 0, n, k * sg, a, m, b, n, 1.0f, (int*)&h->sync[2].ticket, &h->sync[2].error,
                                   h->num_sms, 256));
    }
    return lu_launch_finish_info(st, &h->sync[2], info);
}

// ---------------------------------------------------------------------------
// Tensor-core trailing-update engine for the FP32 blocked factorization.
// ---------------------------------------------------------------------------
namespace {

struct TcEngine final : LuTuEngine {
    lu_context* c = nullptr;
    int prec = LU_TU_BF16;
    int64_t n = 0;
    int nb = 0;
    // packed L21 and U12 (K-major, n x nb each), one pair per panel in flight:
    // two with depth-1 look-ahead, three with depth 2 (panel k's operands are
    // read until TU_right(k) ends, which may be after PF_{k+2} starts)
    static constexpr int kMaxBuf = 3;
    int nbuf = 2;
    char* alo[kMaxBuf] = {nullptr, nullptr, nullptr};
    char* blo[kMaxBuf] = {nullptr, nullptr, nullptr};
    int* counter[2] = {nullptr, nullptr};
    int* error = nullptr;
    int grid_panel = 0, grid_right = 0, grid_steal = 0;
    int band = 0;  // > 0: symmetric (Cholesky) update of the lower block triangle only
    cudaEvent_t ev_ready = nullptr;
    mutable int64_t last_k = -1;
    mutable int64_t last_k0 = 0, last_kb = 0, last_cb = 0, last_ce = 0;

    bool fp8() const { return prec == LU_TU_FP8; }
    int fmt_pack() const { return lu_prec_pack_fmt(prec); }
    int fmt_mma() const { return fp8() ? LU_TC_FMT_E4M3 : (prec == LU_TU_FP16 ? LU_TC_FMT_F16 : LU_TC_FMT_BF16); }
    int segs() const { return fp8() ? 1 : lu_pack_segments(fmt_pack()); }
    int esize() const { return fp8() ? 1 : 2; }
    // FP8: the block scales follow the e4m3 bytes in each operand buffer
    size_t scale_off() const { return al256((size_t)n * nb); }
    float* rscale(int64_t k) const { return reinterpret_cast<float*>(alo[k % nbuf] + scale_off()); }
    float* cscale(int64_t k, int64_t off) const { return reinterpret_cast<float*>(blo[k % nbuf] + scale_off()) + off; }

    bool uses_tc(int64_t kb) const override { return lu_prec_is_tc(prec) && kb % (fp8() ? 128 : 64) == 0; }

    int pack_panel(cudaStream_t st, const float* A, int64_t lda, int64_t k, int64_t k0, int64_t kb) const override {
        if (fp8())
            return lu_launch_pack_rows_e4m3(st, A + (k0 + kb) + k0 * lda, lda, n - (k0 + kb), (int)kb, rscale(k),
                                            alo[k % nbuf]);
        return lu_launch_pack_rows(st, fmt_pack(), A + (k0 + kb) + k0 * lda, lda, n - (k0 + kb), (int)kb, alo[k % nbuf]);
    }

    int launch(cudaStream_t st, float* A, int64_t lda, int64_t k, int64_t k0, int64_t kb, int64_t cb, int64_t ce,
               int which, int grid) const {
        const int64_t m = n - (k0 + kb);
        const int64_t off = cb - (k0 + kb);
        const char* bbuf = blo[k % nbuf] + (size_t)off * kb * esize() * segs();
        return lu_launch_tc_update(st, fp8() ? LU_TC_KIND_F8 : LU_TC_KIND_F16, fmt_mma(), A, lda, k0 + kb, m, cb,
                                   ce - cb, kb * segs(), alo[k % nbuf], m, bbuf, ce - cb, 1.0f, counter[which], error,
                                   grid, 256, fp8() ? rscale(k) : nullptr, fp8() ? cscale(k, off) : nullptr, band);
    }

    int update(cudaStream_t st, float* A, int64_t lda, int64_t k, int64_t k0, int64_t kb, int64_t cb, int64_t ce,
               int which) const override {
        const int64_t off = cb - (k0 + kb);
        char* bbuf = blo[k % nbuf] + (size_t)off * kb * esize() * segs();
        if (fp8())
            LU_TRY(lu_launch_pack_cols_e4m3(st, A + k0 + cb * lda, lda, ce - cb, (int)kb, cscale(k, off), bbuf));
        else
            LU_TRY(lu_launch_pack_cols(st, fmt_pack(), A + k0 + cb * lda, lda, ce - cb, (int)kb, bbuf));
        LU_CHECK_CUDA(cudaMemsetAsync(counter[which], 0, sizeof(int), st));
        if (which == 1) {
            LU_CHECK_CUDA(cudaEventRecord(ev_ready, st));
            last_k = k;
            last_k0 = k0;
            last_kb = kb;
            last_cb = cb;
            last_ce = ce;
        }
        return launch(st, A, lda, k, k0, kb, cb, ce, which,
                      which == 0 ? grid_panel : (c->green_active ? lu_green_rest_sms(c) : grid_right));
    }

    float* A_ = nullptr;
    int64_t lda_ = 0;

    int steal(cudaStream_t st, int64_t k) const override {
        if (last_k != k || grid_steal <= 0) return LU_SUCCESS;
        LU_CHECK_CUDA(cudaStreamWaitEvent(st, ev_ready, 0));
        return launch(st, A_, lda_, k, last_k0, last_kb, last_cb, last_ce, 1, grid_steal);
    }
};

// Operand buffers of the engine for an order-n factorization with options o:
// 2 * nbuf buffers sized for the widest panel of o's schedule.
int engine_nbuf(const lu_opts& o) { return o.lookahead >= 2 ? 3 : 2; }

int engine_width(int64_t n, const lu_opts& o) {
    std::vector<int64_t> s;
    int wmin = 1, wmax = 1;
    lu_panel_bounds(std::max<int64_t>(n, 1), o, &s, &wmin, &wmax);
    return wmax;
}

// Narrowest panel of o's schedule: the handle workspace (interchange plans) is
// sized for it before the engine takes pointers into that workspace.
int narrowest(int64_t n, const lu_opts& o) {
    std::vector<int64_t> s;
    int wmin = 1, wmax = 1;
    lu_panel_bounds(std::max<int64_t>(n, 1), o, &s, &wmin, &wmax);
    return wmin;
}

size_t tc_engine_one(int prec, int64_t n, int nb) {
    if (prec == LU_TU_FP8) return al256(al256((size_t)n * nb) + sizeof(float) * (size_t)n);
    return al256((size_t)n * nb * 2 * lu_pack_segments(lu_prec_pack_fmt(prec)));
}

size_t tc_engine_bytes(int prec, int64_t n, const lu_opts& o) {
    if (!lu_prec_is_tc(prec)) return 256;
    return 2 * (size_t)engine_nbuf(o) * tc_engine_one(prec, n, engine_width(n, o));
}

int setup_engine(TcEngine& e, lu_context* c, int prec, int64_t n, char* base, float* A, int64_t lda,
                 const lu_opts& o) {
    e.c = c;
    e.prec = prec;
    e.n = n;
    e.nb = engine_width(n, o);
    e.nbuf = engine_nbuf(o);
    const size_t one = tc_engine_one(prec, n, e.nb);
    for (int i = 0; i < e.nbuf; ++i) {
        e.alo[i] = base + (size_t)i * one;
        e.blo[i] = base + (size_t)(e.nbuf + i) * one;
    }
    e.counter[0] = (int*)&c->sync[4].ticket;
    e.counter[1] = (int*)&c->sync[5].ticket;
    e.error = &c->sync[0].error;
    e.A_ = A;
    e.lda_ = lda;
    // With look-ahead the right update leaves some SMs to the panel path
    // (opts.tu_reserve, by default a sixth: measured best at n = 16384 among 9,
    // 24, 48, 76 and 100 of 152); with stealing, that many CTAs join the right
    // update once the panel is done.
    const int reserve = o.steal ? lu_resolve_reserve(c, o) : 0;
    e.grid_right = std::max(1, c->num_sms - reserve);
    e.grid_panel = c->num_sms;
    e.grid_steal = reserve;
    e.ev_ready = c->ev_steal;
    return LU_SUCCESS;
}

}  // namespace

// FP32 factorization with a tensor-core trailing update (the factor step of the
// mixed-precision solver).  A32 is overwritten by the FP32 factors.
static int factor_mixed(lu_context* c, int prec, int64_t n, float* A32, int64_t lda, int32_t* ipiv, const lu_opts& o,
                        int32_t* info, char* engine_mem) {
    if (!lu_prec_is_tc(prec)) return lu_factor_blocked<float>(c, n, A32, lda, ipiv, o, info, nullptr);
    TcEngine e;
    LU_TRY(setup_engine(e, c, prec, n, engine_mem, A32, lda, o));
    // panel leaves must fit beside a tensor-core update CTA on the same SM
    const size_t saved = c->pf_smem_budget;
    const int saved_threads = c->pf_threads;
    c->pf_smem_budget = LU_PF_SMEM_BUDGET;
    c->pf_threads = 256;
    // The launch sequence depends only on these arguments, so a repeated call
    // replays it as one CUDA graph (no per-kernel launch gaps on the panel path):
    // a key is run eagerly on first use, captured on its second, replayed after.
    uint64_t sched_hash = 1469598103934665603ull;  // FNV-1a over the schedule
    for (int i = 0; i < o.nsched; ++i) sched_hash = (sched_hash ^ (uint64_t)(uint32_t)o.sched[i]) * 1099511628211ull;
    const uint64_t key[12] = {(uint64_t)(uintptr_t)A32, (uint64_t)lda, (uint64_t)n, (uint64_t)(uintptr_t)ipiv,
                              (uint64_t)(uintptr_t)info, (uint64_t)prec,
                              ((uint64_t)o.nb << 32) | ((uint64_t)o.lookahead << 16) | (uint64_t)o.steal,
                              ((uint64_t)o.leaf << 32) | (uint64_t)o.pf_ctas, (uint64_t)(uintptr_t)engine_mem,
                              (uint64_t)(uintptr_t)c->user,
                              ((uint64_t)(uint32_t)o.tu_reserve << 32) | (uint64_t)(uint32_t)o.nsched,
                              sched_hash ^ ((uint64_t)(uint32_t)o.rtm << 40) ^ ((uint64_t)(uint32_t)o.pf_sms << 48)};
    bool use_graph = !lu_profile_active() && !c->trace_on && n > 0;
    if (use_graph && !c->gs) {
        // the caller's stream may be the legacy default stream, which cannot be
        // captured: the graph is captured on, and replayed from, a stream of its own
        if (cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_g0, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_g1, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            use_graph = false;
        }
    }
    auto replay = [&]() -> int {
        LU_CHECK_CUDA(cudaEventRecord(c->ev_g0, c->user));
        LU_CHECK_CUDA(cudaStreamWaitEvent(c->gs, c->ev_g0, 0));
        if (cudaGraphLaunch(c->fgraph_exec, c->gs) != cudaSuccess) {
            lu_set_error_string("cudaGraphLaunch failed (factorization)", __FILE__, __LINE__);
            return LU_ERR_CUDA;
        }
        LU_CHECK_CUDA(cudaEventRecord(c->ev_g1, c->gs));
        LU_CHECK_CUDA(cudaStreamWaitEvent(c->user, c->ev_g1, 0));
        lu_count_launches(c->fgraph_launches);
        return LU_SUCCESS;
    };
    int r = LU_SUCCESS;
    if (use_graph && c->fgraph_exec && memcmp(key, c->fkey, sizeof(key)) == 0) {
        r = replay();
    } else if (use_graph && memcmp(key, c->fkey_seen, sizeof(key)) == 0) {
        const long long before = lu_launches_so_far();
        cudaGraph_t g = nullptr;
        cudaStream_t user = c->user;
        cudaError_t ce = cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal);
        int rc = LU_SUCCESS;
        if (ce == cudaSuccess) {
            c->user = c->gs;
            rc = lu_factor_blocked<float>(c, n, A32, lda, ipiv, o, info, &e);
            c->user = user;
            const cudaError_t ee = cudaStreamEndCapture(c->gs, &g);
            if (ee != cudaSuccess) ce = ee;
        }
        const long long captured = lu_launches_so_far() - before;
        lu_count_launches(-captured);  // nothing ran yet
        if (ce == cudaSuccess && rc == LU_SUCCESS) {
            if (c->fgraph_exec) cudaGraphExecDestroy(c->fgraph_exec);
            c->fgraph_exec = nullptr;
            ce = cudaGraphInstantiate(&c->fgraph_exec, g, 0);
        }
        if (g) cudaGraphDestroy(g);
        if (ce == cudaSuccess && rc == LU_SUCCESS) {
            memcpy(c->fkey, key, sizeof(key));
            c->fgraph_launches = captured;
            r = replay();
        } else {
            // the capture recorded nothing that ran: fall back to the eager launches
            // (and do not try this key again)
            cudaGetLastError();
            if (c->fgraph_exec) cudaGraphExecDestroy(c->fgraph_exec);
            c->fgraph_exec = nullptr;
            memset(c->fkey_seen, 0, sizeof(c->fkey_seen));
            if (getenv("LU_GB300_TRACE"))
                fprintf(stderr, "[lu] factorization graph capture failed (%s, status %d); eager launches\n",
                        cudaGetErrorString(ce), rc);
            r = lu_factor_blocked<float>(c, n, A32, lda, ipiv, o, info, &e);
        }
    } else {
        r = lu_factor_blocked<float>(c, n, A32, lda, ipiv, o, info, &e);
        memcpy(c->fkey_seen, key, sizeof(key));
    }
    c->pf_smem_budget = saved;
    c->pf_threads = saved_threads;
    return r;
}

extern "C" int lu_factor_mixed_ex(lu_handle h, lu_prec prec, int64_t n, float* A, int64_t lda, int32_t* ipiv,
                                  const lu_opts* opts, int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (!lu_prec_is_tc(prec) && prec != LU_TU_F32) return -2;
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
    if (o.nb == 0 && o.nsched == 0) lu_auto_opts(prec, n, &o);
    std::lock_guard<std::mutex> lk(h->mu);
    LU_TRY(lu_ctx_reserve(h, n, narrowest(n, o)));
    LU_TRY(lu_mx_reserve(h, tc_engine_bytes(prec, std::max<int64_t>(n, 1), o)));
    return factor_mixed(h, prec, n, A, lda, ipiv, o, info, (char*)h->mx);
}

extern "C" int lu_potrf_mixed_ex(lu_handle h, lu_prec prec, int64_t n, float* A, int64_t lda, const lu_opts* opts,
                                 int32_t* info) {
    if (!h) return LU_ERR_HANDLE;
    if (!lu_prec_is_tc(prec) && prec != LU_TU_F32) return -2;
    if (n < 0) return -3;
    if (n > 0 && !A) return -4;
    if (lda < std::max<int64_t>(1, n)) return -5;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -6;
    if (!info) return -7;
    if (n > INT32_MAX / 2) return LU_ERR_UNSUPPORTED;
    if (o.nb == 0 && o.nsched == 0) lu_auto_opts(LU_TUNE_F32, n, &o);
    if (o.rtm && lu_prec_is_tc(prec)) return LU_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(h->mu);
    if (!lu_prec_is_tc(prec)) return lu_chol_factor_f32(h, n, A, lda, o, info, nullptr);
    LU_TRY(lu_ctx_reserve(h, n, narrowest(n, o)));
    LU_TRY(lu_mx_reserve(h, tc_engine_bytes(prec, std::max<int64_t>(n, 1), o)));
    TcEngine e;
    LU_TRY(setup_engine(e, h, prec, n, (char*)h->mx, A, lda, o));
    e.band = o.nsched == 0 ? o.nb : 0;
    return lu_chol_factor_f32(h, n, A, lda, o, info, &e);
}

// ---------------------------------------------------------------------------
// Solver with FP64 iterative refinement.  T is the working precision of the
// factors and of the correction solves: float for the mixed-precision
// variants, double for the plain FP64 reference path (LU_FULL_F64).
// ---------------------------------------------------------------------------
template <typename T>
static int gesv_refined(lu_context* h, int prec, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                        const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int max_iter,
                        const lu_opts& o, int* iters, double* bwd_err) {
    cudaStream_t st = h->user;
    LU_TRY(lu_ctx_reserve(h, n, narrowest(n, o)));
    if (!h->host_eta) LU_CHECK_CUDA(cudaMallocHost(&h->host_eta, 4 * sizeof(double)));
    const int64_t ldw = (n + 31) / 32 * 32;
    const int64_t nch = lu_ir_nchunks(n);
    const int64_t rhs_chunk = std::min<int64_t>(nrhs, 16);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o0 = off; off += al256(bytes); return o0; };
    const size_t o_aw = take(sizeof(T) * (size_t)ldw * n);
    const size_t o_eng = take(sizeof(T) == 4 ? tc_engine_bytes(prec, n, o) : 256);
    const size_t o_ipiv = take(sizeof(int32_t) * n);
    const size_t o_perm = take(sizeof(int32_t) * n);
    const size_t o_r = take(sizeof(double) * n * nrhs);
    const size_t o_xb = take(sizeof(double) * n * nrhs);
    const size_t o_rw = take(sizeof(T) * n * nrhs);
    const size_t o_dw = take(sizeof(T) * n * nrhs);
    const size_t o_part = take(sizeof(double) * nch * rhs_chunk * n);
    const size_t o_sc = take(sizeof(double) * (8 + nrhs) + sizeof(int32_t) * 8);
    const size_t o_dinv = take(lu_trinv_bytes<T>(n));
    const size_t o_xtag = take(sizeof(unsigned long long) * n);
    LU_TRY(lu_mx_reserve(h, off));
    char* base = (char*)h->mx;
    T* Aw = (T*)(base + o_aw);
    int32_t* ipiv = (int32_t*)(base + o_ipiv);
    int32_t* perm = (int32_t*)(base + o_perm);
    double* R = (double*)(base + o_r);
    double* Xb = (double*)(base + o_xb);
    T* rw = (T*)(base + o_rw);
    T* dw = (T*)(base + o_dw);
    double* part = (double*)(base + o_part);
    double* sc = (double*)(base + o_sc);
    T* Dinv = (T*)(base + o_dinv);
    unsigned long long* xtag = (unsigned long long*)(base + o_xtag);
    double* anorm = sc;
    double* eta = sc + 1;
    double* eta_cols = sc + 8;
    int32_t* dinfo = (int32_t*)(sc + 8 + nrhs);
    unsigned int* done = (unsigned int*)(dinfo + 2);
    LU_CHECK_CUDA(cudaMemsetAsync(sc, 0, sizeof(double) * (8 + nrhs) + sizeof(int32_t) * 8, st));
    LU_CHECK_CUDA(cudaMemsetAsync(xtag, 0, sizeof(unsigned long long) * n, st));

    // 1. working copy in T and its factorization
    LU_TRY((lu_launch_cast<double, T>(st, n, n, A, lda, Aw, ldw)));
    if (sizeof(T) == 4)
        LU_TRY(factor_mixed(h, prec, n, (float*)Aw, ldw, ipiv, o, dinfo, base + o_eng));
    else
        LU_TRY(lu_factor_blocked<double>(h, n, (double*)Aw, ldw, ipiv, o, dinfo, nullptr));
    LU_TRY(lu_launch_perm_from_ipiv<T>(st, n, ipiv, perm));
    // inverses of the diagonal blocks of L and U: every correction solve then
    // costs one dense block product per block instead of a substitution chain
    LU_TRY(lu_launch_trinv_diag<T>(st, n, Aw, ldw, Dinv));
    LU_TRY(lu_launch_norm_inf(st, n, A, lda, part, anorm));
    // 2. x0 = U^-1 L^-1 P b in T
    LU_TRY((lu_launch_cast<double, T>(st, n, nrhs, B, ldb, rw, n)));
    LU_TRY(lu_launch_permute_rows<T>(st, n, nrhs, perm, rw, n, dw, n));
    LU_TRY(lu_launch_trsv_blocked<T>(h, st, true, n, nrhs, Aw, ldw, dw, n, Dinv, xtag));
    LU_TRY(lu_launch_trsv_blocked<T>(h, st, false, n, nrhs, Aw, ldw, dw, n, Dinv, xtag));
    LU_TRY((lu_launch_cast<T, double>(st, n, nrhs, dw, n, X, ldx)));
    // 3. refinement: r = b - A x (FP64), eta test on the host, d = (LU)^-1 P r (T), x += d (FP64)
    double best = INFINITY;
    int best_it = -1, it = 0;
    int status = LU_SUCCESS;
    const char* tr = getenv("LU_GB300_TRACE");
    const bool trace = tr && tr[0] == '1';
    for (;; ++it) {
        for (int64_t c0 = 0; c0 < nrhs; c0 += 16) {
            const int64_t nr = std::min<int64_t>(16, nrhs - c0);
            LU_TRY(lu_launch_residual(st, n, nr, A, lda, X + c0 * ldx, ldx, B + c0 * ldb, ldb, R + c0 * n, n, part));
        }
        LU_TRY(lu_launch_eta(st, n, nrhs, R, n, X, ldx, B, ldb, anorm, eta_cols, eta, done));
        LU_CHECK_CUDA(cudaMemcpyAsync(h->host_eta, eta, sizeof(double), cudaMemcpyDeviceToHost, st));
        LU_CHECK_CUDA(cudaMemcpyAsync(h->host_eta + 1, dinfo, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LU_CHECK_CUDA(cudaStreamSynchronize(st));
        const int32_t finfo = *reinterpret_cast<int32_t*>(h->host_eta + 1);
        if (finfo != 0) {
            status = finfo;  // exactly singular U (i > 0) or a device-side timeout (< 0)
            break;
        }
        const double e = h->host_eta[0];
        if (trace) fprintf(stderr, "[lu_gesv_mixed] iteration %d eta %.3e\n", it, e);
        if (e < best) {
            best = e;
            best_it = it;
            if (e > 0.9 * tol && it < max_iter)
                LU_CHECK_CUDA(cudaMemcpy2DAsync(Xb, n * sizeof(double), X, ldx * sizeof(double), n * sizeof(double),
                                                nrhs, cudaMemcpyDeviceToDevice, st));
        }
        // the residual is formed in plain FP64 (rounding ~ sqrt(n) u relative to |A||x|), so
        // convergence is declared with a 10% margin to keep the exact eta below tol
        if (e <= 0.9 * tol) break;
        if (it >= max_iter || !(e == e)) {
            status = LU_WARN_NOT_CONVERGED;
            break;
        }
        LU_TRY((lu_launch_cast<double, T>(st, n, nrhs, R, n, rw, n)));
        LU_TRY(lu_launch_permute_rows<T>(st, n, nrhs, perm, rw, n, dw, n));
        LU_TRY(lu_launch_trsv_blocked<T>(h, st, true, n, nrhs, Aw, ldw, dw, n, Dinv, xtag));
        LU_TRY(lu_launch_trsv_blocked<T>(h, st, false, n, nrhs, Aw, ldw, dw, n, Dinv, xtag));
        LU_TRY(lu_launch_add_to_f64<T>(st, n, nrhs, dw, n, X, ldx));
    }
    if (status == LU_WARN_NOT_CONVERGED && best_it >= 0 && best_it != it) {
        LU_CHECK_CUDA(cudaMemcpy2DAsync(X, ldx * sizeof(double), Xb, n * sizeof(double), n * sizeof(double), nrhs,
                                        cudaMemcpyDeviceToDevice, st));
        LU_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    if (iters) *iters = (status == LU_WARN_NOT_CONVERGED) ? best_it : it;
    if (bwd_err) *bwd_err = best;
    if (status == LU_SUCCESS) {
        int err = 0;
        LU_CHECK_CUDA(cudaMemcpy(&err, &h->sync[1].error, sizeof(int), cudaMemcpyDeviceToHost));
        if (err != 0) {
            cudaMemset(&h->sync[1].error, 0, sizeof(int));
            return err;
        }
    }
    return status;
}

extern "C" int lu_gesv_mixed(lu_handle h, lu_prec prec, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                             const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int max_iter,
                             const lu_opts* opts, int* iters, double* bwd_err) {
    if (!h) return LU_ERR_HANDLE;
    if (!lu_prec_is_tc(prec) && prec != LU_TU_F32 && prec != LU_FULL_F64) return -2;
    if (prec == LU_TU_FP8 && opts && opts->nb % 128 != 0) return -13;
    if (n < 0) return -3;
    if (nrhs < 0) return -4;
    if (n > 0 && !A) return -5;
    if (lda < std::max<int64_t>(1, n)) return -6;
    if (n > 0 && nrhs > 0 && !B) return -7;
    if (ldb < std::max<int64_t>(1, n)) return -8;
    if (n > 0 && nrhs > 0 && !X) return -9;
    if (ldx < std::max<int64_t>(1, n)) return -10;
    if (!(tol >= 0.0)) return -11;
    if (max_iter < 0) return -12;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    if (lu_check_opts(o) != 0) return -13;
    if (iters) *iters = 0;
    if (bwd_err) *bwd_err = 0.0;
    if (n == 0 || nrhs == 0) return LU_SUCCESS;
    if (n > INT32_MAX / 2) return LU_ERR_UNSUPPORTED;
    if (o.nb == 0 && o.nsched == 0) lu_auto_opts(prec == LU_FULL_F64 ? LU_TUNE_F64 : (int)prec, n, &o);
    std::lock_guard<std::mutex> lk(h->mu);
    if (prec == LU_FULL_F64)
        return gesv_refined<double>(h, prec, n, nrhs, A, lda, B, ldb, X, ldx, tol, max_iter, o, iters, bwd_err);
    return gesv_refined<float>(h, prec, n, nrhs, A, lda, B, ldb, X, ldx, tol, max_iter, o, iters, bwd_err);
}
