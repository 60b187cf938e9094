// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

// Upper limits baked into kernels and workspace sizing.
#define LU_PF_MAX_CTAS 128    // CTAs of one panel-factorization leaf launch
#define LU_PF_MAX_LEAF 64     // widest leaf (columns held in shared memory)
#define LU_MAX_NB 1024        // widest panel accepted

// nb for a factorization called with nb = 0: the tuned value for (kind, n) on
// the current device, else 256 (tune.cu).
int lu_auto_nb(int kind, int64_t n);
// The table's value for (kind, n) on the current device, or 0 (tune file loaded first).
int lu_tuned_value(int kind, int64_t n);
// Options of a factorization called with nb = 0 (and no schedule): the plan the
// tuner stored for (kind, n) on the current device -- nb or a per-step schedule,
// the right update's SM reserve (when o->tu_reserve is 0) and the look-ahead
// depth (when look-ahead is on) -- else nb = 256.  A schedule points into
// thread-local storage that stays valid until this thread's next call.
void lu_auto_opts(int kind, int64_t n, lu_opts* o);
#define LU_PF_SMEM_BUDGET (78 * 1024)
#define LU_PF_SMEM_PART (160 * 1024)  // leaf budget on an SM partition of its own (checked at set-up)
#define LU_PF_MAX_CTAS_CLUSTER 16  // CTAs of a cluster panel leaf (non-portable cluster size)

struct LuGreen;  // green-context SM partition of the panel leaves (green.cu)

struct lu_context {
    int device = 0;
    int num_sms = 0;
    cudaStream_t user = nullptr;  // stream set by lu_set_stream
    cudaStream_t hi = nullptr;    // high-priority internal stream (panel path)
    cudaStream_t lo = nullptr;    // low-priority internal stream (right trailing update)
    cudaEvent_t ev_fork = nullptr, ev_pf = nullptr, ev_tu = nullptr, ev_join_hi = nullptr,
                ev_join_lo = nullptr, ev_steal = nullptr, ev_tu2 = nullptr;
    // Workspace: one device buffer carved into fixed regions.
    char* ws = nullptr;
    size_t ws_bytes = 0;
    LuSync* sync = nullptr;   // [0] panel leaves + factorization errors, [1] triangular solves,
                              // [2] standalone tensor-core update, [3] lu_factor info, [4]/[5] tile counters
    void* pf_slots = nullptr; // panel-leaf exchange slots
    int32_t* plans = nullptr; // per-panel interchange plans
    size_t plan_stride = 0;   // int32 entries per plan
    size_t plans_cap = 0;     // number of plans
    int32_t* plan_tmp = nullptr;  // plan used inside the recursive panel
    int32_t* perm = nullptr;  // row permutation for solves
    int32_t* flags = nullptr; // ready flags of the blocked triangular solves
    size_t perm_cap = 0, flags_cap = 0;
    // Scratch for the row gather of a solve.
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // Mixed-precision workspace (FP32 working copy, packed operands, IR vectors).
    void* mx = nullptr;
    size_t mx_bytes = 0;
    double* host_eta = nullptr;  // pinned host word for the convergence test
    // Batched path: matrix order (largest first) and the work counter.
    void* batch_ws = nullptr;
    size_t batch_ws_bytes = 0;
    // Shared memory a panel leaf CTA may use: small enough, on the mixed path, to
    // sit beside a tensor-core trailing-update CTA on the same SM.
    size_t pf_smem_budget = 160 * 1024;
    // threads per CTA of an FP32 cluster leaf: 512 (half the rows per thread of 256)
    // wherever the leaf may take most of an SM, 256 beside the tensor-core update
    int pf_threads = 512;
    // SMs the right trailing update leaves to the panel path (set per factorization).
    int tu_reserve = 0;
    // Symmetric (Cholesky) trailing update: > 0 = the panel width; the updates then
    // form U12 from L21 and touch only the lower block triangle (chol.cu).
    int sym_band = 0;
    // Batched kernel: a tile cut-over forced by lu_tune_batched while it times candidates (0 = none)
    int batched_cut_override = 0;
    // SM partition for the panel leaves (lu_opts.pf_sms); active during a factorization
    LuGreen* green = nullptr;
    bool green_active = false;
    // Per-step trace of the look-ahead schedule (lu_step_trace): timing events
    // around PU(k+1) on the panel stream and TU_right(k) on the update stream.
    struct StepTrace {
        cudaEvent_t pu0 = nullptr, pu1 = nullptr, tu0 = nullptr, tu1 = nullptr;
        int64_t k0 = 0, kb = 0;
        bool has_pu = false, has_tu = false;
    };
    // Runtime-task schedule (rtm.cu): one stream per block-column class, the left
    // interchanges' stream, the capture origin, per-panel and per-column events,
    // and the DAG's instantiated graph with the arguments it was captured for.
    std::vector<cudaStream_t> rtm_cols;
    cudaStream_t rtm_left = nullptr, rtm_origin = nullptr;
    std::vector<cudaEvent_t> rtm_pf, rtm_col, rtm_sev;
    cudaEvent_t rtm_ev = nullptr, rtm_ev2 = nullptr;
    cudaGraphExec_t rtm_exec = nullptr;
    uint64_t rtm_key[12] = {};
    long long rtm_launches = 0;
    bool trace_on = false;
    std::vector<StepTrace> trace;
    int64_t trace_steps = 0;
    // Replay of the mixed factorization as a CUDA graph: the arguments it was
    // captured for (fkey), the instantiated graph, its kernel count, and the key
    // of the previous eager run (a key is captured on its second use).
    cudaGraphExec_t fgraph_exec = nullptr;
    cudaStream_t gs = nullptr;                    // capture/replay stream (non-blocking)
    cudaEvent_t ev_g0 = nullptr, ev_g1 = nullptr; // user -> gs and gs -> user
    long long fgraph_launches = 0;
    uint64_t fkey[12] = {};
    uint64_t fkey_seen[12] = {};
    std::mutex mu;
};

void lu_count_launches(long long k);
long long lu_launches_so_far();
int lu_profile_active();
int lu_ctx_init(lu_context* c);
int lu_ctx_release(lu_context* c);
// Makes sure the workspace can hold a factorization of order n with panel
// width nb (and solves of order n).  May synchronise the user stream.
int lu_ctx_reserve(lu_context* c, int64_t n, int nb);
int lu_mx_reserve(lu_context* c, size_t bytes);

// --- kernels (launchers return LU_SUCCESS or LU_ERR_CUDA) --------------------
bool lu_pf_leaf_shape(int64_t m, int w, int esize, int max_ctas, int64_t* R_out, int64_t* G_out, size_t* smem_out);

template <typename T>
int lu_launch_pf_leaf(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t m, int w,
                      int32_t* ipiv, int64_t ipiv_add, int max_ctas);

int lu_launch_laswp_plan(cudaStream_t st, const int32_t* ipiv, int64_t k1, int64_t k2,
                         int32_t* plan);

// Apply a plan to columns [c1, c1+n1) and [c2, c2+n2) of A.
template <typename T>
int lu_launch_laswp_apply(cudaStream_t st, T* A, int64_t lda, int64_t c1, int64_t n1,
                          int64_t c2, int64_t n2, const int32_t* plan, int64_t K, int num_sms, int max_blocks = 0);

// RL2 + RL3 of a narrow panel node in one launch (w1, w2 <= 32), bit-identical to
// lu_launch_trsm_lunit followed by lu_launch_gemm_update.  arrivals: one zeroed
// counter (left zeroed).
template <typename T>
int lu_launch_trsm_gemm_narrow(cudaStream_t st, int64_t m2, int64_t w2, int64_t w1, const T* L11, T* A12,
                               const T* A21, T* A22, int64_t lda, unsigned* arrivals);
template <typename T>
int lu_launch_trsm_lunit(cudaStream_t st, int64_t m, int64_t n, const T* L, int64_t ldl, T* B,
                         int64_t ldb, int max_ctas = 0);

template <typename T>
int lu_launch_gemm_update(cudaStream_t st, int64_t m, int64_t n, int64_t k, const T* A,
                          int64_t lda, const T* B, int64_t ldb, T* C, int64_t ldc);
// The same with a symmetric band: tiles whose rows all lie above the band-wide
// diagonal block of their first column (absolute indices: C's first row r0,
// first column c0) are skipped (band 0 = none).
template <typename T>
int lu_launch_gemm_update_band(cudaStream_t st, int64_t m, int64_t n, int64_t k, const T* A, int64_t lda,
                               const T* B, int64_t ldb, T* C, int64_t ldc, int64_t r0, int64_t c0, int band);

template <typename T>
int lu_launch_perm_from_ipiv(cudaStream_t st, int64_t n, const int32_t* ipiv, int32_t* perm);

template <typename T>
int lu_launch_permute_rows(cudaStream_t st, int64_t n, int64_t nrhs, const int32_t* perm,
                           const T* B, int64_t ldb, T* X, int64_t ldx);

// Dinv: NULL, or the inverses of the diagonal blocks from lu_launch_trinv_diag,
// which turn each block's substitution into one dense product.
// xtag (FP32, one rhs, with Dinv): n zero-initialised 64-bit words through which the
// blocks pass their solved values tagged with a per-launch id (one global round trip
// per dependency instead of a counter plus a load).
template <typename T>
int lu_launch_trsv_blocked(lu_context* c, cudaStream_t st, bool lower_unit, int64_t n,
                           int64_t nrhs, const T* LU, int64_t lda, T* X, int64_t ldx, const T* Dinv = nullptr,
                           unsigned long long* xtag = nullptr);
template <typename T>
size_t lu_trinv_bytes(int64_t n);
template <typename T>
int lu_launch_trinv_diag(cudaStream_t st, int64_t n, const T* LU, int64_t lda, T* D);

int lu_launch_finish_info(cudaStream_t st, const LuSync* s, int32_t* info);

template <typename T>
// max_c > 0 caps the cluster size; nt = 512 asks for the 512-thread leaf (FP32
// pushed-message leaf only; otherwise 256), the thread count taken goes to nt_out.
bool lu_pf_cluster_shape(int64_t m, int w, size_t budget, int* C_out, int* R_out, size_t* smem_out,
                         int max_c = 0, int nt = 256, int* nt_out = nullptr);
// sib > 0: the leaf also applies L11^-1 to the top rows of the first sib columns to its
// right (its sibling's U12); kprev > 0: the leaf first applies the preceding sibling's
// rank-kprev update to its own columns.  Both need the pushed-message leaf
// (lu_pf_leaf_pairs_supported).
template <typename T>
int lu_launch_pf_leaf_cluster(cudaStream_t st, T* A, int64_t lda, int64_t m, int w, int C, int R, size_t smem,
                              int64_t left_cols, int64_t right_cols, int32_t* ipiv, int64_t ipiv_add, LuSync* sync,
                              int sib = 0, int kprev = 0, int nt = 256);
bool lu_pf_leaf_pairs_supported();
// Pushed-message cluster leaf (pf_push.cu): w columns of a kernel compiled for wc.
size_t lu_pf_push_smem(int esize, int w, int rq, int nt = 256);
template <typename T>
int lu_launch_pf_leaf_push(cudaStream_t st, T* A, int64_t lda, int64_t m, int w, int wc, int C, int R,
                           int64_t left_cols, int64_t right_cols, int32_t* ipiv, int64_t ipiv_add, LuSync* sync,
                           int sib, int kprev, int nt = 256);

// Recursive panel factorization of columns [j0, j0+width) over rows [j0, M)
// of the matrix at A (absolute indices; ipiv absolute, 1-based).
template <typename T>
int lu_panel_recursive(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t M,
                       int64_t j0, int64_t width, int32_t* ipiv, const lu_opts& o);

// Trailing-update engine for the mixed-precision factorization (mixed.cu):
// packs each panel's L21 and, per update, U12, and runs the tensor-core GEMM.
struct LuTuEngine {
    virtual ~LuTuEngine() {}
    virtual bool uses_tc(int64_t kb) const = 0;
    // pack L21 of panel k (rows [k0+kb, n), columns [k0, k0+kb)) on stream st
    virtual int pack_panel(cudaStream_t st, const float* A, int64_t lda, int64_t k, int64_t k0, int64_t kb) const = 0;
    // C[k0+kb.., c_begin..c_end) -= L21 U12 for panel k; which = 0 (panel path) or 1 (right update)
    virtual int update(cudaStream_t st, float* A, int64_t lda, int64_t k, int64_t k0, int64_t kb, int64_t c_begin,
                       int64_t c_end, int which) const = 0;
    // extra CTAs joining the right update of step k once the panel path is done
    virtual int steal(cudaStream_t st, int64_t k) const = 0;
};

int lu_check_opts(const lu_opts& o);
// Green-context partition (green.cu): set up (or keep) a partition of >= part_sms
// SMs for the leaves and the rest for the right update; release it; the rest's
// stream and SM count; make a partition's context current (enter/leave); fork
// the leaf stream from st (entering the leaf context) and join it back.
int lu_green_setup(lu_context* c, int part_sms);
void lu_green_release(lu_context* c);
cudaStream_t lu_green_rest_stream(lu_context* c);
int lu_green_rest_sms(lu_context* c);
int lu_green_enter(lu_context* c, bool leaf);
void lu_green_leave();
int lu_green_leaf_fork(lu_context* c, cudaStream_t st, cudaStream_t* leaf_st);
int lu_green_leaf_join(lu_context* c, cudaStream_t st);
void* lu_current_ctx();
// Column boundaries of the panels: panel k is [s[k], s[k+1]), from the schedule
// (opts.sched) or the fixed nb; wmin/wmax receive the narrowest and widest width.
void lu_panel_bounds(int64_t n, const lu_opts& o, std::vector<int64_t>* s, int* wmin, int* wmax);
// SMs the right update leaves to the panel path (0 without look-ahead).
int lu_resolve_reserve(const lu_context* c, const lu_opts& o);

// One task of the factorization of step k (panel columns [k0, k0+kb)): TU_k on
// columns [cb, ce) plus panel k's interchanges on the `left` leading columns
// (lu_step_tu), and PF(k) with its interchange plan (lu_step_pf).
template <typename T>
int lu_step_tu(lu_context* c, cudaStream_t st, int64_t n, T* A, int64_t lda, int64_t k, int64_t k0, int64_t kb,
               int64_t cb, int64_t ce, int64_t left, bool pivot);
template <typename T>
int lu_step_pf(lu_context* c, cudaStream_t st, T* A, int64_t lda, int64_t n, int64_t k, int64_t k0, int64_t kb,
               int32_t* ipiv, const lu_opts& o, bool pivot);
// Symmetric elimination (chol.cu): U12 := D1 L21^T for block row k (panel columns
// [k0, k0+kb)) on columns [cb, ce), D1 the diagonal of U11, written over A12.
template <typename T>
int lu_launch_sym_u12(cudaStream_t st, T* A, int64_t lda, int64_t k0, int64_t kb, int64_t cb, int64_t ce);
// Cholesky of FP32 A with an optional tensor-core trailing-update engine (chol.cu).
int lu_chol_factor_f32(lu_context* h, int64_t n, float* A, int64_t lda, const lu_opts& o, int32_t* info,
                       const LuTuEngine* eng);
// The runtime-task (dependency DAG) schedule of the same factorization (rtm.cu).
template <typename T>
int lu_factor_rtm(lu_context* c, int64_t n, T* A, int64_t lda, int32_t* ipiv, const lu_opts& o, int32_t* info,
                  bool pivot);

// pivot = false: elimination without interchanges (the Cholesky path, chol.cu):
// panels by lu_panel_nopiv, no interchange plans or row exchanges, ipiv unused.
template <typename T>
int lu_factor_blocked(lu_context* c, int64_t n, T* A, int64_t lda, int32_t* ipiv, const lu_opts& o, int32_t* info,
                      const LuTuEngine* eng, bool pivot = true);

// Panel of columns [j0, j0+width) over rows [j0, M) eliminated without
// interchanges (absolute indices); the first step whose pivot is not positive is
// recorded (1-based) in sync->info.
template <typename T>
int lu_panel_nopiv(cudaStream_t st, T* A, int64_t lda, int64_t M, int64_t j0, int64_t width, LuSync* sync);

// Operand precisions of the tensor-core trailing update.
static inline bool lu_prec_is_tc(int prec) {
    return prec == LU_TU_BF16 || prec == LU_TU_FP16 || prec == LU_TU_BF16X3 || prec == LU_TU_BF16X6 ||
           prec == LU_TU_FP8;
}
// pack.h format code of a tensor-core precision (LU_PACK_BF16 0, FP16 1, BF16X3 2, BF16X6 3)
static inline int lu_prec_pack_fmt(int prec) {
    return prec == LU_TU_FP16 ? 1 : (prec == LU_TU_BF16X3 ? 2 : (prec == LU_TU_BF16X6 ? 3 : 0));
}
