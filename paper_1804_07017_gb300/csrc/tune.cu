// Block-size autotuner.  Sec. 3 leaves the algorithmic block size b to the
// implementation (the paper's experiments fix b = 192 for their processor).  On
// the GPU, b trades the length of the panel chain (n / b panel factorizations,
// each on the critical path of the look-ahead schedule of Sec. 4) against the
// width, and so the efficiency, of the trailing updates; the best value depends
// on n and on the update's precision, so it is measured rather than fixed.
//
// The table maps (device name, factorization kind, ceil(log2 n)) to the plan of
// least measured time: nb, optionally a per-step block-size schedule (the GPU
// form of the early termination of Sec. 4.2: b adjusted from step to step so
// that PU(k+1) and TU_right(k) stay balanced), the SMs the right update leaves
// to the panel path, and the look-ahead depth.  Factorizations called with
// nb = 0 take the table's plan for their kind and n, or nb = 256 when there is
// none.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace {

struct TuneEntry {
    std::string device;
    int kind;
    int bucket;
    int nb;
    float ms;
    int reserve = 0;               // 0: not tuned (automatic)
    int depth = 0;                 // 0: not tuned (the caller's)
    std::vector<int32_t> sched;    // empty: the fixed nb
    int pf_sms = 0;                // SM partition for the panel leaves (0: none)
};

std::mutex g_mu;
std::vector<TuneEntry> g_table;

int bucket_of(int64_t n) {
    int b = 0;
    while (b < 62 && (int64_t(1) << b) < n) ++b;
    return b;
}

bool kind_valid(int kind) {
    return kind == LU_TUNE_F64 || kind == LU_TUNE_F32 || kind == LU_TU_F32 || kind == LU_TUNE_BATCHED_F64 ||
           kind == LU_TUNE_BATCHED_F32 || (kind >= 0 && kind <= LU_TU_BF16X6 && kind != LU_FULL_F64);
}

// Name of the current device (cached per device index).
bool current_device_name(std::string* out) {
    static std::mutex mu;
    static std::vector<std::string> names;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(mu);
    if ((int)names.size() <= dev) names.resize(dev + 1);
    if (names[dev].empty()) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        names[dev] = prop.name;
    }
    *out = names[dev];
    return true;
}

bool resolve_device(const char* device, std::string* out) {
    if (device) {
        *out = device;
        return !out->empty() && out->find('\t') == std::string::npos && out->find('\n') == std::string::npos;
    }
    return current_device_name(out);
}

void put_locked(const TuneEntry& n) {
    for (auto& e : g_table)
        if (e.device == n.device && e.kind == n.kind && e.bucket == n.bucket) {
            e = n;
            return;
        }
    g_table.push_back(n);
}

void put_locked(const std::string& dev, int kind, int bucket, int nb, float ms) {
    TuneEntry e;
    e.device = dev;
    e.kind = kind;
    e.bucket = bucket;
    e.nb = nb;
    e.ms = ms;
    put_locked(e);
}

bool width_ok(int kind, int w) {
    if (kind == LU_TUNE_BATCHED_F64 || kind == LU_TUNE_BATCHED_F32) return w >= 1 && w <= 513;  // a tile cut-over
    return w >= 1 && w <= LU_MAX_NB && !(kind == LU_TU_FP8 && w % 128 != 0);
}

// A seeded n x n matrix with entries iid U[-1, 1): splitmix64 (Steele, Lea and
// Flood, 2014) of the element index, top 53 bits as a fraction.
template <typename T>
__global__ void tune_fill_kernel(T* __restrict__ A, int64_t n, uint64_t seed) {
    const int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        A[e] = (T)(2.0 * u - 1.0);
    }
}

void load_env_table_once() {
    static std::once_flag once;
    std::call_once(once, [] {
        const char* p = std::getenv("LU_GB300_TUNE_FILE");
        if (p && *p) lu_tune_load(p);  // a missing or malformed file leaves the table empty
    });
}

}  // namespace

int lu_tuned_value(int kind, int64_t n) {
    load_env_table_once();
    return lu_tune_get(nullptr, kind, n);
}

int lu_auto_nb(int kind, int64_t n) {
    load_env_table_once();
    const int nb = lu_tune_get(nullptr, kind, n);
    return nb > 0 ? nb : 256;
}

void lu_auto_opts(int kind, int64_t n, lu_opts* o) {
    thread_local std::vector<int32_t> tl_sched;
    load_env_table_once();
    o->nb = 256;
    std::string dev;
    if (n < 1 || !current_device_name(&dev)) return;
    const int b = bucket_of(n);
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& e : g_table)
        if (e.device == dev && e.kind == kind && e.bucket == b) {
            o->nb = e.nb;
            if (!e.sched.empty()) {
                tl_sched = e.sched;
                o->sched = tl_sched.data();
                o->nsched = (int)tl_sched.size();
            }
            if (o->tu_reserve == 0 && e.reserve > 0) o->tu_reserve = e.reserve;
            if (o->lookahead >= 1 && e.depth >= 1) o->lookahead = e.depth;
            if (o->lookahead >= 1 && o->pf_sms == 0 && e.pf_sms > 0) o->pf_sms = e.pf_sms;
            return;
        }
}

extern "C" int lu_tune_plan_set(const char* device, int kind, int64_t n, int nb, int reserve, int depth,
                                const int32_t* sched, int nsched, int pf_sms, float ms) {
    std::string dev;
    if (!resolve_device(device, &dev)) return -1;
    if (!kind_valid(kind)) return -2;
    if (n < 1) return -3;
    if (!width_ok(kind, nb)) return -4;
    if (reserve < 0) return -5;
    if (depth < 0 || depth > 2) return -6;
    if (nsched < 0 || nsched > (1 << 20) || (nsched > 0 && !sched)) return -8;
    for (int i = 0; i < nsched; ++i)
        if (!width_ok(kind, sched[i])) return -7;
    if (pf_sms < 0 || pf_sms > 4096) return -9;
    TuneEntry e;
    e.device = dev;
    e.kind = kind;
    e.bucket = bucket_of(n);
    e.nb = nb;
    e.ms = ms;
    e.reserve = reserve;
    e.depth = depth;
    e.sched.assign(sched, sched + nsched);
    e.pf_sms = pf_sms;
    std::lock_guard<std::mutex> lk(g_mu);
    put_locked(e);
    return LU_SUCCESS;
}

extern "C" int lu_tune_plan_get(const char* device, int kind, int64_t n, int* nb, int* reserve, int* depth,
                                int32_t* sched, int cap, int* nsched, int* pf_sms) {
    if (n < 1) return 0;
    std::string dev;
    if (!resolve_device(device, &dev)) return 0;
    const int b = bucket_of(n);
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& e : g_table)
        if (e.device == dev && e.kind == kind && e.bucket == b) {
            if (nb) *nb = e.nb;
            if (reserve) *reserve = e.reserve;
            if (depth) *depth = e.depth;
            if (nsched) *nsched = (int)e.sched.size();
            if (pf_sms) *pf_sms = e.pf_sms;
            if (sched)
                for (int i = 0; i < cap && i < (int)e.sched.size(); ++i) sched[i] = e.sched[i];
            return 1;
        }
    return 0;
}

extern "C" int lu_tune_get(const char* device, int kind, int64_t n) {
    if (n < 1) return 0;
    std::string dev;
    if (!resolve_device(device, &dev)) return 0;
    const int b = bucket_of(n);
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& e : g_table)
        if (e.device == dev && e.kind == kind && e.bucket == b) return e.nb;
    return 0;
}

extern "C" int lu_tune_set(const char* device, int kind, int64_t n, int nb, float ms) {
    std::string dev;
    if (!resolve_device(device, &dev)) return -1;
    if (!kind_valid(kind)) return -2;
    if (n < 1) return -3;
    if (!width_ok(kind, nb)) return -4;
    std::lock_guard<std::mutex> lk(g_mu);
    put_locked(dev, kind, bucket_of(n), nb, ms);
    return LU_SUCCESS;
}

extern "C" int lu_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.clear();
    return LU_SUCCESS;
}

extern "C" int lu_tune_save(const char* path) {
    if (!path) return -1;
    FILE* f = std::fopen(path, "w");
    if (!f) return LU_ERR_IO;
    bool ok = true;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (const auto& e : g_table) {
            ok = ok && std::fprintf(f, "%s\t%d\t%d\t%d\t%.6g", e.device.c_str(), e.kind, e.bucket, e.nb,
                                    (double)e.ms) > 0;
            if (e.reserve > 0 || e.depth > 0 || !e.sched.empty() || e.pf_sms > 0) {
                ok = ok && std::fprintf(f, "\t%d\t%d\t", e.reserve, e.depth) > 0;
                if (e.sched.empty()) ok = ok && std::fputc('-', f) != EOF;
                for (size_t i = 0; i < e.sched.size(); ++i)
                    ok = ok && std::fprintf(f, i ? ",%d" : "%d", (int)e.sched[i]) > 0;
                if (e.pf_sms > 0) ok = ok && std::fprintf(f, "\t%d", e.pf_sms) > 0;
            }
            ok = ok && std::fputc('\n', f) != EOF;
        }
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LU_SUCCESS : LU_ERR_IO;
}

// Lines "device<TAB>kind<TAB>bucket<TAB>nb<TAB>ms", optionally followed by
// "<TAB>reserve<TAB>depth<TAB>schedule" (the schedule a comma-separated list of
// block sizes, or "-" for none); all are checked before any is merged, so a
// malformed file changes nothing.
static bool parse_line(const std::string& line, TuneEntry* out) {
    const size_t tab = line.find('\t');
    if (tab == std::string::npos || tab == 0) return false;
    TuneEntry e;
    e.device = line.substr(0, tab);
    const char* p = line.c_str() + tab + 1;
    int used = 0;
    if (std::sscanf(p, "%d\t%d\t%d\t%f%n", &e.kind, &e.bucket, &e.nb, &e.ms, &used) != 4) return false;
    p += used;
    if (!kind_valid(e.kind) || e.bucket < 0 || e.bucket > 62 || !width_ok(e.kind, e.nb)) return false;
    if (*p == '\t') {
        if (std::sscanf(p, "\t%d\t%d\t%n", &e.reserve, &e.depth, &used) != 2) return false;
        p += used;
        if (e.reserve < 0 || e.depth < 0 || e.depth > 2) return false;
        if (*p == '-') {
            ++p;
        } else {
            while (true) {
                char* end = nullptr;
                const long w = std::strtol(p, &end, 10);
                if (end == p || !width_ok(e.kind, (int)w) || e.sched.size() >= (1u << 20)) return false;
                e.sched.push_back((int32_t)w);
                p = end;
                if (*p != ',') break;
                ++p;
            }
        }
        if (*p == '\t') {
            if (std::sscanf(p, "\t%d%n", &e.pf_sms, &used) != 1 || e.pf_sms < 0 || e.pf_sms > 4096) return false;
            p += used;
        }
    }
    if (*p != '\0') return false;
    *out = e;
    return true;
}

extern "C" int lu_tune_load(const char* path) {
    if (!path) return -1;
    FILE* f = std::fopen(path, "r");
    if (!f) return LU_ERR_IO;
    std::vector<TuneEntry> rows;
    std::string line;
    char buf[1024];
    bool ok = true, eof = false;
    while (ok && !eof) {
        line.clear();
        while (true) {
            if (!std::fgets(buf, sizeof buf, f)) {
                eof = true;
                break;
            }
            line += buf;
            if (!line.empty() && line.back() == '\n') break;
        }
        if (!line.empty() && line.back() == '\n') line.pop_back();
        if (line.empty()) continue;
        TuneEntry e;
        if (!parse_line(line, &e)) ok = false;
        else rows.push_back(e);
    }
    if (std::ferror(f)) ok = false;
    std::fclose(f);
    if (!ok) return LU_ERR_IO;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& r : rows) put_locked(r);
    return LU_SUCCESS;
}

extern "C" int lu_tune_nb(lu_handle h, int kind, int64_t n, const int* candidates, int count, int reps,
                          const lu_opts* opts, int* best_nb, float* ms) {
    if (!h) return LU_ERR_HANDLE;
    if (!kind_valid(kind)) return -2;
    if (n < 1 || n > INT32_MAX / 2) return -3;
    if (!candidates) return -4;
    if (count < 1) return -5;
    if (reps < 1) return -6;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    o.nb = 256;
    if (lu_check_opts(o) != 0) return -7;
    if (!best_nb) return -8;
    std::string dev;
    if (!current_device_name(&dev)) return LU_ERR_CUDA;
    const bool f64 = kind == LU_TUNE_F64;
    const size_t bytes = (f64 ? sizeof(double) : sizeof(float)) * (size_t)n * (size_t)n;
    void* A = nullptr;
    int32_t* ipiv = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&A, bytes) != cudaSuccess || cudaMalloc(&ipiv, sizeof(int32_t) * ((size_t)n + 4)) != cudaSuccess) {
        cudaGetLastError();
        if (A) cudaFree(A);
        return LU_ERR_NOMEM;
    }
    int32_t* info = ipiv + n;
    int rc = LU_SUCCESS;
    int best = 0;
    float best_ms = INFINITY;
    cudaStream_t st;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        st = h->user;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        rc = LU_ERR_CUDA;
    }
    for (int i = 0; i < count && rc == LU_SUCCESS; ++i) {
        const int nb = candidates[i];
        bool ok = nb >= 1 && nb <= LU_MAX_NB && !(kind == LU_TU_FP8 && nb % 128 != 0);
        float t = -1.f;
        o.nb = nb;
        for (int r = 0; r < reps && ok; ++r) {
            if (f64) tune_fill_kernel<double><<<4 * h->num_sms, 256, 0, st>>>((double*)A, n, 0x5eedull);
            else tune_fill_kernel<float><<<4 * h->num_sms, 256, 0, st>>>((float*)A, n, 0x5eedull);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess) {
                rc = LU_ERR_CUDA;
                break;
            }
            int r2;
            if (f64) r2 = lu_factor_ex(h, LU_F64, n, A, n, ipiv, &o, info);
            else if (kind == LU_TUNE_F32) r2 = lu_factor_ex(h, LU_F32, n, A, n, ipiv, &o, info);
            else r2 = lu_factor_mixed_ex(h, (lu_prec)kind, n, (float*)A, n, ipiv, &o, info);
            if (r2 == LU_ERR_UNSUPPORTED || r2 == LU_ERR_NOMEM || (r2 < 0 && r2 > -100)) {
                ok = false;  // this candidate is rejected; the others still run
                break;
            }
            if (r2 != LU_SUCCESS) {
                rc = r2;
                break;
            }
            int32_t hinfo = -1;
            float el = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaMemcpy(&hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaEventElapsedTime(&el, e0, e1) != cudaSuccess) {
                rc = LU_ERR_CUDA;
                break;
            }
            if (hinfo != 0) {
                ok = false;  // a runtime error inside the factorization, or a zero pivot
                break;
            }
            if (t < 0.f || el < t) t = el;
        }
        if (rc != LU_SUCCESS) break;
        if (ms) ms[i] = ok ? t : -1.f;
        if (ok && t >= 0.f && t < best_ms) {
            best_ms = t;
            best = nb;
        }
    }
    if (rc == LU_ERR_CUDA) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(A);
    cudaFree(ipiv);
    if (rc != LU_SUCCESS) return rc;
    if (best == 0) return LU_ERR_UNSUPPORTED;
    *best_nb = best;
    std::lock_guard<std::mutex> lk(g_mu);
    put_locked(dev, kind, bucket_of(n), best, best_ms);
    return LU_SUCCESS;
}

// ---------------------------------------------------------------------------
// Plan tuning: block size, the right update's SM reserve, look-ahead depth and
// a per-step schedule.
// ---------------------------------------------------------------------------
namespace {

struct TuneRun {
    lu_handle h;
    int kind;
    int64_t n;
    void* A;
    int32_t* ipiv;
    int32_t* info;
    cudaStream_t st;
    cudaEvent_t e0, e1;
};

// One factorization of a freshly filled matrix; *ms its event-timed duration.
// Returns LU_SUCCESS, a hard error, or 1 when these options are rejected.
int run_once(const TuneRun& r, const lu_opts& o, float* ms) {
    if (r.kind == LU_TUNE_F64) tune_fill_kernel<double><<<4 * r.h->num_sms, 256, 0, r.st>>>((double*)r.A, r.n, 0x5eedull);
    else tune_fill_kernel<float><<<4 * r.h->num_sms, 256, 0, r.st>>>((float*)r.A, r.n, 0x5eedull);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(r.e0, r.st) != cudaSuccess) return LU_ERR_CUDA;
    int r2;
    if (r.kind == LU_TUNE_F64) r2 = lu_factor_ex(r.h, LU_F64, r.n, r.A, r.n, r.ipiv, &o, r.info);
    else if (r.kind == LU_TUNE_F32) r2 = lu_factor_ex(r.h, LU_F32, r.n, r.A, r.n, r.ipiv, &o, r.info);
    else r2 = lu_factor_mixed_ex(r.h, (lu_prec)r.kind, r.n, (float*)r.A, r.n, r.ipiv, &o, r.info);
    if (r2 == LU_ERR_UNSUPPORTED || r2 == LU_ERR_NOMEM || (r2 < 0 && r2 > -100)) return 1;
    if (r2 != LU_SUCCESS) return r2;
    int32_t hinfo = -1;
    if (cudaEventRecord(r.e1, r.st) != cudaSuccess || cudaEventSynchronize(r.e1) != cudaSuccess ||
        cudaMemcpy(&hinfo, r.info, sizeof hinfo, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaEventElapsedTime(ms, r.e0, r.e1) != cudaSuccess)
        return LU_ERR_CUDA;
    return hinfo == 0 ? LU_SUCCESS : 1;
}

// Least time over reps runs (a repeated mixed factorization is replayed as a
// graph from its third run on, so reps >= 3 times the replay); < 0 if rejected.
int time_opts(const TuneRun& r, const lu_opts& o, int reps, float* best) {
    *best = -1.f;
    for (int i = 0; i < reps; ++i) {
        float t = 0.f;
        const int rc = run_once(r, o, &t);
        if (rc == 1) {
            *best = -1.f;
            return LU_SUCCESS;
        }
        if (rc != LU_SUCCESS) return rc;
        if (*best < 0.f || t < *best) *best = t;
    }
    return LU_SUCCESS;
}

}  // namespace

extern "C" int lu_tune_plan(lu_handle h, int kind, int64_t n, int reps, const lu_opts* opts, lu_opts* best,
                            int32_t* sched, int cap, float* best_ms, float* fixed_ms) {
    if (!h) return LU_ERR_HANDLE;
    if (!kind_valid(kind)) return -2;
    if (n < 1 || n > INT32_MAX / 2) return -3;
    if (reps < 1) return -4;
    lu_opts o;
    lu_default_opts(&o);
    if (opts) o = *opts;
    o.nb = 256;
    o.nsched = 0;
    o.sched = nullptr;
    o.tu_reserve = 0;
    o.pf_sms = 0;
    if (lu_check_opts(o) != 0) return -5;
    if (!best) return -6;
    if (cap < 0 || (cap > 0 && !sched)) return -8;
    std::string dev;
    if (!current_device_name(&dev)) return LU_ERR_CUDA;
    const bool f64 = kind == LU_TUNE_F64;
    const size_t bytes = (f64 ? sizeof(double) : sizeof(float)) * (size_t)n * (size_t)n;
    TuneRun r{h, kind, n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (cudaMalloc(&r.A, bytes) != cudaSuccess ||
        cudaMalloc(&r.ipiv, sizeof(int32_t) * ((size_t)n + 4)) != cudaSuccess) {
        cudaGetLastError();
        if (r.A) cudaFree(r.A);
        return LU_ERR_NOMEM;
    }
    r.info = r.ipiv + n;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        r.st = h->user;
    }
    int rc = LU_SUCCESS;
    if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) rc = LU_ERR_CUDA;
    const bool tc = kind != LU_TUNE_F64 && kind != LU_TUNE_F32 && kind != LU_TU_F32;
    const int step = kind == LU_TU_FP8 ? 128 : 64;
    std::vector<int32_t> plan;  // the chosen schedule (empty: fixed nb)
    float t_fixed = -1.f, t_best = -1.f;
    lu_opts b = o;
    // 1. block size
    if (rc == LU_SUCCESS) {
        const int cands[] = {128, 192, 256, 320, 384, 512};
        for (int nb : cands) {
            if (tc && nb % step) continue;
            lu_opts t = o;
            t.nb = nb;
            float ms = -1.f;
            if ((rc = time_opts(r, t, reps, &ms)) != LU_SUCCESS) break;
            if (ms >= 0.f && (t_best < 0.f || ms < t_best)) {
                t_best = ms;
                b = t;
            }
        }
    }
    // 2. SMs the right update leaves to the panel path, and 3. look-ahead depth
    if (rc == LU_SUCCESS && t_best >= 0.f && o.lookahead) {
        const int sms = h->num_sms;
        const int res[] = {std::max(4, sms / 12), std::max(4, sms / 6), std::max(4, sms / 4), std::max(4, sms / 3)};
        for (int rv : res) {
            lu_opts t = b;
            t.tu_reserve = rv;
            float ms = -1.f;
            if ((rc = time_opts(r, t, reps, &ms)) != LU_SUCCESS) break;
            if (ms >= 0.f && ms < t_best) {
                t_best = ms;
                b = t;
            }
        }
        for (int d = 1; d <= 2 && rc == LU_SUCCESS; ++d) {
            if (d == b.lookahead) continue;
            lu_opts t = b;
            t.lookahead = d;
            float ms = -1.f;
            if ((rc = time_opts(r, t, reps, &ms)) != LU_SUCCESS) break;
            if (ms >= 0.f && ms < t_best) {
                t_best = ms;
                b = t;
            }
        }
    }
    // 3b. with look-ahead, an SM partition for the panel leaves
    if (rc == LU_SUCCESS && t_best >= 0.f && o.lookahead) {
        const int parts[] = {16, 24, 32};
        for (int pv : parts) {
            lu_opts t = b;
            t.pf_sms = pv;
            float ms = -1.f;
            if ((rc = time_opts(r, t, reps, &ms)) != LU_SUCCESS) break;
            if (ms >= 0.f && ms < t_best) {
                t_best = ms;
                b = t;
            }
        }
    }
    t_fixed = t_best;
    // 4. per-step schedule: trace the steps of the factorization at b/2, b and 2b
    // (per step the span from PU(k+1)'s start to the later of PU(k+1) and
    // TU_right(k), i.e. the critical path the step adds), then walk the columns
    // choosing at each position the width whose measured step there costs the
    // least time per eliminated column.
    if (rc == LU_SUCCESS && t_best >= 0.f) {
        struct Curve {
            int w;
            std::vector<int64_t> k0;
            std::vector<float> per_col;
        };
        std::vector<Curve> curves;
        const int ws[3] = {std::max(step, (b.nb / 2) / step * step), b.nb, std::min(LU_MAX_NB, 2 * b.nb)};
        for (int w : ws) {
            if (!curves.empty() && curves.back().w == w) continue;
            lu_opts t = b;
            t.nb = w;
            {
                std::lock_guard<std::mutex> lk(h->mu);
                h->trace_on = true;
            }
            float ms = 0.f;
            int r1 = run_once(r, t, &ms);
            {
                std::lock_guard<std::mutex> lk(h->mu);
                h->trace_on = false;
            }
            if (r1 == 1) continue;
            if ((rc = r1) != LU_SUCCESS) break;
            const int64_t cnt = lu_step_trace_read(h, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
            if (cnt <= 0) continue;
            std::vector<int64_t> k0((size_t)cnt);
            std::vector<int32_t> kb((size_t)cnt);
            std::vector<float> span((size_t)cnt);
            if (lu_step_trace_read(h, (int)cnt, k0.data(), kb.data(), span.data(), nullptr, nullptr) != cnt) continue;
            Curve cv;
            cv.w = w;
            for (int64_t i = 0; i < cnt; ++i) {
                cv.k0.push_back(k0[(size_t)i]);
                cv.per_col.push_back(span[(size_t)i] / (float)std::max<int32_t>(1, kb[(size_t)i]));
            }
            curves.push_back(cv);
        }
        if (rc == LU_SUCCESS && curves.size() > 1) {
            auto cost_at = [&](const Curve& cv, int64_t c) {
                size_t i = 0;
                while (i + 1 < cv.k0.size() && cv.k0[i + 1] <= c) ++i;
                return cv.per_col[i];
            };
            std::vector<int32_t> sch;
            for (int64_t c = 0; c < n;) {
                int wbest = b.nb;
                float cbest = INFINITY;
                for (const auto& cv : curves) {
                    const float v = cost_at(cv, c);
                    if (v < cbest) {
                        cbest = v;
                        wbest = cv.w;
                    }
                }
                sch.push_back(wbest);
                c += wbest;
            }
            // drop the trailing repeats of the last width (the last entry repeats)
            while (sch.size() > 1 && sch[sch.size() - 1] == sch[sch.size() - 2]) sch.pop_back();
            bool uniform = true;
            for (int32_t w : sch) uniform = uniform && w == b.nb;
            if (!uniform) {
                lu_opts t = b;
                t.sched = sch.data();
                t.nsched = (int)sch.size();
                float ms = -1.f;
                rc = time_opts(r, t, reps, &ms);
                if (rc == LU_SUCCESS && ms >= 0.f && ms < t_best) {
                    t_best = ms;
                    plan = sch;
                }
            }
        }
    }
    if (rc == LU_ERR_CUDA) cudaGetLastError();
    if (r.e0) cudaEventDestroy(r.e0);
    if (r.e1) cudaEventDestroy(r.e1);
    cudaFree(r.A);
    cudaFree(r.ipiv);
    if (rc != LU_SUCCESS) return rc;
    if (t_best < 0.f) return LU_ERR_UNSUPPORTED;
    if ((int)plan.size() > cap) plan.clear();  // the caller has no room: keep the fixed plan
    if (plan.empty()) t_best = t_fixed;
    *best = b;
    best->nsched = (int)plan.size();
    best->sched = plan.empty() ? nullptr : sched;
    for (size_t i = 0; i < plan.size(); ++i) sched[i] = plan[i];
    if (best_ms) *best_ms = t_best;
    if (fixed_ms) *fixed_ms = t_fixed;
    TuneEntry e;
    e.device = dev;
    e.kind = kind;
    e.bucket = bucket_of(n);
    e.nb = b.nb;
    e.ms = t_best;
    e.reserve = o.lookahead ? b.tu_reserve : 0;
    e.depth = o.lookahead ? b.lookahead : 0;
    e.sched = plan;
    e.pf_sms = o.lookahead ? b.pf_sms : 0;
    std::lock_guard<std::mutex> lk(g_mu);
    put_locked(e);
    return LU_SUCCESS;
}
