// Built-in launch profiler: when enabled for a kernel class, every launch of that
// class is bracketed by a pair of CUDA events recorded on the launching stream, tagged
// with its kernel class and its algorithmic bytes and flops.  lu_profile_read
// synchronises, turns the event pairs into durations and aggregates them per
// class.  Off by default; costs two event records per launch when on.
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <vector>

#include "internal.h"
#include "profile.h"

namespace {

struct Rec {
    int cls;
    cudaEvent_t a, b;
    double bytes, flops;
    cudaStream_t st;
};

std::mutex g_mu;
unsigned g_mask = 0;
int g_stride = 1;
long long g_seen[LU_K_COUNT] = {};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
struct Agg {
    long long launches = 0;
    double ms = 0, bytes = 0, flops = 0;
};
Agg g_agg[LU_K_COUNT];

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// LU_GB300_TIMELINE=<file>: every drained launch is also appended to <file> as
// "class stream start_ms duration_ms", start relative to the first launch of the
// drained batch (events of different streams share one device clock).
FILE* timeline_file() {
    static FILE* f = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        const char* path = getenv("LU_GB300_TIMELINE");
        if (path && path[0]) f = fopen(path, "a");
    }
    return f;
}

void drain_locked() {
    if (g_recs.empty()) return;
    cudaDeviceSynchronize();
    if (FILE* f = timeline_file()) {
        const cudaEvent_t base = g_recs.front().a;
        fprintf(f, "# batch of %zu launches\n", g_recs.size());
        for (const Rec& r : g_recs) {
            float t0 = 0.f, d = 0.f;
            if (base && r.a && r.b && cudaEventElapsedTime(&t0, base, r.a) == cudaSuccess &&
                cudaEventElapsedTime(&d, r.a, r.b) == cudaSuccess)
                fprintf(f, "%d %p %.4f %.4f\n", r.cls, (void*)r.st, t0, d);
            else
                cudaGetLastError();
        }
        fflush(f);
    }
    for (Rec& r : g_recs) {
        float ms = 0.f;
        if (r.a && r.b && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            Agg& g = g_agg[r.cls];
            g.launches += 1;
            g.ms += ms;
            g.bytes += r.bytes;
            g.flops += r.flops;
        } else {
            cudaGetLastError();
        }
        if (r.a) g_pool.push_back(r.a);
        if (r.b) g_pool.push_back(r.b);
    }
    g_recs.clear();
}

}  // namespace

static int trace_launches() {
    static int t = -1;
    if (t < 0) {
        const char* e = getenv("LU_GB300_TRACE_LAUNCH");
        t = (e && e[0] == '1') ? 1 : 0;
    }
    return t;
}

LuProfScope::LuProfScope(cudaStream_t st, int cls, double bytes, double flops) : st_(st) {
    if (trace_launches()) {
        fprintf(stderr, "[lu launch] class %d bytes %.0f flops %.0f\n", cls, bytes, flops);
        fflush(stderr);
    }
    if (!(g_mask & (1u << cls))) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!(g_mask & (1u << cls))) return;
    if (g_stride > 1 && (g_seen[cls]++ % g_stride) != 0) return;
    a_ = take_event();
    b_ = take_event();
    cls_ = cls;
    bytes_ = bytes;
    flops_ = flops;
    if (a_) cudaEventRecord(a_, st_);
    active_ = true;
}

LuProfScope::~LuProfScope() {
    if (!active_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (b_) cudaEventRecord(b_, st_);
    g_recs.push_back(Rec{cls_, a_, b_, bytes_, flops_, st_});
}

extern "C" int lu_profile_enable(int mask) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_mask = (unsigned)mask & ((1u << LU_K_COUNT) - 1u);
    return LU_SUCCESS;
}

// Nonzero while any kernel class is profiled (graph replay is then bypassed, so
// that every launch carries its events).
int lu_profile_active() { return g_mask != 0 || timeline_file() != nullptr; }

extern "C" int lu_profile_stride(int every) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_stride = every > 1 ? every : 1;
    for (auto& s : g_seen) s = 0;
    return LU_SUCCESS;
}

extern "C" int lu_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    for (auto& g : g_agg) g = Agg();
    for (auto& s : g_seen) s = 0;
    return LU_SUCCESS;
}

extern "C" int lu_profile_read(int kclass, int64_t* launches, double* ms, double* bytes, double* flops) {
    if (kclass < 0 || kclass >= LU_K_COUNT) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    const Agg& g = g_agg[kclass];
    if (launches) *launches = g.launches;
    if (ms) *ms = g.ms;
    if (bytes) *bytes = g.bytes;
    if (flops) *flops = g.flops;
    return LU_SUCCESS;
}
