// Block-size autotuner.  Sec. 3 leaves the algorithmic block size b to the
// implementation (the paper's experiments fix b = 192 for their processor).  On
// the GPU, b trades the length of the panel chain (n / b panel factorizations,
// each on the critical path of the look-ahead schedule of Sec. 4) against the
// width, and so the efficiency, of the trailing updates; the best value depends
// on n and on the update's precision, so it is measured rather than fixed.
//
// The table maps (device name, factorization kind, ceil(log2 n)) to the nb of
// least measured time.  Factorizations called with nb = 0 take the table's
// value for their kind and n, or 256 when there is none.
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
};

std::mutex g_mu;
std::vector<TuneEntry> g_table;

int bucket_of(int64_t n) {
    int b = 0;
    while (b < 62 && (int64_t(1) << b) < n) ++b;
    return b;
}

bool kind_valid(int kind) {
    return kind == LU_TUNE_F64 || kind == LU_TUNE_F32 || kind == LU_TU_F32 ||
           (kind >= 0 && kind <= LU_TU_BF16X6 && kind != LU_FULL_F64);
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

void put_locked(const std::string& dev, int kind, int bucket, int nb, float ms) {
    for (auto& e : g_table)
        if (e.device == dev && e.kind == kind && e.bucket == bucket) {
            e.nb = nb;
            e.ms = ms;
            return;
        }
    g_table.push_back({dev, kind, bucket, nb, ms});
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

int lu_auto_nb(int kind, int64_t n) {
    load_env_table_once();
    const int nb = lu_tune_get(nullptr, kind, n);
    return nb > 0 ? nb : 256;
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
    if (nb < 1 || nb > LU_MAX_NB || (kind == LU_TU_FP8 && nb % 128 != 0)) return -4;
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
        for (const auto& e : g_table)
            ok = ok && std::fprintf(f, "%s\t%d\t%d\t%d\t%.6g\n", e.device.c_str(), e.kind, e.bucket, e.nb,
                                    (double)e.ms) > 0;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LU_SUCCESS : LU_ERR_IO;
}

// Lines "device<TAB>kind<TAB>bucket<TAB>nb<TAB>ms"; all are checked before any
// is merged, so a malformed file changes nothing.
extern "C" int lu_tune_load(const char* path) {
    if (!path) return -1;
    FILE* f = std::fopen(path, "r");
    if (!f) return LU_ERR_IO;
    std::vector<TuneEntry> rows;
    char line[1024];
    bool ok = true;
    while (ok && std::fgets(line, sizeof line, f)) {
        size_t len = std::strlen(line);
        if (len && line[len - 1] == '\n') line[--len] = '\0';
        if (len == 0) continue;
        char* tab = std::strchr(line, '\t');
        if (!tab || tab == line) {
            ok = false;
            break;
        }
        *tab = '\0';
        int kind = 0, bucket = 0, nb = 0, used = 0;
        float ms = 0.f;
        if (std::sscanf(tab + 1, "%d\t%d\t%d\t%f%n", &kind, &bucket, &nb, &ms, &used) != 4 ||
            tab[1 + used] != '\0' || !kind_valid(kind) || bucket < 0 || bucket > 62 || nb < 1 ||
            nb > LU_MAX_NB || (kind == LU_TU_FP8 && nb % 128 != 0)) {
            ok = false;
            break;
        }
        rows.push_back({std::string(line), kind, bucket, nb, ms});
    }
    if (std::ferror(f)) ok = false;
    std::fclose(f);
    if (!ok) return LU_ERR_IO;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& r : rows) put_locked(r.device, r.kind, r.bucket, r.nb, r.ms);
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
