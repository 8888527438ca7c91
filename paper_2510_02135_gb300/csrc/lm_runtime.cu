// Runtime services around the C ABI (no paper counterpart):
//   * per-call metrics as JSON lines (LM_METRICS_JSONL=<path>);
//   * the persistent autotuner cache (LM_AUTOTUNE_CACHE=<path>) and the
//     automatic-tuning switch (LM_AUTOTUNE=1);
//   * the registry of the device bounds-check words of a build with
//     LM_DEBUG_BOUNDS, read by lm_debug_check.
// NVTX ranges around the ABI calls: TraceRange in lm_runtime.cuh.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lm.h"
#include "lm_internal.cuh"
#include "lm_runtime.cuh"

namespace lmk {
namespace {

std::mutex g_rt_mu;

const char* env(const char* name) {
    const char* v = std::getenv(name);
    return (v != nullptr && v[0] != '\0') ? v : nullptr;
}

// Value of "key": in a one-line JSON object written by this file (numbers and
// plain strings only).
bool json_field(const std::string& line, const char* key, std::string* out) {
    const std::string k = std::string("\"") + key + "\":";
    size_t p = line.find(k);
    if (p == std::string::npos) return false;
    p += k.size();
    while (p < line.size() && line[p] == ' ') ++p;
    if (p < line.size() && line[p] == '"') {
        const size_t e = line.find('"', p + 1);
        if (e == std::string::npos) return false;
        *out = line.substr(p + 1, e - p - 1);
        return true;
    }
    size_t e = p;
    while (e < line.size() && line[e] != ',' && line[e] != '}') ++e;
    *out = line.substr(p, e - p);
    return !out->empty();
}

bool json_int(const std::string& line, const char* key, long long* v) {
    std::string s;
    if (!json_field(line, key, &s)) return false;
    char* end = nullptr;
    *v = std::strtoll(s.c_str(), &end, 10);
    return end != s.c_str();
}

// JSON string escaping for the few characters a GPU name or a message can hold.
std::string json_str(const char* s) {
    std::string o = "\"";
    for (const char* c = s; *c; ++c) {
        if (*c == '"' || *c == '\\') o += '\\';
        if ((unsigned char)*c >= 0x20) o += *c;
    }
    return o + "\"";
}

struct CacheEntry {
    TuneCacheKey key;
    long long n;
    lm_pair_config cfg, adj;
    bool has_adj;
};

bool g_cache_loaded = false;
std::vector<CacheEntry> g_cache;

void load_cache_locked() {
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    const char* path = env("LM_AUTOTUNE_CACHE");
    if (path == nullptr) return;
    FILE* f = std::fopen(path, "r");
    if (f == nullptr) return;
    char buf[1024];
    while (std::fgets(buf, sizeof(buf), f) != nullptr) {
        const std::string line(buf);
        CacheEntry e{};
        std::string gpu;
        long long sms, prec, ang, geom, b, n, t, il, sp, pk;
        if (!json_field(line, "gpu", &gpu) || !json_int(line, "sms", &sms) || !json_int(line, "precision", &prec) ||
            !json_int(line, "angular", &ang) || !json_int(line, "geometry", &geom) ||
            !json_int(line, "log2n", &b) || !json_int(line, "n", &n) || !json_int(line, "threads", &t) ||
            !json_int(line, "ilp", &il) || !json_int(line, "splits", &sp) || !json_int(line, "packed", &pk))
            continue;   // not an entry of this format
        std::snprintf(e.key.gpu, sizeof(e.key.gpu), "%.127s", gpu.c_str());
        e.key.sms = (int)sms;
        e.key.precision = (int)prec;
        e.key.angular = (int)ang;
        e.key.geometry = (int)geom;
        e.key.log2n = (int)b;
        e.n = n;
        e.cfg = lm_pair_config{(int)t, (int)il, (int)sp, (int)pk};
        long long at, ail, asp, apk;
        e.has_adj = json_int(line, "adj_threads", &at) && json_int(line, "adj_ilp", &ail) &&
                    json_int(line, "adj_splits", &asp) && json_int(line, "adj_packed", &apk);
        if (e.has_adj) e.adj = lm_pair_config{(int)at, (int)ail, (int)asp, (int)apk};
        g_cache.push_back(e);   // a later line for the same key wins
    }
    std::fclose(f);
}

bool same_key(const TuneCacheKey& a, const TuneCacheKey& b) {
    return std::strcmp(a.gpu, b.gpu) == 0 && a.sms == b.sms && a.precision == b.precision &&
           a.angular == b.angular && a.geometry == b.geometry && a.log2n == b.log2n;
}

// Bounds-check word readers registered by the translation units of a
// bounds-checked build.
struct BoundsReader {
    BoundsReadFn fn;
    const char* unit;
};

std::vector<BoundsReader>& bounds_readers() {
    static std::vector<BoundsReader> r;
    return r;
}

}  // namespace

bool metrics_enabled() { return env("LM_METRICS_JSONL") != nullptr; }

void metrics_write(const std::string& fields) {
    const char* path = env("LM_METRICS_JSONL");
    if (path == nullptr) return;
    std::lock_guard<std::mutex> lk(g_rt_mu);
    FILE* f = std::fopen(path, "a");
    if (f == nullptr) return;
    std::fprintf(f, "{%s}\n", fields.c_str());
    std::fclose(f);
}

std::string metrics_device_fields(int device) {
    cudaDeviceProp p;
    int clock_khz = 0;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return "\"device\":-1";
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, device);
    char buf[256];
    std::snprintf(buf, sizeof(buf), "\"device\":%d,\"gpu\":%s,\"sms\":%d,\"fp32_peak_tflops\":%.3f", device,
                  json_str(p.name).c_str(), p.multiProcessorCount,
                  (double)p.multiProcessorCount * 128.0 * 2.0 * (double)clock_khz * 1e3 / 1e12);
    return buf;
}

bool tune_cache_key(int device, int precision, int angular, int geometry, int log2n, TuneCacheKey* key) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return false;
    std::snprintf(key->gpu, sizeof(key->gpu), "%.127s", p.name);
    key->sms = p.multiProcessorCount;
    key->precision = precision;
    key->angular = angular;
    key->geometry = geometry;
    key->log2n = log2n;
    return true;
}

bool tune_cache_lookup(const TuneCacheKey& key, long long* n, lm_pair_config* cfg, lm_pair_config* adj,
                       bool* has_adj) {
    std::lock_guard<std::mutex> lk(g_rt_mu);
    load_cache_locked();
    for (size_t i = g_cache.size(); i-- > 0;) {
        if (!same_key(g_cache[i].key, key)) continue;
        *n = g_cache[i].n;
        *cfg = g_cache[i].cfg;
        *has_adj = g_cache[i].has_adj;
        if (g_cache[i].has_adj) *adj = g_cache[i].adj;
        return true;
    }
    return false;
}

void tune_cache_store(const TuneCacheKey& key, long long n, const lm_pair_config& cfg, const lm_pair_config* adj) {
    std::lock_guard<std::mutex> lk(g_rt_mu);
    load_cache_locked();
    CacheEntry e{};
    e.key = key;
    e.n = n;
    e.cfg = cfg;
    e.has_adj = adj != nullptr;
    if (adj) e.adj = *adj;
    g_cache.push_back(e);
    const char* path = env("LM_AUTOTUNE_CACHE");
    if (path == nullptr) return;
    FILE* f = std::fopen(path, "a");
    if (f == nullptr) return;
    std::fprintf(f,
                 "{\"gpu\":%s,\"sms\":%d,\"precision\":%d,\"angular\":%d,\"geometry\":%d,\"log2n\":%d,\"n\":%lld,"
                 "\"threads\":%d,\"ilp\":%d,\"splits\":%d,\"packed\":%d",
                 json_str(key.gpu).c_str(), key.sms, key.precision, key.angular, key.geometry, key.log2n, n,
                 cfg.threads, cfg.ilp, cfg.splits, cfg.packed);
    if (adj)
        std::fprintf(f, ",\"adj_threads\":%d,\"adj_ilp\":%d,\"adj_splits\":%d,\"adj_packed\":%d", adj->threads,
                     adj->ilp, adj->splits, adj->packed);
    std::fprintf(f, "}\n");
    std::fclose(f);
}

int autotune_on_first_use() {
    const char* v = env("LM_AUTOTUNE");
    return (v != nullptr && std::strcmp(v, "1") == 0) ? 1 : 0;
}

void register_bounds_reader(BoundsReadFn fn, const char* unit) {
    std::lock_guard<std::mutex> lk(g_rt_mu);
    bounds_readers().push_back(BoundsReader{fn, unit});
}

}  // namespace lmk

extern "C" int lm_debug_bounds(void) {
#ifdef LM_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

extern "C" lm_status lm_debug_check(void) {
    lmk::set_last_error("");
    std::vector<lmk::BoundsReader> readers;
    {
        std::lock_guard<std::mutex> lk(lmk::g_rt_mu);
        readers = lmk::bounds_readers();
    }
    if (readers.empty()) return LM_OK;   // not a bounds-checked build
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        lmk::set_last_error(cudaGetErrorString(e));
        return LM_ERR_CUDA;
    }
    lm_status st = LM_OK;
    for (const lmk::BoundsReader& r : readers) {
        unsigned long long w = 0;
        e = r.fn(&w);
        if (e != cudaSuccess) {
            lmk::set_last_error(cudaGetErrorString(e));
            return LM_ERR_CUDA;
        }
        if (w != 0 && st == LM_OK) {
            char buf[256];
            std::snprintf(buf, sizeof(buf), "bounds check %llu failed in %s at index %llu (the access was skipped)",
                          w >> 48, r.unit, w & 0xffffffffffffull);
            lmk::set_last_error(buf);
            st = LM_ERR_CUDA;
        }
    }
    return st;
}
