// Runtime services around the C ABI (lm_runtime.cu): NVTX ranges, per-call
// metrics, the persistent autotuner cache.  No paper counterpart.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>

#include "../../include/lm.h"

namespace lmk {

// An NVTX range for the duration of an ABI call (free unless a profiler or a
// tracing tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Per-call metrics: with LM_METRICS_JSONL=<path> set, the heavy calls
// synchronise their stream at the end and append one JSON object per call
// to <path> (fields given without braces).
bool metrics_enabled();
void metrics_write(const std::string& fields);
std::string metrics_device_fields(int device);

// Persistent autotuner cache (LM_AUTOTUNE_CACHE=<path>, JSON lines keyed by
// GPU name, SM count, precision, angular flag, geometry and floor(log2 N)).
struct TuneCacheKey {
    char gpu[128];
    int sms, precision, angular, geometry, log2n;
};
bool tune_cache_key(int device, int precision, int angular, int geometry, int log2n, TuneCacheKey* key);
bool tune_cache_lookup(const TuneCacheKey& key, long long* n, lm_pair_config* cfg, lm_pair_config* adj,
                       bool* has_adj);
void tune_cache_store(const TuneCacheKey& key, long long n, const lm_pair_config& cfg, const lm_pair_config* adj);
// LM_AUTOTUNE=1: a solver without a configuration of its own tunes the first
// time it runs a product at an N bucket that no cache holds.
int autotune_on_first_use();

}  // namespace lmk
