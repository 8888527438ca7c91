// lm_mdot_noalloc: the FP32 mobility product without any device allocation.
//
// Some callers cannot let a library allocate GPU memory:
//   * applications that hand all device memory to their own pool or caching
//     allocator, where a foreign cudaMalloc can fail or fragment the pool;
//   * latency-critical loops, where cudaMalloc / cudaFree would add an
//     implicit device-wide synchronisation to every call;
//   * hosts that forbid runtime allocation inside plugins.
// For them this entry point computes what lm_mdot computes for an FP32 solver
// (same pair kernel, same results up to the order of the split sums), taking
// every buffer from the caller except its scratch.  The scratch (packed
// positions and the j-split partial sums) is one file-scope __device__ array
// of LM_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library keeps
// until the process exits.
//
// The array's name in host code is only a host-side stand-in, never a device
// address: host code must get the address with cudaGetSymbolAddress, which is
// done once per device (with that device current) on the first call and
// cached.  That first call should therefore come before any stream capture.
// Every call reuses the same array and leaves its contents behind; nothing in
// it needs to start at zero (each call overwrites what it reads), but calls
// whose GPU work overlaps (different streams without ordering) race on it.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/lm.h"
#include "lm_internal.cuh"

// The scratch array (device memory; host code uses its address only through
// cudaGetSymbolAddress).
static __device__ __align__(256) unsigned char g_noalloc_scratch[LM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

lm_status noalloc_fail(lm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    lmk::set_last_error(buf);
    return st;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

extern "C" lm_status lm_mdot_noalloc(const float* pos, const float* forces, const float* torques, int64_t N,
                                     double viscosity, double hydrodynamic_radius, int include_angular,
                                     float* lin_out, float* ang_out, void* cuda_stream) {
    lmk::set_last_error("");
    if (N < 1 || N > LM_NOALLOC_MAX_N)
        return noalloc_fail(LM_ERR_INVALID_ARG, "N = %lld is outside [1, %d], the no-allocation limit", (long long)N,
                            (int)LM_NOALLOC_MAX_N);
    if (!(viscosity > 0.0) || !(hydrodynamic_radius > 0.0))
        return noalloc_fail(LM_ERR_INVALID_ARG, "viscosity and radius must be > 0");
    if (pos == nullptr || lin_out == nullptr)
        return noalloc_fail(LM_ERR_INVALID_ARG, "pos and lin_out are required");
    if (include_angular && ang_out == nullptr)
        return noalloc_fail(LM_ERR_INVALID_ARG, "ang_out is required with angular blocks");
    if (!include_angular && (ang_out != nullptr || torques != nullptr))
        return noalloc_fail(LM_ERR_INVALID_ARG, "torques / ang_out given but include_angular is 0");
    const void* ptrs[5] = {pos, forces, torques, lin_out, ang_out};
    for (const void* p : ptrs)
        if (p != nullptr && !on_device(p))
            return noalloc_fail(LM_ERR_INVALID_ARG, "all arrays must be device memory (no staging buffers here)");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LM_ERR_INVALID_ARG, "device index %d too large", dev);
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (g_scratch_addr[dev] == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(LM_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // scratch layout: [flag: 256 B][packed positions: 16 N B][split partials]
    unsigned char* b = static_cast<unsigned char*>(base);
    int* flag = reinterpret_cast<int*>(b);
    float4* pos4 = reinterpret_cast<float4*>(b + 256);
    const size_t part_off = 256 + round_up((size_t)N * sizeof(float4), 256);
    double* partials = reinterpret_cast<double*>(b + part_off);
    const int C = lmk::mdot_partial_components(include_angular ? 1 : 0);
    const size_t per_split = (size_t)C * (size_t)N * sizeof(double);
    const int max_splits = (int)((LM_NOALLOC_SCRATCH_BYTES - part_off) / per_split);

    const int threads = 128, ilp = 4;
    int sms = 1, occ = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    occ = lmk::mdot_ctas_per_sm(0, include_angular ? 1 : 0, threads, ilp);
    if (occ < 1) occ = 1;
    int splits = lmk::auto_splits(N, threads, ilp, occ * sms);
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    // the launcher never launches more splits than requested (at most one per tile)
    if (lmk::mdot_effective_splits(N, threads, splits) > max_splits)
        return noalloc_fail(LM_ERR_INVALID_ARG, "scratch too small for N = %lld", (long long)N);

    e = lmk::launch_pack_positions(pos, 0, N, pos4, 0, flag, stream);
    if (e != cudaSuccess) return noalloc_fail(LM_ERR_CUDA, "packing positions: %s", cudaGetErrorString(e));
    if (forces == nullptr && torques == nullptr) {
        e = cudaMemsetAsync(lin_out, 0, (size_t)N * 3 * sizeof(float), stream);
        if (e == cudaSuccess && include_angular)
            e = cudaMemsetAsync(ang_out, 0, (size_t)N * 3 * sizeof(float), stream);
        if (e != cudaSuccess) return noalloc_fail(LM_ERR_CUDA, "zero output: %s", cudaGetErrorString(e));
        return LM_OK;
    }
    lmk::MdotArgs a;
    a.fp64 = 0;
    a.angular = include_angular ? 1 : 0;
    a.N = N;
    a.pos4 = pos4;
    a.F = forces;
    a.T = include_angular ? torques : nullptr;
    a.in_f64 = 0;
    a.lin = lin_out;
    a.ang = include_angular ? ang_out : nullptr;
    a.out_f64 = 0;
    a.a = hydrodynamic_radius;
    a.eta = viscosity;
    a.threads = threads;
    a.ilp = ilp;
    a.splits = splits;
    a.partials = partials;
    e = lmk::launch_mdot(a, stream);
    if (e != cudaSuccess) return noalloc_fail(LM_ERR_CUDA, "mobility product kernel: %s", cudaGetErrorString(e));
    return LM_OK;
}
