// FP32 throughput probes: the measured ceiling of the FP32 FMA pipe that the
// pair kernels run on (they are bound by it: the RPY pair is a nonlinear
// function of x_i - x_j, not a dense contraction, so it has no tensor-core
// form).  The nominal peak is SMs x 128 lanes x 2 flop x clock; these probes
// measure what FMA streams of different operand patterns reach on the GPU at
// hand (every chain's value is written out, so no work is dead):
//   mode 0  scalar FMA, x = x a + b on 8 independent chains per thread
//           (two operands the same register in every instruction);
//   mode 1  packed f32x2 FMA of the same form (two lanes per instruction,
//           the instruction form of the packed pair kernels);
//   mode 2  packed f32x2 FMA on 12 independent accumulators, each
//           instruction reading two loop-invariant register pairs of its own
//           (three distinct register pairs per instruction, no dependence
//           within 12 instructions);
//   mode 3  packed f32x2 FMA in rotating dependent chains, every operand a
//           value produced a few instructions earlier (the data flow of the
//           pair formulas, where most operands are fresh intermediates);
//   mode 4  FP64 FMA, x = x a + b on 8 independent chains per thread: the
//           ceiling of the Lanczos Gram-Schmidt kernels, which do one FP64
//           FMA per 8-byte basis element.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lm.h"
#include "lm_internal.cuh"

namespace lmk {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(int64_t iters, float a, float b,
                                                                   float* __restrict__ out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-3f * (float)(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma2_kernel(int64_t iters, float a, float b,
                                                                    float* __restrict__ out) {
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(1.0f + 1e-3f * (float)(threadIdx.x + c), 1.0f);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dfma_kernel(int64_t iters, double a, double b,
                                                                   float* __restrict__ out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = (float)s;
}

// Twelve accumulators, each with its own pair of loop-invariant operands.
__global__ void __launch_bounds__(kProbeThreads) probe_ffma2_wide_kernel(int64_t iters, float a, float b,
                                                                         float* __restrict__ out) {
    constexpr int K = 12;
    float2 acc[K], u[K], v[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const float t = 1e-3f * (float)(threadIdx.x + c);
        acc[c] = make_float2(t, -t);
        u[c] = make_float2(a * (1.0f + t), a);
        v[c] = make_float2(b, b * (1.0f - t));
    }
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int c = 0; c < K; ++c) acc[c] = __ffma2_rn(u[c], v[(c + r) % K], acc[c]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < K; ++c) s += acc[c].x + acc[c].y;
    out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

// Three rotating banks of chains: x <- y * z + x, then y <- z * x + y, then
// z <- x * y + z, each on a different chain index, so all three operands of
// every instruction are distinct register pairs produced recently.  The
// recurrence is nonlinear and its values overflow after some iterations; the
// FP32 FMA pipe has no slow path for infinities or NaNs, so the timing does
// not depend on the values.
__global__ void __launch_bounds__(kProbeThreads) probe_ffma2_chain_kernel(int64_t iters, float a, float b,
                                                                          float* __restrict__ out) {
    float2 x[kChains], y[kChains], z[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float t = 1e-3f * (float)(threadIdx.x + c);
        x[c] = make_float2(b + t, -b - t);
        y[c] = make_float2(a, a - t * 1e-3f);
        z[c] = make_float2(1.0f, 1.0f - t * 1e-3f);
    }
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                const int c1 = (c + 1) % kChains, c2 = (c + 3) % kChains;
                x[c] = __ffma2_rn(y[c1], z[c2], x[c]);
                z[c] = __ffma2_rn(x[c2], y[c], z[c1]);
                y[c] = __ffma2_rn(z[c1], x[c], y[c2]);
                x[c1] = __ffma2_rn(y[c], z[c], x[c1]);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y + y[c].x + y[c].y + z[c].x + z[c].y;
    out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace lmk

extern "C" lm_status lm_fp32_probe(int mode, int64_t iters, double* tflops, void* cuda_stream) {
    lmk::set_last_error("");
    if (tflops == nullptr || mode < 0 || mode > 4 || iters < 1 || iters > (int64_t)1 << 24) {
        lmk::set_last_error("lm_fp32_probe: mode in 0..4, 1 <= iters <= 2^24 and tflops are required");
        return LM_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        const int nt = lmk::kProbeThreads;
        if (mode == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lmk::probe_ffma_kernel, nt, 0);
        else if (mode == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lmk::probe_ffma2_kernel, nt, 0);
        else if (mode == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lmk::probe_ffma2_wide_kernel, nt, 0);
        else if (mode == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lmk::probe_ffma2_chain_kernel, nt, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lmk::probe_dfma_kernel, nt, 0);
    }
    if (e != cudaSuccess) {
        lmk::set_last_error(cudaGetErrorString(e));
        return LM_ERR_CUDA;
    }
    const int blocks = sms * (occ > 0 ? occ : 1);
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * lmk::kProbeThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // flops per thread per outer iteration: FFMA and DFMA 16 x 8 x 2; FFMA2
    // 16 x 8 x 4; wide 8 x 12 x 4; chains 4 x 8 x 4 packed FMAs x 4
    const double per_it = (mode == 0 || mode == 4) ? 256.0 : (mode == 2 ? 384.0 : 512.0);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, s);
        if (mode == 0) lmk::probe_ffma_kernel<<<blocks, lmk::kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, out);
        else if (mode == 1) lmk::probe_ffma2_kernel<<<blocks, lmk::kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, out);
        else if (mode == 2) lmk::probe_ffma2_wide_kernel<<<blocks, lmk::kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, out);
        else if (mode == 3) lmk::probe_ffma2_chain_kernel<<<blocks, lmk::kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, out);
        else lmk::probe_dfma_kernel<<<blocks, lmk::kProbeThreads, 0, s>>>(iters, 0.9999, 1e-4, out);
        lmk::count_launches(1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        lmk::set_last_error(cudaGetErrorString(e));
        return LM_ERR_CUDA;
    }
    *tflops = per_it * (double)iters * (double)blocks * lmk::kProbeThreads / (ms * 1e-3) / 1e12;
    return LM_OK;
}
