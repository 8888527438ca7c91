// FP64 vector kernels of the Krylov (Lanczos) square root, M^{1/2} W
// (libMobility paper, Sec. 3.3).  They are HBM-bound: dot products, the
// three-term update, classical Gram-Schmidt against the stored basis
// (full reorthogonalisation), the final combination y = V z and the
// Philox-4x32-10 normal generator for W.
#include <cuda_runtime.h>

#include <cstdint>

#include "lm_internal.cuh"

namespace lmk {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 608;   // 4 x 152 SMs

inline int blocks_for(int64_t n, int per_thread = 4) {
    int64_t b = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
    if (b < 1) b = 1;
    if (b > kMaxBlocks) b = kMaxBlocks;
    return (int)b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kThreads / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < kThreads / 32) ? ws[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void dot_stage1(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                           double* __restrict__ red) {
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kThreads)
        acc = fma(x[e], y[e], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[blockIdx.x] = acc;
}

// mode 0: out[0] = sum ; mode 1: out[0] = sqrt(sum), out[1] = sum
__global__ void sum_stage2(const double* __restrict__ red, int nb, double* __restrict__ out, int mode) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) acc += red[b];
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        if (mode == 0) out[0] = acc;
        else { out[0] = sqrt(acc); out[1] = acc; }
    }
}

__global__ void axpy2_kernel(double* __restrict__ w, const double* __restrict__ vk, const double* __restrict__ alpha,
                             const double* __restrict__ vkm1, const double* __restrict__ beta, int64_t n) {
    const double a = alpha[0];
    const double b = (vkm1 != nullptr) ? beta[0] : 0.0;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kThreads) {
        double v = w[e] - a * vk[e];
        if (vkm1 != nullptr) v -= b * vkm1[e];
        w[e] = v;
    }
}

// Multi-dot: block b owns the chunk [b*cs, min(n, (b+1)*cs)); warp q handles
// rows j = q, q + 8, ...; red[j * nb + b] = partial dot.
// DGKS test for the second Gram-Schmidt pass: h = [h0, h0^2, h1, h1^2], the
// norms before and after the first pass; the pass runs only if h1 < h0 / sqrt(2).
__device__ __forceinline__ bool second_pass_needed(const double* h) {
    return h == nullptr || h[2] < h[0] * 0.70710678118654752440;
}

__global__ void multidot_stage1(const double* __restrict__ V, int m, const double* __restrict__ w, int64_t n,
                                int64_t cs, double* __restrict__ red, const double* __restrict__ cond) {
    if (!second_pass_needed(cond)) return;
    const int64_t e0 = (int64_t)blockIdx.x * cs;
    const int64_t e1 = (e0 + cs < n) ? (e0 + cs) : n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = wid; j < m; j += kThreads / 32) {
        const double* __restrict__ v = V + (int64_t)j * n;
        double acc = 0.0;
        for (int64_t e = e0 + lane; e < e1; e += 32) acc = fma(v[e], w[e], acc);
        acc = warp_sum(acc);
        if (lane == 0) red[(int64_t)j * gridDim.x + blockIdx.x] = acc;
    }
}

__global__ void multidot_stage2(const double* __restrict__ red, int m, int nb, double* __restrict__ c,
                                const double* __restrict__ cond) {
    if (!second_pass_needed(cond)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = blockIdx.x * (kThreads / 32) + wid; j < m; j += gridDim.x * (kThreads / 32)) {
        double acc = 0.0;
        for (int b = lane; b < nb; b += 32) acc += red[(int64_t)j * nb + b];
        acc = warp_sum(acc);
        if (lane == 0) c[j] = acc;
    }
}

// w[e] (+)= sign * sum_j c[j] V[j][e]; accumulate = 0 overwrites (y = V^T z).
__global__ void combine_kernel(const double* __restrict__ V, int m, const double* __restrict__ c,
                               double* __restrict__ w, int64_t n, int accumulate, double sign,
                               const double* __restrict__ cond) {
    if (!second_pass_needed(cond)) return;
    __shared__ double cs[256];
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e - threadIdx.x < n;
         e += (int64_t)gridDim.x * kThreads) {
        double acc = 0.0;
        for (int j0 = 0; j0 < m; j0 += 256) {
            const int mm = (m - j0 < 256) ? (m - j0) : 256;
            __syncthreads();
            if (threadIdx.x < mm) cs[threadIdx.x] = c[j0 + threadIdx.x];
            __syncthreads();
            if (e < n)
                for (int j = 0; j < mm; ++j) acc = fma(cs[j], V[(int64_t)(j0 + j) * n + e], acc);
        }
        if (e < n) w[e] = accumulate ? fma(sign, acc, w[e]) : sign * acc;
    }
}

__global__ void scale_kernel(const double* __restrict__ x, const double* __restrict__ nrm, double* __restrict__ y,
                             int64_t n) {
    const double inv = 1.0 / nrm[0];
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kThreads)
        y[e] = x[e] * inv;
}

__global__ void store_kernel(const double* __restrict__ y, double scale, int64_t N, int angular,
                             void* __restrict__ lin, void* __restrict__ ang, int out_f64) {
    const int64_t n3 = 3 * N;
    const int64_t n = angular ? 2 * n3 : n3;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kThreads) {
        const double v = scale * y[e];
        void* out = (e < n3) ? lin : ang;
        const int64_t idx = (e < n3) ? e : e - n3;
        if (out_f64) static_cast<double*>(out)[idx] = v;
        else static_cast<float*>(out)[idx] = (float)v;
    }
}

// Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of the
// multiply/xor round on four 32-bit words, the key bumped by the Weyl
// constants after every round but the last.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        if (r < 9) { k0 += W0; k1 += W1; }
    }
}

__global__ void philox_normals_kernel(uint64_t seed, uint64_t stream, double* __restrict__ W, int64_t n) {
    const int64_t nq = (n + 3) / 4;
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < nq; q += (int64_t)gridDim.x * kThreads) {
        uint32_t c[4] = {(uint32_t)(q & 0xffffffffu), (uint32_t)((uint64_t)q >> 32),
                         (uint32_t)(stream & 0xffffffffu), (uint32_t)(stream >> 32)};
        philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
        double z[4];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const double u1 = ((double)c[2 * p] + 1.0) * (1.0 / 4294967296.0);
            const double u2 = (double)c[2 * p + 1] * (1.0 / 4294967296.0);
            const double rad = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);
            z[2 * p] = rad * cs;
            z[2 * p + 1] = rad * sn;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (4 * q + t < n) W[4 * q + t] = z[t];
    }
}

// ---------------------------------------------------------------------------
// Single-launch forms: every block writes its partial result, and the last
// block to finish (a device counter, reset by that block) adds the partials
// in block order, so the results are deterministic and equal to the
// two-launch forms'.  They halve the launches of a Lanczos iteration, which
// bound its time at small N.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool last_block_done(unsigned* ctr) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ctr, 1u) == gridDim.x - 1);
    __syncthreads();
    return last;
}

// Sum of red[0, nb) in the order of sum_stage2; called by the last block.
__device__ __forceinline__ double final_sum(const double* red, int nb) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) acc += __ldcg(red + b);
    return block_sum(acc);
}

// mode 0: out[0] = x.y ; mode 1: out[0] = sqrt(x.x), out[1] = x.x
__global__ void dot_fused(const double* __restrict__ x, const double* __restrict__ y, int64_t n, double* red,
                          unsigned* ctr, double* __restrict__ out, int mode) {
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kThreads)
        acc = fma(x[e], y[e], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[blockIdx.x] = acc;
    if (!last_block_done(ctr)) return;
    const double t = final_sum(red, gridDim.x);
    if (threadIdx.x == 0) {
        if (mode == 0) out[0] = t;
        else { out[0] = sqrt(t); out[1] = t; }
        *ctr = 0u;
    }
}

// w -= alpha vk + beta vkm1, then out = (|w|, |w|^2)
__global__ void axpy2_norm_kernel(double* __restrict__ w, const double* __restrict__ vk,
                                  const double* __restrict__ alpha, const double* __restrict__ vkm1,
                                  const double* __restrict__ beta, int64_t n, double* red, unsigned* ctr,
                                  double* __restrict__ out) {
    const double a = alpha[0];
    const double b = (vkm1 != nullptr) ? beta[0] : 0.0;
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < n; e += (int64_t)gridDim.x * kThreads) {
        double v = w[e] - a * vk[e];
        if (vkm1 != nullptr) v -= b * vkm1[e];
        w[e] = v;
        acc = fma(v, v, acc);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[blockIdx.x] = acc;
    if (!last_block_done(ctr)) return;
    const double t = final_sum(red, gridDim.x);
    if (threadIdx.x == 0) { out[0] = sqrt(t); out[1] = t; *ctr = 0u; }
}

// multidot_stage1, then the last block forms c[j] = sum_b red[j nb + b]
// (the order of multidot_stage2).
__global__ void multidot_fused(const double* __restrict__ V, int m, const double* __restrict__ w, int64_t n,
                               int64_t cs, double* red, unsigned* ctr, double* __restrict__ c,
                               const double* __restrict__ cond) {
    if (!second_pass_needed(cond)) return;
    const int64_t e0 = (int64_t)blockIdx.x * cs;
    const int64_t e1 = (e0 + cs < n) ? (e0 + cs) : n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = wid; j < m; j += kThreads / 32) {
        const double* __restrict__ v = V + (int64_t)j * n;
        double acc = 0.0;
        for (int64_t e = e0 + lane; e < e1; e += 32) acc = fma(v[e], w[e], acc);
        acc = warp_sum(acc);
        if (lane == 0) red[(int64_t)j * gridDim.x + blockIdx.x] = acc;
    }
    if (!last_block_done(ctr)) return;
    const int nb = gridDim.x;
    for (int j = wid; j < m; j += kThreads / 32) {
        double acc = 0.0;
        for (int b = lane; b < nb; b += 32) acc += __ldcg(red + (int64_t)j * nb + b);
        acc = warp_sum(acc);
        if (lane == 0) c[j] = acc;
    }
    if (threadIdx.x == 0) *ctr = 0u;
}

// w -= sum_j c[j] V[j] (skipped unless the DGKS test asks for it), then
// out = (|w|, |w|^2) in any case.
__global__ void sub_vc_norm_kernel(const double* __restrict__ V, int m, const double* __restrict__ c,
                                   double* __restrict__ w, int64_t n, const double* __restrict__ cond, double* red,
                                   unsigned* ctr, double* __restrict__ out) {
    const bool apply = second_pass_needed(cond);
    __shared__ double csh[256];
    double nrm = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e - threadIdx.x < n;
         e += (int64_t)gridDim.x * kThreads) {
        double acc = 0.0;
        if (apply) {
            for (int j0 = 0; j0 < m; j0 += 256) {
                const int mm = (m - j0 < 256) ? (m - j0) : 256;
                __syncthreads();
                if (threadIdx.x < mm) csh[threadIdx.x] = c[j0 + threadIdx.x];
                __syncthreads();
                if (e < n)
                    for (int j = 0; j < mm; ++j) acc = fma(csh[j], V[(int64_t)(j0 + j) * n + e], acc);
            }
        }
        if (e < n) {
            const double v = apply ? fma(-1.0, acc, w[e]) : w[e];
            w[e] = v;
            nrm = fma(v, v, nrm);
        }
    }
    nrm = block_sum(nrm);
    if (threadIdx.x == 0) red[blockIdx.x] = nrm;
    if (!last_block_done(ctr)) return;
    const double t = final_sum(red, gridDim.x);
    if (threadIdx.x == 0) { out[0] = sqrt(t); out[1] = t; *ctr = 0u; }
}

inline int64_t md_chunk(int64_t n, int* nb) {
    int64_t cs = (n + kMaxBlocks - 1) / kMaxBlocks;
    cs = (cs + 31) / 32 * 32;
    if (cs < 256) cs = 256;
    *nb = (int)((n + cs - 1) / cs);
    if (*nb < 1) *nb = 1;
    return cs;
}

}  // namespace

size_t lz_red_doubles(int64_t n, int m) {
    int nb = 0;
    md_chunk(n, &nb);
    size_t a = (size_t)nb * (size_t)(m < 1 ? 1 : m);
    return a > (size_t)kMaxBlocks ? a : (size_t)kMaxBlocks;
}

cudaError_t lz_dot(const double* x, const double* y, int64_t n, double* red, double* out, cudaStream_t s) {
    const int nb = blocks_for(n);
    dot_stage1<<<nb, kThreads, 0, s>>>(x, y, n, red);
    sum_stage2<<<1, kThreads, 0, s>>>(red, nb, out, 0);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t lz_norm(const double* x, int64_t n, double* red, double* out, cudaStream_t s) {
    const int nb = blocks_for(n);
    dot_stage1<<<nb, kThreads, 0, s>>>(x, x, n, red);
    sum_stage2<<<1, kThreads, 0, s>>>(red, nb, out, 1);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t lz_axpy2(double* w, const double* vk, const double* alpha, const double* vkm1, const double* beta,
                     int64_t n, cudaStream_t s) {
    axpy2_kernel<<<blocks_for(n), kThreads, 0, s>>>(w, vk, alpha, vkm1, beta, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_multidot(const double* V, int m, const double* w, int64_t n, double* red, double* c,
                        cudaStream_t s, const double* cond) {
    int nb = 0;
    const int64_t cs = md_chunk(n, &nb);
    multidot_stage1<<<nb, kThreads, 0, s>>>(V, m, w, n, cs, red, cond);
    const int g2 = (m + (kThreads / 32) - 1) / (kThreads / 32);
    multidot_stage2<<<g2, kThreads, 0, s>>>(red, m, nb, c, cond);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t lz_sub_vc(const double* V, int m, const double* c, double* w, int64_t n, cudaStream_t s,
                      const double* cond) {
    combine_kernel<<<blocks_for(n, 1), kThreads, 0, s>>>(V, m, c, w, n, 1, -1.0, cond);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_dot1(const double* x, const double* y, int64_t n, double* red, unsigned* ctr, double* out,
                    int mode, cudaStream_t s) {
    dot_fused<<<blocks_for(n), kThreads, 0, s>>>(x, y, n, red, ctr, out, mode);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_axpy2_norm(double* w, const double* vk, const double* alpha, const double* vkm1, const double* beta,
                          int64_t n, double* red, unsigned* ctr, double* out, cudaStream_t s) {
    axpy2_norm_kernel<<<blocks_for(n), kThreads, 0, s>>>(w, vk, alpha, vkm1, beta, n, red, ctr, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_multidot1(const double* V, int m, const double* w, int64_t n, double* red, unsigned* ctr, double* c,
                         cudaStream_t s, const double* cond) {
    int nb = 0;
    const int64_t cs = md_chunk(n, &nb);
    // one block adds the partials: worth it while they are few
    if ((int64_t)nb * m > 8192) return lz_multidot(V, m, w, n, red, c, s, cond);
    multidot_fused<<<nb, kThreads, 0, s>>>(V, m, w, n, cs, red, ctr, c, cond);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_sub_vc_norm(const double* V, int m, const double* c, double* w, int64_t n, double* red,
                           unsigned* ctr, double* out, cudaStream_t s, const double* cond) {
    sub_vc_norm_kernel<<<blocks_for(n, 1), kThreads, 0, s>>>(V, m, c, w, n, cond, red, ctr, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_scale(const double* x, const double* nrm, double* y, int64_t n, cudaStream_t s) {
    scale_kernel<<<blocks_for(n), kThreads, 0, s>>>(x, nrm, y, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_combine(const double* V, int m, const double* z, double* y, int64_t n, cudaStream_t s) {
    combine_kernel<<<blocks_for(n, 1), kThreads, 0, s>>>(V, m, z, y, n, 0, 1.0, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_store(const double* y, double scale, int64_t N, int angular, void* lin, void* ang, int out_f64,
                     cudaStream_t s) {
    const int64_t n = (angular ? 6 : 3) * N;
    store_kernel<<<blocks_for(n), kThreads, 0, s>>>(y, scale, N, angular, lin, ang, out_f64);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lz_philox_normals(uint64_t seed, uint64_t stream, double* W, int64_t n, cudaStream_t s) {
    philox_normals_kernel<<<blocks_for((n + 3) / 4), kThreads, 0, s>>>(seed, stream, W, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lmk
