// FP64 vector kernels of the Krylov (Lanczos) square root, M^{1/2} W
// (libMobility paper, Sec. 3.3): dot products, the three-term update,
// classical Gram-Schmidt against the stored basis (full reorthogonalisation),
// the final combination y = V z and the Philox-4x32-10 normal generator for
// W.  They stream FP64 vectors from HBM; the Gram-Schmidt pair does one FP64
// FMA per 8-byte basis element, so on GB300 (FP64 at 1/64 of the FP32 rate)
// the FP64 pipe, not HBM, bounds it once the basis is long.
#include <cuda_runtime.h>

#include <cstdint>

#include "lm_internal.cuh"
#include "philox.cuh"

namespace lmk {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1216;   // 8 x 152 SMs: one wave of 256-thread blocks

inline int blocks_for(int64_t n, int per_thread = 4) {
    int64_t b = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
    if (b < 1) b = 1;
    if (b > kMaxBlocks) b = kMaxBlocks;
    return (int)b;
}

// Programmatic dependent launch: the per-iteration vector kernels are
// launched with cudaLaunchAttributeProgrammaticStreamSerialization, so that
// each can be scheduled while its predecessor in the stream drains.  Every
// such kernel first waits for its predecessors to complete (griddepcontrol.
// wait: their memory operations are then visible), so the order of all
// memory accesses is that of plain stream order; only the launch latency
// overlaps.  It then allows its own dependent to be scheduled.  In a launch
// without the attribute both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
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

// DGKS test for the second Gram-Schmidt pass: h = [h0, h0^2, h1, h1^2], the
// norms before and after the first pass; the pass runs only if h1 < h0 / sqrt(2).
__device__ __forceinline__ bool second_pass_needed(const double* h) {
    return h == nullptr || h[2] < h[0] * 0.70710678118654752440;
}

// Basis combination for one element e: sum_j c[j] V[j][e], j < m, with c
// staged in shared memory 256 rows at a time.  Eight loads are issued before
// their FMAs and two accumulators alternate, so that a thread keeps eight
// HBM reads and two FP64 FMA chains (64-cycle latency on this GPU) in flight.
__device__ __forceinline__ double basis_combination(const double* __restrict__ V, int m, const double* __restrict__ c,
                                                    int64_t n, int64_t e, double* csh) {
    double a0 = 0.0, a1 = 0.0;
    for (int j0 = 0; j0 < m; j0 += 256) {
        const int mm = (m - j0 < 256) ? (m - j0) : 256;
        __syncthreads();
        if (threadIdx.x < mm) csh[threadIdx.x] = c[j0 + threadIdx.x];
        __syncthreads();
        if (e >= n || !LM_INBOUNDS(j0 + mm <= m, 11, j0 + mm)) continue;
        const double* __restrict__ v = V + (int64_t)j0 * n + e;
        int j = 0;
        for (; j + 8 <= mm; j += 8) {
            double x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = v[(int64_t)(j + q) * n];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                a0 = fma(csh[j + q], x[q], a0);
                a1 = fma(csh[j + q + 1], x[q + 1], a1);
            }
        }
        for (; j < mm; ++j) a0 = fma(csh[j], v[(int64_t)j * n], a0);
    }
    return a0 + a1;
}

// y[e] = sum_j z[j] V[j][e] (the Lanczos iterate y = V z).
__global__ void combine_kernel(const double* __restrict__ V, int m, const double* __restrict__ z,
                               double* __restrict__ y, int64_t n) {
    __shared__ double csh[256];
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e - threadIdx.x < n;
         e += (int64_t)gridDim.x * kThreads) {
        const double acc = basis_combination(V, m, z, n, e, csh);
        if (e < n) y[e] = acc;
    }
}

__global__ void scale_kernel(const double* __restrict__ x, const double* __restrict__ nrm, double* __restrict__ y,
                             int64_t n) {
    pdl_enter();
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

__global__ void philox_normals_kernel(uint64_t seed, uint64_t stream, double* __restrict__ W, int64_t n) {
    const int64_t nq = (n + 3) / 4;
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < nq; q += (int64_t)gridDim.x * kThreads) {
        double z[4];
        philox_normals4(seed, stream, (uint64_t)q, z);
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (4 * q + t < n) W[4 * q + t] = z[t];
    }
}

// Raw Philox-4x32-10 words: out[4 e + t] = word t of philox(ctr[4 e ..], key[2 e ..]).
__global__ void philox_words_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                                    uint32_t* __restrict__ out, int64_t count) {
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < count; e += (int64_t)gridDim.x * kThreads) {
        uint32_t c[4] = {ctr[4 * e], ctr[4 * e + 1], ctr[4 * e + 2], ctr[4 * e + 3]};
        philox4x32_10(c, key[2 * e], key[2 * e + 1]);
#pragma unroll
        for (int t = 0; t < 4; ++t) out[4 * e + t] = c[t];
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
    pdl_enter();
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
    pdl_enter();
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

// Multi-dot c[j] = v_j . w, j < m.  Block (b, g) takes the rows
// [8g, 8g + 8) over the element chunk [b*kMdChunk, (b+1)*kMdChunk): each
// thread accumulates the eight rows over its kMdElems elements (eight
// independent FP64 chains, w read once per element), the warp reduces the
// eight sums by a transposing butterfly (9 shuffles and adds instead of 40),
// the block adds its four warps and writes red[j * nb + b].  The last block
// of row group g (counter ctr[g]) forms c[j] = sum_b red[j * nb + b] in
// lane-strided order followed by a butterfly, so the result is deterministic.
constexpr int kMdThreads = 128;
constexpr int kMdElems = 8;
constexpr int kMdRows = 8;
constexpr int64_t kMdChunk = (int64_t)kMdThreads * kMdElems;

__global__ void __launch_bounds__(kMdThreads) multidot_rows(const double* __restrict__ V, int m,
                                                            const double* __restrict__ w, int64_t n, double* red,
                                                            unsigned* ctr, double* __restrict__ c,
                                                            const double* __restrict__ cond) {
    pdl_enter();
    if (!second_pass_needed(cond)) return;
    const int nb = gridDim.x, g = blockIdx.y;
    const int j0 = g * kMdRows;
    const int rows = (m - j0 < kMdRows) ? (m - j0) : kMdRows;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t eb = (int64_t)blockIdx.x * kMdChunk + threadIdx.x;
    double acc[kMdRows];
#pragma unroll
    for (int r = 0; r < kMdRows; ++r) acc[r] = 0.0;
#pragma unroll 2
    for (int q = 0; q < kMdElems; ++q) {
        const int64_t e = eb + (int64_t)q * kMdThreads;
        if (e < n) {
            const double we = w[e];
            const double* __restrict__ v = V + (int64_t)j0 * n + e;
#pragma unroll
            for (int r = 0; r < kMdRows; ++r)
                if (r < rows && LM_INBOUNDS(j0 + r < m, 10, j0 + r)) acc[r] = fma(v[(int64_t)r * n], we, acc[r]);
        }
    }
    // transposing butterfly: after the offsets 16, 8 and 4 lane l holds the
    // partial of row l >> 2 (bits 4, 3, 2 of l), completed by offsets 2 and 1
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const bool up = lane & 16;
        const double keep = up ? acc[r + 4] : acc[r], send = up ? acc[r] : acc[r + 4];
        acc[r] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const bool up = lane & 8;
        const double keep = up ? acc[r + 2] : acc[r], send = up ? acc[r] : acc[r + 2];
        acc[r] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const bool up = lane & 4;
        const double keep = up ? acc[1] : acc[0], send = up ? acc[0] : acc[1];
        acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    __shared__ double wsum[kMdThreads / 32][kMdRows];
    if ((lane & 3) == 0) wsum[wid][lane >> 2] = acc[0];
    __syncthreads();
    if (threadIdx.x < rows) {
        double t = wsum[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < kMdThreads / 32; ++q) t += wsum[q][threadIdx.x];
        red[(int64_t)(j0 + threadIdx.x) * nb + blockIdx.x] = t;
    }
    // the last block of this row group adds the chunks
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&ctr[g], 1u) == (unsigned)nb - 1u);
    __syncthreads();
    if (!last) return;
    for (int r = wid; r < rows; r += kMdThreads / 32) {
        const double* pr = red + (int64_t)(j0 + r) * nb;
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(pr + b);
        t = warp_sum(t);
        if (lane == 0) c[j0 + r] = t;
    }
    if (threadIdx.x == 0) ctr[g] = 0u;
}

// w -= sum_j c[j] V[j], then out = (|w|, |w|^2).  When the DGKS test skips
// the pass, w is unchanged and its norm is the one the first pass left in
// cond[2], cond[3] (the same kernel over the same w would recompute it bit
// for bit), so one thread copies it.
__global__ void sub_vc_norm_kernel(const double* __restrict__ V, int m, const double* __restrict__ c,
                                   double* __restrict__ w, int64_t n, const double* __restrict__ cond, double* red,
                                   unsigned* ctr, double* __restrict__ out) {
    pdl_enter();
    if (!second_pass_needed(cond)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) { out[0] = cond[2]; out[1] = cond[3]; }
        return;
    }
    __shared__ double csh[256];
    double nrm = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e - threadIdx.x < n;
         e += (int64_t)gridDim.x * kThreads) {
        const double acc = basis_combination(V, m, c, n, e, csh);
        if (e < n) {
            const double v = w[e] - acc;
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

inline int md_blocks(int64_t n) { return (int)((n + kMdChunk - 1) / kMdChunk); }

}  // namespace

size_t lz_red_doubles(int64_t n, int m) {
    const size_t a = (size_t)md_blocks(n) * (size_t)(m < 1 ? 1 : m);
    return a > (size_t)kMaxBlocks ? a : (size_t)kMaxBlocks;
}

size_t lz_ctr_count(int m) { return 1 + (size_t)((m < 1 ? 1 : m) + kMdRows - 1) / kMdRows; }

cudaError_t lz_norm(const double* x, int64_t n, double* red, double* out, cudaStream_t s) {
    const int nb = blocks_for(n);
    dot_stage1<<<nb, kThreads, 0, s>>>(x, x, n, red);
    sum_stage2<<<1, kThreads, 0, s>>>(red, nb, out, 1);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t lz_dot1(const double* x, const double* y, int64_t n, double* red, unsigned* ctr, double* out,
                    int mode, cudaStream_t s) {
    count_launches(1);
    return launch_pdl(dot_fused, dim3(blocks_for(n)), dim3(kThreads), s, x, y, n, red, ctr, out, mode);
}

cudaError_t lz_axpy2_norm(double* w, const double* vk, const double* alpha, const double* vkm1, const double* beta,
                          int64_t n, double* red, unsigned* ctr, double* out, cudaStream_t s) {
    count_launches(1);
    return launch_pdl(axpy2_norm_kernel, dim3(blocks_for(n)), dim3(kThreads), s, w, vk, alpha, vkm1, beta, n, red,
                      ctr, out);
}

cudaError_t lz_multidot1(const double* V, int m, const double* w, int64_t n, double* red, unsigned* ctr, double* c,
                         cudaStream_t s, const double* cond) {
    if (m < 1) return cudaSuccess;
    const int nb = md_blocks(n), ng = (m + kMdRows - 1) / kMdRows;
    if (nb < 1 || ng > 65535) return cudaErrorInvalidConfiguration;
    count_launches(1);
    return launch_pdl(multidot_rows, dim3((unsigned)nb, (unsigned)ng), dim3(kMdThreads), s, V, m, w, n, red, ctr + 1, c,
                      cond);
}

cudaError_t lz_sub_vc_norm(const double* V, int m, const double* c, double* w, int64_t n, double* red,
                           unsigned* ctr, double* out, cudaStream_t s, const double* cond) {
    count_launches(1);
    return launch_pdl(sub_vc_norm_kernel, dim3(blocks_for(n, 1)), dim3(kThreads), s, V, m, c, w, n, cond, red, ctr,
                      out);
}

cudaError_t lz_scale(const double* x, const double* nrm, double* y, int64_t n, cudaStream_t s) {
    count_launches(1);
    return launch_pdl(scale_kernel, dim3(blocks_for(n)), dim3(kThreads), s, x, nrm, y, n);
}

cudaError_t lz_combine(const double* V, int m, const double* z, double* y, int64_t n, cudaStream_t s) {
    combine_kernel<<<blocks_for(n, 1), kThreads, 0, s>>>(V, m, z, y, n);
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

cudaError_t lz_philox_words(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t count,
                            cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    philox_words_kernel<<<blocks_for(count), kThreads, 0, s>>>(ctr, key, out, count);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lmk
