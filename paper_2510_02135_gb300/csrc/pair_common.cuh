// Device helpers shared by the forward pair kernels (pair_kernels.cu) and
// the single-wall pair kernels (wall_kernels.cu): tile element types, the
// free-space RPY pair terms in both branches, the TwoSum fold of tile
// partials, the split reduction and the j-range split plan.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "lm_internal.cuh"

namespace lmk {
namespace {

template <typename R> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = lmk::dvec4; };

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

template <typename R>
__device__ __forceinline__ R load_elem(const void* p, int in_f64, int64_t idx) {
    if (p == nullptr) return R(0);
    return in_f64 ? (R)(static_cast<const double*>(p)[idx]) : (R)(static_cast<const float*>(p)[idx]);
}

// Exact pair coefficients (both branches) for one pair.
template <typename R>
__device__ __forceinline__ void exact_coeffs(R r2, const RpyConst<R>& k, R& A, R& B, R& g, R& ar, R& br) {
    if (r2 >= k.four_a2) {
        const R invr = rsq(r2);
        const R invr2 = invr * invr;
        const R invr3 = invr2 * invr;
        const R invr5 = invr3 * invr2;
        A = invr + k.K1 * invr3;
        B = invr3 - k.K2 * invr5;
        g = invr3;
        ar = R(-0.5) * invr3;
        br = R(1.5) * invr5;
    } else {
        const R invr = (r2 > R(0)) ? rsq(r2) : R(0);
        const R r = r2 * invr;
        A = k.nA0 - k.nA1 * r;
        B = k.nB * invr;
        g = k.ng0 - k.ng1 * r;
        ar = k.inv_a3 * (R(1) - k.rr1 * r + k.rr3 * r * r * r);
        br = k.inv_a3 * (k.rrb0 * invr - k.rrb1 * r);
    }
}

// Current-tile partial sums of one i-particle (registers).  The running
// sums across tiles live in shared memory (FP32: a TwoSum (hi, lo) pair per
// component; FP64: a plain sum), read and written once per tile.
template <typename R, bool ANG>
struct Acc {
    R p[ANG ? 6 : 3];
};

// Far-field pair: u += A F + B (d.F) d + g (T x d) ; w += g (F x d - T/2) + br (d.T) d
// with the tile holding h = -T/2:  T x d = -2 (h x d),  d.T = -2 d.h.
// Written with explicit FMAs: 22 issue slots (tt) / 49 (all blocks) per pair.
template <typename R, bool ANG>
__device__ __forceinline__ void pair_far(R dx, R dy, R dz, R r2, const typename V4<R>::type& f,
                                         const typename V4<R>::type& h, const RpyConst<R>& k,
                                         Acc<R, ANG>& acc) {
    const R invr = rsq(r2);
    const R invr2 = invr * invr;
    const R invr3 = invr2 * invr;
    const R A = fma(k.K1, invr3, invr);
    const R invr5 = invr3 * invr2;
    const R B = fma(-k.K2, invr5, invr3);
    const R dF = fma(dx, f.x, fma(dy, f.y, dz * f.z));
    const R s = B * dF;
    acc.p[0] = fma(s, dx, fma(A, f.x, acc.p[0]));
    acc.p[1] = fma(s, dy, fma(A, f.y, acc.p[1]));
    acc.p[2] = fma(s, dz, fma(A, f.z, acc.p[2]));
    if constexpr (ANG) {
        // u += g (T x d) = (-2 g) (h x d)
        const R m2g = R(-2) * invr3;
        const R cx = fma(h.y, dz, -(h.z * dy));
        const R cy = fma(h.z, dx, -(h.x * dz));
        const R cz = fma(h.x, dy, -(h.y * dx));
        acc.p[0] = fma(m2g, cx, acc.p[0]);
        acc.p[1] = fma(m2g, cy, acc.p[1]);
        acc.p[2] = fma(m2g, cz, acc.p[2]);
        // w += g (F x d + h) + (-2 br) (d.h) d
        const R vx = fma(f.y, dz, fma(-f.z, dy, h.x));
        const R vy = fma(f.z, dx, fma(-f.x, dz, h.y));
        const R vz = fma(f.x, dy, fma(-f.y, dx, h.z));
        const R t = (R(-3) * invr5) * fma(dx, h.x, fma(dy, h.y, dz * h.z));
        acc.p[3] = fma(t, dx, fma(invr3, vx, acc.p[3]));
        acc.p[4] = fma(t, dy, fma(invr3, vy, acc.p[4]));
        acc.p[5] = fma(t, dz, fma(invr3, vz, acc.p[5]));
    }
}

// Exact pair (either branch, including r = 0).
template <typename R, bool ANG>
__device__ __forceinline__ void pair_exact(R dx, R dy, R dz, R r2, const typename V4<R>::type& f,
                                           const typename V4<R>::type& h, const RpyConst<R>& k,
                                           Acc<R, ANG>& acc) {
    R A, B, g, ar, br;
    exact_coeffs<R>(r2, k, A, B, g, ar, br);
    const R s = B * (dx * f.x + dy * f.y + dz * f.z);
    acc.p[0] += A * f.x + s * dx;
    acc.p[1] += A * f.y + s * dy;
    acc.p[2] += A * f.z + s * dz;
    if constexpr (ANG) {
        const R m2g = R(-2) * g;
        acc.p[0] += m2g * (h.y * dz - h.z * dy);
        acc.p[1] += m2g * (h.z * dx - h.x * dz);
        acc.p[2] += m2g * (h.x * dy - h.y * dx);
        const R m2ar = R(-2) * ar;
        const R t = (R(-2) * br) * (dx * h.x + dy * h.y + dz * h.z);
        acc.p[3] += g * (f.y * dz - f.z * dy) + m2ar * h.x + t * dx;
        acc.p[4] += g * (f.z * dx - f.x * dz) + m2ar * h.y + t * dy;
        acc.p[5] += g * (f.x * dy - f.y * dx) + m2ar * h.z + t * dz;
    }
}

// Knuth TwoSum fold of the tile partial p into the shared (hi, lo) pair.
__device__ __forceinline__ void fold(float* hi, float* lo, float& p) {
    const float h = *hi;
    const float s = h + p;
    const float bb = s - h;
    const float err = (h - (s - bb)) + (p - bb);
    *hi = s;
    *lo += err;
    p = 0.0f;
}
__device__ __forceinline__ void fold(double* hi, double* lo, double& p) {
    *hi += p;
    p = 0.0;
    (void)lo;
}

// Dynamic shared memory for the running sums: C x NI x NT values of R
// (FP32 adds the same again for the low parts).
template <typename R, bool ANG, int NT, int NI>
constexpr size_t running_sum_bytes() {
    return (size_t)(ANG ? 6 : 3) * NI * NT * sizeof(R) * (sizeof(R) == 4 ? 2 : 1);
}

// out[3 i + c] = c8 * sum_s partials[s][c][i]
__global__ void reduce_splits_kernel(const double* __restrict__ partials, int splits, int C, int64_t N,
                                     double c8, void* __restrict__ lin, void* __restrict__ ang, int out_f64) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)C * N) return;
    const int64_t i = e / C;
    const int c = (int)(e - i * C);
    double s = 0.0;
    for (int k = 0; k < splits; ++k) {
        const int64_t pidx = ((int64_t)k * C + c) * N + i;
        if (LM_INBOUNDS(pidx < (int64_t)splits * C * N, 5, pidx)) s += partials[pidx];
    }
    void* out = (c < 3) ? lin : ang;
    const int64_t idx = 3 * i + (c % 3);
    if (!LM_INBOUNDS(idx < 3 * N, 6, idx)) return;
    if (out_f64) static_cast<double*>(out)[idx] = c8 * s;
    else static_cast<float*>(out)[idx] = (float)(c8 * s);
}

// Packed FP32 pairs (sm_100-class f32x2 add / mul / fma on a register pair).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// j-range split: `splits` contiguous ranges of whole tiles, as equal as
// possible (split k holds tiles [k T / s, (k + 1) T / s) of the T = ceil(N /
// NT) tiles), so that any split count is exact.  Returns the launched split
// count s = min(splits, T) and the tile count T.
inline int64_t split_plan(int64_t N, int NT, int splits, int64_t* ntiles) {
    if (splits < 1) splits = 1;
    *ntiles = (N + NT - 1) / NT;
    return splits < *ntiles ? splits : *ntiles;
}

// This CTA's j-range [jb, je) for split blockIdx.y of gridDim.y.
__device__ __forceinline__ void split_range(int64_t N, int NT, int64_t ntiles, int64_t* jb, int64_t* je) {
    const int64_t k = blockIdx.y, s = gridDim.y;
    *jb = (k * ntiles / s) * NT;
    const int64_t e = ((k + 1) * ntiles / s) * NT;
    *je = e < N ? e : N;
}

}  // namespace
}  // namespace lmk
