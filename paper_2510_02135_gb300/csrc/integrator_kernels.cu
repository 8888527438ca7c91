// Pieces of the time stepping: the soft steric forces of Eq. (soft_potential)
// and the update of the stochastic Adams-Bashforth scheme (the roller example,
// Sec. 5.1 of the libMobility paper), and the combination of the three terms
// of Eq. (bdhi) into Langevin velocities (Sec. 3.2, LangevinVelocities).
//
// Soft repulsion, a direct O(N^2) sum in the layout of the mobility kernels
// (one i per thread, j-tiles of positions in shared memory):
//   F_i = sum_j (U0 / b) g(r_ij) (x_i - x_j) / r_ij  +  z (U0 / b) g_w(z_i),
//   g(r) = 1 for r < d, exp((d - r) / b) otherwise (d = d_pair; d_wall and
//   the height z_i for the wall), r = 0 pairs skipped.
#include <cuda_runtime.h>

#include <cstdint>

#include "lm_internal.cuh"

namespace lmk {
namespace {

template <typename R> struct P4;
template <> struct P4<float> { using type = float4; };
template <> struct P4<double> { using type = lmk::dvec4; };

template <typename R>
__device__ __forceinline__ R ld3(const void* p, int f64, int64_t idx) {
    return f64 ? (R)(static_cast<const double*>(p)[idx]) : (R)(static_cast<const float*>(p)[idx]);
}
__device__ __forceinline__ float expo(float x) { return expf(x); }
__device__ __forceinline__ double expo(double x) { return exp(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

template <typename R, int NT>
__global__ void __launch_bounds__(NT) soft_repulsion_kernel(const void* __restrict__ pos, int f64, int64_t N, R U0b,
                                                            R inv_b, R d_pair, R d_wall, int wall, R z_wall,
                                                            void* __restrict__ out) {
    using R4 = typename P4<R>::type;
    __shared__ R4 sp[NT];
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    const bool live = i < N;
    const int64_t ii = live ? i : 0;
    const R xi = ld3<R>(pos, f64, 3 * ii), yi = ld3<R>(pos, f64, 3 * ii + 1), zi = ld3<R>(pos, f64, 3 * ii + 2);
    R fx = R(0), fy = R(0), fz = R(0);
    for (int64_t jt = 0; jt < N; jt += NT) {
        const int64_t j = jt + threadIdx.x;
        R4 v;
        if (j < N) {
            v.x = ld3<R>(pos, f64, 3 * j); v.y = ld3<R>(pos, f64, 3 * j + 1); v.z = ld3<R>(pos, f64, 3 * j + 2);
            v.w = R(1);
        } else {
            v.x = v.y = v.z = R(0); v.w = R(0);   // w = 0 marks an empty slot
        }
        __syncthreads();
        sp[threadIdx.x] = v;
        __syncthreads();
        const int cnt = (N - jt < NT) ? (int)(N - jt) : NT;
        for (int jj = 0; jj < cnt; ++jj) {
            const R4 p = sp[jj];
            const R dx = xi - p.x, dy = yi - p.y, dz = zi - p.z;
            const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (r2 > R(0)) {
                const R ir = rsq(r2);
                const R r = r2 * ir;
                const R g = (r < d_pair) ? R(1) : expo((d_pair - r) * inv_b);
                const R c = U0b * g * ir;
                fx = fma(c, dx, fx);
                fy = fma(c, dy, fy);
                fz = fma(c, dz, fz);
            }
        }
    }
    if (!live) return;
    if (wall) {
        const R h = zi - z_wall;   // height above the wall
        fz += U0b * ((h < d_wall) ? R(1) : expo((d_wall - h) * inv_b));
    }
    if (f64) {
        double* o = static_cast<double*>(out);
        o[3 * i] = fx; o[3 * i + 1] = fy; o[3 * i + 2] = fz;
    } else {
        float* o = static_cast<float*>(out);
        o[3 * i] = (float)fx; o[3 * i + 1] = (float)fy; o[3 * i + 2] = (float)fz;
    }
}

// X' = X + dt [(3/2) u - (1/2) u_prev + kT ((3/2) d - (1/2) d_prev)] + y
// (y = sqrt(2 kT dt) (M^{1/2} W)_lin, already scaled, in the position
// precision); u, d FP64 (3N);
// hist = [u_prev (3N); d_prev (3N)] is read unless first, then overwritten
// with (u, d).
__global__ void ab_update_kernel(const void* __restrict__ pos, int f64, const double* __restrict__ u,
                                 const double* __restrict__ d, const void* __restrict__ y,
                                 double* __restrict__ hist, int first, double kT, double dt, int64_t n3,
                                 void* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n3) return;
    const double ue = u[e], de = d ? d[e] : 0.0;
    const double up = first ? ue : hist[e];
    const double dp = first ? de : hist[n3 + e];
    const double x = f64 ? static_cast<const double*>(pos)[e] : (double)static_cast<const float*>(pos)[e];
    const double ye = f64 ? static_cast<const double*>(y)[e] : (double)static_cast<const float*>(y)[e];
    const double xn = x + dt * ((1.5 * ue - 0.5 * up) + kT * (1.5 * de - 0.5 * dp)) + ye;
    hist[e] = ue;
    hist[n3 + e] = de;
    if (f64) static_cast<double*>(out)[e] = xn;
    else static_cast<float*>(out)[e] = (float)xn;
}

// Langevin velocities (Eq. bdhi divided by dt): u + kT d + y over the grand
// vector; lin gets entries [0, 3N), ang [3N, 6N).
__global__ void langevin_combine_kernel(const double* __restrict__ u, const double* __restrict__ d,
                                        const void* __restrict__ y, double kT, int64_t N, int angular,
                                        void* __restrict__ lin, void* __restrict__ ang, int out_f64) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n3 = 3 * N;
    if (e >= (angular ? 2 * n3 : n3)) return;
    const double ye = out_f64 ? static_cast<const double*>(y)[e] : (double)static_cast<const float*>(y)[e];
    const double v = u[e] + (d ? kT * d[e] : 0.0) + ye;
    void* out = (e < n3) ? lin : ang;
    const int64_t k = (e < n3) ? e : e - n3;
    if (out_f64) static_cast<double*>(out)[k] = v;
    else static_cast<float*>(out)[k] = (float)v;
}

}  // namespace

cudaError_t launch_langevin_combine(const double* u, const double* d, const void* y, double kT, int64_t N,
                                    int angular, void* lin, void* ang, int out_f64, cudaStream_t s) {
    const int64_t tot = (angular ? 6 : 3) * N;
    if (tot <= 0) return cudaSuccess;
    langevin_combine_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(u, d, y, kT, N, angular, lin, ang, out_f64);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_soft_repulsion(const void* pos, int f64, int64_t N, double U0, double b, double d_pair,
                                  double d_wall, int wall, double z_wall, void* out, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    constexpr int NT = 256;
    const unsigned blocks = (unsigned)((N + NT - 1) / NT);
    if (f64)
        soft_repulsion_kernel<double, NT><<<blocks, NT, 0, s>>>(pos, 1, N, U0 / b, 1.0 / b, d_pair, d_wall, wall,
                                                                z_wall, out);
    else
        soft_repulsion_kernel<float, NT><<<blocks, NT, 0, s>>>(pos, 0, N, (float)(U0 / b), (float)(1.0 / b),
                                                               (float)d_pair, (float)d_wall, wall, (float)z_wall, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ab_update(const void* pos, int f64, const double* u, const double* d, const void* y,
                             double* hist, int first, double kT, double dt, int64_t N, void* out, cudaStream_t s) {
    const int64_t n3 = 3 * N;
    if (n3 <= 0) return cudaSuccess;
    ab_update_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(pos, f64, u, d, y, hist, first, kT, dt, n3, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lmk
