// Mobility product above a single no-slip wall at z = 0 (NBody with z =
// "single_wall", Sec. 3.5 of the libMobility paper: the Swan-Brady kernel,
// with the damping of particles that overlap the wall).
//
// Each pair block is the free-space RPY block of the open solver plus a wall
// part: the Faxen operators applied to the image system of the Blake Green's
// function.  With R = x_i - x_j* (x_j* the mirror image of the source j),
// rho = |R|, e = R / rho, c = e_z, h = z_j, alpha = a^2 / rho^2, H = h / rho
// and w = e x z, the wall part acting on F_j, T_j is (units 1/(8 pi eta)):
//   u += [A F + (B (e.F) + C F_z) e + (D (e.F) + E F_z) z] / rho
//      + [e x T + K1 z x T + (K2 e + K3 z)(w.T)] / rho^2
//   w += [e x F + L1 z x F + (L2 (e.F) + L3 F_z) w] / rho^2
//      + [(7/2 - 6c^2) T - (9/2)(e.T) e + 3c T_z e + 6c (e.T) z - 3 T_z z] / rho^3
//   A = -1 + 2H^2 - 2cH + alpha (2c^2 - 2/3) + alpha^2 (2/3 - 10c^2/3)
//   B = -1 - 6H^2 + 6cH + alpha (2 - 10c^2) + alpha^2 (70c^2/3 - 10/3)
//   C = 2H + 12cH^2 - 12c^2 H + alpha c (20c^2 - 4) + alpha^2 c (40/3 - 140c^2/3)
//   D = 2H - (20/3) alpha^2 c
//   E = -4H^2 - 4 alpha c^2 + alpha^2 (20c^2 - 8/3)
//   K1 = -2 (alpha c + H), K2 = 2 (5 alpha c - 3c + 3H), K3 = -2 alpha
//   L1 = 2 (alpha c - H),  L2 = 2 (5 alpha c - 3H),      L3 = -2 (10 alpha c^2 - alpha - 6cH)
// The same expressions hold for i = j (R = 2h z): the single-sphere wall
// corrections.
//
// Damping: set_positions stores each particle at height max(z, a) and its
// factor f = clamp(z / a, 0, 1) in the fourth component of the packed
// position.  The j-tile loader multiplies F_j, T_j by f_j and the result is
// multiplied by f_i, which gives M = D M(clamped) D, D = diag(f).
//
// Schedule: as the open kernel (register-blocked i, shared-memory j-tiles,
// warp vote for the overlap branch of the free part, TwoSum fold per tile,
// j-range splits).  The wall part needs no branch: clamped heights keep
// rho >= 2a.
#include <cuda_runtime.h>

#include <cstdint>

#include "lm_internal.cuh"
#include "pair_common.cuh"

namespace lmk {
namespace {

// Wall part of one pair.  th holds -T_j / 2 (the tile convention of the
// free-space part), a2 = a^2.
template <typename R, bool ANG>
__device__ __forceinline__ void wall_pair(R Rx, R Ry, R Rz, R hj, const typename V4<R>::type& f,
                                          const typename V4<R>::type& th, R a2, Acc<R, ANG>& acc) {
    const R u = rsq(fma(Rx, Rx, fma(Ry, Ry, Rz * Rz)));
    const R ex = Rx * u, ey = Ry * u, c = Rz * u;
    const R H = hj * u;
    const R al = a2 * u * u;
    const R al2 = al * al;
    const R c2 = c * c, H2 = H * H, cH = c * H;
    const R A = R(-1) + R(2) * H2 - R(2) * cH + al * (R(2) * c2 - R(2.0 / 3.0)) +
                al2 * (R(2.0 / 3.0) - R(10.0 / 3.0) * c2);
    const R B = R(-1) - R(6) * H2 + R(6) * cH + al * (R(2) - R(10) * c2) + al2 * (R(70.0 / 3.0) * c2 - R(10.0 / 3.0));
    const R C = R(2) * H + R(12) * cH * H - R(12) * c * cH + al * c * (R(20) * c2 - R(4)) +
                al2 * c * (R(40.0 / 3.0) - R(140.0 / 3.0) * c2);
    const R D = R(2) * H - R(20.0 / 3.0) * al2 * c;
    const R E = R(-4) * H2 - R(4) * al * c2 + al2 * (R(20) * c2 - R(8.0 / 3.0));
    const R eF = fma(ex, f.x, fma(ey, f.y, c * f.z));
    const R pe = fma(B, eF, C * f.z);
    const R pz = fma(D, eF, E * f.z);
    acc.p[0] = fma(u, fma(A, f.x, pe * ex), acc.p[0]);
    acc.p[1] = fma(u, fma(A, f.y, pe * ey), acc.p[1]);
    acc.p[2] = fma(u, fma(A, f.z, fma(pe, c, pz)), acc.p[2]);
    if constexpr (ANG) {
        const R Tx = R(-2) * th.x, Ty = R(-2) * th.y, Tz = R(-2) * th.z;
        const R u2 = u * u;
        // u += [e x T + K1 z x T + (K2 e + K3 z)(w.T)] / rho^2
        const R K1 = R(-2) * fma(al, c, H);
        const R K2 = R(2) * (R(5) * al * c - R(3) * c + R(3) * H);
        const R K3 = R(-2) * al;
        const R wT = fma(ey, Tx, -(ex * Ty));
        acc.p[0] = fma(u2, fma(ey, Tz, -(c * Ty)) - K1 * Ty + K2 * wT * ex, acc.p[0]);
        acc.p[1] = fma(u2, fma(c, Tx, -(ex * Tz)) + K1 * Tx + K2 * wT * ey, acc.p[1]);
        acc.p[2] = fma(u2, fma(ex, Ty, -(ey * Tx)) + fma(K2, c, K3) * wT, acc.p[2]);
        // w += [e x F + L1 z x F + (L2 (e.F) + L3 F_z) w] / rho^2
        const R L1 = R(2) * (al * c - H);
        const R L2 = R(2) * (R(5) * al * c - R(3) * H);
        const R L3 = R(-2) * (R(10) * al * c2 - al - R(6) * cH);
        const R q = fma(L2, eF, L3 * f.z);
        acc.p[3] = fma(u2, fma(ey, f.z, -(c * f.y)) - L1 * f.y + q * ey, acc.p[3]);
        acc.p[4] = fma(u2, fma(c, f.x, -(ex * f.z)) + L1 * f.x - q * ex, acc.p[4]);
        acc.p[5] = fma(u2, fma(ex, f.y, -(ey * f.x)), acc.p[5]);
        // w += [(7/2 - 6c^2) T - (9/2)(e.T) e + 3c T_z e + 6c (e.T) z - 3 T_z z] / rho^3
        const R u3 = u2 * u;
        const R eT = fma(ex, Tx, fma(ey, Ty, c * Tz));
        const R Ar = R(3.5) - R(6) * c2;
        const R pr = fma(R(-4.5), eT, R(3) * c * Tz);
        acc.p[3] = fma(u3, fma(Ar, Tx, pr * ex), acc.p[3]);
        acc.p[4] = fma(u3, fma(Ar, Ty, pr * ey), acc.p[4]);
        acc.p[5] = fma(u3, fma(Ar, Tz, fma(pr, c, fma(R(6) * c, eT, R(-3) * Tz))), acc.p[5]);
    }
}

template <typename R, bool ANG, int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_wall_kernel(const typename V4<R>::type* __restrict__ pos4,
                                                      const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                      int in_f64, int64_t N, int64_t jchunk, RpyConst<R> k, R a2,
                                                      double c8, void* __restrict__ lin, void* __restrict__ ang,
                                                      int out_f64, double* __restrict__ partials) {
    using R4 = typename V4<R>::type;
    constexpr int C = ANG ? 6 : 3;
    __shared__ R4 sp[NT];
    __shared__ R4 sf[NT];
    __shared__ R4 sh[ANG ? NT : 1];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    R* s_hi = reinterpret_cast<R*>(dyn_smem);              // [c][q][tid]
    R* s_lo = s_hi + (sizeof(R) == 4 ? C * NI * NT : 0);     // FP32 only

    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * (NT * NI);
    const int64_t jb = (int64_t)blockIdx.y * jchunk;
    const int64_t je = (jb + jchunk < N) ? (jb + jchunk) : N;
    const R pad = (R)kPadCoord;

    R xi[NI], yi[NI], zi[NI], fi[NI];
    Acc<R, ANG> acc[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i < N) {
            const R4 p = pos4[i];
            xi[q] = p.x; yi[q] = p.y; zi[q] = p.z; fi[q] = p.w;
        } else {
            // far from every particle, above the wall
            xi[q] = -pad; yi[q] = -pad; zi[q] = pad; fi[q] = R(0);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            acc[q].p[c] = R(0);
            s_hi[(c * NI + q) * NT + tid] = R(0);
            if (sizeof(R) == 4) s_lo[(c * NI + q) * NT + tid] = R(0);
        }
    }

    // register prefetch of this thread's j in the next tile: position, f F, -f T / 2
    R4 np, nf, nh;
    auto fetch = [&](int64_t j) {
        if (j < je) {
            np = pos4[j];
            const R fj = np.w;
            nf.x = fj * load_elem<R>(Fp, in_f64, 3 * j + 0);
            nf.y = fj * load_elem<R>(Fp, in_f64, 3 * j + 1);
            nf.z = fj * load_elem<R>(Fp, in_f64, 3 * j + 2);
            if constexpr (ANG) {
                const R hf = R(-0.5) * fj;
                nh.x = hf * load_elem<R>(Tp, in_f64, 3 * j + 0);
                nh.y = hf * load_elem<R>(Tp, in_f64, 3 * j + 1);
                nh.z = hf * load_elem<R>(Tp, in_f64, 3 * j + 2);
            }
        } else {
            np.x = pad; np.y = pad; np.z = pad;
            nf.x = R(0); nf.y = R(0); nf.z = R(0);
            nh.x = R(0); nh.y = R(0); nh.z = R(0);
        }
        np.w = R(0); nf.w = R(0); nh.w = R(0);
    };
    fetch(jb + tid);

    for (int64_t jt = jb; jt < je; jt += NT) {
        sp[tid] = np;
        sf[tid] = nf;
        if constexpr (ANG) sh[tid] = nh;
        __syncthreads();
        if (jt + NT < je) fetch(jt + NT + tid);

#pragma unroll 1
        for (int jj = 0; jj < NT; ++jj) {
            const R4 pj = sp[jj];
            const R4 fj = sf[jj];
            R4 hj;
            if constexpr (ANG) hj = sh[jj]; else { hj.x = hj.y = hj.z = hj.w = R(0); }
            R dx[NI], dy[NI], dz[NI], r2[NI];
            R mn;
#pragma unroll
            for (int q = 0; q < NI; ++q) {
                dx[q] = xi[q] - pj.x;
                dy[q] = yi[q] - pj.y;
                dz[q] = zi[q] - pj.z;
                r2[q] = fma(dx[q], dx[q], fma(dy[q], dy[q], dz[q] * dz[q]));
                mn = (q == 0) ? r2[q] : fmin(mn, r2[q]);
            }
            if (__any_sync(0xffffffffu, mn < k.four_a2)) {
#pragma unroll
                for (int q = 0; q < NI; ++q) pair_exact<R, ANG>(dx[q], dy[q], dz[q], r2[q], fj, hj, k, acc[q]);
            } else {
#pragma unroll
                for (int q = 0; q < NI; ++q) pair_far<R, ANG>(dx[q], dy[q], dz[q], r2[q], fj, hj, k, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < NI; ++q) wall_pair<R, ANG>(dx[q], dy[q], zi[q] + pj.z, pj.z, fj, hj, a2, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < NI; ++q) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int o = (c * NI + q) * NT + tid;
                fold(&s_hi[o], &s_lo[o], acc[q].p[c]);
            }
        }
        __syncthreads();
    }

    const bool direct = (gridDim.y == 1);
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int o = (c * NI + q) * NT + tid;
            const double v = (double)fi[q] * ((double)s_hi[o] + (sizeof(R) == 4 ? (double)s_lo[o] : 0.0));
            if (direct) {
                void* out = (c < 3) ? lin : ang;
                const int64_t idx = 3 * i + (c % 3);
                if (out_f64) static_cast<double*>(out)[idx] = c8 * v;
                else static_cast<float*>(out)[idx] = (float)(c8 * v);
            } else {
                partials[((int64_t)blockIdx.y * C + c) * N + i] = v;
            }
        }
    }
}

template <typename R, bool ANG, int NT, int NI>
cudaError_t launch_wall_t(const MdotArgs& a, cudaStream_t s) {
    const int64_t per_cta = (int64_t)NT * NI;
    const int64_t nblk = (a.N + per_cta - 1) / per_cta;
    int64_t jchunk = 0;
    const int splits = (int)split_plan(a.N, NT, a.splits, &jchunk);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<R> k = make_rpy_const<R>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    constexpr size_t dyn = running_sum_bytes<R, ANG, NT, NI>();
    static bool attr_set = false;  // per instantiation; the attribute is process-wide
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(rpy_wall_kernel<R, ANG, NT, NI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
    rpy_wall_kernel<R, ANG, NT, NI><<<grid, NT, dyn, s>>>(
        static_cast<const typename V4<R>::type*>(a.pos4), a.F, ANG ? a.T : nullptr, a.in_f64, a.N, jchunk, k,
        (R)(a.a * a.a), c8, a.lin, a.ang, a.out_f64, a.partials);
    cudaError_t err = cudaGetLastError();
    if (a.ev_end) cudaEventRecord(a.ev_end, s);
    count_launches(1);
    if (err != cudaSuccess || splits == 1) return err;
    constexpr int C = ANG ? 6 : 3;
    const int64_t tot = (int64_t)C * a.N;
    reduce_splits_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.partials, splits, C, a.N, c8, a.lin,
                                                                        a.ang, a.out_f64);
    count_launches(1);
    return cudaGetLastError();
}

// Configurations: FP32 threads {128, 256} x ilp {1, 2, 4}; FP64 threads {128, 256} x ilp 1.
template <typename R, bool ANG>
cudaError_t launch_wall_r(const MdotArgs& a, cudaStream_t s) {
    if (a.threads == 128 && a.ilp == 1) return launch_wall_t<R, ANG, 128, 1>(a, s);
    if (a.threads == 256 && a.ilp == 1) return launch_wall_t<R, ANG, 256, 1>(a, s);
    if constexpr (sizeof(R) == 4) {
        if (a.threads == 128 && a.ilp == 2) return launch_wall_t<R, ANG, 128, 2>(a, s);
        if (a.threads == 128 && a.ilp == 4) return launch_wall_t<R, ANG, 128, 4>(a, s);
        if (a.threads == 256 && a.ilp == 2) return launch_wall_t<R, ANG, 256, 2>(a, s);
        if (a.threads == 256 && a.ilp == 4) return launch_wall_t<R, ANG, 256, 4>(a, s);
    }
    return cudaErrorInvalidConfiguration;
}

template <typename R, bool ANG>
int wall_occupancy_r(int threads, int ilp) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidConfiguration;
#define LM_WOCC(NT, NI)                                                                            \
    if (threads == NT && ilp == NI) {                                                              \
        constexpr size_t dyn = running_sum_bytes<R, ANG, NT, NI>();                                \
        e = cudaFuncSetAttribute(rpy_wall_kernel<R, ANG, NT, NI>,                                  \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);           \
        if (e == cudaSuccess)                                                                      \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_wall_kernel<R, ANG, NT, NI>, \
                                                              NT, dyn);                            \
    }
    LM_WOCC(128, 1) LM_WOCC(256, 1)
    if constexpr (sizeof(R) == 4) {
        LM_WOCC(128, 2) LM_WOCC(128, 4) LM_WOCC(256, 2) LM_WOCC(256, 4)
    }
#undef LM_WOCC
    return e == cudaSuccess ? n : 0;
}

}  // namespace

bool wall_config_supported(int fp64, int threads, int ilp, int packed) {
    if (packed) return false;
    if (threads != 128 && threads != 256) return false;
    return fp64 ? ilp == 1 : (ilp == 1 || ilp == 2 || ilp == 4);
}

int wall_ctas_per_sm(int fp64, int angular, int threads, int ilp) {
    if (fp64) return angular ? wall_occupancy_r<double, true>(threads, ilp) : wall_occupancy_r<double, false>(threads, ilp);
    return angular ? wall_occupancy_r<float, true>(threads, ilp) : wall_occupancy_r<float, false>(threads, ilp);
}

cudaError_t launch_wall_mdot(const MdotArgs& a, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    if (a.packed) return cudaErrorInvalidConfiguration;
    if (a.fp64) return a.angular ? launch_wall_r<double, true>(a, s) : launch_wall_r<double, false>(a, s);
    return a.angular ? launch_wall_r<float, true>(a, s) : launch_wall_r<float, false>(a, s);
}

// --------------------------------------------------------------------------
// Position packing for the wall geometry: clamp heights to a, store the
// damping factor in the fourth component, flag non-finite or too large
// coordinates.
// --------------------------------------------------------------------------
namespace {
template <typename RO>
__global__ void pack_wall_positions_kernel(const void* __restrict__ pos, int in_f64, int64_t N, double a,
                                           typename V4<RO>::type* __restrict__ out, int* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double x, y, z;
    if (in_f64) {
        const double* p = static_cast<const double*>(pos);
        x = p[3 * i]; y = p[3 * i + 1]; z = p[3 * i + 2];
    } else {
        const float* p = static_cast<const float*>(pos);
        x = p[3 * i]; y = p[3 * i + 1]; z = p[3 * i + 2];
    }
    const double m = kMaxAbsCoord;
    if (!(fabs(x) <= m && fabs(y) <= m && fabs(z) <= m)) atomicExch(bad, 1);
    double f = z / a;
    f = f > 0.0 ? (f < 1.0 ? f : 1.0) : 0.0;
    typename V4<RO>::type v;
    v.x = (RO)x; v.y = (RO)y; v.z = (RO)(z > a ? z : a); v.w = (RO)f;
    out[i] = v;
}
// RFD support: pack x + scale * W (W: 3N doubles) the same way, and form
// (P - Q) / delta from two FP64 products.
template <typename RO>
__global__ void displace_pack_wall_kernel(const void* __restrict__ pos, int in_f64, const double* __restrict__ W,
                                          double scale, int64_t N, double a, typename V4<RO>::type* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double x, y, z;
    if (in_f64) {
        const double* p = static_cast<const double*>(pos);
        x = p[3 * i]; y = p[3 * i + 1]; z = p[3 * i + 2];
    } else {
        const float* p = static_cast<const float*>(pos);
        x = p[3 * i]; y = p[3 * i + 1]; z = p[3 * i + 2];
    }
    x = fma(scale, W[3 * i], x);
    y = fma(scale, W[3 * i + 1], y);
    z = fma(scale, W[3 * i + 2], z);
    double f = z / a;
    f = f > 0.0 ? (f < 1.0 ? f : 1.0) : 0.0;
    typename V4<RO>::type v;
    v.x = (RO)x; v.y = (RO)y; v.z = (RO)(z > a ? z : a); v.w = (RO)f;
    out[i] = v;
}

// out (lin: rows [0, 3N), ang: rows [3N, 6N) of P, Q) = (P - Q) * inv_delta
__global__ void rfd_difference_kernel(const double* __restrict__ P, const double* __restrict__ Q, double inv_delta,
                                      int64_t N, int angular, void* __restrict__ lin, void* __restrict__ ang,
                                      int out_f64) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n3 = 3 * N;
    if (e >= (angular ? 2 * n3 : n3)) return;
    const double v = (P[e] - Q[e]) * inv_delta;
    void* out = (e < n3) ? lin : ang;
    const int64_t k = (e < n3) ? e : e - n3;
    if (out_f64) static_cast<double*>(out)[k] = v;
    else static_cast<float*>(out)[k] = (float)v;
}
}  // namespace

cudaError_t launch_displace_pack_wall(const void* pos, int in_f64, const double* W, double scale, int64_t N,
                                      double a, void* pos4, int out_f64, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (out_f64)
        displace_pack_wall_kernel<double><<<blocks, 256, 0, s>>>(pos, in_f64, W, scale, N, a, static_cast<dvec4*>(pos4));
    else
        displace_pack_wall_kernel<float><<<blocks, 256, 0, s>>>(pos, in_f64, W, scale, N, a, static_cast<float4*>(pos4));
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rfd_difference(const double* P, const double* Q, double inv_delta, int64_t N, int angular,
                                  void* lin, void* ang, int out_f64, cudaStream_t s) {
    const int64_t tot = (angular ? 6 : 3) * N;
    if (tot <= 0) return cudaSuccess;
    rfd_difference_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P, Q, inv_delta, N, angular, lin, ang, out_f64);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_wall_positions(const void* pos, int in_f64, int64_t N, double a, void* pos4, int out_f64,
                                       int* bad, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (out_f64)
        pack_wall_positions_kernel<double><<<blocks, 256, 0, s>>>(pos, in_f64, N, a, static_cast<dvec4*>(pos4), bad);
    else
        pack_wall_positions_kernel<float><<<blocks, 256, 0, s>>>(pos, in_f64, N, a, static_cast<float4*>(pos4), bad);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lmk
