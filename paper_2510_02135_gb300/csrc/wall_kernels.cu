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
// Damping: set_positions stores each particle at height max(z - z_wall, a) and its
// factor f = clamp(z / a, 0, 1) in the fourth component of the packed
// position.  The j-tile loader multiplies F_j, T_j by f_j and the result is
// multiplied by f_i, which gives M = D M(clamped) D, D = diag(f).
//
// Schedule: as the open kernel (register-blocked i, shared-memory j-tiles,
// warp vote for the overlap branch of the free part, TwoSum fold per tile,
// j-range splits), in a scalar and a packed f32x2 form.  The wall part needs
// no branch: clamped heights keep rho >= 2a.
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
                                                      int in_f64, int64_t N, int64_t ntiles, RpyConst<R> k, R a2,
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
    int64_t jb, je;
    split_range(N, NT, ntiles, &jb, &je);
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
        if (j < je && LM_INBOUNDS(j >= 0 && j < N, 7, j)) {
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

// ---------------------------------------------------------------------------
// Packed FP32 form of the wall kernel: two i-particles per f32x2
// instruction, as the packed open kernel.  The j-tile holds every operand as
// a plain scalar that enters packed instructions in both lanes (packed
// operands carry no negation): -x_j, f F_j, f T_j, their negatives,
// -f T_j / 2, 3 f T_j / 2 and +z_j (the image height), in the word layout of
// the open kernel with z_j after 3 f Tz / 2 (translation only: (-x, -y, -z,
// f Fx) (f Fy, f Fz, z_j, 0)).  The wall part below is the formula of
// wall_pair with every sign folded into a constant or a tile slot.
// ---------------------------------------------------------------------------
template <bool ANG>
constexpr int wall_x2_words() { return ANG ? 6 : 2; }

template <bool ANG, int NT, int NI>
constexpr size_t wall_x2_smem_bytes() {
    return (size_t)wall_x2_words<ANG>() * NT * sizeof(float4) + running_sum_bytes<float, ANG, NT, NI>();
}

// Wall part of two pairs (one per lane) for the source j.  Rx, Ry: x_i - x_j;
// zi, zj: clamped heights; f*, mf*: f F_j and -f F_j; T*, mT*: f T_j and -f T_j.
template <bool ANG>
__device__ __forceinline__ void wall_pair2(float2 Rx, float2 Ry, float2 zi, float2 zj, float2 a2,
                                           float2 fx, float2 fy, float2 fz, float2 mfx, float2 mfy, float2 mfz,
                                           float2 Tx, float2 Ty, float2 Tz, float2 mTx, float2 mTy, float2 mTz,
                                           float2* acc) {
    const float2 Rz = add2(zi, zj);
    const float2 r2 = fma2(Rx, Rx, fma2(Ry, Ry, mul2(Rz, Rz)));
    const float2 u = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 ex = mul2(Rx, u), ey = mul2(Ry, u), c = mul2(Rz, u);
    const float2 H = mul2(zj, u);
    const float2 al = mul2(mul2(a2, u), u);
    const float2 al2 = mul2(al, al);
    const float2 c2 = mul2(c, c), H2 = mul2(H, H), cH = mul2(c, H);
    const float2 alc = mul2(al, c), al2c = mul2(al2, c);
    // A = -1 + 2H^2 - 2cH + alpha (2c^2 - 2/3) + alpha^2 (2/3 - 10c^2/3)
    const float2 A = fma2(al2, fma2(bc2(-10.f / 3.f), c2, bc2(2.f / 3.f)),
                          fma2(al, fma2(bc2(2.f), c2, bc2(-2.f / 3.f)),
                               fma2(bc2(2.f), H2, fma2(bc2(-2.f), cH, bc2(-1.f)))));
    // B = -1 - 6H^2 + 6cH + alpha (2 - 10c^2) + alpha^2 (70c^2/3 - 10/3)
    const float2 B = fma2(al2, fma2(bc2(70.f / 3.f), c2, bc2(-10.f / 3.f)),
                          fma2(al, fma2(bc2(-10.f), c2, bc2(2.f)),
                               fma2(bc2(-6.f), H2, fma2(bc2(6.f), cH, bc2(-1.f)))));
    // C = 2H + 12 cH (H - c) + alpha c (20c^2 - 4) + alpha^2 c (40/3 - 140c^2/3)
    const float2 C = fma2(al2c, fma2(bc2(-140.f / 3.f), c2, bc2(40.f / 3.f)),
                          fma2(alc, fma2(bc2(20.f), c2, bc2(-4.f)),
                               fma2(mul2(bc2(12.f), cH), fma2(bc2(-1.f), c, H), mul2(bc2(2.f), H))));
    // D = 2H - (20/3) alpha^2 c
    const float2 D = fma2(bc2(-20.f / 3.f), al2c, mul2(bc2(2.f), H));
    // E = -4H^2 - 4 alpha c^2 + alpha^2 (20c^2 - 8/3)
    const float2 E = fma2(al2, fma2(bc2(20.f), c2, bc2(-8.f / 3.f)), fma2(bc2(-4.f), mul2(al, c2), mul2(bc2(-4.f), H2)));
    const float2 eF = fma2(ex, fx, fma2(ey, fy, mul2(c, fz)));
    const float2 pe = fma2(B, eF, mul2(C, fz));
    const float2 pz = fma2(D, eF, mul2(E, fz));
    acc[0] = fma2(u, fma2(A, fx, mul2(pe, ex)), acc[0]);
    acc[1] = fma2(u, fma2(A, fy, mul2(pe, ey)), acc[1]);
    acc[2] = fma2(u, fma2(A, fz, fma2(pe, c, pz)), acc[2]);
    if constexpr (ANG) {
        const float2 u2 = mul2(u, u);
        // u += [e x T + K1 z x T + (K2 e + K3 z)(w.T)] / rho^2, with -K1 = 2 (alpha c + H)
        const float2 K1n = mul2(bc2(2.f), add2(alc, H));
        const float2 K2 = mul2(bc2(2.f), fma2(bc2(5.f), alc, fma2(bc2(-3.f), c, mul2(bc2(3.f), H))));
        const float2 K3 = mul2(bc2(-2.f), al);
        const float2 wT = fma2(ey, Tx, mul2(ex, mTy));
        const float2 K2wT = mul2(K2, wT);
        acc[0] = fma2(u2, fma2(ey, Tz, fma2(c, mTy, fma2(K1n, Ty, mul2(K2wT, ex)))), acc[0]);
        acc[1] = fma2(u2, fma2(c, Tx, fma2(ex, mTz, fma2(K1n, mTx, mul2(K2wT, ey)))), acc[1]);
        acc[2] = fma2(u2, fma2(ex, Ty, fma2(ey, mTx, mul2(fma2(K2, c, K3), wT))), acc[2]);
        // w += [e x F + L1 z x F + (L2 (e.F) + L3 F_z) w] / rho^2
        const float2 L1 = mul2(bc2(2.f), fma2(bc2(-1.f), H, alc));
        const float2 L2 = mul2(bc2(2.f), fma2(bc2(5.f), alc, mul2(bc2(-3.f), H)));
        const float2 L3 = mul2(bc2(-2.f), fma2(bc2(10.f), mul2(al, c2), fma2(bc2(-6.f), cH, mul2(bc2(-1.f), al))));
        const float2 q = fma2(L2, eF, mul2(L3, fz));
        const float2 qn = mul2(bc2(-1.f), q);
        acc[3] = fma2(u2, fma2(ey, fz, fma2(c, mfy, fma2(L1, mfy, mul2(q, ey)))), acc[3]);
        acc[4] = fma2(u2, fma2(c, fx, fma2(ex, mfz, fma2(L1, fx, mul2(qn, ex)))), acc[4]);
        acc[5] = fma2(u2, fma2(ex, fy, mul2(ey, mfx)), acc[5]);
        // w += [(7/2 - 6c^2) T - (9/2)(e.T) e + 3c T_z e + 6c (e.T) z - 3 T_z z] / rho^3
        const float2 u3 = mul2(u2, u);
        const float2 eT = fma2(ex, Tx, fma2(ey, Ty, mul2(c, Tz)));
        const float2 Ar = fma2(bc2(-6.f), c2, bc2(3.5f));
        const float2 pr = fma2(bc2(-4.5f), eT, mul2(mul2(bc2(3.f), c), Tz));
        acc[3] = fma2(u3, fma2(Ar, Tx, mul2(pr, ex)), acc[3]);
        acc[4] = fma2(u3, fma2(Ar, Ty, mul2(pr, ey)), acc[4]);
        acc[5] = fma2(u3, fma2(Ar, Tz, fma2(pr, c, fma2(mul2(bc2(6.f), c), eT, mul2(bc2(-3.f), Tz)))), acc[5]);
    }
}

template <bool ANG, int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_wall_x2_kernel(const float4* __restrict__ pos4,
                                                         const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                         int in_f64, int64_t N, int64_t ntiles, RpyConst<float> k,
                                                         float a2s, double c8, void* __restrict__ lin,
                                                         void* __restrict__ ang, int out_f64,
                                                         double* __restrict__ partials) {
    static_assert(NI % 2 == 0, "packed form needs an even number of i-particles per thread");
    constexpr int NP = NI / 2;
    constexpr int C = ANG ? 6 : 3;
    constexpr int W = wall_x2_words<ANG>();
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    float4* s_t = reinterpret_cast<float4*>(dyn_smem);                 // [w][jj]
    float* s_hi = reinterpret_cast<float*>(s_t + W * NT);              // [c][q][tid]
    float* s_lo = s_hi + C * NI * NT;

    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * (NT * NI);
    int64_t jb, je;
    split_range(N, NT, ntiles, &jb, &je);
    const float pad = (float)kPadCoord;

    float2 xi[NP], yi[NP], zi[NP], fi[NP];
    float2 acc[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float v[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = i0 + (int64_t)(2 * p + h) * NT + tid;
            if (i < N) {
                const float4 q = pos4[i];
                v[h][0] = q.x; v[h][1] = q.y; v[h][2] = q.z; v[h][3] = q.w;
            } else {
                // far from every particle, above the wall
                v[h][0] = -pad; v[h][1] = -pad; v[h][2] = pad; v[h][3] = 0.f;
            }
        }
        xi[p] = make_float2(v[0][0], v[1][0]);
        yi[p] = make_float2(v[0][1], v[1][1]);
        zi[p] = make_float2(v[0][2], v[1][2]);
        fi[p] = make_float2(v[0][3], v[1][3]);
#pragma unroll
        for (int c = 0; c < C; ++c) acc[p][c] = bc2(0.f);
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            s_hi[(c * NI + q) * NT + tid] = 0.f;
            s_lo[(c * NI + q) * NT + tid] = 0.f;
        }
    }
    const float2 K1 = bc2(k.K1);
    const float2 nK2 = bc2(-k.K2);
    const float2 a2 = bc2(a2s);

    // register prefetch of this thread's j of the next tile: position (w = f), f F, f T
    float4 np;
    float3 nf, nt;
    auto fetch = [&](int64_t j) {
        if (j < je && LM_INBOUNDS(j >= 0 && j < N, 7, j)) {
            np = pos4[j];
            const float fj = np.w;
            nf.x = fj * load_elem<float>(Fp, in_f64, 3 * j + 0);
            nf.y = fj * load_elem<float>(Fp, in_f64, 3 * j + 1);
            nf.z = fj * load_elem<float>(Fp, in_f64, 3 * j + 2);
            if constexpr (ANG) {
                nt.x = fj * load_elem<float>(Tp, in_f64, 3 * j + 0);
                nt.y = fj * load_elem<float>(Tp, in_f64, 3 * j + 1);
                nt.z = fj * load_elem<float>(Tp, in_f64, 3 * j + 2);
            }
        } else {
            np = make_float4(pad, pad, pad, 0.f);
            nf = make_float3(0.f, 0.f, 0.f);
            nt = make_float3(0.f, 0.f, 0.f);
        }
    };
    fetch(jb + tid);

    for (int64_t jt = jb; jt < je; jt += NT) {
        s_t[0 * NT + tid] = make_float4(-np.x, -np.y, -np.z, nf.x);
        if constexpr (ANG) {
            s_t[1 * NT + tid] = make_float4(nf.y, nf.z, -nf.x, -nf.y);
            s_t[2 * NT + tid] = make_float4(-nf.z, nt.x, nt.y, nt.z);
            s_t[3 * NT + tid] = make_float4(-nt.x, -nt.y, -nt.z, -0.5f * nt.x);
            s_t[4 * NT + tid] = make_float4(-0.5f * nt.y, -0.5f * nt.z, 1.5f * nt.x, 1.5f * nt.y);
            s_t[5 * NT + tid] = make_float4(1.5f * nt.z, np.z, 0.f, 0.f);
        } else {
            s_t[1 * NT + tid] = make_float4(nf.y, nf.z, np.z, 0.f);
        }
        __syncthreads();
        if (jt + NT < je) fetch(jt + NT + tid);

#pragma unroll 1
        for (int jj = 0; jj < NT; ++jj) {
            const float4 w0 = s_t[0 * NT + jj];
            const float4 w1 = s_t[1 * NT + jj];
            const float2 nx = bc2(w0.x), ny = bc2(w0.y), nz = bc2(w0.z);
            const float2 fx = bc2(w0.w), fy = bc2(w1.x), fz = bc2(w1.y);
            float2 mfx, mfy, mfz, Tx, Ty, Tz, mTx, mTy, mTz, hx, hy, hz, gx, gy, gz, zj;
            if constexpr (ANG) {
                const float4 w2 = s_t[2 * NT + jj];
                const float4 w3 = s_t[3 * NT + jj];
                const float4 w4 = s_t[4 * NT + jj];
                const float4 w5 = s_t[5 * NT + jj];
                mfx = bc2(w1.z); mfy = bc2(w1.w); mfz = bc2(w2.x);
                Tx = bc2(w2.y); Ty = bc2(w2.z); Tz = bc2(w2.w);
                mTx = bc2(w3.x); mTy = bc2(w3.y); mTz = bc2(w3.z);
                hx = bc2(w3.w); hy = bc2(w4.x); hz = bc2(w4.y);
                gx = bc2(w4.z); gy = bc2(w4.w); gz = bc2(w5.x);
                zj = bc2(w5.y);
            } else {
                zj = bc2(w1.z);
                mfx = mfy = mfz = Tx = Ty = Tz = mTx = mTy = mTz = bc2(0.f);
            }
            float2 dx[NP], dy[NP], dz[NP], r2[NP];
            float mn;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                dx[p] = add2(xi[p], nx);
                dy[p] = add2(yi[p], ny);
                dz[p] = add2(zi[p], nz);
                r2[p] = fma2(dx[p], dx[p], fma2(dy[p], dy[p], mul2(dz[p], dz[p])));
                const float m2 = fminf(r2[p].x, r2[p].y);
                mn = (p == 0) ? m2 : fminf(mn, m2);
            }
            // open-space far-field pair of slot p (two i-particles against j)
            auto far_slot = [&](int p) {
                const float2 invr = make_float2(rsqrtf(r2[p].x), rsqrtf(r2[p].y));
                const float2 invr2 = mul2(invr, invr);
                const float2 invr3 = mul2(invr2, invr);
                const float2 A = fma2(K1, invr3, invr);
                const float2 invr5 = mul2(invr3, invr2);
                const float2 B = fma2(nK2, invr5, invr3);
                const float2 dF = fma2(dx[p], fx, fma2(dy[p], fy, mul2(dz[p], fz)));
                const float2 sB = mul2(B, dF);
                acc[p][0] = fma2(sB, dx[p], fma2(A, fx, acc[p][0]));
                acc[p][1] = fma2(sB, dy[p], fma2(A, fy, acc[p][1]));
                acc[p][2] = fma2(sB, dz[p], fma2(A, fz, acc[p][2]));
                if constexpr (ANG) {
                    const float2 cx = fma2(Ty, dz[p], mul2(mTz, dy[p]));
                    const float2 cy = fma2(Tz, dx[p], mul2(mTx, dz[p]));
                    const float2 cz = fma2(Tx, dy[p], mul2(mTy, dx[p]));
                    acc[p][0] = fma2(invr3, cx, acc[p][0]);
                    acc[p][1] = fma2(invr3, cy, acc[p][1]);
                    acc[p][2] = fma2(invr3, cz, acc[p][2]);
                    const float2 vx = fma2(fy, dz[p], fma2(mfz, dy[p], hx));
                    const float2 vy = fma2(fz, dx[p], fma2(mfx, dz[p], hy));
                    const float2 vz = fma2(fx, dy[p], fma2(mfy, dx[p], hz));
                    const float2 t = mul2(invr5, fma2(dx[p], gx, fma2(dy[p], gy, mul2(dz[p], gz))));
                    acc[p][3] = fma2(t, dx[p], fma2(invr3, vx, acc[p][3]));
                    acc[p][4] = fma2(t, dy[p], fma2(invr3, vy, acc[p][4]));
                    acc[p][5] = fma2(t, dz[p], fma2(invr3, vz, acc[p][5]));
                }
            };
            if (__any_sync(0xffffffffu, mn < k.four_a2)) {
                // the exact scalar form only for the slots that hold an
                // overlapping (or self) pair somewhere in the warp
                const float4 fj = make_float4(fx.x, fy.x, fz.x, 0.f);
                float4 hj = make_float4(0.f, 0.f, 0.f, 0.f);
                if constexpr (ANG) hj = make_float4(hx.x, hy.x, hz.x, 0.f);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    if (__any_sync(0xffffffffu, fminf(r2[p].x, r2[p].y) < k.four_a2)) {
                        Acc<float, ANG> t0, t1;
#pragma unroll
                        for (int c = 0; c < C; ++c) { t0.p[c] = 0.f; t1.p[c] = 0.f; }
                        pair_exact<float, ANG>(dx[p].x, dy[p].x, dz[p].x, r2[p].x, fj, hj, k, t0);
                        pair_exact<float, ANG>(dx[p].y, dy[p].y, dz[p].y, r2[p].y, fj, hj, k, t1);
#pragma unroll
                        for (int c = 0; c < C; ++c) acc[p][c] = add2(acc[p][c], make_float2(t0.p[c], t1.p[c]));
                    } else {
                        far_slot(p);
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < NP; ++p) far_slot(p);
            }
            // the wall part: no branch (clamped heights keep rho >= 2a)
#pragma unroll
            for (int p = 0; p < NP; ++p)
                wall_pair2<ANG>(dx[p], dy[p], zi[p], zj, a2, fx, fy, fz, mfx, mfy, mfz, Tx, Ty, Tz, mTx, mTy, mTz,
                                acc[p]);
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int o0 = (c * NI + 2 * p) * NT + tid;
                const int o1 = o0 + NT;
                fold(&s_hi[o0], &s_lo[o0], acc[p][c].x);
                fold(&s_hi[o1], &s_lo[o1], acc[p][c].y);
            }
        }
        __syncthreads();
    }

    const bool direct = (gridDim.y == 1);
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i >= N) continue;
        const float f = (q & 1) ? fi[q >> 1].y : fi[q >> 1].x;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int o = (c * NI + q) * NT + tid;
            const double v = (double)f * ((double)s_hi[o] + (double)s_lo[o]);
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

template <bool ANG, int NT, int NI>
cudaError_t launch_wall_x2_t(const MdotArgs& a, cudaStream_t s) {
    const int64_t per_cta = (int64_t)NT * NI;
    const int64_t nblk = (a.N + per_cta - 1) / per_cta;
    int64_t ntiles = 0;
    const int splits = (int)split_plan(a.N, NT, a.splits, &ntiles);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<float> k = make_rpy_const<float>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    constexpr size_t dyn = wall_x2_smem_bytes<ANG, NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_wall_x2_kernel<ANG, NT, NI>, dyn)) return e;
    if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
    rpy_wall_x2_kernel<ANG, NT, NI><<<grid, NT, dyn, s>>>(static_cast<const float4*>(a.pos4), a.F,
                                                          ANG ? a.T : nullptr, a.in_f64, a.N, ntiles, k,
                                                          (float)(a.a * a.a), c8, a.lin, a.ang, a.out_f64,
                                                          a.partials);
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

// Packed wall configurations (FP32): threads {128, 256} x ilp {2, 4}.
template <bool ANG>
cudaError_t launch_wall_x2(const MdotArgs& a, cudaStream_t s) {
    if (a.threads == 128 && a.ilp == 2) return launch_wall_x2_t<ANG, 128, 2>(a, s);
    if (a.threads == 128 && a.ilp == 4) return launch_wall_x2_t<ANG, 128, 4>(a, s);
    if (a.threads == 256 && a.ilp == 2) return launch_wall_x2_t<ANG, 256, 2>(a, s);
    if (a.threads == 256 && a.ilp == 4) return launch_wall_x2_t<ANG, 256, 4>(a, s);
    return cudaErrorInvalidConfiguration;
}

template <bool ANG>
int wall_x2_occupancy(int threads, int ilp) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidConfiguration;
#define LM_WOCC2(NT, NI)                                                                                 \
    if (threads == NT && ilp == NI) {                                                                    \
        constexpr size_t dyn = wall_x2_smem_bytes<ANG, NT, NI>();                                        \
        e = cudaFuncSetAttribute(rpy_wall_x2_kernel<ANG, NT, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)dyn);                                                              \
        if (e == cudaSuccess)                                                                            \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_wall_x2_kernel<ANG, NT, NI>, NT, dyn); \
    }
    LM_WOCC2(128, 2) LM_WOCC2(128, 4) LM_WOCC2(256, 2) LM_WOCC2(256, 4)
#undef LM_WOCC2
    return e == cudaSuccess ? n : 0;
}

template <typename R, bool ANG, int NT, int NI>
cudaError_t launch_wall_t(const MdotArgs& a, cudaStream_t s) {
    const int64_t per_cta = (int64_t)NT * NI;
    const int64_t nblk = (a.N + per_cta - 1) / per_cta;
    int64_t ntiles = 0;
    const int splits = (int)split_plan(a.N, NT, a.splits, &ntiles);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<R> k = make_rpy_const<R>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    constexpr size_t dyn = running_sum_bytes<R, ANG, NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_wall_kernel<R, ANG, NT, NI>, dyn)) return e;
    if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
    rpy_wall_kernel<R, ANG, NT, NI><<<grid, NT, dyn, s>>>(
        static_cast<const typename V4<R>::type*>(a.pos4), a.F, ANG ? a.T : nullptr, a.in_f64, a.N, ntiles, k,
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
    if (threads != 128 && threads != 256) return false;
    if (packed) return packed == 1 && !fp64 && (ilp == 2 || ilp == 4);
    return fp64 ? ilp == 1 : (ilp == 1 || ilp == 2 || ilp == 4);
}

int wall_ctas_per_sm(int fp64, int angular, int threads, int ilp, int packed) {
    if (!wall_config_supported(fp64, threads, ilp, packed)) return 0;
    if (packed) return angular ? wall_x2_occupancy<true>(threads, ilp) : wall_x2_occupancy<false>(threads, ilp);
    if (fp64) return angular ? wall_occupancy_r<double, true>(threads, ilp) : wall_occupancy_r<double, false>(threads, ilp);
    return angular ? wall_occupancy_r<float, true>(threads, ilp) : wall_occupancy_r<float, false>(threads, ilp);
}

cudaError_t launch_wall_mdot(const MdotArgs& a, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    if (a.packed) {
        if (a.fp64 || a.packed != 1) return cudaErrorInvalidConfiguration;
        return a.angular ? launch_wall_x2<true>(a, s) : launch_wall_x2<false>(a, s);
    }
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
__global__ void pack_wall_positions_kernel(const void* __restrict__ pos, int in_f64, int64_t N, double a, double z0,
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
    z -= z0;   // height above the wall
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
                                          double scale, int64_t N, double a, double z0,
                                          typename V4<RO>::type* __restrict__ out) {
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
    z = fma(scale, W[3 * i + 2], z) - z0;
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
// Diagonal of the grand mobility from the packed positions, for the Jacobi
// preconditioner of the Lanczos square root: p = diag(M)^{-1/2} and
// q = diag(M)^{1/2} (p = 1, q = 0 where the diagonal is 0).  Open: the
// single-sphere drags 1/(6 pi eta a) and 1/(8 pi eta a^3).  Single wall: the
// Swan-Brady single-sphere functions at the clamped height h (xi = a/h),
// 1 - 9/16 xi + 1/8 xi^3 - 1/16 xi^5 (x, y) and 1 - 9/8 xi + 1/2 xi^3 - 1/8 xi^5
// (z) for translation, 1 - 5/16 xi^3 (x, y) and 1 - 1/8 xi^3 (z) for rotation,
// times f^2 (the damping).
template <typename R>
__global__ void mobility_diag_kernel(const typename V4<R>::type* __restrict__ pos4, int64_t N, double a, double eta,
                                     int angular, int wall, double* __restrict__ p, double* __restrict__ q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double pi = 3.14159265358979323846;
    const double mt = 1.0 / (6.0 * pi * eta * a), mr = 1.0 / (8.0 * pi * eta * a * a * a);
    double t[3] = {mt, mt, mt}, r[3] = {mr, mr, mr};
    if (wall) {
        const typename V4<R>::type v = pos4[i];
        const double xi = a / (double)v.z, f = (double)v.w;
        const double x2 = xi * xi, x3 = x2 * xi, x5 = x3 * x2;
        const double f2 = f * f;
        const double tp = 1.0 - 0.5625 * xi + 0.125 * x3 - 0.0625 * x5;
        const double tn = 1.0 - 1.125 * xi + 0.5 * x3 - 0.125 * x5;
        const double rp = 1.0 - 0.3125 * x3, rn = 1.0 - 0.125 * x3;
        t[0] = t[1] = f2 * mt * tp;
        t[2] = f2 * mt * tn;
        r[0] = r[1] = f2 * mr * rp;
        r[2] = f2 * mr * rn;
    }
    for (int c = 0; c < 3; ++c) {
        p[3 * i + c] = t[c] > 0.0 ? 1.0 / sqrt(t[c]) : 1.0;
        q[3 * i + c] = t[c] > 0.0 ? sqrt(t[c]) : 0.0;
        if (angular) {
            p[3 * N + 3 * i + c] = r[c] > 0.0 ? 1.0 / sqrt(r[c]) : 1.0;
            q[3 * N + 3 * i + c] = r[c] > 0.0 ? sqrt(r[c]) : 0.0;
        }
    }
}

// y = a * x (elementwise, FP64)
__global__ void vmul_kernel(const double* __restrict__ a, const double* __restrict__ x, double* __restrict__ y,
                            int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = a[e] * x[e];
}
}  // namespace

cudaError_t launch_mobility_diag(const void* pos4, int fp64, int64_t N, double a, double eta, int angular, int wall,
                                 double* p, double* q, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (fp64)
        mobility_diag_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const dvec4*>(pos4), N, a, eta, angular, wall,
                                                             p, q);
    else
        mobility_diag_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float4*>(pos4), N, a, eta, angular, wall,
                                                            p, q);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_vmul(const double* a, const double* x, double* y, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    vmul_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, x, y, n);
    count_launches(1);
    return cudaGetLastError();
}


cudaError_t launch_displace_pack_wall(const void* pos, int in_f64, const double* W, double scale, int64_t N,
                                      double a, double z0, void* pos4, int out_f64, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (out_f64)
        displace_pack_wall_kernel<double><<<blocks, 256, 0, s>>>(pos, in_f64, W, scale, N, a, z0,
                                                                  static_cast<dvec4*>(pos4));
    else
        displace_pack_wall_kernel<float><<<blocks, 256, 0, s>>>(pos, in_f64, W, scale, N, a, z0,
                                                                 static_cast<float4*>(pos4));
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

cudaError_t launch_pack_wall_positions(const void* pos, int in_f64, int64_t N, double a, double z0, void* pos4,
                                       int out_f64, int* bad, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (out_f64)
        pack_wall_positions_kernel<double><<<blocks, 256, 0, s>>>(pos, in_f64, N, a, z0, static_cast<dvec4*>(pos4),
                                                                   bad);
    else
        pack_wall_positions_kernel<float><<<blocks, 256, 0, s>>>(pos, in_f64, N, a, z0, static_cast<float4*>(pos4),
                                                                  bad);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lmk
