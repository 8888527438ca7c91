// Adjoint of the RPY mobility product (differentiable form of Mdot, Sec. 3.2).
//
// For L = sum_i G_i.u_i + H_i.w_i with [u; w] = M(X) [F; T]:
//   dL/dF = (M [G; H])_u,  dL/dT = (M [G; H])_w      (M is symmetric)
//   dL/dx_i = sum_j grad_d Phi_ij(d),  d = x_i - x_j, with
//   Phi_ij = G_i.tt(d)F_j + F_i.tt(d)G_j + H_i.rr(d)T_j + T_i.rr(d)H_j
//            + g(r) d.(G_i x T_j + H_i x F_j - G_j x T_i - H_j x F_i)
// (tt, rr even in d; the tr/rt coupling odd, hence the signs).  With
// tt = A I + B d d^T and rr = ar I + br d d^T (B, br multiply (d.f) d):
//   grad_d [g.tt f] = (A'/r)(g.f) d + (B'/r)(g.d)(f.d) d + B[(f.d) g + (g.d) f]
//   grad_d [g(r) d.P] = (g'/r)(d.P) d + g P.
// One pass over j per i recomputes every pair term; nothing of size N^2 is
// stored.  The i-side vectors (G_i, F_i, H_i, T_i) multiply sums of scalars
// or vectors accumulated over a tile, so their products are applied once per
// tile.  FP32 partial sums are folded per tile with TwoSum, as in the forward
// kernel.  Units: coefficients in 1/(8 pi eta), applied once per particle.
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
__device__ __forceinline__ R ld(const void* p, int f64, int64_t idx) {
    if (p == nullptr) return R(0);
    return f64 ? (R)(static_cast<const double*>(p)[idx]) : (R)(static_cast<const float*>(p)[idx]);
}

// Coefficients and their derivatives divided by r.
template <typename R>
struct Coef {
    R A, B, g, ar, br;       // values
    R Ap, Bp, gp, arp, brp;  // d/dr divided by r
};

template <typename R, bool ANG>
__device__ __forceinline__ void far_coef(R r2, const RpyConst<R>& k, Coef<R>& c) {
    const R invr = rsq(r2);
    const R invr2 = invr * invr;
    const R invr3 = invr2 * invr;
    const R invr5 = invr3 * invr2;
    const R invr7 = invr5 * invr2;
    c.A = fma(k.K1, invr3, invr);
    c.B = fma(-k.K2, invr5, invr3);
    c.Ap = fma(R(-3) * k.K1, invr5, -invr3);
    c.Bp = fma(R(5) * k.K2, invr7, R(-3) * invr5);
    if constexpr (ANG) {
        c.g = invr3;
        c.gp = R(-3) * invr5;
        c.ar = R(-0.5) * invr3;
        c.arp = R(1.5) * invr5;
        c.br = R(1.5) * invr5;
        c.brp = R(-7.5) * invr7;
    }
}

// Exact coefficients; returns false at r = 0 (self / coincident pair), where
// the gradient is taken as zero and only the mobility part contributes.
template <typename R, bool ANG>
__device__ __forceinline__ bool exact_coef(R r2, const RpyConst<R>& k, Coef<R>& c) {
    if (r2 >= k.four_a2) {
        far_coef<R, ANG>(r2, k, c);
        return true;
    }
    const R invr = (r2 > R(0)) ? rsq(r2) : R(0);
    const R r = r2 * invr;
    const R invr3 = invr * invr * invr;
    c.A = k.nA0 - k.nA1 * r;
    c.B = k.nB * invr;
    c.Ap = -k.nA1 * invr;
    c.Bp = -k.nB * invr3;
    if constexpr (ANG) {
        c.g = k.ng0 - k.ng1 * r;
        c.gp = -k.ng1 * invr;
        c.ar = k.inv_a3 * (R(1) - k.rr1 * r + k.rr3 * r * r * r);
        c.arp = k.inv_a3 * (-k.rr1 * invr + R(3) * k.rr3 * r);
        c.br = k.inv_a3 * (k.rrb0 * invr - k.rrb1 * r);
        c.brp = k.inv_a3 * (-k.rrb0 * invr3 - k.rrb1 * invr);
    }
    if (!(r2 > R(0))) {
        c.Ap = c.Bp = R(0);
        if constexpr (ANG) { c.gp = c.arp = c.brp = R(0); }
        return false;
    }
    return true;
}

// j-range split (as in the forward kernels): `splits` contiguous ranges of
// whole tiles, as equal as possible; split k holds tiles [k T / s, (k + 1) T / s).
inline int64_t adj_split_plan(int64_t N, int NT, int splits, int64_t* ntiles) {
    if (splits < 1) splits = 1;
    *ntiles = (N + NT - 1) / NT;
    return splits < *ntiles ? splits : *ntiles;
}

__device__ __forceinline__ void split_range(int64_t N, int NT, int64_t ntiles, int64_t* jb, int64_t* je) {
    const int64_t k = blockIdx.y, s = gridDim.y;
    *jb = (k * ntiles / s) * NT;
    const int64_t e = ((k + 1) * ntiles / s) * NT;
    *je = e < N ? e : N;
}

template <typename R, bool ANG>
struct IData {
    R x, y, z;
    R F[3], G[3];
    R T[ANG ? 3 : 1], H[ANG ? 3 : 1];
};

template <typename R, bool ANG>
struct AAcc {
    static constexpr int C = ANG ? 9 : 6;   // dX(3) dF(3) [dT(3)]
    R p[C];                                 // current-tile partials (running sums in shared memory)
    R sG, sF;                               // scalars multiplying G_i, F_i
    R sH, sT;                               // scalars multiplying H_i, T_i
    R gT[3], gF[3], gG[3], gH[3];           // g-weighted sums of j vectors
};

// One pair.  grad = false skips the gradient (r = 0).
template <typename R, bool ANG>
__device__ __forceinline__ void adj_pair(R dx, R dy, R dz, const Coef<R>& c, bool grad,
                                         const typename V4<R>::type& Fj, const typename V4<R>::type& Gj,
                                         const typename V4<R>::type& Tj, const typename V4<R>::type& Hj,
                                         const IData<R, ANG>& I, AAcc<R, ANG>& a) {
    const R b1 = fma(Fj.x, dx, fma(Fj.y, dy, Fj.z * dz));   // F_j.d
    const R b2 = fma(Gj.x, dx, fma(Gj.y, dy, Gj.z * dz));   // G_j.d
    const R Bb2 = c.B * b2;
    // dF += A G_j + B (G_j.d) d
    a.p[3] = fma(Bb2, dx, fma(c.A, Gj.x, a.p[3]));
    a.p[4] = fma(Bb2, dy, fma(c.A, Gj.y, a.p[4]));
    a.p[5] = fma(Bb2, dz, fma(c.A, Gj.z, a.p[5]));
    if (grad) {
        const R a1 = fma(I.G[0], dx, fma(I.G[1], dy, I.G[2] * dz));  // G_i.d
        const R a2 = fma(I.F[0], dx, fma(I.F[1], dy, I.F[2] * dz));  // F_i.d
        const R S1 = fma(I.G[0], Fj.x, fma(I.G[1], Fj.y, fma(I.G[2], Fj.z,
                     fma(I.F[0], Gj.x, fma(I.F[1], Gj.y, I.F[2] * Gj.z)))));
        const R S2 = fma(a1, b1, a2 * b2);
        R cd = fma(c.Ap, S1, c.Bp * S2);
        const R Ba2 = c.B * a2, Ba1 = c.B * a1;
        a.sG = fma(c.B, b1, a.sG);
        a.sF += Bb2;
        if constexpr (ANG) {
            const R e1 = fma(Tj.x, dx, fma(Tj.y, dy, Tj.z * dz));    // T_j.d
            const R e2 = fma(Hj.x, dx, fma(Hj.y, dy, Hj.z * dz));    // H_j.d
            const R c1 = fma(I.H[0], dx, fma(I.H[1], dy, I.H[2] * dz));
            const R c2 = fma(I.T[0], dx, fma(I.T[1], dy, I.T[2] * dz));
            const R R1 = fma(I.H[0], Tj.x, fma(I.H[1], Tj.y, fma(I.H[2], Tj.z,
                         fma(I.T[0], Hj.x, fma(I.T[1], Hj.y, I.T[2] * Hj.z)))));
            const R R2 = fma(c1, e1, c2 * e2);
            cd = fma(c.arp, R1, fma(c.brp, R2, cd));
            // d.P with P = G_i x T_j + H_i x F_j - G_j x T_i - H_j x F_i
            //   = T_j.(d x G_i) + F_j.(d x H_i) + G_j.(d x T_i) + H_j.(d x F_i)
            const R dP =
                Tj.x * (dy * I.G[2] - dz * I.G[1]) + Tj.y * (dz * I.G[0] - dx * I.G[2]) + Tj.z * (dx * I.G[1] - dy * I.G[0]) +
                Fj.x * (dy * I.H[2] - dz * I.H[1]) + Fj.y * (dz * I.H[0] - dx * I.H[2]) + Fj.z * (dx * I.H[1] - dy * I.H[0]) +
                Gj.x * (dy * I.T[2] - dz * I.T[1]) + Gj.y * (dz * I.T[0] - dx * I.T[2]) + Gj.z * (dx * I.T[1] - dy * I.T[0]) +
                Hj.x * (dy * I.F[2] - dz * I.F[1]) + Hj.y * (dz * I.F[0] - dx * I.F[2]) + Hj.z * (dx * I.F[1] - dy * I.F[0]);
            cd = fma(c.gp, dP, cd);
            const R bc2 = c.br * c2, bc1 = c.br * c1;
            a.p[0] = fma(bc2, Hj.x, fma(bc1, Tj.x, a.p[0]));
            a.p[1] = fma(bc2, Hj.y, fma(bc1, Tj.y, a.p[1]));
            a.p[2] = fma(bc2, Hj.z, fma(bc1, Tj.z, a.p[2]));
            a.sH = fma(c.br, e1, a.sH);
            a.sT = fma(c.br, e2, a.sT);
            a.gT[0] = fma(c.g, Tj.x, a.gT[0]); a.gT[1] = fma(c.g, Tj.y, a.gT[1]); a.gT[2] = fma(c.g, Tj.z, a.gT[2]);
            a.gF[0] = fma(c.g, Fj.x, a.gF[0]); a.gF[1] = fma(c.g, Fj.y, a.gF[1]); a.gF[2] = fma(c.g, Fj.z, a.gF[2]);
            a.gG[0] = fma(c.g, Gj.x, a.gG[0]); a.gG[1] = fma(c.g, Gj.y, a.gG[1]); a.gG[2] = fma(c.g, Gj.z, a.gG[2]);
            a.gH[0] = fma(c.g, Hj.x, a.gH[0]); a.gH[1] = fma(c.g, Hj.y, a.gH[1]); a.gH[2] = fma(c.g, Hj.z, a.gH[2]);
        }
        a.p[0] = fma(cd, dx, fma(Ba2, Gj.x, fma(Ba1, Fj.x, a.p[0])));
        a.p[1] = fma(cd, dy, fma(Ba2, Gj.y, fma(Ba1, Fj.y, a.p[1])));
        a.p[2] = fma(cd, dz, fma(Ba2, Gj.z, fma(Ba1, Fj.z, a.p[2])));
    }
    if constexpr (ANG) {
        // dF += g (H_j x d) ; dT += g (G_j x d) + ar H_j + br (H_j.d) d
        const R e2 = fma(Hj.x, dx, fma(Hj.y, dy, Hj.z * dz));
        a.p[3] = fma(c.g, Hj.y * dz - Hj.z * dy, a.p[3]);
        a.p[4] = fma(c.g, Hj.z * dx - Hj.x * dz, a.p[4]);
        a.p[5] = fma(c.g, Hj.x * dy - Hj.y * dx, a.p[5]);
        const R be2 = c.br * e2;
        a.p[6] = fma(be2, dx, fma(c.ar, Hj.x, fma(c.g, Gj.y * dz - Gj.z * dy, a.p[6])));
        a.p[7] = fma(be2, dy, fma(c.ar, Hj.y, fma(c.g, Gj.z * dx - Gj.x * dz, a.p[7])));
        a.p[8] = fma(be2, dz, fma(c.ar, Hj.z, fma(c.g, Gj.x * dy - Gj.y * dx, a.p[8])));
    }
}

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

// Apply the tile's i-side products to dX and fold into the running sums
// (shared memory, [c][q][tid]).
template <typename R, bool ANG, int NT, int NI>
__device__ __forceinline__ void flush_tile(const IData<R, ANG>& I, AAcc<R, ANG>& a, R* s_hi, R* s_lo, int q) {
#pragma unroll
    for (int q = 0; q < 3; ++q) a.p[q] = fma(a.sG, I.G[q], fma(a.sF, I.F[q], a.p[q]));
    a.sG = a.sF = R(0);
    if constexpr (ANG) {
#pragma unroll
        for (int q = 0; q < 3; ++q) a.p[q] = fma(a.sH, I.H[q], fma(a.sT, I.T[q], a.p[q]));
        a.sH = a.sT = R(0);
        // + G_i x gT + H_i x gF - gG x T_i - gH x F_i
        a.p[0] += (I.G[1] * a.gT[2] - I.G[2] * a.gT[1]) + (I.H[1] * a.gF[2] - I.H[2] * a.gF[1]) -
                  (a.gG[1] * I.T[2] - a.gG[2] * I.T[1]) - (a.gH[1] * I.F[2] - a.gH[2] * I.F[1]);
        a.p[1] += (I.G[2] * a.gT[0] - I.G[0] * a.gT[2]) + (I.H[2] * a.gF[0] - I.H[0] * a.gF[2]) -
                  (a.gG[2] * I.T[0] - a.gG[0] * I.T[2]) - (a.gH[2] * I.F[0] - a.gH[0] * I.F[2]);
        a.p[2] += (I.G[0] * a.gT[1] - I.G[1] * a.gT[0]) + (I.H[0] * a.gF[1] - I.H[1] * a.gF[0]) -
                  (a.gG[0] * I.T[1] - a.gG[1] * I.T[0]) - (a.gH[0] * I.F[1] - a.gH[1] * I.F[0]);
#pragma unroll
        for (int q = 0; q < 3; ++q) a.gT[q] = a.gF[q] = a.gG[q] = a.gH[q] = R(0);
    }
#pragma unroll
    for (int c = 0; c < AAcc<R, ANG>::C; ++c) {
        const int o = (c * NI + q) * NT + threadIdx.x;
        fold(&s_hi[o], &s_lo[o], a.p[c]);
    }
}

template <typename R, bool ANG, int NT, int NI>
constexpr size_t adj_running_bytes() {
    return (size_t)(ANG ? 9 : 6) * NI * NT * sizeof(R) * (sizeof(R) == 4 ? 2 : 1);
}

template <typename R, bool ANG, int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_adjoint_kernel(const typename V4<R>::type* __restrict__ pos4,
                                                         const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                         const void* __restrict__ Gp, const void* __restrict__ Hp,
                                                         int f64, int64_t N, int64_t ntiles, RpyConst<R> k, double c8,
                                                         void* __restrict__ dX, void* __restrict__ dF,
                                                         void* __restrict__ dT, double* __restrict__ partials) {
    using R4 = typename V4<R>::type;
    constexpr int C = AAcc<R, ANG>::C;
    __shared__ R4 sp[NT], sF[NT], sG[NT];
    __shared__ R4 sT[ANG ? NT : 1], sH[ANG ? NT : 1];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    R* s_hi = reinterpret_cast<R*>(dyn_smem);
    R* s_lo = s_hi + (sizeof(R) == 4 ? C * NI * NT : 0);
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * (NT * NI);
    int64_t jb, je;
    split_range(N, NT, ntiles, &jb, &je);
    const R pad = (R)kPadCoord;

    IData<R, ANG> I[NI];
    AAcc<R, ANG> a[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i < N) {
            const R4 p = pos4[i];
            I[q].x = p.x; I[q].y = p.y; I[q].z = p.z;
        } else {
            I[q].x = I[q].y = I[q].z = -pad;
        }
        const int64_t ii = (i < N) ? i : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            I[q].F[c] = ld<R>(Fp, f64, 3 * ii + c);
            I[q].G[c] = ld<R>(Gp, f64, 3 * ii + c);
            if constexpr (ANG) {
                I[q].T[c] = ld<R>(Tp, f64, 3 * ii + c);
                I[q].H[c] = ld<R>(Hp, f64, 3 * ii + c);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            a[q].p[c] = R(0);
            s_hi[(c * NI + q) * NT + tid] = R(0);
            if (sizeof(R) == 4) s_lo[(c * NI + q) * NT + tid] = R(0);
        }
        a[q].sG = a[q].sF = a[q].sH = a[q].sT = R(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) a[q].gT[c] = a[q].gF[c] = a[q].gG[c] = a[q].gH[c] = R(0);
    }

    R4 np, nF, nG, nT, nH;
    auto fetch = [&](int64_t j) {
        const bool in = j < je;
        if (in) np = pos4[j]; else { np.x = pad; np.y = pad; np.z = pad; }
        const int64_t jj = in ? j : 0;
        const R z = R(0);
        nF.x = in ? ld<R>(Fp, f64, 3 * jj) : z; nF.y = in ? ld<R>(Fp, f64, 3 * jj + 1) : z; nF.z = in ? ld<R>(Fp, f64, 3 * jj + 2) : z;
        nG.x = in ? ld<R>(Gp, f64, 3 * jj) : z; nG.y = in ? ld<R>(Gp, f64, 3 * jj + 1) : z; nG.z = in ? ld<R>(Gp, f64, 3 * jj + 2) : z;
        if constexpr (ANG) {
            nT.x = in ? ld<R>(Tp, f64, 3 * jj) : z; nT.y = in ? ld<R>(Tp, f64, 3 * jj + 1) : z; nT.z = in ? ld<R>(Tp, f64, 3 * jj + 2) : z;
            nH.x = in ? ld<R>(Hp, f64, 3 * jj) : z; nH.y = in ? ld<R>(Hp, f64, 3 * jj + 1) : z; nH.z = in ? ld<R>(Hp, f64, 3 * jj + 2) : z;
        }
        np.w = nF.w = nG.w = nT.w = nH.w = z;
    };
    fetch(jb + tid);

    for (int64_t jt = jb; jt < je; jt += NT) {
        sp[tid] = np; sF[tid] = nF; sG[tid] = nG;
        if constexpr (ANG) { sT[tid] = nT; sH[tid] = nH; }
        __syncthreads();
        if (jt + NT < je) fetch(jt + NT + tid);
#pragma unroll 2
        for (int jj = 0; jj < NT; ++jj) {
            const R4 pj = sp[jj];
            const R4 Fj = sF[jj];
            const R4 Gj = sG[jj];
            R4 Tj, Hj;
            if constexpr (ANG) { Tj = sT[jj]; Hj = sH[jj]; } else { Tj = Fj; Hj = Fj; }
            R dx[NI], dy[NI], dz[NI], r2[NI];
            R mn = R(0);
#pragma unroll
            for (int q = 0; q < NI; ++q) {
                dx[q] = I[q].x - pj.x; dy[q] = I[q].y - pj.y; dz[q] = I[q].z - pj.z;
                r2[q] = fma(dx[q], dx[q], fma(dy[q], dy[q], dz[q] * dz[q]));
                mn = (q == 0) ? r2[q] : fmin(mn, r2[q]);
            }
            if (__any_sync(0xffffffffu, mn < k.four_a2)) {
#pragma unroll
                for (int q = 0; q < NI; ++q) {
                    Coef<R> c;
                    const bool g = exact_coef<R, ANG>(r2[q], k, c);
                    adj_pair<R, ANG>(dx[q], dy[q], dz[q], c, g, Fj, Gj, Tj, Hj, I[q], a[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < NI; ++q) {
                    Coef<R> c;
                    far_coef<R, ANG>(r2[q], k, c);
                    adj_pair<R, ANG>(dx[q], dy[q], dz[q], c, true, Fj, Gj, Tj, Hj, I[q], a[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NI; ++q) flush_tile<R, ANG, NT, NI>(I[q], a[q], s_hi, s_lo, q);
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
            const double v = (double)s_hi[o] + (sizeof(R) == 4 ? (double)s_lo[o] : 0.0);
            if (direct) {
                void* out = (c < 3) ? dX : (c < 6 ? dF : dT);
                if (out == nullptr) continue;
                const int64_t idx = 3 * i + (c % 3);
                if (f64) static_cast<double*>(out)[idx] = c8 * v;
                else static_cast<float*>(out)[idx] = (float)(c8 * v);
            } else {
                partials[((int64_t)blockIdx.y * C + c) * N + i] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Packed FP32 adjoint, translation blocks only: two i-particles per f32x2
// instruction (same scheme as the packed forward kernel).  The j-tile holds
// -x_j, F_j and G_j duplicated into both halves of a float2.  Per far-field
// pair (units 1/(8 pi eta)):
//   dF_i += A G_j + B (G_j.d) d
//   dX_i += [A'/r (G_i.F_j + F_i.G_j) + B'/r ((G_i.d)(F_j.d) + (F_i.d)(G_j.d))] d
//           + B (F_i.d) G_j + B (G_i.d) F_j
//           + [B (F_j.d)] G_i + [B (G_j.d)] F_i        (scalars summed per tile)
// with A'/r = -1/r^3 - 3 K1/r^5 and B'/r = -3/r^5 + 5 K2/r^7.  UJ consecutive
// j share one overlap vote, so that the far-field work of UJ j-particles is
// one block of independent instructions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// float4 words per j, plain scalars (a j-value enters a packed instruction as
// the same scalar in both lanes): (-x,-y,-z,Fx) (Fy,Fz,Gx,Gy) (Gz,0,0,0)
constexpr int kAdjX2Words = 3;

template <int NT, int NI>
constexpr size_t adj_x2_smem_bytes() {
    return (size_t)kAdjX2Words * NT * sizeof(float4) + adj_running_bytes<float, false, NT, NI>();
}

template <int NT, int NI, int UJ, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) rpy_adjoint_x2_kernel(const float4* __restrict__ pos4,
                                                            const void* __restrict__ Fp, const void* __restrict__ Gp,
                                                            int f64, int64_t N, int64_t ntiles, RpyConst<float> k,
                                                            double c8, void* __restrict__ dX, void* __restrict__ dF,
                                                            double* __restrict__ partials) {
    static_assert(NI % 2 == 0, "packed form needs an even number of i-particles per thread");
    static_assert(NT % UJ == 0, "the j tile must hold whole groups of UJ");
    constexpr int NP = NI / 2;
    constexpr int C = 6;   // dX(3) dF(3)
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    float4* s_t = reinterpret_cast<float4*>(dyn_smem);
    float* s_hi = reinterpret_cast<float*>(s_t + kAdjX2Words * NT);
    float* s_lo = s_hi + C * NI * NT;
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * (NT * NI);
    int64_t jb, je;
    split_range(N, NT, ntiles, &jb, &je);
    const float pad = (float)kPadCoord;

    float2 xi[NP], yi[NP], zi[NP], Fi[NP][3], Gi[NP][3];
    float2 p[NP][C], sG[NP], sF[NP];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
        float v[2][9];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = i0 + (int64_t)(2 * pp + h) * NT + tid;
            if (i < N) {
                const float4 q = pos4[i];
                v[h][0] = q.x; v[h][1] = q.y; v[h][2] = q.z;
            } else {
                v[h][0] = v[h][1] = v[h][2] = -pad;
            }
            const int64_t ii = (i < N) ? i : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[h][3 + c] = ld<float>(Fp, f64, 3 * ii + c);
                v[h][6 + c] = ld<float>(Gp, f64, 3 * ii + c);
            }
        }
        xi[pp] = make_float2(v[0][0], v[1][0]);
        yi[pp] = make_float2(v[0][1], v[1][1]);
        zi[pp] = make_float2(v[0][2], v[1][2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Fi[pp][c] = make_float2(v[0][3 + c], v[1][3 + c]);
            Gi[pp][c] = make_float2(v[0][6 + c], v[1][6 + c]);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) p[pp][c] = bc2(0.f);
        sG[pp] = sF[pp] = bc2(0.f);
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            s_hi[(c * NI + q) * NT + tid] = 0.f;
            s_lo[(c * NI + q) * NT + tid] = 0.f;
        }
    }
    const float2 K1 = bc2(k.K1), nK2 = bc2(-k.K2), m3K1 = bc2(-3.f * k.K1), K2x5 = bc2(5.f * k.K2);
    const float2 m1 = bc2(-1.f), m3 = bc2(-3.f);

    float4 np;
    float3 nF, nG;
    auto fetch = [&](int64_t j) {
        if (j < je && LM_INBOUNDS(j >= 0 && j < N, 8, j)) {
            np = pos4[j];
            nF = make_float3(ld<float>(Fp, f64, 3 * j), ld<float>(Fp, f64, 3 * j + 1), ld<float>(Fp, f64, 3 * j + 2));
            nG = make_float3(ld<float>(Gp, f64, 3 * j), ld<float>(Gp, f64, 3 * j + 1), ld<float>(Gp, f64, 3 * j + 2));
        } else {
            np = make_float4(pad, pad, pad, 0.f);
            nF = nG = make_float3(0.f, 0.f, 0.f);
        }
    };
    fetch(jb + tid);

    for (int64_t jt = jb; jt < je; jt += NT) {
        s_t[0 * NT + tid] = make_float4(-np.x, -np.y, -np.z, nF.x);
        s_t[1 * NT + tid] = make_float4(nF.y, nF.z, nG.x, nG.y);
        s_t[2 * NT + tid] = make_float4(nG.z, 0.f, 0.f, 0.f);
        __syncthreads();
        if (jt + NT < je) fetch(jt + NT + tid);
        // UJ consecutive j share one overlap vote (more independent work per warp)
#pragma unroll 1
        for (int jj = 0; jj < NT; jj += UJ) {
            float2 dx[UJ][NP], dy[UJ][NP], dz[UJ][NP], r2[UJ][NP];
            float mn;
#pragma unroll
            for (int u = 0; u < UJ; ++u) {
                const float4 w0 = s_t[0 * NT + jj + u];
                const float2 nx = bc2(w0.x), ny = bc2(w0.y), nz = bc2(w0.z);
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                    dx[u][pp] = add2(xi[pp], nx);
                    dy[u][pp] = add2(yi[pp], ny);
                    dz[u][pp] = add2(zi[pp], nz);
                    r2[u][pp] = fma2(dx[u][pp], dx[u][pp], fma2(dy[u][pp], dy[u][pp], mul2(dz[u][pp], dz[u][pp])));
                    const float m2 = fminf(r2[u][pp].x, r2[u][pp].y);
                    mn = (u == 0 && pp == 0) ? m2 : fminf(mn, m2);
                }
            }
            if (__any_sync(0xffffffffu, mn < k.four_a2)) {
#pragma unroll
                for (int u = 0; u < UJ; ++u) {
                    const float4 w0 = s_t[0 * NT + jj + u], w1 = s_t[1 * NT + jj + u];
                    const float4 w2 = s_t[2 * NT + jj + u];
                    const float4 Fj = make_float4(w0.w, w1.x, w1.y, 0.f), Gj = make_float4(w1.z, w1.w, w2.x, 0.f);
#pragma unroll
                    for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            IData<float, false> I;
                            AAcc<float, false> t;
                            I.x = I.y = I.z = 0.f;
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                I.F[c] = h ? Fi[pp][c].y : Fi[pp][c].x;
                                I.G[c] = h ? Gi[pp][c].y : Gi[pp][c].x;
                            }
#pragma unroll
                            for (int c = 0; c < C; ++c) t.p[c] = 0.f;
                            t.sG = t.sF = 0.f;
                            Coef<float> cf;
                            const float ddx = h ? dx[u][pp].y : dx[u][pp].x, ddy = h ? dy[u][pp].y : dy[u][pp].x;
                            const float ddz = h ? dz[u][pp].y : dz[u][pp].x, rr = h ? r2[u][pp].y : r2[u][pp].x;
                            const bool g = exact_coef<float, false>(rr, k, cf);
                            adj_pair<float, false>(ddx, ddy, ddz, cf, g, Fj, Gj, Fj, Fj, I, t);
                            if (h) {
#pragma unroll
                                for (int c = 0; c < C; ++c) p[pp][c].y += t.p[c];
                                sG[pp].y += t.sG;
                                sF[pp].y += t.sF;
                            } else {
#pragma unroll
                                for (int c = 0; c < C; ++c) p[pp][c].x += t.p[c];
                                sG[pp].x += t.sG;
                                sF[pp].x += t.sF;
                            }
                        }
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < UJ; ++u) {
                    const float4 w0 = s_t[0 * NT + jj + u], w1 = s_t[1 * NT + jj + u];
                    const float4 w2 = s_t[2 * NT + jj + u];
                    const float2 Fx = bc2(w0.w), Fy = bc2(w1.x), Fz = bc2(w1.y);
                    const float2 Gx = bc2(w1.z), Gy = bc2(w1.w), Gz = bc2(w2.x);
#pragma unroll
                    for (int pp = 0; pp < NP; ++pp) {
                        const float2 ddx = dx[u][pp], ddy = dy[u][pp], ddz = dz[u][pp];
                        const float2 invr = make_float2(rsqrtf(r2[u][pp].x), rsqrtf(r2[u][pp].y));
                        const float2 invr2 = mul2(invr, invr);
                        const float2 invr3 = mul2(invr2, invr);
                        const float2 invr5 = mul2(invr3, invr2);
                        const float2 A = fma2(K1, invr3, invr);
                        const float2 B = fma2(nK2, invr5, invr3);
                        const float2 Ap = mul2(invr3, fma2(m3K1, invr2, m1));    // -1/r^3 - 3 K1/r^5
                        const float2 Bp = mul2(invr5, fma2(K2x5, invr2, m3));    // -3/r^5 + 5 K2/r^7
                        const float2 b1 = fma2(Fx, ddx, fma2(Fy, ddy, mul2(Fz, ddz)));   // F_j.d
                        const float2 b2 = fma2(Gx, ddx, fma2(Gy, ddy, mul2(Gz, ddz)));   // G_j.d
                        const float2 Bb2 = mul2(B, b2);
                        p[pp][3] = fma2(Bb2, ddx, fma2(A, Gx, p[pp][3]));
                        p[pp][4] = fma2(Bb2, ddy, fma2(A, Gy, p[pp][4]));
                        p[pp][5] = fma2(Bb2, ddz, fma2(A, Gz, p[pp][5]));
                        const float2 a1 = fma2(Gi[pp][0], ddx, fma2(Gi[pp][1], ddy, mul2(Gi[pp][2], ddz)));
                        const float2 a2 = fma2(Fi[pp][0], ddx, fma2(Fi[pp][1], ddy, mul2(Fi[pp][2], ddz)));
                        const float2 S1 = fma2(Gi[pp][0], Fx, fma2(Gi[pp][1], Fy, fma2(Gi[pp][2], Fz,
                                          fma2(Fi[pp][0], Gx, fma2(Fi[pp][1], Gy, mul2(Fi[pp][2], Gz))))));
                        const float2 S2 = fma2(a1, b1, mul2(a2, b2));
                        const float2 cd = fma2(Ap, S1, mul2(Bp, S2));
                        const float2 Ba2 = mul2(B, a2), Ba1 = mul2(B, a1);
                        sG[pp] = fma2(B, b1, sG[pp]);
                        sF[pp] = add2(sF[pp], Bb2);
                        p[pp][0] = fma2(cd, ddx, fma2(Ba2, Gx, fma2(Ba1, Fx, p[pp][0])));
                        p[pp][1] = fma2(cd, ddy, fma2(Ba2, Gy, fma2(Ba1, Fy, p[pp][1])));
                        p[pp][2] = fma2(cd, ddz, fma2(Ba2, Gz, fma2(Ba1, Fz, p[pp][2])));
                    }
                }
            }
        }
        // apply the tile's i-side scalars and fold into the running sums
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
            for (int c = 0; c < 3; ++c) p[pp][c] = fma2(sG[pp], Gi[pp][c], fma2(sF[pp], Fi[pp][c], p[pp][c]));
            sG[pp] = sF[pp] = bc2(0.f);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int o0 = (c * NI + 2 * pp) * NT + tid;
                const int o1 = o0 + NT;
                fold(&s_hi[o0], &s_lo[o0], p[pp][c].x);
                fold(&s_hi[o1], &s_lo[o1], p[pp][c].y);
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
            const double v = (double)s_hi[o] + (double)s_lo[o];
            if (direct) {
                void* out = (c < 3) ? dX : dF;
                if (out == nullptr) continue;
                const int64_t idx = 3 * i + (c % 3);
                if (f64) static_cast<double*>(out)[idx] = c8 * v;
                else static_cast<float*>(out)[idx] = (float)(c8 * v);
            } else {
                partials[((int64_t)blockIdx.y * C + c) * N + i] = v;
            }
        }
    }
}

__global__ void adj_reduce_kernel(const double* __restrict__ partials, int splits, int C, int64_t N, double c8,
                                  void* __restrict__ dX, void* __restrict__ dF, void* __restrict__ dT, int f64) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)C * N) return;
    const int64_t i = e / C;
    const int c = (int)(e - i * C);
    void* out = (c < 3) ? dX : (c < 6 ? dF : dT);
    if (out == nullptr) return;
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += partials[((int64_t)k * C + c) * N + i];
    const int64_t idx = 3 * i + (c % 3);
    if (f64) static_cast<double*>(out)[idx] = c8 * s;
    else static_cast<float*>(out)[idx] = (float)(c8 * s);
}


template <typename R, bool ANG, int NI>
cudaError_t launch_adj_t(const AdjointArgs& a, cudaStream_t s) {
    constexpr int NT = 128;
    const int64_t nblk = (a.N + NT * NI - 1) / (NT * NI);
    int64_t ntiles = 0;
    const int splits = (int)adj_split_plan(a.N, NT, a.splits, &ntiles);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<R> k = make_rpy_const<R>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    constexpr size_t dyn = adj_running_bytes<R, ANG, NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_adjoint_kernel<R, ANG, NT, NI>, dyn)) return e;
    rpy_adjoint_kernel<R, ANG, NT, NI><<<grid, NT, dyn, s>>>(static_cast<const typename V4<R>::type*>(a.pos4), a.F,
                                                       ANG ? a.T : nullptr, a.G, ANG ? a.H : nullptr, a.fp64, a.N,
                                                       ntiles, k, c8, a.dX, a.dF, ANG ? a.dT : nullptr, a.partials);
    cudaError_t err = cudaGetLastError();
    count_launches(1);
    if (err != cudaSuccess || splits == 1) return err;
    constexpr int C = ANG ? 9 : 6;
    const int64_t tot = (int64_t)C * a.N;
    adj_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.partials, splits, C, a.N, c8, a.dX, a.dF,
                                                                     ANG ? a.dT : nullptr, a.fp64);
    count_launches(1);
    return cudaGetLastError();
}

template <int NT, int NI, int UJ>
cudaError_t launch_adj_x2_t(const AdjointArgs& a, cudaStream_t s) {
    const int64_t nblk = (a.N + NT * NI - 1) / (NT * NI);
    int64_t ntiles = 0;
    const int splits = (int)adj_split_plan(a.N, NT, a.splits, &ntiles);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<float> k = make_rpy_const<float>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    constexpr size_t dyn = adj_x2_smem_bytes<NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_adjoint_x2_kernel<NT, NI, UJ>, dyn)) return e;
    rpy_adjoint_x2_kernel<NT, NI, UJ><<<grid, NT, dyn, s>>>(static_cast<const float4*>(a.pos4), a.F, a.G, a.fp64, a.N,
                                                        ntiles, k, c8, a.dX, a.dF, a.partials);
    cudaError_t err = cudaGetLastError();
    count_launches(1);
    if (err != cudaSuccess || splits == 1) return err;
    const int64_t tot = 6 * a.N;
    adj_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.partials, splits, 6, a.N, c8, a.dX, a.dF,
                                                                     nullptr, a.fp64);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Symmetric form of the packed translation adjoint (AdjointArgs::uj == 3).
//
// The pair term is symmetric: with d = x_i - x_j and g_ij its gradient,
// dL/dx_j receives -g_ij, and dL/dF_j receives M(d) G_i = A G_i + B (G_i.d) d
// (M is even in d).  So each unordered pair is evaluated once and added to
// both particles: 57 + 18 packed instructions per two pairs for both
// directions against 2 x 57 for the one-sided kernel.  The j-side terms are
//   dX_j -= cd d + B (F_j.d) G_i + B (G_j.d) F_i   (summed as a vector)
//          + [B (F_i.d)] G_j + [B (G_i.d)] F_j     (scalars, applied per tile)
//   dF_j += A G_i + B (G_i.d) d.
// Work item (i-block b, tiles [t0, t1)): the tiles of the block's own range
// [b NI, (b + 1) NI) are diagonal and run one-sided (all ordered pairs,
// self pairs included); every later tile runs symmetric, and no i-block
// visits tiles before its own.  Per j, the eight j-side sums of a warp are
// added across its lanes by a transposing butterfly (9 shuffles) and into
// the tile's shared sums with one atomic per value; at the end of a tile and
// of the item, both sides go to FP64 accumulators acc[particle][dX 3, dF 3]
// by atomic adds, so the summation order of those FP64 adds (not of any
// FP32 sum) varies from run to run.  A final kernel scales acc into the
// outputs.
// ---------------------------------------------------------------------------
constexpr int kAdjSymVals = 8;   // j-side sums per j: dX vector (3), dF (3), scalars of G_j and F_j

template <int NT, int NI>
constexpr size_t adj_sym_smem_bytes() {
    return (size_t)kAdjX2Words * NT * sizeof(float4) + (size_t)kAdjSymVals * (NT + 1) * sizeof(float) +
           adj_running_bytes<float, false, NT, NI>();
}

// Eight per-lane values reduced over the warp: on return lane l holds the
// sum of value (l >> 2) over all 32 lanes.
__device__ __forceinline__ float warp_transpose_sum8(float v[8], int lane) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const bool up = lane & 16;
        const float keep = up ? v[r + 4] : v[r], send = up ? v[r] : v[r + 4];
        v[r] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const bool up = lane & 8;
        const float keep = up ? v[r + 2] : v[r], send = up ? v[r] : v[r + 2];
        v[r] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const bool up = lane & 4;
        const float keep = up ? v[1] : v[0], send = up ? v[0] : v[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

template <int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_adjoint_sym_kernel(const float4* __restrict__ pos4,
                                                             const void* __restrict__ Fp, const void* __restrict__ Gp,
                                                             int f64, int64_t N, const int4* __restrict__ items,
                                                             RpyConst<float> k, double* __restrict__ acc) {
    static_assert(NI % 2 == 0, "packed form needs an even number of i-particles per thread");
    constexpr int NP = NI / 2;
    constexpr int C = 6;   // dX(3) dF(3)
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    float4* s_t = reinterpret_cast<float4*>(dyn_smem);
    // j-side sums [v][jj], rows NT + 1 apart so that the eight lanes adding
    // values 0..7 of one j hit eight different banks
    constexpr int SJ = NT + 1;
    float* s_j = reinterpret_cast<float*>(s_t + kAdjX2Words * NT);
    float* s_hi = s_j + kAdjSymVals * SJ;
    float* s_lo = s_hi + C * NI * NT;
    const int tid = threadIdx.x, lane = tid & 31;
    const int4 item = items[blockIdx.x];
    const int64_t b = item.x, t_begin = item.y, t_end = item.z;
    const int64_t i0 = b * (NT * NI);
    const int64_t diag_end = (b + 1) * NI;   // first tile after the block's own range
    const float pad = (float)kPadCoord;

    float2 xi[NP], yi[NP], zi[NP], Fi[NP][3], Gi[NP][3];
    float2 p[NP][C], sG[NP], sF[NP];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
        float v[2][9];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = i0 + (int64_t)(2 * pp + h) * NT + tid;
            if (i < N && LM_INBOUNDS(i >= 0, 12, i)) {
                const float4 q = pos4[i];
                v[h][0] = q.x; v[h][1] = q.y; v[h][2] = q.z;
            } else {
                v[h][0] = v[h][1] = v[h][2] = -pad;
            }
            const int64_t ii = (i < N) ? i : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[h][3 + c] = (i < N) ? ld<float>(Fp, f64, 3 * ii + c) : 0.f;
                v[h][6 + c] = (i < N) ? ld<float>(Gp, f64, 3 * ii + c) : 0.f;
            }
        }
        xi[pp] = make_float2(v[0][0], v[1][0]);
        yi[pp] = make_float2(v[0][1], v[1][1]);
        zi[pp] = make_float2(v[0][2], v[1][2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Fi[pp][c] = make_float2(v[0][3 + c], v[1][3 + c]);
            Gi[pp][c] = make_float2(v[0][6 + c], v[1][6 + c]);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) p[pp][c] = bc2(0.f);
        sG[pp] = sF[pp] = bc2(0.f);
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            s_hi[(c * NI + q) * NT + tid] = 0.f;
            s_lo[(c * NI + q) * NT + tid] = 0.f;
        }
    }
#pragma unroll
    for (int v = 0; v < kAdjSymVals; ++v) s_j[v * SJ + tid] = 0.f;
    const float2 K1 = bc2(k.K1), nK2 = bc2(-k.K2), m3K1 = bc2(-3.f * k.K1), K2x5 = bc2(5.f * k.K2);
    const float2 m1 = bc2(-1.f), m3 = bc2(-3.f);

    const int64_t jlo = t_begin * NT;
    const int64_t jhi = (t_end * NT < N) ? t_end * NT : N;
    float4 np;
    float3 nF, nG;
    auto fetch = [&](int64_t j) {
        if (j < jhi && LM_INBOUNDS(j >= 0 && j < N, 13, j)) {
            np = pos4[j];
            nF = make_float3(ld<float>(Fp, f64, 3 * j), ld<float>(Fp, f64, 3 * j + 1), ld<float>(Fp, f64, 3 * j + 2));
            nG = make_float3(ld<float>(Gp, f64, 3 * j), ld<float>(Gp, f64, 3 * j + 1), ld<float>(Gp, f64, 3 * j + 2));
        } else {
            np = make_float4(pad, pad, pad, 0.f);
            nF = nG = make_float3(0.f, 0.f, 0.f);
        }
    };
    fetch(jlo + tid);

    for (int64_t t = t_begin; t < t_end; ++t) {
        const int64_t jt = t * NT;
        const bool sym = t >= diag_end;
        s_t[0 * NT + tid] = make_float4(-np.x, -np.y, -np.z, nF.x);
        s_t[1 * NT + tid] = make_float4(nF.y, nF.z, nG.x, nG.y);
        s_t[2 * NT + tid] = make_float4(nG.z, 0.f, 0.f, 0.f);
        __syncthreads();
        if (jt + NT < jhi) fetch(jt + NT + tid);
#pragma unroll 1
        for (int jj = 0; jj < NT; ++jj) {
            const float4 w0 = s_t[0 * NT + jj], w1 = s_t[1 * NT + jj], w2 = s_t[2 * NT + jj];
            const float2 nx = bc2(w0.x), ny = bc2(w0.y), nz = bc2(w0.z);
            const float2 Fx = bc2(w0.w), Fy = bc2(w1.x), Fz = bc2(w1.y);
            const float2 Gx = bc2(w1.z), Gy = bc2(w1.w), Gz = bc2(w2.x);
            float2 dx[NP], dy[NP], dz[NP], r2[NP];
            float mn;
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
                dx[pp] = add2(xi[pp], nx);
                dy[pp] = add2(yi[pp], ny);
                dz[pp] = add2(zi[pp], nz);
                r2[pp] = fma2(dx[pp], dx[pp], fma2(dy[pp], dy[pp], mul2(dz[pp], dz[pp])));
                const float m2 = fminf(r2[pp].x, r2[pp].y);
                mn = (pp == 0) ? m2 : fminf(mn, m2);
            }
            const bool near = __any_sync(0xffffffffu, mn < k.four_a2);
            // j-side sums of this lane for j (packed over the lane's i pairs)
            float2 jX[3], jF[3], jSG, jSF;
#pragma unroll
            for (int c = 0; c < 3; ++c) jX[c] = jF[c] = bc2(0.f);
            jSG = jSF = bc2(0.f);
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
                const float2 ddx = dx[pp], ddy = dy[pp], ddz = dz[pp];
                float2 A, B, Ap, Bp;
                if (!near) {
                    const float2 invr = make_float2(rsqrtf(r2[pp].x), rsqrtf(r2[pp].y));
                    const float2 invr2 = mul2(invr, invr);
                    const float2 invr3 = mul2(invr2, invr);
                    const float2 invr5 = mul2(invr3, invr2);
                    A = fma2(K1, invr3, invr);
                    B = fma2(nK2, invr5, invr3);
                    Ap = mul2(invr3, fma2(m3K1, invr2, m1));    // -1/r^3 - 3 K1/r^5
                    Bp = mul2(invr5, fma2(K2x5, invr2, m3));    // -3/r^5 + 5 K2/r^7
                } else {
                    // exact coefficients of either branch per lane; at r = 0
                    // (self or coincident pairs) A is the self mobility and
                    // B = A' = B' = 0, so the pair adds only A G_j to dF
                    Coef<float> c0, c1;
                    exact_coef<float, false>(r2[pp].x, k, c0);
                    exact_coef<float, false>(r2[pp].y, k, c1);
                    A = make_float2(c0.A, c1.A);
                    B = make_float2(c0.B, c1.B);
                    Ap = make_float2(c0.Ap, c1.Ap);
                    Bp = make_float2(c0.Bp, c1.Bp);
                }
                const float2 b1 = fma2(Fx, ddx, fma2(Fy, ddy, mul2(Fz, ddz)));   // F_j.d
                const float2 b2 = fma2(Gx, ddx, fma2(Gy, ddy, mul2(Gz, ddz)));   // G_j.d
                const float2 Bb2 = mul2(B, b2);
                p[pp][3] = fma2(Bb2, ddx, fma2(A, Gx, p[pp][3]));
                p[pp][4] = fma2(Bb2, ddy, fma2(A, Gy, p[pp][4]));
                p[pp][5] = fma2(Bb2, ddz, fma2(A, Gz, p[pp][5]));
                const float2 a1 = fma2(Gi[pp][0], ddx, fma2(Gi[pp][1], ddy, mul2(Gi[pp][2], ddz)));
                const float2 a2 = fma2(Fi[pp][0], ddx, fma2(Fi[pp][1], ddy, mul2(Fi[pp][2], ddz)));
                const float2 S1 = fma2(Gi[pp][0], Fx, fma2(Gi[pp][1], Fy, fma2(Gi[pp][2], Fz,
                                  fma2(Fi[pp][0], Gx, fma2(Fi[pp][1], Gy, mul2(Fi[pp][2], Gz))))));
                const float2 S2 = fma2(a1, b1, mul2(a2, b2));
                const float2 cd = fma2(Ap, S1, mul2(Bp, S2));
                const float2 Ba2 = mul2(B, a2), Ba1 = mul2(B, a1), Bb1 = mul2(B, b1);
                sG[pp] = add2(sG[pp], Bb1);
                sF[pp] = add2(sF[pp], Bb2);
                p[pp][0] = fma2(cd, ddx, fma2(Ba2, Gx, fma2(Ba1, Fx, p[pp][0])));
                p[pp][1] = fma2(cd, ddy, fma2(Ba2, Gy, fma2(Ba1, Fy, p[pp][1])));
                p[pp][2] = fma2(cd, ddz, fma2(Ba2, Gz, fma2(Ba1, Fz, p[pp][2])));
                if (sym) {
                    jX[0] = fma2(cd, ddx, fma2(Bb1, Gi[pp][0], fma2(Bb2, Fi[pp][0], jX[0])));
                    jX[1] = fma2(cd, ddy, fma2(Bb1, Gi[pp][1], fma2(Bb2, Fi[pp][1], jX[1])));
                    jX[2] = fma2(cd, ddz, fma2(Bb1, Gi[pp][2], fma2(Bb2, Fi[pp][2], jX[2])));
                    jSG = add2(jSG, Ba2);
                    jSF = add2(jSF, Ba1);
                    jF[0] = fma2(Ba1, ddx, fma2(A, Gi[pp][0], jF[0]));
                    jF[1] = fma2(Ba1, ddy, fma2(A, Gi[pp][1], jF[1]));
                    jF[2] = fma2(Ba1, ddz, fma2(A, Gi[pp][2], jF[2]));
                }
            }
            if (sym) {
                float v[kAdjSymVals] = {jX[0].x + jX[0].y, jX[1].x + jX[1].y, jX[2].x + jX[2].y,
                                        jF[0].x + jF[0].y, jF[1].x + jF[1].y, jF[2].x + jF[2].y,
                                        jSG.x + jSG.y, jSF.x + jSF.y};
                const float tot = warp_transpose_sum8(v, lane);
                if ((lane & 3) == 0) atomicAdd(&s_j[(lane >> 2) * SJ + jj], tot);
            }
        }
        // apply the tile's i-side scalars and fold into the running sums
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
            for (int c = 0; c < 3; ++c) p[pp][c] = fma2(sG[pp], Gi[pp][c], fma2(sF[pp], Fi[pp][c], p[pp][c]));
            sG[pp] = sF[pp] = bc2(0.f);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int o0 = (c * NI + 2 * pp) * NT + tid;
                const int o1 = o0 + NT;
                fold(&s_hi[o0], &s_lo[o0], p[pp][c].x);
                fold(&s_hi[o1], &s_lo[o1], p[pp][c].y);
            }
        }
        __syncthreads();
        if (sym) {
            // this tile's j-side sums of the CTA: dX_j -= vector + sG_j G_j + sF_j F_j, dF_j += sums
            const int64_t j = jt + tid;
            if (j < N && LM_INBOUNDS(j >= 0, 14, j)) {
                const float4 w0 = s_t[0 * NT + tid], w1 = s_t[1 * NT + tid], w2 = s_t[2 * NT + tid];
                const float Fj[3] = {w0.w, w1.x, w1.y}, Gj[3] = {w1.z, w1.w, w2.x};
                const float sgj = s_j[6 * SJ + tid], sfj = s_j[7 * SJ + tid];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float dxj = s_j[c * SJ + tid] + sgj * Gj[c] + sfj * Fj[c];
                    atomicAdd(&acc[6 * j + c], -(double)dxj);
                    atomicAdd(&acc[6 * j + 3 + c], (double)s_j[(3 + c) * SJ + tid]);
                }
            }
#pragma unroll
            for (int v = 0; v < kAdjSymVals; ++v) s_j[v * SJ + tid] = 0.f;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int o = (c * NI + q) * NT + tid;
            atomicAdd(&acc[6 * i + c], (double)s_hi[o] + (double)s_lo[o]);
        }
    }
}

// out = c8 * acc[N][C] (dX from components 0..2, dF from 3..5, dT from
// 6..8 when C = 9), nullable outputs.
__global__ void adj_sym_store_kernel(const double* __restrict__ acc, int C, int64_t N, double c8,
                                     void* __restrict__ dX, void* __restrict__ dF, void* __restrict__ dT,
                                     int out_f64) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)C * N) return;
    const int64_t i = e / C;
    const int c = (int)(e - (int64_t)C * i);
    void* out = (c < 3) ? dX : (c < 6 ? dF : dT);
    if (out == nullptr) return;
    const int64_t idx = 3 * i + (c % 3);
    if (out_f64) static_cast<double*>(out)[idx] = c8 * acc[e];
    else static_cast<float*>(out)[idx] = (float)(c8 * acc[e]);
}

template <int NT, int NI>
cudaError_t launch_adj_sym_t(const AdjointArgs& a, cudaStream_t s) {
    if (a.sym_items == nullptr || a.sym_acc == nullptr || a.n_sym_items < 1) return cudaErrorInvalidValue;
    if (a.n_sym_items > 0x7fffffff) return cudaErrorInvalidConfiguration;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<float> k = make_rpy_const<float>(a.a);
    constexpr size_t dyn = adj_sym_smem_bytes<NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_adjoint_sym_kernel<NT, NI>, dyn)) return e;
    cudaError_t e = cudaMemsetAsync(a.sym_acc, 0, (size_t)6 * a.N * sizeof(double), s);
    if (e != cudaSuccess) return e;
    rpy_adjoint_sym_kernel<NT, NI><<<(unsigned)a.n_sym_items, NT, dyn, s>>>(
        static_cast<const float4*>(a.pos4), a.F, a.G, a.fp64, a.N, static_cast<const int4*>(a.sym_items), k,
        a.sym_acc);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_sym_store_kernel<<<(unsigned)((6 * a.N + 255) / 256), 256, 0, s>>>(a.sym_acc, 6, a.N, c8, a.dX, a.dF, nullptr,
                                                                         a.fp64);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adj_sym(const AdjointArgs& a, cudaStream_t s) {
    if (a.threads == 128 && a.ilp == 2) return launch_adj_sym_t<128, 2>(a, s);
    if (a.threads == 128 && a.ilp == 4) return launch_adj_sym_t<128, 4>(a, s);
    if (a.threads == 256 && a.ilp == 2) return launch_adj_sym_t<256, 2>(a, s);
    if (a.threads == 256 && a.ilp == 4) return launch_adj_sym_t<256, 4>(a, s);
    return cudaErrorInvalidConfiguration;
}

template <int NT, int NI>
int adj_sym_occupancy() {
    int n = 0;
    constexpr size_t dyn = adj_sym_smem_bytes<NT, NI>();
    cudaError_t e = cudaFuncSetAttribute(rpy_adjoint_sym_kernel<NT, NI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_adjoint_sym_kernel<NT, NI>, NT, dyn);
    return e == cudaSuccess ? n : 0;
}

// ---------------------------------------------------------------------------
// Symmetric form of the scalar adjoint (AdjointArgs::uj == 3 with angular
// blocks, or in FP64).  Each unordered pair {i, j} is evaluated once, with
// d = x_i - x_j.  The pair term Phi_ij of the header satisfies
// Phi_ji(-d) = Phi_ij(d), so its gradient g_ij goes to dX_i and -g_ij to
// dX_j; the mobility parts of both directions come from the same
// coefficients (tt and rr even in d, the coupling odd):
//   dF_i += A G_j + B (G_j.d) d + g H_j x d,  dT_i += g G_j x d + ar H_j + br (H_j.d) d
//   dF_j += A G_i + B (G_i.d) d - g H_i x d,  dT_j += -g G_i x d + ar H_i + br (H_i.d) d.
// With P = G_i x T_j + H_i x F_j + T_i x G_j + F_i x H_j and
// cd = (A'/r) S1 + (B'/r) S2 + (ar'/r) R1 + (br'/r) R2 + (g'/r) d.P (S1, S2,
// R1, R2 as in adj_pair):
//   g_ij = cd d + g P + B [(F_j.d) G_i + (G_i.d) F_j + (G_j.d) F_i + (F_i.d) G_j]
//                     + br [(T_j.d) H_i + (H_i.d) T_j + (H_j.d) T_i + (T_i.d) H_j].
// A term that multiplies an i-vector is summed as a scalar over the tile on
// the i-side, one that multiplies a j-vector as a scalar per j on the j-side.
// The j-side sums of a warp for one j (13 with angular blocks, 8 without)
// are added across its lanes by a transposing butterfly and into the tile's
// shared sums with one atomic per value.  Work items, diagonal tiles and the
// FP64 accumulators acc[particle][C] are those of the packed translation
// form above.  At r = 0 (self or coincident pairs) the gradient is taken as
// zero, as in the one-sided form; only the mobility parts contribute.
// ---------------------------------------------------------------------------

// V per-lane values (V = 8 or 16) reduced over the warp: on return lane l
// holds the sum over all 32 lanes of value l / (32 / V).
template <typename R, int V>
__device__ __forceinline__ R warp_transpose_sum(R (&v)[V], int lane) {
    static_assert(V == 8 || V == 16, "butterfly width");
#pragma unroll
    for (int h = V / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int r = 0; r < h; ++r) {
            const R keep = up ? v[r + h] : v[r], send = up ? v[r] : v[r + h];
            v[r] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = 16 / V; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    return v[0];
}

template <bool ANG> constexpr int sym_s_words() { return ANG ? 4 : 3; }    // R4 words per j in the tile
template <bool ANG> constexpr int sym_s_vals() { return ANG ? 13 : 8; }    // j-side sums per j
template <bool ANG> constexpr int sym_s_width() { return ANG ? 16 : 8; }   // butterfly width

template <typename R, bool ANG, int NT, int NI>
constexpr size_t adj_sym_s_smem_bytes() {
    return (size_t)sym_s_words<ANG>() * NT * sizeof(typename V4<R>::type) +
           (size_t)sym_s_vals<ANG>() * (NT + 1) * sizeof(R) + adj_running_bytes<R, ANG, NT, NI>();
}

template <typename R, bool ANG>
struct SymAcc {
    static constexpr int C = ANG ? 9 : 6;
    R p[C];             // current-tile partials: dX(3) dF(3) [dT(3)]
    R sG, sF, sH, sT;   // scalars multiplying G_i, F_i, H_i, T_i
};

// One pair of the symmetric form: the i-side partials and scalars and, for
// SYM, the j-side sums v = jX(3) jF(3) [jT(3)] then the scalars of F_j, G_j
// [, T_j, H_j].  gg is g where the gradient is taken (r > 0), else 0.
template <typename R, bool ANG, bool SYM>
__device__ __forceinline__ void sym_pair(R dx, R dy, R dz, const Coef<R>& c, R gg, const IData<R, ANG>& I,
                                         const IData<R, ANG>& J, SymAcc<R, ANG>& a, R* v) {
    const R a1 = fma(I.G[0], dx, fma(I.G[1], dy, I.G[2] * dz));   // G_i.d
    const R a2 = fma(I.F[0], dx, fma(I.F[1], dy, I.F[2] * dz));   // F_i.d
    const R b1 = fma(J.F[0], dx, fma(J.F[1], dy, J.F[2] * dz));   // F_j.d
    const R b2 = fma(J.G[0], dx, fma(J.G[1], dy, J.G[2] * dz));   // G_j.d
    const R S1 = fma(I.G[0], J.F[0], fma(I.G[1], J.F[1], fma(I.G[2], J.F[2],
                 fma(I.F[0], J.G[0], fma(I.F[1], J.G[1], I.F[2] * J.G[2])))));
    R cd = fma(c.Ap, S1, c.Bp * fma(a1, b1, a2 * b2));
    const R BA1 = c.B * a1, BA2 = c.B * a2, BB1 = c.B * b1, BB2 = c.B * b2;
    R V[3] = {R(0), R(0), R(0)};
    R rC1 = R(0), rC2 = R(0), rE1 = R(0), rE2 = R(0);
    if constexpr (ANG) {
        const R c1 = fma(I.H[0], dx, fma(I.H[1], dy, I.H[2] * dz));   // H_i.d
        const R c2 = fma(I.T[0], dx, fma(I.T[1], dy, I.T[2] * dz));   // T_i.d
        const R e1 = fma(J.T[0], dx, fma(J.T[1], dy, J.T[2] * dz));   // T_j.d
        const R e2 = fma(J.H[0], dx, fma(J.H[1], dy, J.H[2] * dz));   // H_j.d
        const R R1 = fma(I.H[0], J.T[0], fma(I.H[1], J.T[1], fma(I.H[2], J.T[2],
                     fma(I.T[0], J.H[0], fma(I.T[1], J.H[1], I.T[2] * J.H[2])))));
        // P = G_i x T_j + H_i x F_j + T_i x G_j + F_i x H_j
        R P[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int u = (q + 1) % 3, w = (q + 2) % 3;
            P[q] = fma(I.G[u], J.T[w], fma(-I.G[w], J.T[u], fma(I.H[u], J.F[w], fma(-I.H[w], J.F[u],
                   fma(I.T[u], J.G[w], fma(-I.T[w], J.G[u], fma(I.F[u], J.H[w], -I.F[w] * J.H[u])))))));
        }
        cd = fma(c.arp, R1, fma(c.brp, fma(c1, e1, c2 * e2), fma(c.gp, fma(dx, P[0], fma(dy, P[1], dz * P[2])), cd)));
#pragma unroll
        for (int q = 0; q < 3; ++q) V[q] = gg * P[q];
        rC1 = c.br * c1; rC2 = c.br * c2; rE1 = c.br * e1; rE2 = c.br * e2;
    }
    V[0] = fma(cd, dx, V[0]);
    V[1] = fma(cd, dy, V[1]);
    V[2] = fma(cd, dz, V[2]);
    const R d[3] = {dx, dy, dz};
    // i-side
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        R t = fma(BA2, J.G[q], fma(BA1, J.F[q], V[q]));
        if constexpr (ANG) t = fma(rC2, J.H[q], fma(rC1, J.T[q], t));
        a.p[q] += t;
        a.p[3 + q] = fma(BB2, d[q], fma(c.A, J.G[q], a.p[3 + q]));
    }
    a.sG += BB1;
    a.sF += BB2;
    if constexpr (ANG) {
        a.sH += rE1;
        a.sT += rE2;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int u = (q + 1) % 3, w = (q + 2) % 3;
            // dF_i += g H_j x d ; dT_i += g G_j x d + ar H_j + br (H_j.d) d
            a.p[3 + q] = fma(c.g, fma(J.H[u], d[w], -J.H[w] * d[u]), a.p[3 + q]);
            a.p[6 + q] = fma(rE2, d[q], fma(c.ar, J.H[q], fma(c.g, fma(J.G[u], d[w], -J.G[w] * d[u]), a.p[6 + q])));
        }
    }
    if constexpr (SYM) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            R t = fma(BB2, I.F[q], fma(BB1, I.G[q], V[q]));
            if constexpr (ANG) t = fma(rE2, I.T[q], fma(rE1, I.H[q], t));
            v[q] += t;
            v[3 + q] = fma(BA1, d[q], fma(c.A, I.G[q], v[3 + q]));
        }
        if constexpr (ANG) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int u = (q + 1) % 3, w = (q + 2) % 3;
                // dF_j -= g H_i x d ; dT_j += -g G_i x d + ar H_i + br (H_i.d) d
                v[3 + q] = fma(-c.g, fma(I.H[u], d[w], -I.H[w] * d[u]), v[3 + q]);
                v[6 + q] = fma(rC1, d[q], fma(c.ar, I.H[q], fma(-c.g, fma(I.G[u], d[w], -I.G[w] * d[u]), v[6 + q])));
            }
            v[9] += BA1;    // x F_j
            v[10] += BA2;   // x G_j
            v[11] += rC1;   // x T_j
            v[12] += rC2;   // x H_j
        } else {
            v[6] += BA1;
            v[7] += BA2;
        }
    }
}

template <typename R, bool ANG, int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_adjoint_sym_s_kernel(const typename V4<R>::type* __restrict__ pos4,
                                                               const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                               const void* __restrict__ Gp, const void* __restrict__ Hp,
                                                               int f64, int64_t N, const int4* __restrict__ items,
                                                               RpyConst<R> k, double* __restrict__ acc) {
    using R4 = typename V4<R>::type;
    constexpr int C = SymAcc<R, ANG>::C;
    constexpr int W = sym_s_words<ANG>();
    constexpr int NV = sym_s_vals<ANG>();
    constexpr int VW = sym_s_width<ANG>();
    constexpr int SJ = NT + 1;   // j-side rows one word apart in bank
    extern __shared__ __align__(32) unsigned char adj_sym_s_smem[];
    R4* s_t = reinterpret_cast<R4*>(adj_sym_s_smem);   // [w][jj]
    R* s_j = reinterpret_cast<R*>(s_t + W * NT);       // [v][jj]
    R* s_hi = s_j + NV * SJ;                           // [c][q][tid]
    R* s_lo = s_hi + (sizeof(R) == 4 ? C * NI * NT : 0);
    const int tid = threadIdx.x, lane = tid & 31;
    const int4 item = items[blockIdx.x];
    const int64_t b = item.x, t_begin = item.y, t_end = item.z;
    const int64_t i0 = b * (NT * NI);
    const int64_t diag_end = (b + 1) * NI;   // first tile after the block's own range
    const R pad = (R)kPadCoord;

    IData<R, ANG> I[NI];
    SymAcc<R, ANG> a[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        const bool in = i < N && LM_INBOUNDS(i >= 0, 12, i);
        if (in) {
            const R4 p = pos4[i];
            I[q].x = p.x; I[q].y = p.y; I[q].z = p.z;
        } else {
            I[q].x = I[q].y = I[q].z = -pad;
        }
        const int64_t ii = in ? i : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            I[q].F[c] = in ? ld<R>(Fp, f64, 3 * ii + c) : R(0);
            I[q].G[c] = in ? ld<R>(Gp, f64, 3 * ii + c) : R(0);
            if constexpr (ANG) {
                I[q].T[c] = in ? ld<R>(Tp, f64, 3 * ii + c) : R(0);
                I[q].H[c] = in ? ld<R>(Hp, f64, 3 * ii + c) : R(0);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            a[q].p[c] = R(0);
            s_hi[(c * NI + q) * NT + tid] = R(0);
            if (sizeof(R) == 4) s_lo[(c * NI + q) * NT + tid] = R(0);
        }
        a[q].sG = a[q].sF = a[q].sH = a[q].sT = R(0);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) s_j[v * SJ + tid] = R(0);

    const int64_t jlo = t_begin * NT;
    const int64_t jhi = (t_end * NT < N) ? t_end * NT : N;
    // register prefetch of this thread's j of the next tile
    R nv[4 * W];
    auto fetch = [&](int64_t j) {
        const bool in = j < jhi && LM_INBOUNDS(j >= 0 && j < N, 13, j);
        const int64_t jj = in ? j : 0;
        if (in) {
            const R4 p = pos4[jj];
            nv[0] = p.x; nv[1] = p.y; nv[2] = p.z;
        } else {
            nv[0] = nv[1] = nv[2] = pad;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            nv[3 + c] = in ? ld<R>(Fp, f64, 3 * jj + c) : R(0);
            nv[6 + c] = in ? ld<R>(Gp, f64, 3 * jj + c) : R(0);
            if constexpr (ANG) {
                nv[9 + c] = in ? ld<R>(Tp, f64, 3 * jj + c) : R(0);
                nv[12 + c] = in ? ld<R>(Hp, f64, 3 * jj + c) : R(0);
            }
        }
#pragma unroll
        for (int c = ANG ? 15 : 9; c < 4 * W; ++c) nv[c] = R(0);
    };
    fetch(jlo + tid);

    for (int64_t t = t_begin; t < t_end; ++t) {
        const int64_t jt = t * NT;
        const bool sym = t >= diag_end;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            R4 q;
            q.x = nv[4 * w]; q.y = nv[4 * w + 1]; q.z = nv[4 * w + 2]; q.w = nv[4 * w + 3];
            s_t[w * NT + tid] = q;
        }
        __syncthreads();
        if (jt + NT < jhi) fetch(jt + NT + tid);
#pragma unroll 1
        for (int jj = 0; jj < NT; ++jj) {
            R wv[4 * W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const R4 q = s_t[w * NT + jj];
                wv[4 * w] = q.x; wv[4 * w + 1] = q.y; wv[4 * w + 2] = q.z; wv[4 * w + 3] = q.w;
            }
            IData<R, ANG> J;
            J.x = wv[0]; J.y = wv[1]; J.z = wv[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                J.F[c] = wv[3 + c];
                J.G[c] = wv[6 + c];
                if constexpr (ANG) { J.T[c] = wv[9 + c]; J.H[c] = wv[12 + c]; }
            }
            R dx[NI], dy[NI], dz[NI], r2[NI];
            R mn = R(0);
#pragma unroll
            for (int q = 0; q < NI; ++q) {
                dx[q] = I[q].x - J.x; dy[q] = I[q].y - J.y; dz[q] = I[q].z - J.z;
                r2[q] = fma(dx[q], dx[q], fma(dy[q], dy[q], dz[q] * dz[q]));
                mn = (q == 0) ? r2[q] : fmin(mn, r2[q]);
            }
            const bool near = __any_sync(0xffffffffu, mn < k.four_a2);
            R v[VW];
#pragma unroll
            for (int c = 0; c < VW; ++c) v[c] = R(0);
#pragma unroll
            for (int q = 0; q < NI; ++q) {
                Coef<R> c;
                bool g = true;
                if (near) g = exact_coef<R, ANG>(r2[q], k, c);
                else far_coef<R, ANG>(r2[q], k, c);
                R gg = R(0);
                if constexpr (ANG) gg = g ? c.g : R(0);
                if (sym) sym_pair<R, ANG, true>(dx[q], dy[q], dz[q], c, gg, I[q], J, a[q], v);
                else sym_pair<R, ANG, false>(dx[q], dy[q], dz[q], c, gg, I[q], J, a[q], v);
            }
            if (sym) {
                const R tot = warp_transpose_sum<R, VW>(v, lane);
                constexpr int per = 32 / VW;
                if (lane % per == 0 && lane / per < NV) atomicAdd(&s_j[(lane / per) * SJ + jj], tot);
            }
        }
        // apply the tile's i-side scalars and fold into the running sums
#pragma unroll
        for (int q = 0; q < NI; ++q) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                R t = fma(a[q].sG, I[q].G[c], fma(a[q].sF, I[q].F[c], a[q].p[c]));
                if constexpr (ANG) t = fma(a[q].sH, I[q].H[c], fma(a[q].sT, I[q].T[c], t));
                a[q].p[c] = t;
            }
            a[q].sG = a[q].sF = a[q].sH = a[q].sT = R(0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int o = (c * NI + q) * NT + tid;
                fold(&s_hi[o], &s_lo[o], a[q].p[c]);
            }
        }
        __syncthreads();
        if (sym) {
            // this tile's j-side sums of the CTA: dX_j -= vector + scalars x (F_j, G_j[, T_j, H_j])
            const int64_t j = jt + tid;
            if (j < N && LM_INBOUNDS(j >= 0, 14, j)) {
                R wv[4 * W];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const R4 q = s_t[w * NT + tid];
                    wv[4 * w] = q.x; wv[4 * w + 1] = q.y; wv[4 * w + 2] = q.z; wv[4 * w + 3] = q.w;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    R x = s_j[c * SJ + tid];
                    if constexpr (ANG) {
                        x = fma(s_j[9 * SJ + tid], wv[3 + c], fma(s_j[10 * SJ + tid], wv[6 + c], x));
                        x = fma(s_j[11 * SJ + tid], wv[9 + c], fma(s_j[12 * SJ + tid], wv[12 + c], x));
                    } else {
                        x = fma(s_j[6 * SJ + tid], wv[3 + c], fma(s_j[7 * SJ + tid], wv[6 + c], x));
                    }
                    atomicAdd(&acc[C * j + c], -(double)x);
                }
#pragma unroll
                for (int c = 3; c < C; ++c) atomicAdd(&acc[C * j + c], (double)s_j[c * SJ + tid]);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) s_j[v * SJ + tid] = R(0);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int o = (c * NI + q) * NT + tid;
            atomicAdd(&acc[C * i + c], (double)s_hi[o] + (sizeof(R) == 4 ? (double)s_lo[o] : 0.0));
        }
    }
}

template <typename R, bool ANG, int NI>
cudaError_t launch_adj_sym_s_t(const AdjointArgs& a, cudaStream_t s) {
    constexpr int NT = 128;
    constexpr int C = SymAcc<R, ANG>::C;
    if (a.sym_items == nullptr || a.sym_acc == nullptr || a.n_sym_items < 1) return cudaErrorInvalidValue;
    if (a.n_sym_items > 0x7fffffff) return cudaErrorInvalidConfiguration;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<R> k = make_rpy_const<R>(a.a);
    constexpr size_t dyn = adj_sym_s_smem_bytes<R, ANG, NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_adjoint_sym_s_kernel<R, ANG, NT, NI>, dyn)) return e;
    cudaError_t e = cudaMemsetAsync(a.sym_acc, 0, (size_t)C * a.N * sizeof(double), s);
    if (e != cudaSuccess) return e;
    rpy_adjoint_sym_s_kernel<R, ANG, NT, NI><<<(unsigned)a.n_sym_items, NT, dyn, s>>>(
        static_cast<const typename V4<R>::type*>(a.pos4), a.F, ANG ? a.T : nullptr, a.G, ANG ? a.H : nullptr, a.fp64,
        a.N, static_cast<const int4*>(a.sym_items), k, a.sym_acc);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t tot = (int64_t)C * a.N;
    adj_sym_store_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.sym_acc, C, a.N, c8, a.dX, a.dF,
                                                                       ANG ? a.dT : nullptr, a.fp64);
    count_launches(1);
    return cudaGetLastError();
}

// i-particles per thread of the symmetric scalar form: FP64 1; FP32 with
// angular blocks 2 or 4.
inline bool sym_s_ilp_supported(int fp64, int ilp) { return fp64 ? ilp == 1 : (ilp == 2 || ilp == 4); }

cudaError_t launch_adj_sym_s(const AdjointArgs& a, cudaStream_t s) {
    if (a.fp64) return a.angular ? launch_adj_sym_s_t<double, true, 1>(a, s) : launch_adj_sym_s_t<double, false, 1>(a, s);
    if (!a.angular) return cudaErrorInvalidConfiguration;   // FP32 translation: the packed symmetric form
    return a.ilp == 4 ? launch_adj_sym_s_t<float, true, 4>(a, s) : launch_adj_sym_s_t<float, true, 2>(a, s);
}

template <typename R, bool ANG, int NI>
int adj_sym_s_occupancy() {
    int n = 0;
    constexpr size_t dyn = adj_sym_s_smem_bytes<R, ANG, 128, NI>();
    cudaError_t e = cudaFuncSetAttribute(rpy_adjoint_sym_s_kernel<R, ANG, 128, NI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_adjoint_sym_s_kernel<R, ANG, 128, NI>, 128, dyn);
    return e == cudaSuccess ? n : 0;
}

// ---------------------------------------------------------------------------
// Packed (f32x2) form of the symmetric adjoint with angular blocks
// (AdjointArgs::uj == 4, FP32): the pair of rpy_adjoint_sym_s_kernel with
// two i-particles per packed instruction; the j-words enter as the same
// scalar in both lanes.  Packed operands take no negation, so the cross
// products with d use g d and -g d, and P is formed as the difference of
// its two halves.  Same work items, j-side butterfly and FP64 accumulators.
// ---------------------------------------------------------------------------
struct PCoef2 {
    float2 A, B, Ap, Bp, g, gp, ar, arp, br, brp;
};

struct Sym6Acc2 {
    float2 p[9];             // dX(3) dF(3) dT(3) of the tile, two i-particles
    float2 sG, sF, sH, sT;   // scalars multiplying G_i, F_i, H_i, T_i
};

// j-side sums v (SYM): jX(3) jF(3) jT(3), then the scalars of F_j, G_j, T_j, H_j.
template <bool SYM>
__device__ __forceinline__ void sym6_pair2(const float2 (&d)[3], const PCoef2& c, float2 gg, const float2 (&Fi)[3],
                                           const float2 (&Gi)[3], const float2 (&Ti)[3], const float2 (&Hi)[3],
                                           const float (&jw)[16], Sym6Acc2& a, float2 (&v)[13]) {
    // j-words: (-x, -y, -z, Fx) (Fy, Fz, Gx, Gy) (Gz, Tx, Ty, Tz) (Hx, Hy, Hz, 0)
    const float* Fj = jw + 3;
    const float* Gj = jw + 6;
    const float* Tj = jw + 9;
    const float* Hj = jw + 12;
    auto doti = [&](const float2 (&w)[3]) { return fma2(w[0], d[0], fma2(w[1], d[1], mul2(w[2], d[2]))); };
    auto dotj = [&](const float* w) { return fma2(bc2(w[0]), d[0], fma2(bc2(w[1]), d[1], mul2(bc2(w[2]), d[2]))); };
    const float2 a1 = doti(Gi), a2 = doti(Fi), c1 = doti(Hi), c2 = doti(Ti);
    const float2 b1 = dotj(Fj), b2 = dotj(Gj), e1 = dotj(Tj), e2 = dotj(Hj);
    const float2 S1 = fma2(Gi[0], bc2(Fj[0]), fma2(Gi[1], bc2(Fj[1]), fma2(Gi[2], bc2(Fj[2]),
                      fma2(Fi[0], bc2(Gj[0]), fma2(Fi[1], bc2(Gj[1]), mul2(Fi[2], bc2(Gj[2])))))));
    const float2 R1 = fma2(Hi[0], bc2(Tj[0]), fma2(Hi[1], bc2(Tj[1]), fma2(Hi[2], bc2(Tj[2]),
                      fma2(Ti[0], bc2(Hj[0]), fma2(Ti[1], bc2(Hj[1]), mul2(Ti[2], bc2(Hj[2])))))));
    // P = G_i x T_j + H_i x F_j + T_i x G_j + F_i x H_j = X - Y
    float2 P[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int u = (q + 1) % 3, w = (q + 2) % 3;
        const float2 X = fma2(Gi[u], bc2(Tj[w]), fma2(Hi[u], bc2(Fj[w]), fma2(Ti[u], bc2(Gj[w]), mul2(Fi[u], bc2(Hj[w])))));
        const float2 Y = fma2(Gi[w], bc2(Tj[u]), fma2(Hi[w], bc2(Fj[u]), fma2(Ti[w], bc2(Gj[u]), mul2(Fi[w], bc2(Hj[u])))));
        P[q] = fma2(bc2(-1.f), Y, X);
    }
    const float2 dP = fma2(d[0], P[0], fma2(d[1], P[1], mul2(d[2], P[2])));
    const float2 cd = fma2(c.Ap, S1, fma2(c.Bp, fma2(a1, b1, mul2(a2, b2)),
                      fma2(c.arp, R1, fma2(c.brp, fma2(c1, e1, mul2(c2, e2)), mul2(c.gp, dP)))));
    const float2 BA1 = mul2(c.B, a1), BA2 = mul2(c.B, a2), BB1 = mul2(c.B, b1), BB2 = mul2(c.B, b2);
    const float2 rC1 = mul2(c.br, c1), rC2 = mul2(c.br, c2), rE1 = mul2(c.br, e1), rE2 = mul2(c.br, e2);
    const float2 ng = mul2(bc2(-1.f), c.g);
    float2 V[3], gd[3], ngd[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        V[q] = fma2(cd, d[q], mul2(gg, P[q]));
        gd[q] = mul2(c.g, d[q]);
        ngd[q] = mul2(ng, d[q]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int u = (q + 1) % 3, w = (q + 2) % 3;
        a.p[q] = fma2(BA2, bc2(Gj[q]), fma2(BA1, bc2(Fj[q]), fma2(rC2, bc2(Hj[q]), fma2(rC1, bc2(Tj[q]),
                 add2(a.p[q], V[q])))));
        // dF_i += A G_j + B (G_j.d) d + g H_j x d ;  dT_i += g G_j x d + ar H_j + br (H_j.d) d
        a.p[3 + q] = fma2(BB2, d[q], fma2(c.A, bc2(Gj[q]), fma2(bc2(Hj[u]), gd[w], fma2(bc2(Hj[w]), ngd[u],
                     a.p[3 + q]))));
        a.p[6 + q] = fma2(rE2, d[q], fma2(c.ar, bc2(Hj[q]), fma2(bc2(Gj[u]), gd[w], fma2(bc2(Gj[w]), ngd[u],
                     a.p[6 + q]))));
    }
    a.sG = add2(a.sG, BB1);
    a.sF = add2(a.sF, BB2);
    a.sH = add2(a.sH, rE1);
    a.sT = add2(a.sT, rE2);
    if constexpr (SYM) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int u = (q + 1) % 3, w = (q + 2) % 3;
            v[q] = fma2(BB2, Fi[q], fma2(BB1, Gi[q], fma2(rE2, Ti[q], fma2(rE1, Hi[q], add2(v[q], V[q])))));
            // dF_j += A G_i + B (G_i.d) d - g H_i x d ;  dT_j += -g G_i x d + ar H_i + br (H_i.d) d
            v[3 + q] = fma2(BA1, d[q], fma2(c.A, Gi[q], fma2(Hi[u], ngd[w], fma2(Hi[w], gd[u], v[3 + q]))));
            v[6 + q] = fma2(rC1, d[q], fma2(c.ar, Hi[q], fma2(Gi[u], ngd[w], fma2(Gi[w], gd[u], v[6 + q]))));
        }
        v[9] = add2(v[9], BA1);     // x F_j
        v[10] = add2(v[10], BA2);   // x G_j
        v[11] = add2(v[11], rC1);   // x T_j
        v[12] = add2(v[12], rC2);   // x H_j
    }
}

template <int NT, int NI>
constexpr size_t adj_sym6_x2_smem_bytes() { return adj_sym_s_smem_bytes<float, true, NT, NI>(); }

template <int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_adjoint_sym6_x2_kernel(const float4* __restrict__ pos4,
                                                                 const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                                 const void* __restrict__ Gp, const void* __restrict__ Hp,
                                                                 int f64, int64_t N, const int4* __restrict__ items,
                                                                 RpyConst<float> k, double* __restrict__ acc) {
    static_assert(NI % 2 == 0, "packed form needs an even number of i-particles per thread");
    constexpr int NP = NI / 2;
    constexpr int C = 9;
    constexpr int W = 4;
    constexpr int NV = 13;
    constexpr int SJ = NT + 1;
    extern __shared__ __align__(16) unsigned char adj_sym6_smem[];
    float4* s_t = reinterpret_cast<float4*>(adj_sym6_smem);   // [w][jj]
    float* s_j = reinterpret_cast<float*>(s_t + W * NT);      // [v][jj]
    float* s_hi = s_j + NV * SJ;                              // [c][q][tid]
    float* s_lo = s_hi + C * NI * NT;
    const int tid = threadIdx.x, lane = tid & 31;
    const int4 item = items[blockIdx.x];
    const int64_t b = item.x, t_begin = item.y, t_end = item.z;
    const int64_t i0 = b * (NT * NI);
    const int64_t diag_end = (b + 1) * NI;
    const float pad = (float)kPadCoord;

    float2 xi[NP][3], Fi[NP][3], Gi[NP][3], Ti[NP][3], Hi[NP][3];
    Sym6Acc2 a[NP];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
        float v[2][15];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = i0 + (int64_t)(2 * pp + h) * NT + tid;
            const bool in = i < N && LM_INBOUNDS(i >= 0, 12, i);
            if (in) {
                const float4 q = pos4[i];
                v[h][0] = q.x; v[h][1] = q.y; v[h][2] = q.z;
            } else {
                v[h][0] = v[h][1] = v[h][2] = -pad;
            }
            const int64_t ii = in ? i : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[h][3 + c] = in ? ld<float>(Fp, f64, 3 * ii + c) : 0.f;
                v[h][6 + c] = in ? ld<float>(Gp, f64, 3 * ii + c) : 0.f;
                v[h][9 + c] = in ? ld<float>(Tp, f64, 3 * ii + c) : 0.f;
                v[h][12 + c] = in ? ld<float>(Hp, f64, 3 * ii + c) : 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xi[pp][c] = make_float2(v[0][c], v[1][c]);
            Fi[pp][c] = make_float2(v[0][3 + c], v[1][3 + c]);
            Gi[pp][c] = make_float2(v[0][6 + c], v[1][6 + c]);
            Ti[pp][c] = make_float2(v[0][9 + c], v[1][9 + c]);
            Hi[pp][c] = make_float2(v[0][12 + c], v[1][12 + c]);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) a[pp].p[c] = bc2(0.f);
        a[pp].sG = a[pp].sF = a[pp].sH = a[pp].sT = bc2(0.f);
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            s_hi[(c * NI + q) * NT + tid] = 0.f;
            s_lo[(c * NI + q) * NT + tid] = 0.f;
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) s_j[v * SJ + tid] = 0.f;
    const float2 K1 = bc2(k.K1), nK2 = bc2(-k.K2), m3K1 = bc2(-3.f * k.K1), K2x5 = bc2(5.f * k.K2);
    const float2 m1 = bc2(-1.f), m3 = bc2(-3.f), mhalf = bc2(-0.5f), p15 = bc2(1.5f), m75 = bc2(-7.5f);

    const int64_t jlo = t_begin * NT;
    const int64_t jhi = (t_end * NT < N) ? t_end * NT : N;
    float nv[16];
    auto fetch = [&](int64_t j) {
        const bool in = j < jhi && LM_INBOUNDS(j >= 0 && j < N, 13, j);
        const int64_t jj = in ? j : 0;
        if (in) {
            const float4 p = pos4[jj];
            nv[0] = -p.x; nv[1] = -p.y; nv[2] = -p.z;
        } else {
            nv[0] = nv[1] = nv[2] = -pad;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            nv[3 + c] = in ? ld<float>(Fp, f64, 3 * jj + c) : 0.f;
            nv[6 + c] = in ? ld<float>(Gp, f64, 3 * jj + c) : 0.f;
            nv[9 + c] = in ? ld<float>(Tp, f64, 3 * jj + c) : 0.f;
            nv[12 + c] = in ? ld<float>(Hp, f64, 3 * jj + c) : 0.f;
        }
        nv[15] = 0.f;
    };
    fetch(jlo + tid);

    for (int64_t t = t_begin; t < t_end; ++t) {
        const int64_t jt = t * NT;
        const bool sym = t >= diag_end;
#pragma unroll
        for (int w = 0; w < W; ++w) s_t[w * NT + tid] = make_float4(nv[4 * w], nv[4 * w + 1], nv[4 * w + 2], nv[4 * w + 3]);
        __syncthreads();
        if (jt + NT < jhi) fetch(jt + NT + tid);
#pragma unroll 1
        for (int jj = 0; jj < NT; ++jj) {
            float jw[16];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const float4 q = s_t[w * NT + jj];
                jw[4 * w] = q.x; jw[4 * w + 1] = q.y; jw[4 * w + 2] = q.z; jw[4 * w + 3] = q.w;
            }
            float2 d[NP][3], r2[NP];
            float mn = 0.f;
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
                for (int c = 0; c < 3; ++c) d[pp][c] = add2(xi[pp][c], bc2(jw[c]));
                r2[pp] = fma2(d[pp][0], d[pp][0], fma2(d[pp][1], d[pp][1], mul2(d[pp][2], d[pp][2])));
                const float m2 = fminf(r2[pp].x, r2[pp].y);
                mn = (pp == 0) ? m2 : fminf(mn, m2);
            }
            const bool near = __any_sync(0xffffffffu, mn < k.four_a2);
            float2 v[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) v[c] = bc2(0.f);
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) {
                PCoef2 c;
                float2 gg;
                if (!near) {
                    const float2 invr = make_float2(rsqrtf(r2[pp].x), rsqrtf(r2[pp].y));
                    const float2 invr2 = mul2(invr, invr);
                    const float2 invr3 = mul2(invr2, invr);
                    const float2 invr5 = mul2(invr3, invr2);
                    const float2 invr7 = mul2(invr5, invr2);
                    c.A = fma2(K1, invr3, invr);
                    c.B = fma2(nK2, invr5, invr3);
                    c.Ap = mul2(invr3, fma2(m3K1, invr2, m1));   // -1/r^3 - 3 K1/r^5
                    c.Bp = mul2(invr5, fma2(K2x5, invr2, m3));   // -3/r^5 + 5 K2/r^7
                    c.g = invr3;
                    c.gp = mul2(m3, invr5);
                    c.ar = mul2(mhalf, invr3);
                    c.arp = mul2(p15, invr5);
                    c.br = c.arp;
                    c.brp = mul2(m75, invr7);
                    gg = c.g;
                } else {
                    // exact coefficients of either branch per lane; at r = 0 the
                    // gradient is taken as zero (gg = 0, the derivatives vanish)
                    Coef<float> c0, c1;
                    const bool g0 = exact_coef<float, true>(r2[pp].x, k, c0);
                    const bool g1 = exact_coef<float, true>(r2[pp].y, k, c1);
                    c.A = make_float2(c0.A, c1.A);
                    c.B = make_float2(c0.B, c1.B);
                    c.Ap = make_float2(c0.Ap, c1.Ap);
                    c.Bp = make_float2(c0.Bp, c1.Bp);
                    c.g = make_float2(c0.g, c1.g);
                    c.gp = make_float2(c0.gp, c1.gp);
                    c.ar = make_float2(c0.ar, c1.ar);
                    c.arp = make_float2(c0.arp, c1.arp);
                    c.br = make_float2(c0.br, c1.br);
                    c.brp = make_float2(c0.brp, c1.brp);
                    gg = make_float2(g0 ? c0.g : 0.f, g1 ? c1.g : 0.f);
                }
                if (sym) sym6_pair2<true>(d[pp], c, gg, Fi[pp], Gi[pp], Ti[pp], Hi[pp], jw, a[pp], v);
                else sym6_pair2<false>(d[pp], c, gg, Fi[pp], Gi[pp], Ti[pp], Hi[pp], jw, a[pp], v);
            }
            if (sym) {
                float s[16];
#pragma unroll
                for (int c = 0; c < NV; ++c) s[c] = v[c].x + v[c].y;
#pragma unroll
                for (int c = NV; c < 16; ++c) s[c] = 0.f;
                const float tot = warp_transpose_sum<float, 16>(s, lane);
                if ((lane & 1) == 0 && (lane >> 1) < NV) atomicAdd(&s_j[(lane >> 1) * SJ + jj], tot);
            }
        }
        // apply the tile's i-side scalars and fold into the running sums
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                a[pp].p[c] = fma2(a[pp].sG, Gi[pp][c], fma2(a[pp].sF, Fi[pp][c], fma2(a[pp].sH, Hi[pp][c],
                             fma2(a[pp].sT, Ti[pp][c], a[pp].p[c]))));
            a[pp].sG = a[pp].sF = a[pp].sH = a[pp].sT = bc2(0.f);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int o0 = (c * NI + 2 * pp) * NT + tid;
                const int o1 = o0 + NT;
                fold(&s_hi[o0], &s_lo[o0], a[pp].p[c].x);
                fold(&s_hi[o1], &s_lo[o1], a[pp].p[c].y);
            }
        }
        __syncthreads();
        if (sym) {
            const int64_t j = jt + tid;
            if (j < N && LM_INBOUNDS(j >= 0, 14, j)) {
                float wv[16];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const float4 q = s_t[w * NT + tid];
                    wv[4 * w] = q.x; wv[4 * w + 1] = q.y; wv[4 * w + 2] = q.z; wv[4 * w + 3] = q.w;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float x = s_j[c * SJ + tid];
                    x = fmaf(s_j[9 * SJ + tid], wv[3 + c], fmaf(s_j[10 * SJ + tid], wv[6 + c], x));
                    x = fmaf(s_j[11 * SJ + tid], wv[9 + c], fmaf(s_j[12 * SJ + tid], wv[12 + c], x));
                    atomicAdd(&acc[C * j + c], -(double)x);
                }
#pragma unroll
                for (int c = 3; c < C; ++c) atomicAdd(&acc[C * j + c], (double)s_j[c * SJ + tid]);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) s_j[v * SJ + tid] = 0.f;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int o = (c * NI + q) * NT + tid;
            atomicAdd(&acc[C * i + c], (double)s_hi[o] + (double)s_lo[o]);
        }
    }
}

template <int NI>
cudaError_t launch_adj_sym6_x2_t(const AdjointArgs& a, cudaStream_t s) {
    constexpr int NT = 128;
    constexpr int C = 9;
    if (a.sym_items == nullptr || a.sym_acc == nullptr || a.n_sym_items < 1) return cudaErrorInvalidValue;
    if (a.n_sym_items > 0x7fffffff) return cudaErrorInvalidConfiguration;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<float> k = make_rpy_const<float>(a.a);
    constexpr size_t dyn = adj_sym6_x2_smem_bytes<NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_adjoint_sym6_x2_kernel<NT, NI>, dyn)) return e;
    cudaError_t e = cudaMemsetAsync(a.sym_acc, 0, (size_t)C * a.N * sizeof(double), s);
    if (e != cudaSuccess) return e;
    rpy_adjoint_sym6_x2_kernel<NT, NI><<<(unsigned)a.n_sym_items, NT, dyn, s>>>(
        static_cast<const float4*>(a.pos4), a.F, a.T, a.G, a.H, a.fp64, a.N, static_cast<const int4*>(a.sym_items), k,
        a.sym_acc);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t tot = (int64_t)C * a.N;
    adj_sym_store_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.sym_acc, C, a.N, c8, a.dX, a.dF, a.dT,
                                                                       a.fp64);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adj_sym6_x2(const AdjointArgs& a, cudaStream_t s) {
    if (a.fp64 || !a.angular) return cudaErrorInvalidConfiguration;
    return a.ilp == 4 ? launch_adj_sym6_x2_t<4>(a, s) : launch_adj_sym6_x2_t<2>(a, s);
}

template <int NI>
int adj_sym6_x2_occupancy() {
    int n = 0;
    constexpr size_t dyn = adj_sym6_x2_smem_bytes<128, NI>();
    cudaError_t e = cudaFuncSetAttribute(rpy_adjoint_sym6_x2_kernel<128, NI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_adjoint_sym6_x2_kernel<128, NI>, 128, dyn);
    return e == cudaSuccess ? n : 0;
}

// Packed translation adjoint configurations: threads {128, 256} x ilp {2, 4}
// x j per vote {1, 2} (AdjointArgs::uj).
template <int NT, int NI>
cudaError_t launch_adj_x2_u(const AdjointArgs& a, cudaStream_t s) {
    return a.uj == 2 ? launch_adj_x2_t<NT, NI, 2>(a, s) : launch_adj_x2_t<NT, NI, 1>(a, s);
}

cudaError_t launch_adj_x2(const AdjointArgs& a, cudaStream_t s) {
    if (a.threads == 128 && a.ilp == 2) return launch_adj_x2_u<128, 2>(a, s);
    if (a.threads == 128 && a.ilp == 4) return launch_adj_x2_u<128, 4>(a, s);
    if (a.threads == 256 && a.ilp == 2) return launch_adj_x2_u<256, 2>(a, s);
    if (a.threads == 256 && a.ilp == 4) return launch_adj_x2_u<256, 4>(a, s);
    return cudaErrorInvalidConfiguration;
}

template <int NT, int NI, int UJ>
int adj_x2_occupancy() {
    int n = 0;
    constexpr size_t dyn = adj_x2_smem_bytes<NT, NI>();
    cudaError_t e = cudaFuncSetAttribute(rpy_adjoint_x2_kernel<NT, NI, UJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_adjoint_x2_kernel<NT, NI, UJ>, NT, dyn);
    return e == cudaSuccess ? n : 0;
}

}  // namespace

int adjoint_partial_components(int angular) { return angular ? 9 : 6; }

// i-particles per thread: FP32 translation 4 (packed; tunable), FP32 with
// angular blocks 2, FP64 1 (register budget of the heavier angular and FP64
// adjoints).
int adjoint_ilp(int fp64, int angular) { return fp64 ? 1 : (angular ? 2 : 4); }

bool adjoint_config_supported(int fp64, int angular, int threads, int ilp, int uj) {
    if (fp64 || angular) {
        if (uj == 3) return threads == 128 && sym_s_ilp_supported(fp64, ilp);   // symmetric scalar form
        if (uj == 4) return !fp64 && threads == 128 && (ilp == 2 || ilp == 4);   // symmetric packed form
        return threads == 128 && ilp == adjoint_ilp(fp64, angular) && uj >= 0 && uj <= 1;
    }
    return (threads == 128 || threads == 256) && (ilp == 2 || ilp == 4) && uj >= 0 && uj <= 3;
}

cudaError_t launch_adjoint(const AdjointArgs& a, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    if (!adjoint_config_supported(a.fp64, a.angular, a.threads, a.ilp, a.uj)) return cudaErrorInvalidConfiguration;
    // FP64, and FP32 with angular blocks: the scalar kernels, one-sided or symmetric
    if (a.fp64 || a.angular) {
        if (a.uj == 3) return launch_adj_sym_s(a, s);
        if (a.uj == 4) return launch_adj_sym6_x2(a, s);
        if (a.fp64) return a.angular ? launch_adj_t<double, true, 1>(a, s) : launch_adj_t<double, false, 1>(a, s);
        return launch_adj_t<float, true, 2>(a, s);
    }
    // FP32 translation blocks: the packed (f32x2) kernels, one-sided or symmetric
    return a.uj == 3 ? launch_adj_sym(a, s) : launch_adj_x2(a, s);
}

int adjoint_ctas_per_sm(int fp64, int angular, int threads, int ilp, int uj) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidConfiguration;
    if (!adjoint_config_supported(fp64, angular, threads, ilp, uj)) return 0;
#define LM_AOCC(R, ANG, NI)                                                                       \
    {                                                                                             \
        constexpr size_t dyn = adj_running_bytes<R, ANG, 128, NI>();                              \
        e = cudaFuncSetAttribute(rpy_adjoint_kernel<R, ANG, 128, NI>,                             \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);          \
        if (e == cudaSuccess)                                                                     \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_adjoint_kernel<R, ANG, 128, NI>, 128, dyn); \
    }
    if (angular && !fp64 && uj == 4) return ilp == 4 ? adj_sym6_x2_occupancy<4>() : adj_sym6_x2_occupancy<2>();
    if ((fp64 || angular) && uj == 3) {
        if (fp64) return angular ? adj_sym_s_occupancy<double, true, 1>() : adj_sym_s_occupancy<double, false, 1>();
        return ilp == 4 ? adj_sym_s_occupancy<float, true, 4>() : adj_sym_s_occupancy<float, true, 2>();
    }
    if (fp64 && angular) LM_AOCC(double, true, 1)
    else if (fp64) LM_AOCC(double, false, 1)
    else if (angular) LM_AOCC(float, true, 2)
    else if (uj == 3) {
        if (threads == 128 && ilp == 2) return adj_sym_occupancy<128, 2>();
        if (threads == 128 && ilp == 4) return adj_sym_occupancy<128, 4>();
        if (threads == 256 && ilp == 2) return adj_sym_occupancy<256, 2>();
        if (threads == 256 && ilp == 4) return adj_sym_occupancy<256, 4>();
        return 0;
    } else {
        const bool two = uj == 2;
        if (threads == 128 && ilp == 2) return two ? adj_x2_occupancy<128, 2, 2>() : adj_x2_occupancy<128, 2, 1>();
        if (threads == 128 && ilp == 4) return two ? adj_x2_occupancy<128, 4, 2>() : adj_x2_occupancy<128, 4, 1>();
        if (threads == 256 && ilp == 2) return two ? adj_x2_occupancy<256, 2, 2>() : adj_x2_occupancy<256, 2, 1>();
        if (threads == 256 && ilp == 4) return two ? adj_x2_occupancy<256, 4, 2>() : adj_x2_occupancy<256, 4, 1>();
        return 0;
    }
#undef LM_AOCC
    return e == cudaSuccess ? n : 0;
}

}  // namespace lmk
