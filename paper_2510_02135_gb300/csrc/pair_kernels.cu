// Direct-sum RPY mobility product [u; w] = M(X) [F; T] (libMobility paper,
// Eq. block_mobility; NBody solver of Sec. 3.5: the O(N^2) pairwise sum).
//
// Layout and schedule (sm_103a):
//   * Each thread owns NI i-particles (register blocking); a CTA owns
//     NT * NI consecutive particles, i = i0 + k * NT + tid.
//   * The j-range [0, N) is cut into `splits` equal chunks (a multiple of the
//     tile length) so that small N still fills the 152 SMs; blockIdx.y picks
//     the chunk.
//   * j-particles stream through shared memory in tiles of NT: position,
//     force and -T/2 as float4 (double4 in FP64).  Each thread loads one j of
//     the next tile into registers while the current tile is computed.
//   * Per (thread, j) the NI squared distances are reduced to their minimum;
//     a warp vote takes the exact branch only if some lane sees an
//     overlapping pair (r < 2a, including the self pair).  Otherwise all lanes
//     run the branch-free far-field formula.
//   * FP32: each tile is summed in plain FP32 and folded into a (hi, lo)
//     pair with Knuth's TwoSum, so the compensation costs O(1) per tile.
//   * One split writes the result directly; several splits write FP64
//     partial sums that a second kernel adds in FP64 and scales by
//     1/(8 pi eta).
#include <cuda_runtime.h>

#include <cstdint>

#include "lm_internal.cuh"
#include "pair_common.cuh"

namespace lmk {
namespace {

// Shared memory of the scalar kernels: the j-tile (static) and the running
// sums (dynamic, [c][q][tid]; FP32 adds the low parts).
template <typename R, bool ANG, int NT>
struct ScalarTile {
    typename V4<R>::type p[NT];
    typename V4<R>::type f[NT];
    typename V4<R>::type h[ANG ? NT : 1];
};

// Sums of the i-block starting at i0 against j in [jb, je) into s_hi / s_lo
// (zeroed here); every thread leaves its own entries.
template <typename R, bool ANG, int NT, int NI>
__device__ __forceinline__ void scalar_segment(const typename V4<R>::type* __restrict__ pos4,
                                               const void* __restrict__ Fp, const void* __restrict__ Tp,
                                               int in_f64, int64_t N, int64_t i0, int64_t jb, int64_t je,
                                               const RpyConst<R>& k, ScalarTile<R, ANG, NT>& tile, R* s_hi,
                                               R* s_lo) {
    using R4 = typename V4<R>::type;
    constexpr int C = ANG ? 6 : 3;
    R4* sp = tile.p;
    R4* sf = tile.f;
    R4* sh = tile.h;
    const int tid = threadIdx.x;
    const R pad = (R)kPadCoord;

    R xi[NI], yi[NI], zi[NI];
    Acc<R, ANG> acc[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i < N) {
            const R4 p = pos4[i];
            xi[q] = p.x; yi[q] = p.y; zi[q] = p.z;
        } else {
            xi[q] = -pad; yi[q] = -pad; zi[q] = -pad;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            acc[q].p[c] = R(0);
            s_hi[(c * NI + q) * NT + tid] = R(0);
            if (sizeof(R) == 4) s_lo[(c * NI + q) * NT + tid] = R(0);
        }
    }

    // register prefetch of this thread's j in the first tile
    R4 np, nf, nh;
    auto fetch = [&](int64_t j) {
        if (j < je && LM_INBOUNDS(j >= 0 && j < N, 1, j)) {
            np = pos4[j];
            nf.x = load_elem<R>(Fp, in_f64, 3 * j + 0);
            nf.y = load_elem<R>(Fp, in_f64, 3 * j + 1);
            nf.z = load_elem<R>(Fp, in_f64, 3 * j + 2);
            if constexpr (ANG) {
                nh.x = R(-0.5) * load_elem<R>(Tp, in_f64, 3 * j + 0);
                nh.y = R(-0.5) * load_elem<R>(Tp, in_f64, 3 * j + 1);
                nh.z = R(-0.5) * load_elem<R>(Tp, in_f64, 3 * j + 2);
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

#pragma unroll 2
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

}

template <typename R, bool ANG, int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_mdot_kernel(const typename V4<R>::type* __restrict__ pos4,
                                                      const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                      int in_f64, int64_t N, int64_t ntiles, RpyConst<R> k,
                                                      double c8, void* __restrict__ lin, void* __restrict__ ang,
                                                      int out_f64, double* __restrict__ partials) {
    constexpr int C = ANG ? 6 : 3;
    __shared__ ScalarTile<R, ANG, NT> tile;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    R* s_hi = reinterpret_cast<R*>(dyn_smem);              // [c][q][tid]
    R* s_lo = s_hi + (sizeof(R) == 4 ? C * NI * NT : 0);     // FP32 only
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * (NT * NI);
    int64_t jb, je;
    split_range(N, NT, ntiles, &jb, &je);
    scalar_segment<R, ANG, NT, NI>(pos4, Fp, Tp, in_f64, N, i0, jb, je, k, tile, s_hi, s_lo);
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
                void* out = (c < 3) ? lin : ang;
                const int64_t idx = 3 * i + (c % 3);
                if (out_f64) static_cast<double*>(out)[idx] = c8 * v;
                else static_cast<float*>(out)[idx] = (float)(c8 * v);
            } else {
                const int64_t pidx = ((int64_t)blockIdx.y * C + c) * N + i;
                if (LM_INBOUNDS(pidx < (int64_t)gridDim.y * C * N, 3, pidx)) partials[pidx] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Packed FP32 form: two i-particles per f32x2 instruction.
//
// sm_100-class SMs execute add / mul / fma on a pair of FP32 values held in an
// adjacent register pair as one instruction.  The pair sum is the same for
// every i and one j, so i-particles q = 2p and 2p + 1 of a thread share each
// instruction: the far-field pair costs 21 (translation) / 46 (all blocks)
// packed instructions per two pairs, plus one scalar rsqrt per pair.
//
// Packed operands carry no negation, so the j-tile holds every signed and
// scaled value a pair needs, as plain scalars (21 per j, 6 float4 words):
//   word 0  (-x_j, -y_j, -z_j, Fx)          (d = x_i + (-x_j))
//   word 1  (Fy, Fz, -Fx, -Fy)              (F x d without negation)
//   word 2  (-Fz, Tx, Ty, Tz)
//   word 3  (-Tx, -Ty, -Tz, -Tx/2)          (T x d; the -T/2 term of w)
//   word 4  (-Ty/2, -Tz/2, 3Tx/2, 3Ty/2)    (d.T term of w: t = (d.(3T/2)) / r^5)
//   word 5  (3Tz/2, 0, 0, 0)
// A j-value enters a packed instruction as the same scalar in both lanes
// (make_float2(v, v)); the compiler feeds it to both halves without a
// duplicated register pair.  On GB300 this beat a tile of pre-duplicated
// float2 values (11 words per j) by 2-5% at equal results: half the shared
// loads and fewer register operands per packed instruction, which is what
// bounds packed FMA streams there (lm_fp32_probe).
// Translation-only solvers use words 0..1.  Far field (r >= 2a), per pair:
//   u += A F + B (d.F) d + (T x d) / r^3
//   w += (F x d - T/2) / r^3 + (3/2) (d.T) d / r^5
// The exact branch (some pair of the warp at r < 2a) unpacks the two lanes
// and runs the scalar formula.
// ---------------------------------------------------------------------------

// float4 words of one j in the packed tile
template <bool ANG>
constexpr int x2_words() { return ANG ? 6 : 2; }

template <bool ANG, int NT, int NI>
constexpr size_t x2_smem_bytes() {
    return (size_t)x2_words<ANG>() * NT * sizeof(float4) + running_sum_bytes<float, ANG, NT, NI>();
}

// Sums of the i-block starting at i0 against j in [jb, je) into the running
// sums s_hi / s_lo (zeroed here); every thread leaves its own entries.
template <bool ANG, int NT, int NI, int UJ>
__device__ __forceinline__ void x2_segment(const float4* __restrict__ pos4, const void* __restrict__ Fp,
                                           const void* __restrict__ Tp, int in_f64, int64_t N, int64_t i0,
                                           int64_t jb, int64_t je, const RpyConst<float>& k, float4* s_t,
                                           float* s_hi, float* s_lo) {
    static_assert(NI % 2 == 0, "packed form needs an even number of i-particles per thread");
    static_assert(NT % UJ == 0, "the j tile must hold whole groups of UJ");
    constexpr int NP = NI / 2;
    constexpr int C = ANG ? 6 : 3;
    const int tid = threadIdx.x;
    const float pad = (float)kPadCoord;

    float2 xi[NP], yi[NP], zi[NP];
    float2 acc[NP][C];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float x2[2], y2[2], z2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = i0 + (int64_t)(2 * p + h) * NT + tid;
            if (i < N) {
                const float4 v = pos4[i];
                x2[h] = v.x; y2[h] = v.y; z2[h] = v.z;
            } else {
                x2[h] = -pad; y2[h] = -pad; z2[h] = -pad;
            }
        }
        xi[p] = make_float2(x2[0], x2[1]);
        yi[p] = make_float2(y2[0], y2[1]);
        zi[p] = make_float2(z2[0], z2[1]);
#pragma unroll
        for (int c = 0; c < C; ++c) acc[p][c] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            s_hi[(c * NI + q) * NT + tid] = 0.f;
            s_lo[(c * NI + q) * NT + tid] = 0.f;
        }
    }
    const float2 K1 = make_float2(k.K1, k.K1);
    const float2 nK2 = make_float2(-k.K2, -k.K2);

    // register prefetch of this thread's j of the next tile (raw values)
    float4 np;
    float3 nf, nt;
    auto fetch = [&](int64_t j) {
        if (j < je && LM_INBOUNDS(j >= 0 && j < N, 1, j)) {
            np = pos4[j];
            nf.x = load_elem<float>(Fp, in_f64, 3 * j + 0);
            nf.y = load_elem<float>(Fp, in_f64, 3 * j + 1);
            nf.z = load_elem<float>(Fp, in_f64, 3 * j + 2);
            if constexpr (ANG) {
                nt.x = load_elem<float>(Tp, in_f64, 3 * j + 0);
                nt.y = load_elem<float>(Tp, in_f64, 3 * j + 1);
                nt.z = load_elem<float>(Tp, in_f64, 3 * j + 2);
            }
        } else {
            np = make_float4(pad, pad, pad, 0.f);
            nf = make_float3(0.f, 0.f, 0.f);
            nt = make_float3(0.f, 0.f, 0.f);
        }
    };
    fetch(jb + tid);

    for (int64_t jt = jb; jt < je; jt += NT) {
        // scalar tile words: (-x,-y,-z,Fx) (Fy,Fz,-Fx,-Fy) (-Fz,Tx,Ty,Tz) (-Tx,-Ty,-Tz,-Tx/2)
        //                    (-Ty/2,-Tz/2,1.5Tx,1.5Ty) (1.5Tz,0,0,0)
        s_t[0 * NT + tid] = make_float4(-np.x, -np.y, -np.z, nf.x);
        s_t[1 * NT + tid] = make_float4(nf.y, nf.z, -nf.x, -nf.y);
        if constexpr (ANG) {
            s_t[2 * NT + tid] = make_float4(-nf.z, nt.x, nt.y, nt.z);
            s_t[3 * NT + tid] = make_float4(-nt.x, -nt.y, -nt.z, -0.5f * nt.x);
            s_t[4 * NT + tid] = make_float4(-0.5f * nt.y, -0.5f * nt.z, 1.5f * nt.x, 1.5f * nt.y);
            s_t[5 * NT + tid] = make_float4(1.5f * nt.z, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        if (jt + NT < je) fetch(jt + NT + tid);

        // UJ consecutive j share one overlap vote, so that the far-field work
        // of UJ j-particles forms one block of independent instructions.
#pragma unroll 1
        for (int jj = 0; jj < NT; jj += UJ) {
            float2 dx[UJ][NP], dy[UJ][NP], dz[UJ][NP], r2[UJ][NP];
            float mn;
#pragma unroll
            for (int u = 0; u < UJ; ++u) {
                const float4 w0 = s_t[0 * NT + jj + u];
                const float2 nx = bc2(w0.x), ny = bc2(w0.y), nz = bc2(w0.z);
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    dx[u][p] = add2(xi[p], nx);
                    dy[u][p] = add2(yi[p], ny);
                    dz[u][p] = add2(zi[p], nz);
                    r2[u][p] = fma2(dx[u][p], dx[u][p], fma2(dy[u][p], dy[u][p], mul2(dz[u][p], dz[u][p])));
                    const float m2 = fminf(r2[u][p].x, r2[u][p].y);
                    mn = (u == 0 && p == 0) ? m2 : fminf(mn, m2);
                }
            }
            // far-field pair of slot (u, p): two i-particles against j = jj + u
            auto far_slot = [&](int u, int p) {
                const float4 w0 = s_t[0 * NT + jj + u];
                const float4 w1 = s_t[1 * NT + jj + u];
                const float2 fx = bc2(w0.w), fy = bc2(w1.x), fz = bc2(w1.y);
                const float2 ddx = dx[u][p], ddy = dy[u][p], ddz = dz[u][p];
                const float2 invr = make_float2(rsqrtf(r2[u][p].x), rsqrtf(r2[u][p].y));
                const float2 invr2 = mul2(invr, invr);
                const float2 invr3 = mul2(invr2, invr);
                const float2 A = fma2(K1, invr3, invr);
                const float2 invr5 = mul2(invr3, invr2);
                const float2 B = fma2(nK2, invr5, invr3);
                const float2 dF = fma2(ddx, fx, fma2(ddy, fy, mul2(ddz, fz)));
                const float2 sB = mul2(B, dF);
                acc[p][0] = fma2(sB, ddx, fma2(A, fx, acc[p][0]));
                acc[p][1] = fma2(sB, ddy, fma2(A, fy, acc[p][1]));
                acc[p][2] = fma2(sB, ddz, fma2(A, fz, acc[p][2]));
                if constexpr (ANG) {
                    const float4 w2 = s_t[2 * NT + jj + u];
                    const float4 w3 = s_t[3 * NT + jj + u];
                    const float4 w4 = s_t[4 * NT + jj + u];
                    const float4 w5 = s_t[5 * NT + jj + u];
                    const float2 mfx = bc2(w1.z), mfy = bc2(w1.w), mfz = bc2(w2.x);
                    const float2 Tx = bc2(w2.y), Ty = bc2(w2.z), Tz = bc2(w2.w);
                    const float2 mTx = bc2(w3.x), mTy = bc2(w3.y), mTz = bc2(w3.z);
                    const float2 hx = bc2(w3.w), hy = bc2(w4.x), hz = bc2(w4.y);
                    const float2 gx = bc2(w4.z), gy = bc2(w4.w), gz = bc2(w5.x);
                    // u += (T x d) / r^3
                    const float2 cx = fma2(Ty, ddz, mul2(mTz, ddy));
                    const float2 cy = fma2(Tz, ddx, mul2(mTx, ddz));
                    const float2 cz = fma2(Tx, ddy, mul2(mTy, ddx));
                    acc[p][0] = fma2(invr3, cx, acc[p][0]);
                    acc[p][1] = fma2(invr3, cy, acc[p][1]);
                    acc[p][2] = fma2(invr3, cz, acc[p][2]);
                    // w += (F x d - T/2) / r^3 + (d.(3T/2)) d / r^5
                    const float2 vx = fma2(fy, ddz, fma2(mfz, ddy, hx));
                    const float2 vy = fma2(fz, ddx, fma2(mfx, ddz, hy));
                    const float2 vz = fma2(fx, ddy, fma2(mfy, ddx, hz));
                    const float2 t = mul2(invr5, fma2(ddx, gx, fma2(ddy, gy, mul2(ddz, gz))));
                    acc[p][3] = fma2(t, ddx, fma2(invr3, vx, acc[p][3]));
                    acc[p][4] = fma2(t, ddy, fma2(invr3, vy, acc[p][4]));
                    acc[p][5] = fma2(t, ddz, fma2(invr3, vz, acc[p][5]));
                }
            };
            if (__any_sync(0xffffffffu, mn < k.four_a2)) {
                // some pair of the warp overlaps (or is the self pair): the exact
                // scalar form only for the slots that hold one, the packed far
                // field for the others
#pragma unroll
                for (int u = 0; u < UJ; ++u) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (__any_sync(0xffffffffu, fminf(r2[u][p].x, r2[u][p].y) < k.four_a2)) {
                            const float4 w0 = s_t[0 * NT + jj + u];
                            const float4 w1 = s_t[1 * NT + jj + u];
                            const float4 fj = make_float4(w0.w, w1.x, w1.y, 0.f);
                            float4 hj = make_float4(0.f, 0.f, 0.f, 0.f);
                            if constexpr (ANG) {
                                const float4 w3 = s_t[3 * NT + jj + u];
                                const float4 w4 = s_t[4 * NT + jj + u];
                                hj = make_float4(w3.w, w4.x, w4.y, 0.f);
                            }
                            Acc<float, ANG> t0, t1;
#pragma unroll
                            for (int c = 0; c < C; ++c) { t0.p[c] = 0.f; t1.p[c] = 0.f; }
                            pair_exact<float, ANG>(dx[u][p].x, dy[u][p].x, dz[u][p].x, r2[u][p].x, fj, hj, k, t0);
                            pair_exact<float, ANG>(dx[u][p].y, dy[u][p].y, dz[u][p].y, r2[u][p].y, fj, hj, k, t1);
#pragma unroll
                            for (int c = 0; c < C; ++c) acc[p][c] = add2(acc[p][c], make_float2(t0.p[c], t1.p[c]));
                        } else {
                            far_slot(u, p);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < UJ; ++u) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) far_slot(u, p);
                }
            }
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

}

// Dynamic shared memory of the packed kernels: [w][jj] tile words, then the
// running sums [c][q][tid] (hi, then lo).
template <bool ANG, int NT, int NI>
struct X2Smem {
    float4* t;
    float* hi;
    float* lo;
    __device__ explicit X2Smem(unsigned char* base) {
        t = reinterpret_cast<float4*>(base);
        hi = reinterpret_cast<float*>(t + x2_words<ANG>() * NT);
        lo = hi + (ANG ? 6 : 3) * NI * NT;
    }
};

// Split schedule: CTA (blockIdx.x, blockIdx.y) takes i-block blockIdx.x and
// j-split blockIdx.y; several splits write FP64 partials that a second kernel
// adds.
template <bool ANG, int NT, int NI, int UJ>
__global__ void __launch_bounds__(NT) rpy_mdot_x2_kernel(const float4* __restrict__ pos4,
                                                         const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                         int in_f64, int64_t N, int64_t ntiles, RpyConst<float> k,
                                                         double c8, void* __restrict__ lin, void* __restrict__ ang,
                                                         int out_f64, double* __restrict__ partials) {
    constexpr int C = ANG ? 6 : 3;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    X2Smem<ANG, NT, NI> sm(dyn_smem);
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * (NT * NI);
    int64_t jb, je;
    split_range(N, NT, ntiles, &jb, &je);
    x2_segment<ANG, NT, NI, UJ>(pos4, Fp, Tp, in_f64, N, i0, jb, je, k, sm.t, sm.hi, sm.lo);
    const bool direct = (gridDim.y == 1);
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t i = i0 + (int64_t)q * NT + tid;
        if (i >= N) continue;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int o = (c * NI + q) * NT + tid;
            const double v = (double)sm.hi[o] + (double)sm.lo[o];
            if (direct) {
                void* out = (c < 3) ? lin : ang;
                const int64_t idx = 3 * i + (c % 3);
                if (out_f64) static_cast<double*>(out)[idx] = c8 * v;
                else static_cast<float*>(out)[idx] = (float)(c8 * v);
            } else {
                const int64_t pidx = ((int64_t)blockIdx.y * C + c) * N + i;
                if (LM_INBOUNDS(pidx < (int64_t)gridDim.y * C * N, 3, pidx)) partials[pidx] = v;
            }
        }
    }
}

template <typename R, bool ANG, int NT, int NI>
cudaError_t launch_t(const MdotArgs& a, cudaStream_t s) {
    const int64_t per_cta = (int64_t)NT * NI;
    const int64_t nblk = (a.N + per_cta - 1) / per_cta;
    int64_t ntiles = 0;
    const int splits = (int)split_plan(a.N, NT, a.splits, &ntiles);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<R> k = make_rpy_const<R>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    constexpr size_t dyn = running_sum_bytes<R, ANG, NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_mdot_kernel<R, ANG, NT, NI>, dyn)) return e;
    if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
    rpy_mdot_kernel<R, ANG, NT, NI><<<grid, NT, dyn, s>>>(
        static_cast<const typename V4<R>::type*>(a.pos4), a.F, ANG ? a.T : nullptr, a.in_f64, a.N, ntiles, k, c8,
        a.lin, a.ang, a.out_f64, a.partials);
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

template <bool ANG, int NT, int NI, int UJ>
cudaError_t launch_x2_t(const MdotArgs& a, cudaStream_t s) {
    const int64_t per_cta = (int64_t)NT * NI;
    const int64_t nblk = (a.N + per_cta - 1) / per_cta;
    int64_t ntiles = 0;
    const int splits = (int)split_plan(a.N, NT, a.splits, &ntiles);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<float> k = make_rpy_const<float>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    constexpr size_t dyn = x2_smem_bytes<ANG, NT, NI>();
    static std::atomic<unsigned long long> attr_devs{0};  // devices whose limit is raised
    if (cudaError_t e = smem_attr_once(attr_devs, rpy_mdot_x2_kernel<ANG, NT, NI, UJ>, dyn)) return e;
    if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
    rpy_mdot_x2_kernel<ANG, NT, NI, UJ><<<grid, NT, dyn, s>>>(static_cast<const float4*>(a.pos4), a.F,
                                                          ANG ? a.T : nullptr, a.in_f64, a.N, ntiles, k, c8,
                                                          a.lin, a.ang, a.out_f64, a.partials);
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

// Packed configurations (FP32 only): threads {128, 256} x ilp {2, 4, 8};
// packed = UJ, the j-particles per overlap vote: 1, 2, or 4 (ilp 4 and 8
// only; more independent work per warp where a CTA of 8 warps fills an SM).
template <bool ANG, int UJ>
cudaError_t launch_x2_u(const MdotArgs& a, cudaStream_t s) {
    if constexpr (UJ != 4) {
        if (a.threads == 128 && a.ilp == 2) return launch_x2_t<ANG, 128, 2, UJ>(a, s);
        if (a.threads == 256 && a.ilp == 2) return launch_x2_t<ANG, 256, 2, UJ>(a, s);
    }
    if (a.threads == 128 && a.ilp == 4) return launch_x2_t<ANG, 128, 4, UJ>(a, s);
    if (a.threads == 128 && a.ilp == 8) return launch_x2_t<ANG, 128, 8, UJ>(a, s);
    if (a.threads == 256 && a.ilp == 4) return launch_x2_t<ANG, 256, 4, UJ>(a, s);
    if (a.threads == 256 && a.ilp == 8) return launch_x2_t<ANG, 256, 8, UJ>(a, s);
    return cudaErrorInvalidConfiguration;
}

template <bool ANG>
cudaError_t launch_x2(const MdotArgs& a, cudaStream_t s) {
    if (a.packed == 4) return launch_x2_u<ANG, 4>(a, s);
    return a.packed == 2 ? launch_x2_u<ANG, 2>(a, s) : launch_x2_u<ANG, 1>(a, s);
}

template <typename K>
int occupancy_of(K kernel, int threads, size_t dyn) {
    int n = 0;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, dyn);
    return e == cudaSuccess ? n : 0;
}

template <bool ANG, int UJ>
int occupancy_x2(int threads, int ilp) {
#define LM_OCC2(NT, NI) \
    if (threads == NT && ilp == NI) return occupancy_of(rpy_mdot_x2_kernel<ANG, NT, NI, UJ>, NT, x2_smem_bytes<ANG, NT, NI>());
    if constexpr (UJ != 4) { LM_OCC2(128, 2) LM_OCC2(256, 2) }
    LM_OCC2(128, 4) LM_OCC2(128, 8) LM_OCC2(256, 4) LM_OCC2(256, 8)
#undef LM_OCC2
    return 0;
}

// Instantiated configurations: FP32 threads {128, 256} x ilp {1, 2, 4, 8};
// FP64 (parity path) threads {128, 256} x ilp {1, 2}.
template <typename R>
constexpr bool ilp_ok(int ilp) {
    return sizeof(R) == 4 ? (ilp == 1 || ilp == 2 || ilp == 4 || ilp == 8) : (ilp == 1 || ilp == 2);
}

template <typename R, bool ANG>
cudaError_t launch_r(const MdotArgs& a, cudaStream_t s) {
    if (a.threads == 128 && a.ilp == 1) return launch_t<R, ANG, 128, 1>(a, s);
    if (a.threads == 128 && a.ilp == 2) return launch_t<R, ANG, 128, 2>(a, s);
    if (a.threads == 256 && a.ilp == 1) return launch_t<R, ANG, 256, 1>(a, s);
    if (a.threads == 256 && a.ilp == 2) return launch_t<R, ANG, 256, 2>(a, s);
    if constexpr (sizeof(R) == 4) {
        if (a.threads == 128 && a.ilp == 4) return launch_t<R, ANG, 128, 4>(a, s);
        if (a.threads == 128 && a.ilp == 8) return launch_t<R, ANG, 128, 8>(a, s);
        if (a.threads == 256 && a.ilp == 4) return launch_t<R, ANG, 256, 4>(a, s);
        if (a.threads == 256 && a.ilp == 8) return launch_t<R, ANG, 256, 8>(a, s);
    }
    return cudaErrorInvalidConfiguration;
}

template <typename R, bool ANG>
int occupancy_r(int threads, int ilp) {
#define LM_OCC(NT, NI) \
    if (threads == NT && ilp == NI) return occupancy_of(rpy_mdot_kernel<R, ANG, NT, NI>, NT, running_sum_bytes<R, ANG, NT, NI>());
    LM_OCC(128, 1) LM_OCC(128, 2) LM_OCC(256, 1) LM_OCC(256, 2)
    if constexpr (sizeof(R) == 4) {
        LM_OCC(128, 4) LM_OCC(128, 8) LM_OCC(256, 4) LM_OCC(256, 8)
    }
#undef LM_OCC
    return 0;
}

}  // namespace

int64_t mdot_effective_splits(int64_t N, int threads, int splits) {
    int64_t nt = 0;
    return split_plan(N, threads, splits, &nt);
}

int mdot_ctas_per_sm(int fp64, int angular, int threads, int ilp, int packed) {
    if (packed) {
        if (fp64 || !mdot_config_supported(fp64, angular, threads, ilp, packed)) return 0;
        if (packed == 4) return angular ? occupancy_x2<true, 4>(threads, ilp) : occupancy_x2<false, 4>(threads, ilp);
        if (packed == 2) return angular ? occupancy_x2<true, 2>(threads, ilp) : occupancy_x2<false, 2>(threads, ilp);
        return angular ? occupancy_x2<true, 1>(threads, ilp) : occupancy_x2<false, 1>(threads, ilp);
    }
    if (fp64) return angular ? occupancy_r<double, true>(threads, ilp) : occupancy_r<double, false>(threads, ilp);
    return angular ? occupancy_r<float, true>(threads, ilp) : occupancy_r<float, false>(threads, ilp);
}

bool mdot_config_supported(int fp64, int angular, int threads, int ilp, int packed) {
    (void)angular;
    if (packed) return (packed == 1 || packed == 2 || (packed == 4 && ilp >= 4)) && !fp64 &&
                       (threads == 128 || threads == 256) && (ilp == 2 || ilp == 4 || ilp == 8);
    return (threads == 128 || threads == 256) && (fp64 ? ilp_ok<double>(ilp) : ilp_ok<float>(ilp));
}

int mdot_partial_components(int angular) { return angular ? 6 : 3; }

cudaError_t launch_mdot(const MdotArgs& a, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
    if (a.packed) {
        if (a.fp64) return cudaErrorInvalidConfiguration;
        return a.angular ? launch_x2<true>(a, s) : launch_x2<false>(a, s);
    }
    if (a.fp64) return a.angular ? launch_r<double, true>(a, s) : launch_r<double, false>(a, s);
    return a.angular ? launch_r<float, true>(a, s) : launch_r<float, false>(a, s);
}

// --------------------------------------------------------------------------
// Position packing with a finiteness / range check.
// --------------------------------------------------------------------------
namespace {
template <typename RO>
__global__ void pack_positions_kernel(const void* __restrict__ pos, int in_f64, int64_t N,
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
    // written as a negated "inside" test so that NaN counts as bad
    if (!(fabs(x) <= m && fabs(y) <= m && fabs(z) <= m)) atomicExch(bad, 1);
    typename V4<RO>::type v;
    v.x = (RO)x; v.y = (RO)y; v.z = (RO)z; v.w = (RO)0;
    out[i] = v;
}
}  // namespace

cudaError_t launch_pack_positions(const void* pos, int in_f64, int64_t N, void* pos4, int out_f64, int* bad,
                                  cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (out_f64)
        pack_positions_kernel<double><<<blocks, 256, 0, s>>>(pos, in_f64, N, static_cast<dvec4*>(pos4), bad);
    else
        pack_positions_kernel<float><<<blocks, 256, 0, s>>>(pos, in_f64, N, static_cast<float4*>(pos4), bad);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lmk
