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

template <typename R, bool ANG, int NT, int NI>
__global__ void __launch_bounds__(NT) rpy_mdot_kernel(const typename V4<R>::type* __restrict__ pos4,
                                                      const void* __restrict__ Fp, const void* __restrict__ Tp,
                                                      int in_f64, int64_t N, int64_t jchunk, RpyConst<R> k,
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
        if (j < je) {
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
                partials[((int64_t)blockIdx.y * C + c) * N + i] = v;
            }
        }
    }
}

// out[3 i + c] = c8 * sum_s partials[s][c][i]
__global__ void reduce_splits_kernel(const double* __restrict__ partials, int splits, int C, int64_t N,
                                     double c8, void* __restrict__ lin, void* __restrict__ ang, int out_f64) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)C * N) return;
    const int64_t i = e / C;
    const int c = (int)(e - i * C);
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += partials[((int64_t)k * C + c) * N + i];
    void* out = (c < 3) ? lin : ang;
    const int64_t idx = 3 * i + (c % 3);
    if (out_f64) static_cast<double*>(out)[idx] = c8 * s;
    else static_cast<float*>(out)[idx] = (float)(c8 * s);
}

// j-range split: equal chunks of whole tiles; returns the launched split count.
int64_t split_plan(int64_t N, int NT, int splits, int64_t* jchunk) {
    if (splits < 1) splits = 1;
    const int64_t ntiles = (N + NT - 1) / NT;
    if (splits > ntiles) splits = (int)ntiles;
    const int64_t tps = (ntiles + splits - 1) / splits;
    *jchunk = tps * NT;
    return (N + *jchunk - 1) / *jchunk;
}

template <typename R, bool ANG, int NT, int NI>
cudaError_t launch_t(const MdotArgs& a, cudaStream_t s) {
    const int64_t per_cta = (int64_t)NT * NI;
    const int64_t nblk = (a.N + per_cta - 1) / per_cta;
    int64_t jchunk = 0;
    const int splits = (int)split_plan(a.N, NT, a.splits, &jchunk);
    if (nblk > 0x7fffffff || splits > 65535) return cudaErrorInvalidConfiguration;
    const double c8 = 1.0 / (8.0 * 3.14159265358979323846 * a.eta);
    const RpyConst<R> k = make_rpy_const<R>(a.a);
    dim3 grid((unsigned)nblk, (unsigned)splits);
    if (splits > 1 && a.partials == nullptr) return cudaErrorInvalidValue;
    constexpr size_t dyn = running_sum_bytes<R, ANG, NT, NI>();
    static bool attr_set = false;  // per instantiation; the attribute is process-wide
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(rpy_mdot_kernel<R, ANG, NT, NI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
    rpy_mdot_kernel<R, ANG, NT, NI><<<grid, NT, dyn, s>>>(
        static_cast<const typename V4<R>::type*>(a.pos4), a.F, ANG ? a.T : nullptr, a.in_f64, a.N, jchunk, k, c8,
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
    int n = 0;
    cudaError_t e = cudaErrorInvalidConfiguration;
#define LM_OCC(NT, NI)                                                                             \
    if (threads == NT && ilp == NI) {                                                              \
        constexpr size_t dyn = running_sum_bytes<R, ANG, NT, NI>();                                \
        e = cudaFuncSetAttribute(rpy_mdot_kernel<R, ANG, NT, NI>,                                  \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);           \
        if (e == cudaSuccess)                                                                      \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rpy_mdot_kernel<R, ANG, NT, NI>, \
                                                              NT, dyn);                            \
    }
    LM_OCC(128, 1) LM_OCC(128, 2) LM_OCC(256, 1) LM_OCC(256, 2)
    if constexpr (sizeof(R) == 4) {
        LM_OCC(128, 4) LM_OCC(128, 8) LM_OCC(256, 4) LM_OCC(256, 8)
    }
#undef LM_OCC
    return e == cudaSuccess ? n : 0;
}

}  // namespace

int64_t mdot_effective_splits(int64_t N, int threads, int splits) {
    int64_t jc = 0;
    return split_plan(N, threads, splits, &jc);
}

int mdot_ctas_per_sm(int fp64, int angular, int threads, int ilp) {
    if (fp64) return angular ? occupancy_r<double, true>(threads, ilp) : occupancy_r<double, false>(threads, ilp);
    return angular ? occupancy_r<float, true>(threads, ilp) : occupancy_r<float, false>(threads, ilp);
}

bool mdot_config_supported(int fp64, int angular, int threads, int ilp) {
    (void)angular;
    return (threads == 128 || threads == 256) && (fp64 ? ilp_ok<double>(ilp) : ilp_ok<float>(ilp));
}

int mdot_partial_components(int angular) { return angular ? 6 : 3; }

cudaError_t launch_mdot(const MdotArgs& a, cudaStream_t s) {
    if (a.N <= 0) return cudaSuccess;
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
