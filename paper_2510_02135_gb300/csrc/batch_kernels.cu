// Batched Brownian dynamics of many independent open-boundary suspensions in
// one persistent cooperative launch (libMobility paper, Eq. bdhi with the
// Euler-Maruyama step of Sec. 3.2; Lanczos square root of Sec. 3.3; the drift
// term is zero in the open geometry, Sec. 2).
//
// One BD step, every system s at once:
//   A1  chunks   W_s (Philox) -> V_s[0], |W_s|^2 partials, F_s = -k x_s
//   A2  chunks   v_0 = W_s / |W_s|
//   for k = 0, 1, ...                       (systems drop out as they converge)
//     B   items    partial products of w = M_s v_k over one j-part (k = 0: also
//                  u = M_s F_s, a second right-hand side sharing the pair
//                  coefficients); v_k = w_{k-1} / beta_{k-1} is formed while
//                  loading (and stored for the own rows); partial v_k . w
//     C2  chunks   w = sum of the j-parts; alpha_k = sum of the item partials;
//                  w -= alpha_k v_k + beta_{k-1} v_{k-1}; dots V_s^T w
//     C3  chunks   w -= V_s c; |w|^2 after the pass.  The system's last chunk
//                  makes the DGKS test (|w| below 1/sqrt(2) of its value
//                  before C3) and, without a second pass, ends the iteration:
//                  beta_k, a solve request for z_k = |W| f(T_k) e1 (served by
//                  the solver warps), the stopping rule on the results that
//                  have arrived (in BD runs the relative-change test is first
//                  made one iteration before the count of the system's
//                  previous step)
//     C4  chunks   only if some system needs it: dots V_s^T w, then
//                  w -= V_s c', |w|^2, and the end of the iteration by the
//                  last chunk of each such system
//   D   chunks   y = V_s z; x += dt u + sqrt(2 kT dt) y
// Phases are separated by a grid barrier whose waits are bounded in clock
// cycles: an expired wait sets an error flag and every CTA returns.
// Items are (system, block of NT*NI particles, j-part of kBatchJPart) in
// decreasing system size, handed out through a ticket counter, so that the
// largest systems are cut into several short items; chunks are kBatchChunk
// vector elements
// of one system, assigned round-robin.  Every reduction is a fixed-order sum
// of per-item or per-chunk partials, so results do not depend on timing.
#include <cuda_runtime.h>

#include <cstdint>

#include "lm_internal.cuh"
#include "philox.cuh"
#include "tridiag.cuh"
#include "tridiag_dev.cuh"

namespace lmk {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Phase end times of the last step of the run (CTA 0, thread 0), for profiling.
__device__ __forceinline__ void stamp(const BatchParams& P, int step, int& slot) {
    const int last = (P.mode == kBatchBD) ? P.nsteps - 1 : 0;
    if (P.timeline != nullptr && step == last && blockIdx.x == 0 && threadIdx.x == 0 && slot < P.timeline_len)
        P.timeline[slot] = global_ns();
    ++slot;
}

// Grid barrier with a bounded wait.  Returns false if the run must stop.
// Two levels: a CTA adds itself to its group's counter; the last CTA of a
// group resets that counter and adds the group to bar[0]; the last group's
// CTA resets bar[0] and advances the generation, which every other CTA waits
// for.  Same-address atomics are what a one-counter barrier pays for (one
// per CTA, serialised in one L2 slice); here each counter takes at most
// kBarGroup of them and the group counters sit in separate lines.
__device__ bool grid_sync(const BatchParams& P) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = P.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const int grp = blockIdx.x / kBarGroup;
        const int ngrp = (P.n_main + kBarGroup - 1) / kBarGroup;
        const unsigned gsize = (unsigned)min(kBarGroup, P.n_main - grp * kBarGroup);
        unsigned* gc = P.bar + kBarStride * (1 + grp);
        bool release = false;
        if (atomicAdd(gc, 1u) == gsize - 1u) {
            // every CTA of the group has arrived: none can arrive again before
            // the generation advances, so the counter can be reset now
            atomicExch(gc, 0u);
            __threadfence();
            if (atomicAdd(P.bar, 1u) == (unsigned)ngrp - 1u) {
                atomicExch(P.bar, 0u);
                __threadfence();
                atomicAdd(P.bar + 1, 1u);
                release = true;
            }
        }
        if (!release) {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*(volatile int*)P.err != kBatchOk) break;
                if (clock64() - t0 > P.spin_limit) {
                    atomicCAS(P.err, kBatchOk, kBatchTimeout);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)P.err == kBatchOk;
}

__device__ __forceinline__ double* basis(const BatchParams& P, int s, int j) {
    const int64_t o = P.off[s];
    return P.V + (int64_t)P.m_max * 3 * o + (int64_t)j * 3 * (P.off[s + 1] - o);
}

// ---------------------------------------------------------------------------
// Phase B: pair products for one item (system s, particles [i0, i0 + NT*NI)).
// Right-hand side A: F_in (float, mdot mode) or a double vector times scaleA;
// right-hand side B (NRHS = 2): the forces Fbuf (float).
// ---------------------------------------------------------------------------
template <int NT, int NI, int NRHS>
__device__ void pair_item(const BatchParams& P, int s, int i0, int jb, int je, const float* srcA_f,
                          const double* srcA_d, double scaleA, double* outA_d, double* outB, double* Vrow_store,
                          double* part_slot, float* st, double* sred) {
    const int tid = threadIdx.x;
    const int64_t o = P.off[s];
    const int Ns = (int)(P.off[s + 1] - o);
    const float pad = (float)kPadCoord;
    const RpyConst<float>& k = P.k;
    // Packed form: each f32x2 instruction evaluates one i against two
    // consecutive j (j-paired), so any i-blocking works; the j-tile is stored
    // as structure-of-arrays floats (x[NT], y[NT], z[NT] in the float4 arrays'
    // memory) so that a float2 load yields the pair (x_j, x_j+1).
    // two tile buffers of nine NT-float arrays (x, y, z, A, B), used in turn:
    // the next tile is written into the idle buffer after the current one is
    // computed, so one barrier per tile separates its writes from the reads of
    // both neighbours
    float *tx, *ty, *tz, *ax, *ay, *az, *bx, *by, *bz;
    auto use_buffer = [&](int b) {
        tx = st + b * 9 * NT; ty = tx + NT; tz = ty + NT;
        ax = tz + NT; ay = ax + NT; az = ay + NT;
        bx = az + NT; by = bx + NT; bz = by + NT;
    };
    float2 xi[NI], yi[NI], zi[NI];
    float2 pA[NI][3], pB[NRHS == 2 ? NI : 1][3];
    float hA[NI][3], lA[NI][3];
    float hB[NRHS == 2 ? NI : 1][3], lB[NRHS == 2 ? NI : 1][3];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int i = i0 + q * NT + tid;
        float x = -pad, y = -pad, z = -pad;
        if (i < Ns) {
            const float4 p = P.pos4[o + i];
            x = p.x; y = p.y; z = p.z;
        }
        // -x_i: d = x_j - x_i is the negated separation (exact); the tt terms are even in d
        xi[q] = make_float2(-x, -x); yi[q] = make_float2(-y, -y); zi[q] = make_float2(-z, -z);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pA[q][c] = make_float2(0.f, 0.f);
            hA[q][c] = lA[q][c] = 0.f;
            if (NRHS == 2) { pB[q][c] = make_float2(0.f, 0.f); hB[q][c] = lB[q][c] = 0.f; }
        }
    }
    const float2 K1 = make_float2(k.K1, k.K1), nK2 = make_float2(-k.K2, -k.K2);
    // this thread's j of the next tile, loaded into registers one tile ahead so
    // that the global-load latency hides behind the current tile's pairs
    float nj[NRHS == 2 ? 9 : 6];
    auto fetch = [&](int j) {
        if (j < je && LM_INBOUNDS(o + j >= 0 && o + j < P.Ntot, 9, o + j)) {
            const float4 pj = P.pos4[o + j];
            nj[0] = pj.x; nj[1] = pj.y; nj[2] = pj.z;
            if (srcA_f) {
                nj[3] = srcA_f[3 * (o + j)]; nj[4] = srcA_f[3 * (o + j) + 1]; nj[5] = srcA_f[3 * (o + j) + 2];
            } else {
                nj[3] = (float)(srcA_d[3 * (o + j)] * scaleA);
                nj[4] = (float)(srcA_d[3 * (o + j) + 1] * scaleA);
                nj[5] = (float)(srcA_d[3 * (o + j) + 2] * scaleA);
            }
            if constexpr (NRHS == 2) {
                nj[6] = P.Fbuf[3 * (o + j)]; nj[7] = P.Fbuf[3 * (o + j) + 1]; nj[8] = P.Fbuf[3 * (o + j) + 2];
            }
        } else {
            nj[0] = nj[1] = nj[2] = pad;
            nj[3] = nj[4] = nj[5] = 0.f;
            if constexpr (NRHS == 2) nj[6] = nj[7] = nj[8] = 0.f;
        }
    };
    auto store_tile = [&](int b) {
        float* t = st + b * 9 * NT;
        t[0 * NT + tid] = nj[0]; t[1 * NT + tid] = nj[1]; t[2 * NT + tid] = nj[2];
        t[3 * NT + tid] = nj[3]; t[4 * NT + tid] = nj[4]; t[5 * NT + tid] = nj[5];
        if constexpr (NRHS == 2) { t[6 * NT + tid] = nj[6]; t[7 * NT + tid] = nj[7]; t[8 * NT + tid] = nj[8]; }
    };
    fetch(jb + tid);
    __syncthreads();   // the previous item's last reads of buffer 0 are done
    store_tile(0);
    __syncthreads();
    int buf = 0;
    for (int jt = jb; jt < je; jt += NT) {
        const bool more = jt + NT < je;
        if (more) fetch(jt + NT + tid);
        use_buffer(buf);
        static_assert(NT % 4 == 0, "the j tile holds whole groups of four");
        // two j-pairs (four j) per overlap vote: two independent packed chains
        // per i-particle; a slot (one i against one j-pair) that holds an
        // overlapping or self pair takes the exact scalar coefficients
        for (int jj = 0; jj < NT; jj += 4) {
            float2 dx[2][NI], dy[2][NI], dz[2][NI], r2[2][NI];
            float mn = 0.f;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int j2 = jj + 2 * u;
                const float2 xj = *reinterpret_cast<const float2*>(tx + j2);
                const float2 yj = *reinterpret_cast<const float2*>(ty + j2);
                const float2 zj = *reinterpret_cast<const float2*>(tz + j2);
#pragma unroll
                for (int q = 0; q < NI; ++q) {
                    dx[u][q] = __fadd2_rn(xj, xi[q]); dy[u][q] = __fadd2_rn(yj, yi[q]); dz[u][q] = __fadd2_rn(zj, zi[q]);
                    r2[u][q] = __ffma2_rn(dx[u][q], dx[u][q], __ffma2_rn(dy[u][q], dy[u][q], __fmul2_rn(dz[u][q], dz[u][q])));
                    const float m2 = fminf(r2[u][q].x, r2[u][q].y);
                    mn = (u == 0 && q == 0) ? m2 : fminf(mn, m2);
                }
            }
            auto slot = [&](int u, int q, bool exact) {
                const int j2 = jj + 2 * u;
                float2 A, B;
                if (exact) {
                    float a_[2], b_[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float rr = h ? r2[u][q].y : r2[u][q].x;
                        if (rr < k.four_a2) {
                            const float invr = (rr > 0.f) ? rsqrtf(rr) : 0.f;
                            const float r = rr * invr;
                            a_[h] = k.nA0 - k.nA1 * r;
                            b_[h] = k.nB * invr;
                        } else {
                            const float invr = rsqrtf(rr);
                            const float invr2 = invr * invr;
                            const float invr3 = invr2 * invr;
                            a_[h] = fmaf(k.K1, invr3, invr);
                            b_[h] = fmaf(-k.K2, invr3 * invr2, invr3);
                        }
                    }
                    A = make_float2(a_[0], a_[1]);
                    B = make_float2(b_[0], b_[1]);
                } else {
                    const float2 invr = make_float2(rsqrtf(r2[u][q].x), rsqrtf(r2[u][q].y));
                    const float2 invr2 = __fmul2_rn(invr, invr);
                    const float2 invr3 = __fmul2_rn(invr2, invr);
                    A = __ffma2_rn(K1, invr3, invr);
                    B = __ffma2_rn(nK2, __fmul2_rn(invr3, invr2), invr3);
                }
                const float2 fx = *reinterpret_cast<const float2*>(ax + j2);
                const float2 fy = *reinterpret_cast<const float2*>(ay + j2);
                const float2 fz = *reinterpret_cast<const float2*>(az + j2);
                const float2 ddx = dx[u][q], ddy = dy[u][q], ddz = dz[u][q];
                const float2 sa_ = __fmul2_rn(B, __ffma2_rn(ddx, fx, __ffma2_rn(ddy, fy, __fmul2_rn(ddz, fz))));
                pA[q][0] = __ffma2_rn(sa_, ddx, __ffma2_rn(A, fx, pA[q][0]));
                pA[q][1] = __ffma2_rn(sa_, ddy, __ffma2_rn(A, fy, pA[q][1]));
                pA[q][2] = __ffma2_rn(sa_, ddz, __ffma2_rn(A, fz, pA[q][2]));
                if constexpr (NRHS == 2) {
                    const float2 gx = *reinterpret_cast<const float2*>(bx + j2);
                    const float2 gy = *reinterpret_cast<const float2*>(by + j2);
                    const float2 gz = *reinterpret_cast<const float2*>(bz + j2);
                    const float2 sb_ = __fmul2_rn(B, __ffma2_rn(ddx, gx, __ffma2_rn(ddy, gy, __fmul2_rn(ddz, gz))));
                    pB[q][0] = __ffma2_rn(sb_, ddx, __ffma2_rn(A, gx, pB[q][0]));
                    pB[q][1] = __ffma2_rn(sb_, ddy, __ffma2_rn(A, gy, pB[q][1]));
                    pB[q][2] = __ffma2_rn(sb_, ddz, __ffma2_rn(A, gz, pB[q][2]));
                }
            };
            if (__any_sync(0xffffffffu, mn < k.four_a2)) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
#pragma unroll
                    for (int q = 0; q < NI; ++q)
                        slot(u, q, __any_sync(0xffffffffu, fminf(r2[u][q].x, r2[u][q].y) < k.four_a2));
                }
            } else {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
#pragma unroll
                    for (int q = 0; q < NI; ++q) slot(u, q, false);
                }
            }
        }
        // TwoSum fold of the tile partials (the two j-lanes first added in FP32)
#pragma unroll
        for (int q = 0; q < NI; ++q) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float pa = pA[q][c].x + pA[q][c].y;
                float sm = hA[q][c] + pa, bb = sm - hA[q][c];
                lA[q][c] += (hA[q][c] - (sm - bb)) + (pa - bb);
                hA[q][c] = sm; pA[q][c] = make_float2(0.f, 0.f);
                if (NRHS == 2) {
                    const float pb = pB[q][c].x + pB[q][c].y;
                    sm = hB[q][c] + pb; bb = sm - hB[q][c];
                    lB[q][c] += (hB[q][c] - (sm - bb)) + (pb - bb);
                    hB[q][c] = sm; pB[q][c] = make_float2(0.f, 0.f);
                }
            }
        }
        if (more) store_tile(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    if (P.pair_count != nullptr && tid == 0)
        atomicAdd(P.pair_count, (unsigned long long)min(NT * NI, Ns - i0) * (unsigned long long)(je - jb));
    // outputs and the partial v_k . w of this item
    double dot = 0.0;
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int i = i0 + q * NT + tid;
        if (i >= Ns) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t g = 3 * (o + i) + c;
            const double wv = P.c8 * ((double)hA[q][c] + (double)lA[q][c]);
            outA_d[3 * i + c] = wv;
            if (part_slot) {
                const double vk = srcA_d[g] * scaleA;
                if (Vrow_store) Vrow_store[3 * i + c] = vk;
                dot = fma(vk, wv, dot);
            }
            if (NRHS == 2) outB[3 * i + c] = P.c8 * ((double)hB[q][c] + (double)lB[q][c]);
        }
    }
    if (part_slot) {
        dot = warp_sum_d(dot);
        if ((tid & 31) == 0) sred[tid >> 5] = dot;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += sred[w];
            *part_slot = t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Vector phases on one chunk (system s, elements [e0, e1) of the system).
// ---------------------------------------------------------------------------
template <int NT>
__device__ void chunk_dots(const BatchParams& P, int s, int e0, int e1, const double* w, int nrows,
                           double* part_out) {
    // Each warp takes eight rows at a time: every lane runs eight independent
    // FP64 chains over its elements (w read once per element; the element
    // loop unrolled twice keeps eighteen loads in flight, which halves the
    // chain of DRAM round trips of one chunk), then a transposing butterfly reduces the eight sums
    // (after the offsets 16, 8 and 4 lane l holds row l >> 2; 9 shuffles and
    // adds instead of 40).
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ns = 3 * (P.off[s + 1] - P.off[s]);
    for (int j0 = wid * 8; j0 < nrows; j0 += NW * 8) {
        const int nr = min(8, nrows - j0);
        const double* v = basis(P, s, 0) + j0 * ns;
        double acc[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r] = 0.0;
#pragma unroll 2
        for (int e = e0 + lane; e < e1; e += 32) {
            const double we = w[e];
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (r < nr) acc[r] = fma(v[r * ns + e], we, acc[r]);
        }
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
        if ((lane & 3) == 0 && (lane >> 2) < nr) part_out[j0 + (lane >> 2)] = acc[0];
    }
}

// Sum of base[c * stride] over c = c0, c0 + step, ... < ce with four
// independent accumulators (four loads in flight; the order depends only on
// c0, step and ce, so every caller with the same range gets the same bits).
__device__ __forceinline__ double strided_sum4(const double* base, int64_t stride, int c0, int step, int ce) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    int c = c0;
    for (; c + 3 * step < ce; c += 4 * step) {
        t0 += base[(int64_t)c * stride];
        t1 += base[(int64_t)(c + step) * stride];
        t2 += base[(int64_t)(c + 2 * step) * stride];
        t3 += base[(int64_t)(c + 3 * step) * stride];
    }
    for (; c < ce; c += step) t0 += base[(int64_t)c * stride];
    return (t0 + t1) + (t2 + t3);
}

// Deterministic warp sum of base[c * stride] for c in [cb, ce): lane-strided
// partial sums, then a butterfly (every lane returns the same value).
__device__ __forceinline__ double warp_range_sum(const double* base, int64_t stride, int cb, int ce) {
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int c = cb + lane; c < ce; c += 32) t += base[(int64_t)c * stride];
    return warp_sum_d(t);
}

// The same sum through L2 (partials that other CTAs wrote since the last
// grid barrier).
__device__ __forceinline__ double warp_range_sum_cg(const double* base, int64_t stride, int cb, int ce) {
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int c = cb + lane; c < ce; c += 32) t += __ldcg(base + (int64_t)c * stride);
    return warp_sum_d(t);
}

// cvec[j] = sum over the chunks of system s of part[c][j], j < nrows.  With
// few rows, G = NT / nrows threads (a power of two, at most 8) share a row
// and combine their partial sums by a butterfly; the order depends only on
// nrows, so every chunk of the system obtains the same coefficients.
template <int NT>
__device__ void chunk_sum_coeffs(const BatchParams& P, int s, const double* part, int nrows, double* cvec) {
    const int cb = P.chunk_range[2 * s], ce = P.chunk_range[2 * s + 1];
    const int64_t M1 = P.m_max + 1;
    int G = 1;
    while (G < 8 && 2 * G * nrows <= NT) G *= 2;
    const int rows_per_pass = NT / G;
    for (int j0 = 0; j0 < nrows; j0 += rows_per_pass) {
        const int j = j0 + threadIdx.x / G, q = threadIdx.x % G;
        double t = 0.0;
        if (j < nrows) t = strided_sum4(part + j, M1, cb + q, G, ce);
        for (int o = 1; o < G; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (j < nrows && q == 0) cvec[j] = t;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Asynchronous tridiagonal solves.  The main CTAs post a request (step,
// system, k) once beta_k is known and keep iterating; each warp of the solver
// CTAs takes one posted request at a time, computes |W| f(T_{k+1}) e1 with
// T_{k+1} = tridiag(beta_0..k-1, alpha_0..k, beta_0..k-1) with all its lanes
// (tridiag_sqrt_e1_warp; the QR form on lane 0 where the quadrature declines)
// and publishes it in the system's result ring under a tag; the main CTAs
// apply the stopping rule in iteration order as results arrive.  Requests of an earlier step are dropped.  Every wait is bounded by
// spin_limit clock cycles without progress of the other side.
// ---------------------------------------------------------------------------
// Requests in flight per system beyond the next pending stopping test.
constexpr int kSpecDepth = 8;

__device__ __forceinline__ unsigned long long res_tag(uint64_t gstep, int k) {
    return (unsigned long long)gstep * 128ull + (unsigned long long)k + 1ull;
}

__device__ __forceinline__ size_t res_index(const BatchParams& P, int s, uint64_t gstep, int k) {
    return ((size_t)s * 2 + (size_t)(gstep & 1)) * (size_t)P.R + (size_t)(k % P.R);
}

__device__ __forceinline__ unsigned long long vload(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

// Post request (gstep, s, k).  Returns false on a timeout.
__device__ bool post_request(const BatchParams& P, uint64_t gstep, int s, int k) {
    atomicAdd(&P.inflight[gstep & 1], 1);
    __threadfence();   // alpha / beta of the request visible before it is posted
    const unsigned long long idx = atomicAdd(&P.q_ctr[1], 1ull);
    const int slot = (int)(idx % (unsigned long long)P.q_cap);
    if (idx >= (unsigned long long)P.q_cap) {
        // the slot's previous request must have been read
        const unsigned long long want = idx - (unsigned long long)P.q_cap + 1ull;
        long long t0 = clock64();
        unsigned long long seen = vload(&P.q_ctr[2]);
        while (vload(&P.q_ack[slot]) != want) {
            if (*(volatile int*)P.err != kBatchOk) return false;
            const unsigned long long now = vload(&P.q_ctr[2]);
            if (now != seen) { seen = now; t0 = clock64(); }
            if (clock64() - t0 > P.spin_limit) { atomicCAS(P.err, kBatchOk, kBatchTimeout); return false; }
            __nanosleep(200);
        }
    }
    P.q_req[slot] = (long long)((gstep << 28) | ((uint64_t)s << 7) | (uint64_t)k);
    __threadfence();
    atomicExch(&P.q_seq[slot], idx + 1ull);
    return true;
}

// Solve the request of ticket idx with the whole warp (every lane calls it
// with the same idx; scr is the warp's scratch, wid its solver-warp index).
// Returns false on an error (the same value on every lane).
__device__ bool serve_request(const BatchParams& P, unsigned long long idx, int lane, int wid, double* scr) {
    const int slot = (int)(idx % (unsigned long long)P.q_cap);
    unsigned long long req = 0;
    int got = 1;
    if (lane == 0) {
        const long long t0 = clock64();
        while (vload(&P.q_seq[slot]) != idx + 1ull) {   // the poster is between its two writes
            if (clock64() - t0 > P.spin_limit) {
                atomicCAS(P.err, kBatchOk, kBatchTimeout);
                got = 0;
                break;
            }
            __nanosleep(100);
        }
        if (got) {
            __threadfence();
            req = (unsigned long long)*(volatile long long*)&P.q_req[slot];
            __threadfence();
            atomicExch(&P.q_ack[slot], idx + 1ull);
        }
    }
    if (!__shfl_sync(0xffffffffu, got, 0)) return false;
    req = __shfl_sync(0xffffffffu, req, 0);
    const uint64_t gstep = req >> 28;
    const int s = (int)((req >> 7) & ((1u << 21) - 1));
    const int k = (int)(req & 127);
    bool ok = true;
    int current = 0;
    if (lane == 0) current = (long long)gstep == *(volatile long long*)P.cur_step;
    if (__shfl_sync(0xffffffffu, current, 0)) {
        const int m = k + 1;
        const double* al = P.alpha + (size_t)s * P.m_max;
        const double* be = P.beta + (size_t)s * P.m_max;
        double* z = scr + 4 * (size_t)P.m_max;
        int rcode = tridiag_sqrt_e1_warp(m, P.m_max, al, be, scr, z, lane);
        if (rcode == 1) {
            // not certified positive definite: the QR form on lane 0
            if (lane == 0) {
                df* d = reinterpret_cast<df*>(scr + 5 * (size_t)P.m_max);
                rcode = tridiag_sqrt_e1_df<1>(m, al, be, d, d + P.m_max, d + 2 * P.m_max,
                                              P.trk + (size_t)wid * P.max_rot,
                                              reinterpret_cast<df*>(P.trc + (size_t)wid * P.max_rot),
                                              reinterpret_cast<df*>(P.trs + (size_t)wid * P.max_rot), P.max_rot, z);
            }
            rcode = __shfl_sync(0xffffffffu, rcode, 0);
            __syncwarp();
        }
        // a request that became stale during the solve may have read the next
        // step's coefficients: its result and status are dropped
        int still = 0;
        if (lane == 0) still = (long long)gstep == *(volatile long long*)P.cur_step;
        if (__shfl_sync(0xffffffffu, still, 0)) {
            if (rcode != 0) {
                if (lane == 0) atomicCAS(P.err, kBatchOk, kBatchTridiag);
                ok = false;
            } else {
                const size_t ri = res_index(P, s, gstep, k);
                double* zr = P.zres + ri * P.m_max;
                const double nw = __ldcg(P.normW + s);
                for (int i = lane; i < m; i += 32) zr[i] = z[i] * nw;
                __threadfence();
                __syncwarp();
                if (lane == 0) atomicExch(&P.zdone[ri], res_tag(gstep, k));
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        atomicSub(&P.inflight[gstep & 1], 1);
        atomicAdd(&P.q_ctr[2], 1ull);
    }
    return ok;
}

__device__ void solver_loop(const BatchParams& P) {
    // every solver warp serves one request at a time with all its lanes
    const int lane = threadIdx.x & 31;
    const int wid = ((blockIdx.x - P.n_main) * blockDim.x + threadIdx.x) >> 5;
    double* scr = P.sv_w + (size_t)wid * tridiag_warp_scratch_doubles(P.m_max);
    // idle wait: bounded by spin_limit cycles without any sign of progress of
    // the main CTAs (barrier generation, item tickets, posted requests)
    unsigned hb_bar = 0;
    unsigned long long hb_ticket = 0, hb_tail = 0;
    long long t0 = clock64();
    while (true) {
        unsigned long long first = 0;
        int n = 0, quit = 0;
        if (lane == 0) {
            const unsigned long long h = vload(&P.q_ctr[0]);
            const unsigned long long t = vload(&P.q_ctr[1]);
            if (t > h && atomicCAS(&P.q_ctr[0], h, h + 1ull) == h) {
                n = 1;
                first = h;
            }
            if (n == 0) {
                if (*(volatile int*)P.main_done || *(volatile int*)P.err != kBatchOk) {
                    quit = 1;
                } else {
                    const unsigned b = *(volatile unsigned*)(P.bar + 1);
                    const unsigned long long tk = vload(P.ticket);
                    if (b != hb_bar || tk != hb_ticket || t != hb_tail) {
                        hb_bar = b; hb_ticket = tk; hb_tail = t;
                        t0 = clock64();
                    } else if (clock64() - t0 > P.spin_limit) {
                        atomicCAS(P.err, kBatchOk, kBatchTimeout);
                        quit = 1;
                    }
                }
            }
        }
        n = __shfl_sync(0xffffffffu, n, 0);
        quit = __shfl_sync(0xffffffffu, quit, 0);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (quit) return;
        if (n == 0) {
            __nanosleep(256);
            continue;
        }
        serve_request(P, first, lane, wid, scr);
        if (lane == 0) t0 = clock64();
    }
}

// Stopping rule of one system on the results that have arrived, in iteration
// order (thread 0 of the system's CTA).  Returns true when the system stops.
__device__ bool evaluate_results(const BatchParams& P, int s, uint64_t gstep, int upto) {
    const int k0 = P.k0s[s];
    while (P.next_check[s] <= upto) {
        const int j = P.next_check[s];
        if (j < k0) { P.next_check[s] = j + 1; continue; }
        const size_t rj = res_index(P, s, gstep, j);
        if (vload(&P.zdone[rj]) != res_tag(gstep, j)) return false;   // not there yet
        __threadfence();
        const double* zj = P.zres + rj * P.m_max;
        const int m = j + 1;
        bool stop = false;
        if (j >= 1 && j >= k0 + 1) {
            const double* zp = P.zres + res_index(P, s, gstep, j - 1) * P.m_max;
            double dn = 0.0, zn = 0.0;
            for (int i = 0; i < m; ++i) {
                const double zi = __ldcg(zj + i);
                const double dd = zi - (i < m - 1 ? __ldcg(zp + i) : 0.0);
                dn += dd * dd;
                zn += zi * zi;
            }
            const double rel = (zn > 0.0) ? sqrt(dn / zn) : 0.0;
            P.rel[s] = rel;
            if (rel < P.tol) stop = true;
        }
        if (!stop && P.state[s] >= 2 && j == P.last_k[s]) {
            stop = true;
            if (P.state[s] == 2) P.notconv[s] = 1;   // max_iter reached; a breakdown is converged
        }
        if (stop) {
            double* zf = P.z + (size_t)s * P.m_max;
            for (int i = 0; i < m; ++i) zf[i] = __ldcg(zj + i);
            P.msys[s] = m;
            P.itsum[s] += m;
            P.kprev[s] = m;
            P.state[s] = 0;
            P.active[s] = 0;
            return true;
        }
        P.next_check[s] = j + 1;
    }
    return false;
}

// Post the due requests of system s: iterations after the last one posted,
// from k0 on, up to kmax and at most kSpecDepth beyond the next iteration
// whose stopping test is pending (bounded speculation: a system that keeps
// iterating while its results are pending does not flood the solvers).
__device__ bool post_due(const BatchParams& P, int s, uint64_t gstep, int kmax) {
    const int hi = min(kmax, P.next_check[s] + kSpecDepth);
    for (int j = max(P.posted[s] + 1, P.k0s[s]); j <= hi; ++j) {
        if (!post_request(P, gstep, s, j)) return false;
        P.posted[s] = j;
    }
    return true;
}

// End of Lanczos iteration k of system s (one thread, once per iteration:
// the thread that closed the system's last chunk), with b2 = |w|^2 after the
// reorthogonalisation: beta_k, breakdown and max_iter, the stopping rule on
// the results that have arrived, the due solve requests, and the count of
// systems that iterate on.  Warm start (BD mode): with kprev the iteration
// count of the system's previous step, solves begin at (0-based) iteration
// k0 = kprev - 3 and the relative-change test one iteration later, at the
// count kprev - 1 (one below the previous count, so that counts can also
// fall), since counts change little from one step to the next; breakdown and
// max_iter end the iteration at once.  A system keeps iterating while its
// results are pending; iterations past its stopping point are discarded.
__device__ void end_iteration(const BatchParams& P, int s, int k, uint64_t gstep, double b2) {
    const double b = sqrt(b2);
    P.beta[s * P.m_max + k] = b;
    const int m = k + 1;
    const bool breakdown = b <= P.brk_rel * __ldcg(P.amax + s);
    const bool last = (m == P.m_max);
    if (breakdown || last) {
        if (k < P.k0s[s]) P.k0s[s] = k;   // the last iteration is always solved
        P.state[s] = breakdown ? 3 : 2;
        P.last_k[s] = k;
        P.active[s] = 0;
    }
    if (evaluate_results(P, s, gstep, k)) return;
    if (!post_due(P, s, gstep, k)) return;   // a timeout: the error flag is set
    if (P.state[s] == 1) atomicAdd(&P.nact[k + 1], 1);
}

// Evaluate and post for system s (states 2, 3: iteration ended) until it
// stops.  The wait is bounded by spin_limit cycles without a finished
// request.  Returns false on a timeout or an error.
__device__ bool drain_system(const BatchParams& P, int s, uint64_t gstep) {
    long long t0 = clock64();
    unsigned long long seen = vload(&P.q_ctr[2]);
    while (P.state[s] != 0) {
        if (evaluate_results(P, s, gstep, P.last_k[s])) break;
        if (!post_due(P, s, gstep, P.last_k[s])) return false;
        if (*(volatile int*)P.err != kBatchOk) return false;
        const unsigned long long now = vload(&P.q_ctr[2]);
        if (now != seen) { seen = now; t0 = clock64(); }
        if (clock64() - t0 > P.spin_limit) { atomicCAS(P.err, kBatchOk, kBatchTimeout); return false; }
        __nanosleep(200);
    }
    return true;
}

template <int NT, int NI>
__global__ void __launch_bounds__(NT) batch_kernel(BatchParams P) {
    if (blockIdx.x >= P.n_main) {
        solver_loop(P);
        return;
    }
    __shared__ float s_tile[2 * 9 * NT];
    __shared__ double sred[NT / 32];
    __shared__ double cvec[129];
    __shared__ unsigned long long s_ticket;
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int G = P.n_main;
    const int per_item = NT * NI;
    unsigned long long base = 0;

    // dynamic item loop: calls fn(t) for items t handed out by the ticket counter
    auto for_items = [&](auto&& fn) {
        while (true) {
            if (tid == 0) s_ticket = atomicAdd(P.ticket, 1ull);
            __syncthreads();
            const unsigned long long t = s_ticket;
            __syncthreads();
            if (t - base >= (unsigned long long)P.n_items) break;
            fn((int)(t - base));
        }
        base += (unsigned long long)P.n_items + (unsigned long long)G;
    };

    // item t: system, first particle, j-part [jp * kBatchJPart, ...)
    auto item_args = [&](int t, int& s, int& i0, int& jp, int& jb, int& je, double*& wout, double*& uout) {
        s = P.items[3 * t];
        i0 = P.items[3 * t + 1];
        jp = P.items[3 * t + 2];
        const int ns = (int)(P.off[s + 1] - P.off[s]);
        jb = jp * kBatchJPart;
        je = min(jb + kBatchJPart, ns);
        wout = P.wsplit + P.woff[s] + (int64_t)jp * 3 * ns;
        uout = P.usplit + P.woff[s] + (int64_t)jp * 3 * ns;
    };
    // sum of the j-part partials of system s at element e
    auto sum_parts = [&](const double* split, int s, int e) {
        const int ns = (int)(P.off[s + 1] - P.off[s]);
        const int parts = (ns + kBatchJPart - 1) / kBatchJPart;
        const double* b = split + P.woff[s];
        double t = 0.0;
        for (int p = 0; p < parts; ++p) t += b[(int64_t)p * 3 * ns + e];
        return t;
    };

    if (P.mode == kBatchMdot) {
        for_items([&](int t) {
            int s, i0, jp, jb, je;
            double *wout, *uout;
            item_args(t, s, i0, jp, jb, je, wout, uout);
            pair_item<NT, NI, 1>(P, s, i0, jb, je, P.F_in, nullptr, 1.0, wout, nullptr, nullptr, nullptr, s_tile, sred);
        });
        if (!grid_sync(P)) return;
        if (blockIdx.x == 0 && tid == 0) atomicExch(P.main_done, 1);
        for (int c = blockIdx.x; c < P.n_chunks; c += G) {
            const int s = P.chunks[2 * c], e0 = P.chunks[2 * c + 1];
            const int64_t o = P.off[s];
            const int ns3 = 3 * (int)(P.off[s + 1] - o);
            const int e1 = min(e0 + kBatchChunk, ns3);
            for (int e = e0 + tid; e < e1; e += NT) P.lin_out[3 * o + e] = (float)sum_parts(P.wsplit, s, e);
        }
        (void)per_item;
        return;
    }

    const int nsteps = (P.mode == kBatchBD) ? P.nsteps : 1;
    const double sq = sqrt(2.0 * P.kT * P.dt);
    const int M1 = P.m_max + 1;
    double* partA = P.part_chunk;
    double* partB = P.part_chunk + (int64_t)P.n_chunks * M1;

    for (int step = 0; step < nsteps; ++step) {
        const uint64_t gstep = (uint64_t)(P.step0 + step);
        int slot = 0;
        stamp(P, step, slot);
        // ---- A1: noise, forces, |W|^2 partials
        if (blockIdx.x == 0) {
            for (int k = tid; k <= P.m_max; k += NT) {
                P.nact[k] = 0;
                P.pass2[k] = 0;
            }
            if (tid == 0) {
                atomicExch((unsigned long long*)P.cur_step, (unsigned long long)gstep);
                // requests of two steps ago (same result-ring parity) all finished:
                // no stale result can land in a slot of this step
                long long t0 = clock64();
                unsigned long long seen = vload(&P.q_ctr[2]);
                while (*(volatile int*)&P.inflight[gstep & 1] != 0) {
                    const unsigned long long now = vload(&P.q_ctr[2]);
                    if (now != seen) { seen = now; t0 = clock64(); }
                    if (clock64() - t0 > P.spin_limit) { atomicCAS(P.err, kBatchOk, kBatchTimeout); break; }
                    __nanosleep(200);
                }
            }
        }
        for (int c = blockIdx.x; c < P.n_chunks; c += G) {
            const int s = P.chunks[2 * c], e0 = P.chunks[2 * c + 1];
            const int64_t o = P.off[s];
            const int ns = 3 * (int)(P.off[s + 1] - o);
            const int e1 = min(e0 + kBatchChunk, ns);
            double* v0 = basis(P, s, 0);
            double acc = 0.0;
            if (P.W_in != nullptr) {
                for (int e = e0 + tid; e < e1; e += NT) {
                    const double wv = P.W_in[3 * o + e];
                    v0[e] = wv;
                    acc = fma(wv, wv, acc);
                }
            } else {
                const uint64_t stream = (P.mode == kBatchBD) ? ((gstep << 32) | (uint64_t)s) : (uint64_t)s;
                for (int q = e0 / 4 + tid; 4 * q < e1; q += NT) {
                    double zz[4];
                    philox_normals4(P.seed, stream, (uint64_t)q, zz);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int e = 4 * q + t;
                        if (e < e1) { v0[e] = zz[t]; acc = fma(zz[t], zz[t], acc); }
                    }
                }
            }
            if (P.mode == kBatchBD)
                for (int e = e0 + tid; e < e1; e += NT) P.Fbuf[3 * o + e] = (float)(-P.k_trap * P.x64[3 * o + e]);
            acc = warp_sum_d(acc);
            if ((tid & 31) == 0) sred[tid >> 5] = acc;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < NT / 32; ++w) t += sred[w];
                partA[(int64_t)c * M1] = t;
                if (e0 == 0) {
                    P.sys_cnt[s] = 0;
                    P.amax[s] = 0.0;
                    P.active[s] = 1;
                    P.state[s] = 1;
                    P.msys[s] = 0;
                    P.next_check[s] = 0;
                    P.last_k[s] = -1;
                    P.posted[s] = -1;
                    P.k0s[s] = (P.warm_start && P.kprev[s] > 0) ? max(0, P.kprev[s] - 3) : 0;
                }
            }
            __syncthreads();
        }
        if (!grid_sync(P)) return;
        stamp(P, step, slot);
        // ---- A2: normalise
        for (int c = blockIdx.x; c < P.n_chunks; c += G) {
            const int s = P.chunks[2 * c], e0 = P.chunks[2 * c + 1];
            const int ns = 3 * (int)(P.off[s + 1] - P.off[s]);
            const int e1 = min(e0 + kBatchChunk, ns);
            chunk_sum_coeffs<NT>(P, s, partA, 1, cvec);
            const double nw = sqrt(cvec[0]);
            if (e0 == 0 && tid == 0) {
                P.normW[s] = nw;
                if (!(nw > 0.0)) { P.active[s] = 0; P.state[s] = 0; }   // W = 0: zero output, no iterations
            }
            if (nw > 0.0) {
                double* v0 = basis(P, s, 0);
                const double inv = 1.0 / nw;
                for (int e = e0 + tid; e < e1; e += NT) v0[e] *= inv;
            }
            __syncthreads();
        }
        if (!grid_sync(P)) return;
        stamp(P, step, slot);
        // ---- Lanczos iterations
        for (int k = 0; k < P.m_max; ++k) {
            double* wcur = (k & 1) ? P.w1 : P.w0;
            double* wprev = (k & 1) ? P.w0 : P.w1;
            // B: products
            for_items([&](int t) {
                int s, i0, jp, jb, je;
                double *wout, *uout;
                item_args(t, s, i0, jp, jb, je, wout, uout);
                if (!P.active[s]) return;
                const int64_t o = P.off[s];
                if (k == 0) {
                    const double* v0 = basis(P, s, 0) - 3 * o;  // indexed by global element
                    if (P.mode == kBatchBD)
                        pair_item<NT, NI, 2>(P, s, i0, jb, je, nullptr, v0, 1.0, wout, uout, nullptr,
                                             &P.part_item[t], s_tile, sred);
                    else
                        pair_item<NT, NI, 1>(P, s, i0, jb, je, nullptr, v0, 1.0, wout, nullptr, nullptr,
                                             &P.part_item[t], s_tile, sred);
                } else {
                    const double invb = 1.0 / P.beta[s * P.m_max + k - 1];
                    pair_item<NT, NI, 1>(P, s, i0, jb, je, nullptr, wprev, invb, wout, nullptr,
                                         jp == 0 ? basis(P, s, k) : nullptr, &P.part_item[t], s_tile, sred);
                }
            });
            if (!grid_sync(P)) return;
            stamp(P, step, slot);
            // C2: alpha, three-term update, first Gram-Schmidt dots
            for (int c = blockIdx.x; c < P.n_chunks; c += G) {
                const int s = P.chunks[2 * c], e0 = P.chunks[2 * c + 1];
                if (!P.active[s]) continue;
                const int64_t o = P.off[s];
                const int ns = 3 * (int)(P.off[s + 1] - o);
                const int e1 = min(e0 + kBatchChunk, ns);
                const double alpha = warp_range_sum(P.part_item, 1, P.item_range[2 * s], P.item_range[2 * s + 1]);
                if (e0 == 0 && tid == 0) {
                    P.alpha[s * P.m_max + k] = alpha;
                    P.amax[s] = fmax(P.amax[s], fabs(alpha));
                }
                const double bprev = (k > 0) ? P.beta[s * P.m_max + k - 1] : 0.0;
                const double* vk = basis(P, s, k);
                const double* vkm1 = (k > 0) ? basis(P, s, k - 1) : vk;
                double* w = wcur + 3 * o;
                double h0 = 0.0;
                for (int e = e0 + tid; e < e1; e += NT) {
                    const double we = sum_parts(P.wsplit, s, e) - (alpha * vk[e] + bprev * vkm1[e]);
                    w[e] = we;
                    h0 = fma(we, we, h0);
                    if (k == 0 && P.mode == kBatchBD) P.u[3 * o + e] = sum_parts(P.usplit, s, e);
                }
                // |w|^2 before the Gram-Schmidt pass, in the spare last slot
                h0 = warp_sum_d(h0);
                if ((tid & 31) == 0) sred[tid >> 5] = h0;
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    for (int ww = 0; ww < NT / 32; ++ww) t += sred[ww];
                    partA[(int64_t)c * M1 + P.m_max] = t;
                }
                chunk_dots<NT>(P, s, e0, e1, w, k + 1, partA + (int64_t)c * M1);
                __syncthreads();
            }
            if (!grid_sync(P)) return;
            stamp(P, step, slot);
            // C3: first Gram-Schmidt pass and |w|^2 after it.  The CTA that
            // finishes a system's last chunk makes the system's DGKS test: a
            // system that needs no second pass (the usual case) ends its
            // iteration there (end_iteration), the others raise pass2[k].
            // C4, only when pass2[k] is set: the second pass of the systems whose
            // |w| dropped below |w_before| / sqrt(2): its dots (C4a), then the
            // subtraction and the |w|^2 partials, and the end of the iteration by
            // each such system's last chunk (C4b).
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) {
                    if (*(volatile int*)&P.pass2[k] == 0) {
                        stamp(P, step, slot);
                        break;
                    }
                    for (int c = blockIdx.x; c < P.n_chunks; c += G) {
                        const int s = P.chunks[2 * c], e0 = P.chunks[2 * c + 1];
                        if (!P.active[s]) continue;
                        const int cb = P.chunk_range[2 * s], ce = P.chunk_range[2 * s + 1];
                        const double h0 = warp_range_sum(partA + P.m_max, M1, cb, ce);
                        const double h1 = warp_range_sum(partB + P.m_max, M1, cb, ce);
                        if (!(P.reorth || h1 < 0.5 * h0)) continue;
                        const int64_t o = P.off[s];
                        const int ns = 3 * (int)(P.off[s + 1] - o);
                        const int e1 = min(e0 + kBatchChunk, ns);
                        chunk_dots<NT>(P, s, e0, e1, wcur + 3 * o, k + 1, partB + (int64_t)c * M1);
                        __syncthreads();
                    }
                    if (!grid_sync(P)) return;
                }
                const double* pin = pass == 0 ? partA : partB;
                double* pout = pass == 0 ? partB : partA;
                for (int c = blockIdx.x; c < P.n_chunks; c += G) {
                    const int s = P.chunks[2 * c], e0 = P.chunks[2 * c + 1];
                    if (!P.active[s]) continue;
                    const int64_t o = P.off[s];
                    const int ns = 3 * (int)(P.off[s + 1] - o);
                    const int e1 = min(e0 + kBatchChunk, ns);
                    const int cb = P.chunk_range[2 * s], ce = P.chunk_range[2 * s + 1];
                    if (pass == 1) {
                        const double h0 = warp_range_sum(partA + P.m_max, M1, cb, ce);
                        const double h1 = warp_range_sum(partB + P.m_max, M1, cb, ce);
                        if (!(P.reorth || h1 < 0.5 * h0)) continue;   // squared norms: |w1| < |w0| / sqrt(2)
                    }
                    double* w = wcur + 3 * o;
                    const double* V0 = basis(P, s, 0);
                    double nrm = 0.0;
                    chunk_sum_coeffs<NT>(P, s, pin, k + 1, cvec);
                    // the thread's kBatchChunk / NT elements advance together:
                    // independent FP64 chains and loads in flight per row
                    static_assert(kBatchChunk % NT == 0, "a chunk is a whole number of elements per thread");
                    constexpr int EPT = kBatchChunk / NT;
                    double acc[EPT];
#pragma unroll
                    for (int q = 0; q < EPT; ++q) {
                        const int e = e0 + tid + q * NT;
                        acc[q] = (e < e1) ? w[e] : 0.0;
                    }
#pragma unroll 2
                    for (int j = 0; j <= k; ++j) {
                        const double cj = cvec[j];
                        const double* vj = V0 + (int64_t)j * ns;
#pragma unroll
                        for (int q = 0; q < EPT; ++q) {
                            const int e = e0 + tid + q * NT;
                            if (e < e1) acc[q] = fma(-cj, vj[e], acc[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < EPT; ++q) {
                        const int e = e0 + tid + q * NT;
                        if (e < e1) {
                            w[e] = acc[q];
                            nrm = fma(acc[q], acc[q], nrm);
                        }
                    }
                    __syncthreads();
                    nrm = warp_sum_d(nrm);
                    if ((tid & 31) == 0) sred[tid >> 5] = nrm;
                    __syncthreads();
                    if (tid == 0) {
                        double t = 0.0;
                        for (int ww = 0; ww < NT / 32; ++ww) t += sred[ww];
                        pout[(int64_t)c * M1 + (pass == 0 ? P.m_max : 0)] = t;
                        // the system's last chunk of this pass (its partials are all written)
                        __threadfence();
                        s_last = atomicAdd(&P.sys_cnt[s], 1) == ce - cb - 1;
                        if (s_last) P.sys_cnt[s] = 0;
                    }
                    __syncthreads();
                    if (s_last && tid < 32) {
                        __threadfence();
                        if (pass == 0) {
                            const double h0 = warp_range_sum_cg(partA + P.m_max, M1, cb, ce);
                            const double h1 = warp_range_sum_cg(partB + P.m_max, M1, cb, ce);
                            if (tid == 0) {
                                if (P.reorth || h1 < 0.5 * h0) atomicExch(&P.pass2[k], 1);
                                else end_iteration(P, s, k, gstep, h1);   // w unchanged: beta from the first pass
                            }
                        } else {
                            const double b2 = warp_range_sum_cg(partA, M1, cb, ce);
                            if (tid == 0) end_iteration(P, s, k, gstep, b2);
                        }
                    }
                    __syncthreads();
                }
                if (!grid_sync(P)) return;
                stamp(P, step, slot);
            }
            stamp(P, step, slot);   // the end-of-iteration work ran inside C3 / C4
            if (*(volatile int*)&P.nact[k + 1] == 0) break;
        }
        // ---- wait for the last results of every system
        for (int s = blockIdx.x; s < P.S; s += G) {
            if (tid != 0 || P.state[s] == 0) continue;
            if (!drain_system(P, s, gstep)) break;
        }
        if (!grid_sync(P)) return;
        stamp(P, step, slot);
        // ---- D: combine and update
        for (int c = blockIdx.x; c < P.n_chunks; c += G) {
            const int s = P.chunks[2 * c], e0 = P.chunks[2 * c + 1];
            const int64_t o = P.off[s];
            const int ns = 3 * (int)(P.off[s + 1] - o);
            const int e1 = min(e0 + kBatchChunk, ns);
            const int m = P.msys[s];
            for (int j = tid; j < m; j += NT) cvec[j] = P.z[s * P.m_max + j];
            __syncthreads();
            const double* V0 = basis(P, s, 0);
            for (int e = e0 + tid; e < e1; e += NT) {
                double y = 0.0;
                for (int j = 0; j < m; ++j) y = fma(cvec[j], V0[(int64_t)j * ns + e], y);
                if (P.mode == kBatchBD) {
                    const double xn = P.x64[3 * o + e] + P.dt * P.u[3 * o + e] + sq * y;
                    P.x64[3 * o + e] = xn;
                    float* pf = reinterpret_cast<float*>(P.pos4 + o + e / 3);
                    pf[e % 3] = (float)xn;
                } else {
                    P.lin_out[3 * o + e] = (float)(P.prefactor * y);
                }
            }
            __syncthreads();
        }
        if (!grid_sync(P)) return;
        stamp(P, step, slot);
    }
    if (blockIdx.x == 0 && tid == 0) atomicExch(P.main_done, 1);
}

__global__ void batch_pack_kernel(const float* __restrict__ pos, int64_t N, float4* __restrict__ pos4,
                                  double* __restrict__ x64, int* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    const float m = (float)kMaxAbsCoord;
    if (!(fabsf(x) <= m && fabsf(y) <= m && fabsf(z) <= m)) atomicExch(bad, 1);
    pos4[i] = make_float4(x, y, z, 0.f);
    x64[3 * i] = x; x64[3 * i + 1] = y; x64[3 * i + 2] = z;
}

__global__ void batch_unpack_kernel(const double* __restrict__ x64, int64_t n, float* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = (float)x64[e];
}

// Every CTA waits at a barrier that expects one CTA more than the grid has.
__global__ void timeout_probe_kernel(BatchParams P) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = P.bar + 1;
        const unsigned g = *gen;
        atomicAdd(P.bar, 1u);   // never reaches gridDim.x + 1
        const long long t0 = clock64();
        while (*gen == g) {
            if (clock64() - t0 > P.spin_limit) {
                atomicCAS(P.err, kBatchOk, kBatchTimeout);
                break;
            }
            __nanosleep(100);
        }
    }
    __syncthreads();
}

// One thread per system: out = sqrt(T) e1 with the device tridiagonal step.
// One warp per system: the warp form of the tridiagonal step, the QR form on
// lane 0 where it declines (path[c] = 1), exactly as the solver warps of the
// batched kernel run it.
__global__ void tridiag_warp_kernel(int count, int m, const double* alpha, const double* beta, double* scratch,
                                    int* rk, double* rc, double* rs, int max_rot, double* out, int* status,
                                    int* path) {
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= count) return;   // whole warps
    double* scr = scratch + (size_t)w * tridiag_warp_scratch_doubles(m);
    const double* al = alpha + (size_t)w * m;
    const double* be = beta + (size_t)w * m;
    double* o = out + (size_t)w * m;
    int rcode = tridiag_sqrt_e1_warp(m, m, al, be, scr, o, lane);
    const int qr = rcode == 1;
    if (qr) {
        if (lane == 0) {
            df* d = reinterpret_cast<df*>(scr + 5 * (size_t)m);
            rcode = tridiag_sqrt_e1_df<1>(m, al, be, d, d + m, d + 2 * m, rk + (size_t)w * max_rot,
                                          reinterpret_cast<df*>(rc + (size_t)w * max_rot),
                                          reinterpret_cast<df*>(rs + (size_t)w * max_rot), max_rot, o);
        }
        rcode = __shfl_sync(0xffffffffu, rcode, 0);
    }
    if (lane == 0) {
        if (rcode != 0) atomicCAS(status, 0, rcode);
        if (path != nullptr) path[w] = qr;
    }
}

template <int NT, int NI>
cudaError_t launch_nt(const BatchParams& p, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel<NT, NI>, p);
}

template <int NT, int NI>
int occ_nt() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<NT, NI>, NT, 0) != cudaSuccess) return 0;
    return n;
}

}  // namespace

bool batch_tiling_supported(int threads, int ilp) {
    return (threads == 64 || threads == 128) && (ilp == 1 || ilp == 2);
}

int batch_ctas_per_sm(int threads, int ilp) {
    if (threads == 64 && ilp == 1) return occ_nt<64, 1>();
    if (threads == 64 && ilp == 2) return occ_nt<64, 2>();
    if (threads == 128 && ilp == 1) return occ_nt<128, 1>();
    if (threads == 128 && ilp == 2) return occ_nt<128, 2>();
    return 0;
}

cudaError_t launch_batch(const BatchParams& p, int threads, int ilp, int grid, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidConfiguration;
    if (threads == 64 && ilp == 1) e = launch_nt<64, 1>(p, grid, s);
    else if (threads == 64 && ilp == 2) e = launch_nt<64, 2>(p, grid, s);
    else if (threads == 128 && ilp == 1) e = launch_nt<128, 1>(p, grid, s);
    else if (threads == 128 && ilp == 2) e = launch_nt<128, 2>(p, grid, s);
    count_launches(1);
    return e;
}

cudaError_t launch_batch_pack(const float* pos, int64_t N, float4* pos4, double* x64, int* bad, cudaStream_t s) {
    batch_pack_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(pos, N, pos4, x64, bad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batch_unpack(const double* x64, int64_t N, float* out, cudaStream_t s) {
    batch_unpack_kernel<<<(unsigned)((3 * N + 255) / 256), 256, 0, s>>>(x64, 3 * N, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tridiag_dev(int count, int m, const double* alpha, const double* beta, double* scratch, int* rk,
                               double* rc, double* rs, int max_rot, double* out, int* status, int* path,
                               cudaStream_t s) {
    tridiag_warp_kernel<<<(count + 3) / 4, 128, 0, s>>>(count, m, alpha, beta, scratch, rk, rc, rs, max_rot, out,
                                                        status, path);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batch_timeout_probe(unsigned* bar, int* err, long long spin_limit, int grid, cudaStream_t s) {
    BatchParams p = {};
    p.bar = bar;
    p.err = err;
    p.spin_limit = spin_limit;
    timeout_probe_kernel<<<grid, 32, 0, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lmk
