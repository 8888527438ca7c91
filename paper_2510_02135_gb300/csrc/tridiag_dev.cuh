// Device forms of the tridiagonal step f(T) e1, f = sqrt (the last step of the
// Krylov square root M^{1/2} W ~ |W| V_m T_m^{1/2} e1, libMobility paper,
// Sec. 3.3): the warp-parallel quadrature at the end of this file, and, for a
// T that it declines, the QR form on one thread.  The QR form is the algorithm of tridiag.cuh (implicit
// symmetric QR with Wilkinson shifts, Golub & Van Loan Sec. 8.3; the
// rotations' product Q applied to e1 during the sweeps and, in reverse, to
// f(Lambda) Q^T e1 afterwards), in double-float arithmetic.
//
// Why double-float: on this GPU FP64 instructions issue at about one per 64
// cycles per SM sub-partition whether or not they depend on each other, so a
// QR sweep in FP64 costs ~64 cycles for every FP64 operation (about 30 per
// rotation).  A double-float number is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi) / 2, 48 significant bits); its operations are short
// sequences of FP32 instructions (error-free transformations: Knuth's TwoSum,
// Dekker's FastTwoSum, the FMA-based exact product; Dekker 1971, "A
// floating-point technique for extending the available precision"), which the
// FP32 pipes issue every cycle.  Additions use the form whose error is bounded
// by a few units of 2^-48 relative to the operands' magnitudes (like FP64
// rounding of inexact operands), which is what the backward stability of the
// QR iteration needs.
//
// Scaling: T is multiplied by 4^-k (exact) so that its largest entry lies in
// [1/4, 1) and every product stays inside the FP32 exponent range; the result
// is multiplied by 2^k.  Deflation and shift decisions are made on the hi
// parts.  1/t and 1/sqrt(t) start from the FP32 hardware estimates and take
// one third-order correction, y (1 + e + e^2) with e = 1 - t y for 1/t and
// y (1 + h/2 + 3 h^2 / 8) with h = 1 - t y^2 for 1/sqrt(t) (the binomial
// series of (1 - e)^-1 and (1 - h)^-1/2 to second order: the estimates'
// relative error of about 2^-22 becomes about 2^-66, below double-float
// precision).
#pragma once

#include <cstdint>

#include "lm_internal.cuh"
#include "tridiag.cuh"

namespace lmk {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}

__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = a.hi * b;
    const float e = fmaf(a.hi, b, -p);
    return fast_two_sum(p, fmaf(a.lo, b, e));
}

__device__ __forceinline__ df df_sqr(df a) {
    const float p = a.hi * a.hi;
    const float e = fmaf(a.hi, a.hi, -p);
    return fast_two_sum(p, fmaf(2.f * a.hi, a.lo, e));
}

__device__ __forceinline__ float approx_rcp_f32(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float approx_rsqrt_f32(float x) {
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1 / a, a != 0, |a.hi| a normal FP32 number.
__device__ __forceinline__ df df_rcp(df a) {
    const float y = approx_rcp_f32(a.hi);
    const df e = df_add({1.f, 0.f}, df_neg(df_mulf(a, y)));       // 1 - a y, about 2^-22
    const df c = df_mulf(df_add(e, {e.hi * e.hi, 0.f}), y);       // y (e + e^2)
    return df_add({y, 0.f}, c);
}

// 1 / sqrt(a), a > 0, a.hi a normal FP32 number.
__device__ __forceinline__ df df_rsqrt(df a) {
    const float y = approx_rsqrt_f32(a.hi);
    const float p = y * y;
    const df yy = {p, fmaf(y, y, -p)};                             // y^2 exactly
    const df h = df_add({1.f, 0.f}, df_neg(df_mul(a, yy)));       // 1 - a y^2, about 2^-22
    const df t = df_add(df_mulf(h, 0.5f), {0.375f * h.hi * h.hi, 0.f});
    return df_add({y, 0.f}, df_mulf(t, y));
}

__device__ __forceinline__ df df_from_scaled(double x, int two_k) {   // x 4^-k = x 2^-two_k
    const double xs = ldexp(x, -two_k);
    const float h = (float)xs;
    return {h, (float)(xs - (double)h)};
}

// |e| <= eps (|d1| + |d2|) with eps = 2^-48, the double-float unit roundoff.
__device__ __forceinline__ bool df_negligible(df e, df d1, df d2) {
    return fabsf(e.hi) <= 3.5527136788005009e-15f * (fabsf(d1.hi) + fabsf(d2.hi));
}

// out = sqrt(T) e1 for T = tridiag(beta[0..m-2], alpha[0..m-1], beta[0..m-2]).
// Element i of d, e, r and entry t of rk, rc, rs are at [i * ST], [t * ST];
// out[i * ST] is FP64.  d, e, r: m entries of scratch; rk, rc, rs: max_rot
// entries.  Eigenvalues below zero (round-off) are clamped to 0.  Returns 0;
// -1 if 30 m QR steps did not converge; -2 if more than max_rot rotations
// were needed; -3 if T has a non-finite entry.
template <int ST>
__device__ int tridiag_sqrt_e1_df(int m, const double* alpha, const double* beta, df* __restrict__ d,
                                  df* __restrict__ e, df* __restrict__ r, int* __restrict__ rk, df* __restrict__ rc,
                                  df* __restrict__ rs, int max_rot, double* __restrict__ out) {
    // scale: 4^-k with the largest |entry| in [1/4, 1)
    float amax = 0.f;
    #pragma unroll 1
    for (int i = 0; i < m; ++i) amax = fmaxf(amax, fabsf((float)load_coef(alpha + i)));
    #pragma unroll 1
    for (int i = 0; i + 1 < m; ++i) amax = fmaxf(amax, fabsf((float)load_coef(beta + i)));
    if (!(amax <= 3.0e38f)) return -3;
    if (amax == 0.f) {
        #pragma unroll 1
        for (int i = 0; i < m; ++i) out[i * ST] = 0.0;
        return 0;
    }
    int ex = 0;
    frexpf(amax, &ex);                     // amax in [2^(ex-1), 2^ex)
    const int k = (ex + 1) >> 1;           // 4^-k amax in [2^(ex-1-2k), 2^(ex-2k)), ex - 2k in {-1, 0}
    #pragma unroll 1
    for (int i = 0; i < m; ++i) {
        d[i * ST] = df_from_scaled(load_coef(alpha + i), 2 * k);
        r[i * ST] = {(i == 0) ? 1.f : 0.f, 0.f};
    }
    #pragma unroll 1
    for (int i = 0; i + 1 < m; ++i) e[i * ST] = df_from_scaled(load_coef(beta + i), 2 * k);

    int steps = 0, nr = 0;
    int hi = m - 1;
    while (hi > 0) {
        if (df_negligible(e[(hi - 1) * ST], d[(hi - 1) * ST], d[hi * ST])) {
            e[(hi - 1) * ST] = {0.f, 0.f};
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && !df_negligible(e[(lo - 1) * ST], d[(lo - 1) * ST], d[lo * ST])) --lo;
        if (lo > 0) e[(lo - 1) * ST] = {0.f, 0.f};
        if (++steps > 30 * m) return -1;
        if (nr + (hi - lo) > max_rot) return -2;
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
        const df dh = d[hi * ST];
        const df delta = df_mulf(df_sub(d[(hi - 1) * ST], dh), 0.5f);
        const df bb = e[(hi - 1) * ST];
        const df b2 = df_sqr(bb);
        const df h2 = df_add(df_sqr(delta), b2);                   // > 0: bb is not negligible
        df hyp = df_mul(h2, df_rsqrt(h2));
        if (delta.hi < 0.f) hyp = df_neg(hyp);
        const df mu = df_sub(dh, df_mul(b2, df_rcp(df_add(delta, hyp))));
        // bulge chase over [lo, hi]: (ak, bk) = current d[k], e[k]; ra = r[k]
        df ak = d[lo * ST], bk = e[lo * ST], ra = r[lo * ST];
        df x = df_sub(ak, mu), z = bk;
        #pragma unroll 1
        for (int kk = lo; kk < hi; ++kk) {
            const df ak1 = d[(kk + 1) * ST];
            const df bk1 = (kk + 1 < hi) ? e[(kk + 1) * ST] : df{0.f, 0.f};
            const df rb = r[(kk + 1) * ST];
            const df zz = df_sqr(z);
            const df x2 = df_sqr(x);
            const df t2 = df_add(x2, zz);
            df c, s, nrm, ek, dk, dk1;
            if (t2.hi > 1e-37f) {
                const df u = df_rcp(t2);
                const df q = df_rsqrt(t2);
                c = df_mul(x, q);
                s = df_mul(z, q);
                nrm = df_mul(t2, q);
                const df xz = df_mul(x, z);
                // e_k' = (x z (ak1 - ak) + (x^2 - z^2) bk) / t2 = c s (ak1 - ak) + (c^2 - s^2) bk
                const df pq = df_add(df_mul(xz, df_sub(ak1, ak)), df_mul(df_sub(x2, zz), bk));
                // d_k' = ak - g / t2, d_k+1' = ak1 + g / t2, g = z^2 (ak - ak1) - 2 x z bk
                const df g = df_sub(df_mul(zz, df_sub(ak, ak1)), df_mulf(df_mul(xz, bk), 2.f));
                const df gu = df_mul(g, u);
                ek = df_mul(pq, u);
                dk1 = df_add(ak1, gu);
                dk = df_sub(ak, gu);
            } else {   // |x|, |z| below about 3e-19 of the largest entry: identity rotation
                c = {1.f, 0.f};
                s = {0.f, 0.f};
                nrm = {0.f, 0.f};
                ek = bk;
                dk = ak;
                dk1 = ak1;
            }
            if (kk > lo) e[(kk - 1) * ST] = nrm;
            d[kk * ST] = dk;
            r[kk * ST] = df_add(df_mul(c, ra), df_mul(s, rb));     // r <- J^T r on (kk, kk+1)
            ra = df_sub(df_mul(c, rb), df_mul(s, ra));
            rk[nr * ST] = kk;
            rc[nr * ST] = c;
            rs[nr * ST] = s;
            ++nr;
            if (kk + 1 < hi) {
                x = ek;
                z = df_mul(s, bk1);
                bk = df_mul(c, bk1);
            } else {
                e[kk * ST] = ek;
            }
            ak = dk1;
        }
        d[hi * ST] = ak;
        r[hi * ST] = ra;
    }
    // v = sqrt(Lambda) Q^T e1 (into r), then out = Q v: the rotations in
    // reverse; within a sweep out[kk + 1] of one rotation is out[kk] of the
    // one replayed just before, carried in a register.
    #pragma unroll 1
    for (int i = 0; i < m; ++i) {
        const df lam = d[i * ST];
        df v = {0.f, 0.f};
        if (lam.hi > 1e-36f) v = df_mul(r[i * ST], df_mul(lam, df_rsqrt(lam)));
        r[i * ST] = v;
    }
    int cidx = -1;
    df cval = {0.f, 0.f};
    #pragma unroll 1
    for (int t = nr - 1; t >= 0; --t) {
        const int kk = rk[t * ST];
        const df c = rc[t * ST], s = rs[t * ST];
        const df a = r[kk * ST];
        df b;
        if (cidx == kk + 1) b = cval;
        else b = r[(kk + 1) * ST];
        const df na = df_sub(df_mul(c, a), df_mul(s, b));
        const df nb = df_add(df_mul(s, a), df_mul(c, b));
        r[(kk + 1) * ST] = nb;
        r[kk * ST] = na;
        cidx = kk;
        cval = na;
    }
    #pragma unroll 1
    for (int i = 0; i < m; ++i) {
        const df v = r[i * ST];
        out[i * ST] = ldexp((double)v.hi + (double)v.lo, k);
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Warp form of the same step: one warp computes sqrt(T) e1 for one T.
//
// The QR iteration above is a chain of dependent rotations: about m^2 of
// them, so one solve at m = 48 takes milliseconds on one thread.  For a
// symmetric positive definite T the warp form uses the integral
//   T^{-1/2} e1 = (2/pi) int_0^inf (T + t^2 I)^{-1} e1 dt
// (for a scalar lambda > 0 it is the elementary arctan integral).  With t = e^u
// the integrand of one eigen-component becomes (1 / (2 sqrt(lambda)))
// sech(u - log sqrt(lambda)), analytic in the strip |Im u| < pi/2, so the
// trapezoid rule of step h converges geometrically: the sum of h sech(k h - c)
// over all k equals pi (1 + 2 sum_n cos(2 pi n c / h) / cosh(pi^2 n / h))
// (Poisson summation), a relative error of at most about 4 exp(-pi^2 / h).
// The rule is truncated L beyond the spectrum on both sides, where the
// neglected tails are about 2 exp(-L) relative.  Each node is one tridiagonal
// solve (T + t_k^2 I) x_k = e1, independent of the others: the 32 lanes take
// the nodes in turn, u = sum_k w_k x_k with w_k = (2/pi) h t_k, and
// sqrt(T) e1 = T u.
//
// The lower end of the spectrum comes from FP32 Sturm counts (multisection:
// 32 points per round, five rounds); a count in floating point is exact for a
// matrix whose entries differ from T's by a few units of roundoff relative
// (Kahan; Demmel, Applied Numerical Linear Algebra, Sec. 5.3.4), so the bound
// is lowered by a margin of that size.  If the bound cannot certify that T is
// positive definite with lambda_min at least twice that margin, the warp
// form declines and the caller runs the QR form (which also clamps negative
// eigenvalues to zero).
// ---------------------------------------------------------------------------

// Trapezoid step and truncation margin for a relative error of about 1e-13:
// h = pi^2 / ln(4 / 1e-13), L = ln(2 / (pi 1e-13)).
constexpr double kQuadH = 0.31512246914760783;
constexpr double kQuadL = 29.48202350363314;
// Margin of the FP32 Sturm bound, relative to the largest |entry| of the
// scaled T (a few units of FP32 roundoff on each entry, with room to spare).
constexpr float kSturmMargin = 4e-6f;

// Number of eigenvalues of T below x (count of negative pivots of T - x I),
// FP32, on the hi parts; a zero pivot is replaced by a tiny negative one.
__device__ __forceinline__ int sturm_count_f32(int m, const df* __restrict__ d, const df* __restrict__ b2, float x) {
    float q = d[0].hi - x;
    int c = q < 0.f;
    for (int i = 1; i < m; ++i) {
        if (fabsf(q) < 1e-30f) q = -1e-30f;
        q = (d[i].hi - x) - b2[i - 1].hi * approx_rcp_f32(q);
        c += q < 0.f;
    }
    return c;
}

__device__ __forceinline__ df df_from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// exp(32 h) and (2 / pi) h for the node recurrence t_{k+32} = t_k exp(32 h)
// and the weights w_k = (2 / pi) h t_k.
constexpr double kQuadR32 = 23954.68052402656;
constexpr double kQuadW = 0.20061319457666027;

// out[i] = (sqrt(T) e1)_i, i < m, for T = tridiag(beta[0..m-2], alpha[0..m-1],
// beta[0..m-2]), 1 <= m <= m_max, by the quadrature above.  Called by all 32
// lanes of a warp with the same arguments (lane = its lane index); scr is the
// warp's scratch of tridiag_warp_scratch_doubles(m_max) doubles (lm_internal.cuh),
// out holds m doubles: the z slot of scr (scr + 4 m_max) or memory outside it.  Returns 0 (out written), 1 (declined: T not certified
// positive definite; out untouched) or -3 (a non-finite entry).
__device__ int tridiag_sqrt_e1_warp(int m, int m_max, const double* alpha, const double* beta, double* scr,
                                    double* out, int lane) {
    df* d = reinterpret_cast<df*>(scr);
    df* bb = d + m_max;
    df* b2 = bb + m_max;
    df* u = b2 + m_max;
    df* inv = reinterpret_cast<df*>(scr + 5 * (size_t)m_max);   // [row][lane]
    df* acc = inv + 32 * (size_t)m_max;                          // [row][lane]
    if (!LM_INBOUNDS(m >= 1 && m <= m_max, 15, m)) return -3;   // the scratch holds m_max rows

    // scale by 4^-k as the QR form does (largest |entry| in [1/4, 1))
    float amax = 0.f;
    bool bad = false;
    for (int i = lane; i < m; i += 32) {
        const double a = load_coef(alpha + i);
        const double b = (i + 1 < m) ? load_coef(beta + i) : 0.0;
        bad |= !isfinite(a) || !isfinite(b);
        amax = fmaxf(amax, fmaxf(fabsf((float)a), fabsf((float)b)));
    }
    if (__any_sync(0xffffffffu, bad || !(amax <= 3.0e38f))) return -3;
    amax = warp_max_f(amax);
    if (amax == 0.f) {
        for (int i = lane; i < m; i += 32) out[i] = 0.0;
        return 0;
    }
    int ex = 0;
    frexpf(amax, &ex);
    const int k = (ex + 1) >> 1;
    for (int i = lane; i < m; i += 32) {
        d[i] = df_from_scaled(load_coef(alpha + i), 2 * k);
        const df b = (i + 1 < m) ? df_from_scaled(load_coef(beta + i), 2 * k) : df{0.f, 0.f};
        bb[i] = b;
        b2[i] = df_sqr(b);
    }
    __syncwarp();

    // Gershgorin interval, widened by the Sturm margin
    const float margin = kSturmMargin * ldexpf(amax, -2 * k);
    float glo = 3.0e38f, ghi = -3.0e38f;
    for (int i = lane; i < m; i += 32) {
        const float r = fabsf(bb[i].hi) + (i > 0 ? fabsf(bb[i - 1].hi) : 0.f);
        glo = fminf(glo, d[i].hi - r);
        ghi = fmaxf(ghi, d[i].hi + r);
    }
    glo = warp_min_f(glo) - margin;
    ghi = warp_max_f(ghi) + margin;
    if (!(ghi > 0.f)) return 1;

    // lower end of the spectrum: lo keeps a computed count of zero
    float lo = glo, hi = ghi;
    for (int round = 0; round < 5; ++round) {
        const float step = (hi - lo) * (1.f / 33.f);
        const float x = lo + step * (float)(lane + 1);
        const unsigned zero = __ballot_sync(0xffffffffu, sturm_count_f32(m, d, b2, x) == 0);
        const int j = 32 - __clz((int)zero);   // highest lane with a zero count, plus one
        const float nlo = (j == 0) ? lo : lo + step * (float)j;
        const float nhi = (j == 32) ? hi : lo + step * (float)(j + 1);
        lo = nlo;
        hi = nhi;
    }
    const float a_lo = lo - margin;   // lambda_min >= a_lo
    if (!(a_lo >= margin)) return 1;

    // nodes t_k = exp(u0 + k h), k = 0 .. n-1, lane l takes k = l, l + 32, ...
    const float u0 = 0.5f * logf(a_lo) - (float)kQuadL;
    const float u1 = 0.5f * logf(ghi) + (float)kQuadL;
    const int n = (int)ceilf((u1 - u0) / (float)kQuadH) + 1;
    for (int r = 0; r < m; ++r) acc[r * 32 + lane] = df{0.f, 0.f};
    const df r32 = df_from_double(kQuadR32), cw = df_from_double(kQuadW);
    df t = df_from_double(exp((double)u0 + (double)lane * kQuadH));
    for (int kk = lane; kk < n; kk += 32) {
        const df s = df_sqr(t);
        const df w = df_mul(cw, t);
        // pivots from the bottom: D_{m-1} = d_{m-1} + s, D_r = d_r + s - b_r^2 / D_{r+1}
        df iv = df_rcp(df_add(d[m - 1], s));
        inv[(m - 1) * 32 + lane] = iv;
        for (int r = m - 2; r >= 0; --r) {
            iv = df_rcp(df_sub(df_add(d[r], s), df_mul(b2[r], iv)));
            inv[r * 32 + lane] = iv;
        }
        // (T + s I)^{-1} e1 from the top: x_0 = 1 / D_0, x_{r+1} = -b_r x_r / D_{r+1}
        df x = iv;
        acc[lane] = df_add(acc[lane], df_mul(w, x));
        for (int r = 0; r + 1 < m; ++r) {
            x = df_neg(df_mul(df_mul(bb[r], x), inv[(r + 1) * 32 + lane]));
            acc[(r + 1) * 32 + lane] = df_add(acc[(r + 1) * 32 + lane], df_mul(w, x));
        }
        t = df_mul(t, r32);
    }
    __syncwarp();

    // u = sum over the lanes (fixed order), then sqrt(T) e1 = T u, unscaled by 2^k
    for (int r = lane; r < m; r += 32) {
        df sum = acc[r * 32];
#pragma unroll 1
        for (int l = 1; l < 32; ++l) sum = df_add(sum, acc[r * 32 + l]);
        u[r] = sum;
    }
    __syncwarp();
    for (int r = lane; r < m; r += 32) {
        df zr = df_mul(d[r], u[r]);
        if (r > 0) zr = df_add(zr, df_mul(bb[r - 1], u[r - 1]));
        if (r + 1 < m) zr = df_add(zr, df_mul(bb[r], u[r + 1]));
        out[r] = ldexp((double)zr.hi + (double)zr.lo, k);
    }
    return 0;
}

}  // namespace lmk
