// f(T) e1 with f = sqrt for a small symmetric tridiagonal T, the last step
// of the Krylov square root M^{1/2} W ~ |W| V_m T_m^{1/2} e1 (libMobility
// paper, Sec. 3.3).  Eigenvalues by implicit symmetric QR steps with
// Wilkinson shifts and bulge chasing (Golub & Van Loan, "Matrix
// Computations", Sec. 8.3).  The eigenvector matrix Q is the product of the
// Givens rotations of all QR steps, Q = J_1 J_2 ... J_K; instead of forming it
// (O(m^3)), the rotations are recorded and applied to two vectors:
//   r = Q^T e1 = J_K^T ... J_1^T e1,   z = Q (f(Lambda) r) = J_1 ... J_K (f(Lambda) r),
// which costs O(K) = O(m^2).  Host and device.
#pragma once

#include <cmath>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace lmk {

// 1 / sqrt(t) for t > 0.  On the device FP64 square root and division are
// long dependent sequences, so the rotation uses Newton-Raphson iteration for
// the reciprocal square root, y <- y (3 - t y^2) / 2, from the FP32 estimate:
// two steps take the ~2^-22 relative error of the seed below FP64 rounding
// (quadratic convergence).  Outside the FP32 range, and on the host, it is
// the plain quotient.
__host__ __device__ inline double inv_sqrt(double t) {
#ifdef __CUDA_ARCH__
    if (t > 1e-36 && t < 1e36) {
        double y = (double)rsqrtf((float)t);
        y = y * fma(-0.5 * t, y * y, 1.5);
        y = y * fma(-0.5 * t, y * y, 1.5);
        return y;
    }
#endif
    return 1.0 / sqrt(t);
}

// Load of a coefficient that another CTA may have written (on the device
// through L2, bypassing the SM's L1).
__host__ __device__ inline double load_coef(const double* p) {
#ifdef __CUDA_ARCH__
    return __ldcg(p);
#else
    return *p;
#endif
}

// d[0..m-1] diagonal, e[0..m-2] off-diagonal (both destroyed; d receives the
// eigenvalues).  Rotation t acts on (rk[t], rk[t]+1) with (rc[t], rs[t]).
// Returns 0; -1 if 30 m QR steps did not converge; -2 if more than max_rot
// rotations were needed.  Element i of every array is at [i * ST]: ST = 1 for
// a plain array, ST = 32 for the lane-interleaved scratch of a warp whose 32
// lanes solve 32 systems side by side (coalesced accesses).
// Deflation test |e| <= eps (|d1| + |d2|).  On the device the comparison is
// made in FP32 (a dependent FP64 compare costs ~130 cycles there); it only
// decides when an off-diagonal entry is negligible, and the FP32 operands
// differ from the FP64 ones by one rounding, far below the threshold's scale.
__host__ __device__ inline bool negligible(double e, double d1, double d2) {
#ifdef __CUDA_ARCH__
    return fabsf((float)e) <= 2.220446049250313e-16f * (fabsf((float)d1) + fabsf((float)d2));
#else
    return fabs(e) <= 2.220446049250313e-16 * (fabs(d1) + fabs(d2));
#endif
}

template <int ST = 1>
__host__ __device__ inline int tridiag_qr_rotations(int m, double* d, double* e, int* rk, double* rc, double* rs,
                                                    int max_rot, int* nrot) {
    int steps = 0, nr = 0;
    int hi = m - 1;
    while (hi > 0) {
        if (negligible(e[(hi - 1) * ST], d[(hi - 1) * ST], d[hi * ST])) {
            e[(hi - 1) * ST] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && !negligible(e[(lo - 1) * ST], d[(lo - 1) * ST], d[lo * ST])) --lo;
        if (lo > 0) e[(lo - 1) * ST] = 0.0;
        if (++steps > 30 * m) { *nrot = nr; return -1; }
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
        const double delta = 0.5 * (d[(hi - 1) * ST] - d[hi * ST]);
        const double bb = e[(hi - 1) * ST];
        const double den = delta + copysign(sqrt(delta * delta + bb * bb), delta);
        const double mu = d[hi * ST] - bb * bb / den;
        double x = d[lo * ST] - mu;
        double z = e[lo * ST];
        for (int k = lo; k < hi; ++k) {
            // rotation J = [[c, -s], [s, c]] on (k, k+1) with J^T [x; z] = [r; 0]
            // entries of T are of the order of the mobility: no over/underflow in x^2 + z^2
            const double t2 = x * x + z * z;
            double c = 1.0, s = 0.0, r = 0.0;
            if (t2 > 0.0) {
                const double inv = inv_sqrt(t2);
                c = x * inv;
                s = z * inv;
                r = t2 * inv;
            }
            if (k > lo) e[(k - 1) * ST] = r;
            const double ak = d[k * ST], ak1 = d[(k + 1) * ST], bk = e[k * ST];
            d[k * ST] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
            d[(k + 1) * ST] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
            e[k * ST] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
            if (k < hi - 1) {
                x = e[k * ST];
                z = s * e[(k + 1) * ST];
                e[(k + 1) * ST] = c * e[(k + 1) * ST];
            }
            if (nr >= max_rot) { *nrot = nr; return -2; }
            rk[nr * ST] = k; rc[nr * ST] = c; rs[nr * ST] = s;
            ++nr;
        }
    }
    *nrot = nr;
    return 0;
}

// out = f(T) e1, f = sqrt, eigenvalues below zero (round-off) clamped to 0
// and counted in *clamped.  d, e: m doubles of scratch each; rk, rc, rs:
// max_rot entries of scratch.
// alpha, beta: plain arrays (stride 1); d, e, rk, rc, rs, out: stride ST.
template <int ST = 1>
__host__ __device__ inline int tridiag_sqrt_e1(int m, const double* alpha, const double* beta, double* d, double* e,
                                               int* rk, double* rc, double* rs, int max_rot, double* out,
                                               int* clamped) {
    for (int i = 0; i < m; ++i) d[i * ST] = load_coef(alpha + i);
    for (int i = 0; i + 1 < m; ++i) e[i * ST] = load_coef(beta + i);
    int nr = 0;
    const int rc_ = tridiag_qr_rotations<ST>(m, d, e, rk, rc, rs, max_rot, &nr);
    if (rc_ != 0) return rc_;
    // r = Q^T e1
    for (int i = 0; i < m; ++i) out[i * ST] = (i == 0) ? 1.0 : 0.0;
    for (int t = 0; t < nr; ++t) {
        const int k = rk[t * ST];
        const double c = rc[t * ST], s = rs[t * ST];
        const double a = out[k * ST], b = out[(k + 1) * ST];
        out[k * ST] = c * a + s * b;
        out[(k + 1) * ST] = -s * a + c * b;
    }
    int nclamp = 0;
    for (int i = 0; i < m; ++i) {
        double lam = d[i * ST];
        if (lam < 0.0) { lam = 0.0; ++nclamp; }
        out[i * ST] *= sqrt(lam);
    }
    // z = Q v
    for (int t = nr - 1; t >= 0; --t) {
        const int k = rk[t * ST];
        const double c = rc[t * ST], s = rs[t * ST];
        const double a = out[k * ST], b = out[(k + 1) * ST];
        out[k * ST] = c * a - s * b;
        out[(k + 1) * ST] = s * a + c * b;
    }
    if (clamped) *clamped = nclamp;
    return 0;
}

}  // namespace lmk
