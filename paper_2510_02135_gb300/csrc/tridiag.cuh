// f(T) e1 with f = sqrt for a small symmetric tridiagonal T, the last step
// of the Krylov square root M^{1/2} W ~ |W| V_m T_m^{1/2} e1 (libMobility
// paper, Sec. 3.3).  Eigen-decomposition by implicit symmetric QR steps with
// Wilkinson shifts and bulge chasing (Golub & Van Loan, "Matrix
// Computations", Sec. 8.3), written for host and device.
#pragma once

#include <cmath>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace lmk {

// d[0..m-1] diagonal, e[0..m-2] off-diagonal (destroyed); Q is m x m
// row-major and receives the eigenvectors in its columns; on return d holds
// the eigenvalues.  Returns 0, or -1 if 30 m QR steps did not converge.
__host__ __device__ inline int tridiag_eig(int m, double* d, double* e, double* Q) {
    const double eps = 2.220446049250313e-16;
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) Q[r * m + c] = (r == c) ? 1.0 : 0.0;
    int steps = 0;
    int hi = m - 1;
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        if (++steps > 30 * m) return -1;
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
        const double delta = 0.5 * (d[hi - 1] - d[hi]);
        const double bb = e[hi - 1];
        const double den = delta + copysign(hypot(delta, bb), delta);
        const double mu = d[hi] - bb * bb / den;
        double x = d[lo] - mu;
        double z = e[lo];
        for (int k = lo; k < hi; ++k) {
            // rotation J = [[c, -s], [s, c]] with J^T [x; z] = [r; 0]
            const double r = hypot(x, z);
            double c = 1.0, s = 0.0;
            if (r > 0.0) { c = x / r; s = z / r; }
            if (k > lo) e[k - 1] = r;
            const double ak = d[k], ak1 = d[k + 1], bk = e[k];
            d[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
            d[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
            e[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
            if (k < hi - 1) {
                x = e[k];
                z = s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
            for (int rr = 0; rr < m; ++rr) {
                const double q0 = Q[rr * m + k], q1 = Q[rr * m + k + 1];
                Q[rr * m + k] = c * q0 + s * q1;
                Q[rr * m + k + 1] = -s * q0 + c * q1;
            }
        }
    }
    return 0;
}

// out = f(T) e1, f = sqrt, with eigenvalues below zero (round-off) clamped
// to zero; *clamped counts them.  work needs m*m + 2m doubles.
__host__ __device__ inline int tridiag_sqrt_e1(int m, const double* alpha, const double* beta, double* work,
                                               double* out, int* clamped) {
    double* Q = work;
    double* d = work + m * m;
    double* e = d + m;
    for (int i = 0; i < m; ++i) d[i] = alpha[i];
    for (int i = 0; i + 1 < m; ++i) e[i] = beta[i];
    const int rc = tridiag_eig(m, d, e, Q);
    int nclamp = 0;
    for (int r = 0; r < m; ++r) out[r] = 0.0;
    for (int i = 0; i < m; ++i) {
        double lam = d[i];
        if (lam < 0.0) { lam = 0.0; ++nclamp; }
        const double w = sqrt(lam) * Q[0 * m + i];
        for (int r = 0; r < m; ++r) out[r] += w * Q[r * m + i];
    }
    if (clamped) *clamped = nclamp;
    return rc;
}

}  // namespace lmk
