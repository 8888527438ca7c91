/*
 * FP64 CPU oracle for the open-boundary Rotne-Prager-Yamakawa (RPY) mobility.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA library.
 *
 * What it computes (libMobility paper, Sec. 2):
 *   - the grand mobility M of Eq. (block_mobility): a 6N x 6N matrix acting on
 *     [F;T] (all forces, then all torques) and giving [u;w] (all linear, then
 *     all angular velocities);
 *   - each 3x3 pair block is the double envelope integral of the free-space
 *     Stokes Green's function, Eq. (stokestomob), with the RPY envelopes:
 *     delta_F uniform on the sphere surface, delta_T uniform in the ball.
 *     The closed forms written below are the classical ones (Rotne & Prager
 *     1969; Yamakawa 1970) and, for overlapping spheres r < 2a, those of
 *     Wajnryb, Mizerski, Zuk & Szymczak (J. Fluid Mech. 2013).  The paper
 *     names the RPY kernel (Sec. 3.5, NBody) but does not print it; the tests
 *     pin these forms to a numerical quadrature of Eq. (stokestomob).
 *   - the self blocks are the single-sphere Stokes drags, (6 pi eta a)^-1 I
 *     (Sec. 3.5, SelfMobility) and (8 pi eta a^3)^-1 I.
 *
 * Conventions: d = x_i - x_j, r = |d|, e = d / r, [e]x v = e x v.
 *   uF (M_uF)  = att I + btt e e^T
 *   uT (M_uT)  = g [e]x          (u_i from T_j)
 *   wF (M_wF)  = g [e]x          (w_i from F_j; equal to uT for the same pair)
 *   wT (M_wT)  = arr I + brr e e^T
 * The full matrix is symmetric because uT(i,j) = wF(j,i)^T ([e]x is odd in e
 * and antisymmetric).
 *
 * Coincident distinct particles (r = 0, i != j) take the r -> 0 limit of the
 * overlap forms, which equals the self blocks.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* Scalar coefficient functions of the pair blocks and their r-derivatives.
 * c[0]=att c[1]=btt c[2]=g c[3]=arr c[4]=brr ; dc[k] = d c[k] / dr. */
static void orc_coefficients(double r, double a, double eta, double c[5], double dc[5])
{
    const double pi = ORC_PI;
    if (r >= 2.0 * a) {
        /* far field, r >= 2a (Rotne-Prager-Yamakawa) */
        const double k8 = 1.0 / (8.0 * pi * eta);
        const double r2 = r * r, r3 = r2 * r, r4 = r2 * r2;
        c[0] = k8 * (1.0 / r + 2.0 * a * a / (3.0 * r3));
        c[1] = k8 * (1.0 / r - 2.0 * a * a / r3);
        c[2] = -k8 / r2;
        c[3] = -1.0 / (16.0 * pi * eta * r3);
        c[4] = 3.0 / (16.0 * pi * eta * r3);
        dc[0] = k8 * (-1.0 / r2 - 2.0 * a * a / r4);
        dc[1] = k8 * (-1.0 / r2 + 6.0 * a * a / r4);
        dc[2] = 2.0 * k8 / r3;
        dc[3] = 3.0 / (16.0 * pi * eta * r4);
        dc[4] = -9.0 / (16.0 * pi * eta * r4);
    } else {
        /* overlapping spheres, r < 2a (Wajnryb et al. 2013) */
        const double k6 = 1.0 / (6.0 * pi * eta * a);
        const double kc = 1.0 / (16.0 * pi * eta * a * a);
        const double kr = 1.0 / (8.0 * pi * eta * a * a * a);
        const double s = r / a;
        c[0] = k6 * (1.0 - 9.0 * s / 32.0);
        c[1] = k6 * (3.0 * s / 32.0);
        c[2] = -kc * s * (1.0 - 3.0 * s / 8.0);
        c[3] = kr * (1.0 - 27.0 * s / 32.0 + 5.0 * s * s * s / 64.0);
        c[4] = kr * (9.0 * s / 32.0 - 3.0 * s * s * s / 64.0);
        dc[0] = k6 * (-9.0 / 32.0) / a;
        dc[1] = k6 * (3.0 / 32.0) / a;
        dc[2] = -kc * (1.0 - 3.0 * s / 4.0) / a;
        dc[3] = kr * (-27.0 / 32.0 + 15.0 * s * s / 64.0) / a;
        dc[4] = kr * (9.0 / 32.0 - 9.0 * s * s / 64.0) / a;
    }
}

/* ([v]x)_{ab} such that ([v]x) w = v x w */
static void orc_cross_matrix(const double v[3], double m[9])
{
    m[0] = 0.0;   m[1] = -v[2]; m[2] = v[1];
    m[3] = v[2];  m[4] = 0.0;   m[5] = -v[0];
    m[6] = -v[1]; m[7] = v[0];  m[8] = 0.0;
}

/* The four 3x3 pair blocks (row-major) for separation d = x_i - x_j. */
void orc_pair_blocks(const double d[3], double a, double eta,
                     double uF[9], double uT[9], double wF[9], double wT[9])
{
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double e[3] = {0.0, 0.0, 0.0};
    if (r > 0.0) {
        e[0] = d[0] / r; e[1] = d[1] / r; e[2] = d[2] / r;
    }
    double c[5], dc[5];
    orc_coefficients(r, a, eta, c, dc);
    double ex[9];
    orc_cross_matrix(e, ex);
    for (int p = 0; p < 3; ++p) {
        for (int q = 0; q < 3; ++q) {
            const double id = (p == q) ? 1.0 : 0.0;
            uF[3 * p + q] = c[0] * id + c[1] * e[p] * e[q];
            wT[3 * p + q] = c[3] * id + c[4] * e[p] * e[q];
            uT[3 * p + q] = c[2] * ex[3 * p + q];
            wF[3 * p + q] = c[2] * ex[3 * p + q];
        }
    }
}

/* Derivatives of the four pair blocks with respect to d_k, k = 0..2:
 * dB[k*9 + 3p + q] = d B_pq / d d_k.  Undefined at r = 0; returns zeros there
 * (the self block does not depend on the positions). */
void orc_pair_blocks_grad(const double d[3], double a, double eta,
                          double duF[27], double duT[27], double dwF[27], double dwT[27])
{
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    memset(duF, 0, 27 * sizeof(double));
    memset(duT, 0, 27 * sizeof(double));
    memset(dwF, 0, 27 * sizeof(double));
    memset(dwT, 0, 27 * sizeof(double));
    if (!(r > 0.0)) return;
    const double e[3] = {d[0] / r, d[1] / r, d[2] / r};
    double c[5], dc[5];
    orc_coefficients(r, a, eta, c, dc);
    double ex[9];
    orc_cross_matrix(e, ex);
    for (int k = 0; k < 3; ++k) {
        /* de_p / dd_k = (delta_pk - e_p e_k) / r */
        double de[3];
        for (int p = 0; p < 3; ++p) de[p] = (((p == k) ? 1.0 : 0.0) - e[p] * e[k]) / r;
        double dex[9];
        orc_cross_matrix(de, dex);
        for (int p = 0; p < 3; ++p) {
            for (int q = 0; q < 3; ++q) {
                const double id = (p == q) ? 1.0 : 0.0;
                const double eeq = e[p] * e[q];
                const double deeq = de[p] * e[q] + e[p] * de[q];
                duF[9 * k + 3 * p + q] = dc[0] * e[k] * id + dc[1] * e[k] * eeq + c[1] * deeq;
                dwT[9 * k + 3 * p + q] = dc[3] * e[k] * id + dc[4] * e[k] * eeq + c[4] * deeq;
                duT[9 * k + 3 * p + q] = dc[2] * e[k] * ex[3 * p + q] + c[2] * dex[3 * p + q];
                dwF[9 * k + 3 * p + q] = duT[9 * k + 3 * p + q];
            }
        }
    }
}

/*
 * Single no-slip wall at z = 0 (NBody with z = "single_wall", Sec. 3.5: the
 * Swan-Brady kernel).
 *
 * Definition.  With G_B(x, y) the Blake (1971) Green's function of a point
 * force at y above the wall (Stokeslet, minus its mirror image, plus the
 * image Stokes doublet and source dipole at y* = (y1, y2, -y3)), the
 * Swan & Brady (2007) RPY blocks for field particle i at x and source
 * particle j at y are
 *   uF = (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y) G_B / (8 pi eta)
 *   wF = 1/2 curl_x (1 + a^2/6 Lap_y) G_B / (8 pi eta)
 *   uT = 1/2 curl_y (1 + a^2/6 Lap_x) G_B / (8 pi eta)   (curl on the column)
 *   wT = 1/4 curl_x curl_y G_B / (8 pi eta).
 * The free-space Stokeslet part of G_B gives the open RPY blocks above; this
 * function returns the remainder (the wall part), including i = j.
 *
 * Closed forms (derived by hand from the definition and pinned to it by the
 * tests), in units 1/(8 pi eta): R = x - y* = rho e, c = e_z, s = sqrt(1 - c^2),
 * h = y_z (height of the source).  In the frame (t, n, z) with t the
 * horizontal direction of R (any horizontal unit vector when s = 0) and
 * n = z x t the nonzero components are
 *   uF: tt = -2/rho + c^2/rho + 4ch/rho^2 - 4h^2/rho^3 - 6c^3 h/rho^2 + 6c^2h^2/rho^3
 *            + a^2 (10c^4 - 10c^2 + 4/3)/rho^3 + a^4 (-70c^4/3 + 70c^2/3 - 8/3)/rho^5
 *       tz = s [-c/rho + 2h/rho^2 - 6c^2 h/rho^2 + 6ch^2/rho^3 + a^2 (10c^3 - 2c)/rho^3
 *               + a^4 (-70c^3/3 + 10c)/rho^5]
 *       nn = -1/rho - 2ch/rho^2 + 2h^2/rho^3 + a^2 (2c^2 - 2/3)/rho^3 + a^4 (2/3 - 10c^2/3)/rho^5
 *       zt = s [-c/rho + 2h/rho^2 + 6c^2 h/rho^2 - 6ch^2/rho^3 - a^2 (10c^3 - 2c)/rho^3
 *               + a^4 (70c^3/3 - 10c)/rho^5]
 *       zz = -1/rho - c^2/rho + 2ch/rho^2 - 2h^2/rho^3 - 6c^3 h/rho^2 + 6c^2h^2/rho^3
 *            + a^2 (10c^4 - 4c^2 - 2/3)/rho^3 + a^4 (-70c^4/3 + 20c^2 - 2)/rho^5
 *   wF: tn = -c/rho^2 + 2h/rho^3 - 2a^2 c/rho^4
 *       nt = c/rho^2 + 4h/rho^3 - 6c^2 h/rho^3 + a^2 (10c^3 - 8c)/rho^4
 *       nz = s [-1/rho^2 - 6ch/rho^3 + a^2 (10c^2 - 2)/rho^4]
 *       zn = s/rho^2
 *   uT: tn = 5c/rho^2 - 6c^3/rho^2 - 4h/rho^3 + 6c^2 h/rho^3 + a^2 (10c^3 - 8c)/rho^4
 *       nt = c/rho^2 - 2h/rho^3 - 2a^2 c/rho^4
 *       nz = -s/rho^2
 *       zn = s [1/rho^2 + 6c^2/rho^2 - 6ch/rho^3 + a^2 (2 - 10c^2)/rho^4]
 *   wT: tt = -(1 + 3c^2/2)/rho^3, tz = -(3/2) c s/rho^3, nn = (7/2 - 6c^2)/rho^3,
 *       zt = (3/2) c s/rho^3, zz = (1/2 - 3c^2/2)/rho^3.
 * At i = j (R = 2h z) these reduce to the single-sphere wall corrections of
 * Swan & Brady (2007): 1 - 9/16 xi + 1/8 xi^3 - 1/16 xi^5 (translation parallel
 * to the wall), 1 - 9/8 xi + 1/2 xi^3 - 1/8 xi^5 (normal), 1 - 5/16 xi^3 and
 * 1 - 1/8 xi^3 (rotation about a parallel and the normal axis), xi = a / h.
 */
void orc_wall_blocks(const double x[3], const double y[3], double a, double eta,
                     double uF[9], double uT[9], double wF[9], double wT[9])
{
    const double R[3] = {x[0] - y[0], x[1] - y[1], x[2] + y[2]};
    const double h = y[2];
    const double rho = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    const double rh = sqrt(R[0] * R[0] + R[1] * R[1]);
    const double c = R[2] / rho, s = rh / rho;
    const double a2 = a * a, a4 = a2 * a2;
    const double r1 = 1.0 / rho, r2 = r1 * r1, r3 = r2 * r1, r4 = r2 * r2, r5 = r4 * r1;
    const double c2 = c * c, c3 = c2 * c, c4 = c2 * c2;
    const double k8 = 1.0 / (8.0 * ORC_PI * eta);
    /* local frame (t, n, z) */
    double t[3] = {1.0, 0.0, 0.0};
    if (rh > 0.0) { t[0] = R[0] / rh; t[1] = R[1] / rh; }
    const double n[3] = {-t[1], t[0], 0.0};
    const double z[3] = {0.0, 0.0, 1.0};
    const double *fr[3] = {t, n, z};
    double LuF[9] = {0}, LwF[9] = {0}, LuT[9] = {0}, LwT[9] = {0};
    LuF[0] = -2.0 * r1 + c2 * r1 + 4.0 * c * h * r2 - 4.0 * h * h * r3 - 6.0 * c3 * h * r2 + 6.0 * c2 * h * h * r3
             + a2 * (10.0 * c4 - 10.0 * c2 + 4.0 / 3.0) * r3 + a4 * (-70.0 * c4 / 3.0 + 70.0 * c2 / 3.0 - 8.0 / 3.0) * r5;
    LuF[2] = s * (-c * r1 + 2.0 * h * r2 - 6.0 * c2 * h * r2 + 6.0 * c * h * h * r3 + a2 * (10.0 * c3 - 2.0 * c) * r3
                  + a4 * (-70.0 * c3 / 3.0 + 10.0 * c) * r5);
    LuF[4] = -r1 - 2.0 * c * h * r2 + 2.0 * h * h * r3 + a2 * (2.0 * c2 - 2.0 / 3.0) * r3
             + a4 * (2.0 / 3.0 - 10.0 * c2 / 3.0) * r5;
    LuF[6] = s * (-c * r1 + 2.0 * h * r2 + 6.0 * c2 * h * r2 - 6.0 * c * h * h * r3 - a2 * (10.0 * c3 - 2.0 * c) * r3
                  + a4 * (70.0 * c3 / 3.0 - 10.0 * c) * r5);
    LuF[8] = -r1 - c2 * r1 + 2.0 * c * h * r2 - 2.0 * h * h * r3 - 6.0 * c3 * h * r2 + 6.0 * c2 * h * h * r3
             + a2 * (10.0 * c4 - 4.0 * c2 - 2.0 / 3.0) * r3 + a4 * (-70.0 * c4 / 3.0 + 20.0 * c2 - 2.0) * r5;
    LwF[1] = -c * r2 + 2.0 * h * r3 - 2.0 * a2 * c * r4;
    LwF[3] = c * r2 + 4.0 * h * r3 - 6.0 * c2 * h * r3 + a2 * (10.0 * c3 - 8.0 * c) * r4;
    LwF[5] = s * (-r2 - 6.0 * c * h * r3 + a2 * (10.0 * c2 - 2.0) * r4);
    LwF[7] = s * r2;
    LuT[1] = 5.0 * c * r2 - 6.0 * c3 * r2 - 4.0 * h * r3 + 6.0 * c2 * h * r3 + a2 * (10.0 * c3 - 8.0 * c) * r4;
    LuT[3] = c * r2 - 2.0 * h * r3 - 2.0 * a2 * c * r4;
    LuT[5] = -s * r2;
    LuT[7] = s * (r2 + 6.0 * c2 * r2 - 6.0 * c * h * r3 + a2 * (2.0 - 10.0 * c2) * r4);
    LwT[0] = -(1.0 + 1.5 * c2) * r3;
    LwT[2] = -1.5 * c * s * r3;
    LwT[4] = (3.5 - 6.0 * c2) * r3;
    LwT[6] = 1.5 * c * s * r3;
    LwT[8] = (0.5 - 1.5 * c2) * r3;
    /* B_pq = sum_{k,l} L_kl f_k[p] f_l[q] */
    for (int p = 0; p < 3; ++p) {
        for (int q = 0; q < 3; ++q) {
            double su = 0.0, sw = 0.0, st = 0.0, sr = 0.0;
            for (int k = 0; k < 3; ++k) {
                for (int l = 0; l < 3; ++l) {
                    const double b = fr[k][p] * fr[l][q];
                    su += LuF[3 * k + l] * b;
                    sw += LwF[3 * k + l] * b;
                    st += LuT[3 * k + l] * b;
                    sr += LwT[3 * k + l] * b;
                }
            }
            uF[3 * p + q] = k8 * su;
            wF[3 * p + q] = k8 * sw;
            uT[3 * p + q] = k8 * st;
            wT[3 * p + q] = k8 * sr;
        }
    }
}

/* Wall damping (the SPD-preserving treatment of particles overlapping the
 * wall that Sec. 3.5 adopts from the magnetic-roller work, in the reading
 * used here): a particle at height z is evaluated at height max(z, a) and its
 * rows and columns of M are scaled by f = min(max(z / a, 0), 1), so that
 * M_damped = D M(clamped) D with D = diag(f).  Returns f and writes the
 * clamped position. */
double orc_wall_clamp(const double x[3], double a, double xc[3])
{
    xc[0] = x[0];
    xc[1] = x[1];
    xc[2] = x[2] > a ? x[2] : a;
    double f = x[2] / a;
    if (!(f > 0.0)) f = 0.0;
    if (f > 1.0) f = 1.0;
    return f;
}

/* The four blocks of M for particles i (field, at x) and j (source, at y)
 * in the chosen geometry: open (wall = 0) or single wall (wall = 1, with
 * the damping above).  pair_self: 1 when i and j are the same particle. */
static void orc_blocks(const double *x, const double *y, double a, double eta, int wall,
                       double uF[9], double uT[9], double wF[9], double wT[9])
{
    if (!wall) {
        const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
        orc_pair_blocks(d, a, eta, uF, uT, wF, wT);
        return;
    }
    double xc[3], yc[3];
    const double fi = orc_wall_clamp(x, a, xc), fj = orc_wall_clamp(y, a, yc);
    const double d[3] = {xc[0] - yc[0], xc[1] - yc[1], xc[2] - yc[2]};
    double vF[9], vT[9], zF[9], zT[9];
    orc_pair_blocks(d, a, eta, uF, uT, wF, wT);
    orc_wall_blocks(xc, yc, a, eta, vF, vT, zF, zT);
    const double ff = fi * fj;
    for (int k = 0; k < 9; ++k) {
        uF[k] = ff * (uF[k] + vF[k]);
        uT[k] = ff * (uT[k] + vT[k]);
        wF[k] = ff * (wF[k] + zF[k]);
        wT[k] = ff * (wT[k] + zT[k]);
    }
}

/* Dense grand mobility, Eq. (block_mobility): dim = 3N (angular = 0) or 6N,
 * row-major, ordering [u_1..u_N ; w_1..w_N] x [F_1..F_N ; T_1..T_N]. */
void orc_assemble(int64_t n, const double *pos, double a, double eta, int angular, int wall, double *M)
{
    const int64_t dim = angular ? 6 * n : 3 * n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double uF[9], uT[9], wF[9], wT[9];
        for (int64_t j = 0; j < n; ++j) {
            orc_blocks(pos + 3 * i, pos + 3 * j, a, eta, wall, uF, uT, wF, wT);
            for (int p = 0; p < 3; ++p) {
                for (int q = 0; q < 3; ++q) {
                    M[(3 * i + p) * dim + 3 * j + q] = uF[3 * p + q];
                    if (angular) {
                        M[(3 * i + p) * dim + 3 * n + 3 * j + q] = uT[3 * p + q];
                        M[(3 * n + 3 * i + p) * dim + 3 * j + q] = wF[3 * p + q];
                        M[(3 * n + 3 * i + p) * dim + 3 * n + 3 * j + q] = wT[3 * p + q];
                    }
                }
            }
        }
    }
}

/* Matrix-free product [u;w] = M [F;T] for the listed rows (rows == NULL means
 * all N rows, in order).  Output row k is particle rows[k].  T may be NULL
 * (zero torques); W may be NULL when angular == 0. */
void orc_mdot(int64_t n, const double *pos, const double *F, const double *T,
              double a, double eta, int angular, int wall, const int64_t *rows, int64_t nrows,
              double *U, double *W)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t i = rows ? rows[k] : k;
        double u[3] = {0.0, 0.0, 0.0}, w[3] = {0.0, 0.0, 0.0};
        double uF[9], uT[9], wF[9], wT[9];
        for (int64_t j = 0; j < n; ++j) {
            orc_blocks(pos + 3 * i, pos + 3 * j, a, eta, wall, uF, uT, wF, wT);
            for (int p = 0; p < 3; ++p) {
                for (int q = 0; q < 3; ++q) {
                    u[p] += uF[3 * p + q] * F[3 * j + q];
                    if (angular) {
                        if (T) u[p] += uT[3 * p + q] * T[3 * j + q];
                        w[p] += wF[3 * p + q] * F[3 * j + q];
                        if (T) w[p] += wT[3 * p + q] * T[3 * j + q];
                    }
                }
            }
        }
        for (int p = 0; p < 3; ++p) {
            U[3 * k + p] = u[p];
            if (angular && W) W[3 * k + p] = w[p];
        }
    }
}

/* Gradient of L = sum_i G_i . u_i + H_i . w_i, with [u;w] = M(X) [F;T], with
 * respect to the positions, for the listed rows (rows == NULL: all).
 * With phi_kl(d) = [G_k;H_k]^T B(d) [F_l;T_l] (B the 6x6 pair block), the
 * chain rule gives dL/dx_i = sum_l grad phi_il(x_i - x_l) - sum_k grad phi_ki(x_k - x_i).
 * H, T may be NULL (zero). */
void orc_grad(int64_t n, const double *pos, const double *F, const double *T,
              const double *G, const double *H, double a, double eta, int angular,
              const int64_t *rows, int64_t nrows, double *dX)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t kk = 0; kk < nrows; ++kk) {
        const int64_t i = rows ? rows[kk] : kk;
        double acc[3] = {0.0, 0.0, 0.0};
        double duF[27], duT[27], dwF[27], dwT[27];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            for (int side = 0; side < 2; ++side) {
                /* side 0: phi_ij at d = x_i - x_j, sign +; side 1: phi_ji at d = x_j - x_i, sign - */
                const int64_t k = side == 0 ? i : j;  /* row particle (G, H) */
                const int64_t l = side == 0 ? j : i;  /* column particle (F, T) */
                const double sgn = side == 0 ? 1.0 : -1.0;
                const double d[3] = {pos[3 * k] - pos[3 * l], pos[3 * k + 1] - pos[3 * l + 1],
                                     pos[3 * k + 2] - pos[3 * l + 2]};
                orc_pair_blocks_grad(d, a, eta, duF, duT, dwF, dwT);
                for (int c = 0; c < 3; ++c) {
                    double s = 0.0;
                    for (int p = 0; p < 3; ++p) {
                        for (int q = 0; q < 3; ++q) {
                            s += G[3 * k + p] * duF[9 * c + 3 * p + q] * F[3 * l + q];
                            if (angular) {
                                if (T) s += G[3 * k + p] * duT[9 * c + 3 * p + q] * T[3 * l + q];
                                if (H) s += H[3 * k + p] * dwF[9 * c + 3 * p + q] * F[3 * l + q];
                                if (H && T) s += H[3 * k + p] * dwT[9 * c + 3 * p + q] * T[3 * l + q];
                            }
                        }
                    }
                    acc[c] += sgn * s;
                }
            }
        }
        for (int c = 0; c < 3; ++c) dX[3 * kk + c] = acc[c];
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
