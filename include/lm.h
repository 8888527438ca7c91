/*
 * lm.h -- C ABI of the GB300 open-boundary RPY mobility library.
 *
 * The operations follow the solver interface of the libMobility paper
 * (Sec. 3.2): a solver is created for a periodicity ("open" in x, y, z: the
 * NBody solver of Sec. 3.5), initialised with the viscosity and hydrodynamic
 * radius, given positions, and then applies the grand mobility M of
 * Eq. (block_mobility) to forces and torques (Mdot), or its square root to a
 * Gaussian vector (sqrtMdotW, Sec. 3.3, by the Lanczos method).  divM is zero
 * for the open geometry (Sec. 2, after Eq. fdt).
 *
 * Common conventions
 *   - Every call returns an lm_status; LM_OK is 0.  No call aborts, throws or
 *     exits.  On failure lm_last_error() returns a message for the calling
 *     thread.
 *   - Arrays are row-major N x 3 (x, y, z per particle).  The element type is
 *     float for LM_FP32C solvers and double for LM_FP64 solvers, except W and
 *     the Lanczos state, which are always double.
 *   - A grand vector (W) is ordered [F-part (3N); T-part (3N)], the ordering of
 *     Eq. (block_mobility); without angular blocks it has 3N entries.
 *   - Any array argument may live in device memory or in host memory (pinned
 *     or pageable).  Host arrays are copied to and from the GPU by the
 *     library (Sec. 3.2: numpy inputs are moved automatically); device arrays
 *     are used in place.  The caller keeps ownership of every array it passes.
 *   - Calls are ordered on the solver's CUDA stream and return before the GPU
 *     work finishes, except where a host value must be returned (lm_sqrt_mdot:
 *     the Lanczos iteration count and convergence) or a host output array is
 *     written; those synchronise the stream.
 *   - The library owns its scratch memory (packed positions, split partial
 *     sums, the Krylov basis) and frees it in lm_destroy.
 */
#ifndef LM_GB300_H
#define LM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lm_solver lm_solver; /* opaque, owned by the library */

typedef enum {
    LM_OK = 0,
    LM_ERR_INVALID_ARG = 1,          /* bad pointer, size, value or combination */
    LM_ERR_UNSUPPORTED_GEOMETRY = 2, /* periodicity other than "open" */
    LM_ERR_STATE = 3,                /* call out of order (e.g. mdot before set_positions) */
    LM_ERR_NONFINITE = 4,            /* NaN or Inf in positions */
    LM_ERR_NOT_CONVERGED = 5,        /* Lanczos hit max_iter; outputs hold the last iterate */
    LM_ERR_TIMEOUT = 6,              /* a bounded device-side wait expired */
    LM_ERR_OOM = 7,                  /* device allocation failed */
    LM_ERR_CUDA = 8                  /* any other CUDA runtime error */
} lm_status;

typedef enum {
    LM_FP32C = 0, /* FP32 pair arithmetic, compensated (two-float) accumulation */
    LM_FP64 = 1   /* FP64 throughout */
} lm_precision;

/*
 * lm_create -- the solver constructor and `initialize` of Sec. 3.2.
 *   px, py, pz: periodicity strings (NBody, Sec. 3.5; Table
 *     tab:solver_summary): px = py = "open"; pz = "open" (free-space RPY) or
 *     "single_wall" (a no-slip wall at z = 0: the Swan-Brady kernel, with the
 *     damping of particles that overlap the wall, see below).  Other valid
 *     names ("periodic", "two_walls", or a wall in x or y) give
 *     LM_ERR_UNSUPPORTED_GEOMETRY, unknown names LM_ERR_INVALID_ARG.
 *   Single wall: each block is the open RPY block plus the Faxen operators
 *     applied to the image system of the Blake Green's function (Swan & Brady
 *     2007).  A particle at height z is evaluated at height max(z, a) and its
 *     rows and columns of M are scaled by f = clamp(z / a, 0, 1), so that M
 *     stays symmetric positive semi-definite and the mobility of a particle
 *     goes to zero as it reaches the wall (Sec. 3.5).
 *   viscosity (eta > 0), hydrodynamic_radius (a > 0): the parameters of the
 *     RPY kernel.
 *   include_angular: nonzero to accept torques and return angular
 *     velocities (the 6N grand mobility); zero for forces only (3N).
 *   cuda_stream: a cudaStream_t, or NULL for the legacy default stream.
 *   *out receives the solver; it is NULL on failure.
 */
lm_status lm_create(lm_solver **out, const char *px, const char *py, const char *pz,
                    double viscosity, double hydrodynamic_radius, int include_angular,
                    lm_precision precision, void *cuda_stream);

/* lm_destroy -- frees the solver and all its device memory.  NULL is allowed. */
lm_status lm_destroy(lm_solver *solver);

/* lm_set_stream -- change the CUDA stream used by later calls. */
lm_status lm_set_stream(lm_solver *solver, void *cuda_stream);

/*
 * lm_set_positions -- setPositions of Sec. 3.2.
 *   pos: N x 3 positions (float for LM_FP32C, double for LM_FP64), host or
 *     device.  The library copies them into its own packed buffer, so the
 *     caller may reuse pos immediately after the call returns.
 *   N >= 1.  Non-finite coordinates give LM_ERR_NONFINITE (this check
 *   synchronises the stream) and leave the solver without positions.
 */
lm_status lm_set_positions(lm_solver *solver, const void *pos, int64_t N);

/*
 * lm_mdot -- Mdot of Sec. 3.2: [lin; ang] = M(X) [F; T] with the blocks of
 * Eq. (block_mobility), a direct O(N^2) sum over all ordered pairs including
 * the self term (NBody, Sec. 3.5).
 *   forces, torques: N x 3 or NULL (NULL means zero; "one or both").
 *     torques must be NULL unless include_angular.
 *   lin_out: N x 3, required.  ang_out: N x 3, required iff include_angular,
 *     must be NULL otherwise.
 */
lm_status lm_mdot(lm_solver *solver, const void *forces, const void *torques, void *lin_out,
                  void *ang_out);

/*
 * lm_sqrt_mdot -- sqrtMdotW of Sec. 3.2 by the Krylov/Lanczos method of
 * Sec. 3.3: [lin; ang] = prefactor * M^{1/2} W.
 *   W: 3N (or 6N with angular) doubles, host or device; NULL draws W from
 *     the library's Philox-4x32-10 generator keyed by seed (normals by
 *     Box-Muller, element e from counter e / 4).
 *   prefactor: scale applied to the result, e.g. sqrt(2 kT dt) for the
 *     Brownian term of Eq. (bdhi); 1 gives M^{1/2} W.
 *   tol: stop when the relative change of successive iterates is below tol
 *     (checked from the second iteration).  tol >= 0.
 *   max_iter: iteration cap, 1 <= max_iter (values above the dimension are
 *     clamped to it).
 *   iters_out: optional; receives the number of Lanczos iterations.
 *   Returns LM_ERR_NOT_CONVERGED when max_iter is reached first; the outputs
 *   then hold the last iterate.  W = 0 gives zero outputs and 0 iterations.
 *   Synchronises the stream once per iteration (scalar read-back).
 */
lm_status lm_sqrt_mdot(lm_solver *solver, const double *W, uint64_t seed, double prefactor,
                       double tol, int max_iter, void *lin_out, void *ang_out, int *iters_out);

/*
 * lm_set_sqrt_preconditioner -- preconditioning of the Lanczos square root
 * (Sec. 3.3 notes that the Krylov method can be preconditioned; the paper's
 * release does not).  kind 0: none (the default; lm_sqrt_mdot approximates
 * the principal root M^{1/2} W).  kind 1: Jacobi, P = diag(M)^{-1/2} from the
 * single-sphere mobilities (Swan-Brady and the damping with a single wall):
 * lm_sqrt_mdot then approximates B W with B = P^{-1} (P M P)^{1/2}, another
 * square root of M (B B^T = M, so the noise has the covariance of Eq. fdt),
 * by the Lanczos iteration on P M P, whose spectrum is better conditioned when
 * the diagonal of M varies (particles near or touching a wall).  The stopping
 * rule applies to the iterates of (P M P)^{1/2} W.  kind other than 0, 1
 * gives LM_ERR_INVALID_ARG.
 */
lm_status lm_set_sqrt_preconditioner(lm_solver *solver, int kind);

/*
 * lm_set_reorthogonalization -- the Gram-Schmidt passes of the Lanczos
 * square root (full reorthogonalisation of each new Krylov vector against the
 * stored basis, as in the Krylov square-root method of Ando, Chow, Saad &
 * Skolnick 2012 that Sec. 3.3 cites).  mode 0 (the default): one classical pass, and a
 * second only when the first removed more than 1 - 1/sqrt(2) of the norm of
 * w (the DGKS criterion, Daniel, Gragg, Kaufman & Stewart 1976).  mode 1:
 * always two passes (costs one more pass over the basis per iteration; the
 * iterates agree with mode 0 to rounding).  Other modes give
 * LM_ERR_INVALID_ARG.  lm_batch_set_reorthogonalization does the same for a
 * batch.
 */
lm_status lm_set_reorthogonalization(lm_solver *solver, int mode);

/*
 * lm_div_m -- divM of Sec. 3.2: lin_i = sum_j d/dx_j . M_uF(i, j),
 * ang_i = sum_j d/dx_j . M_wF(i, j) (the thermal drift of Eq. bdhi is kT
 * times this).  For the open geometry the mobility is translation invariant
 * and isotropic, so it is identically zero (Sec. 2, discussion after Eq.
 * fdt) and the outputs are set to zero.  With a single wall it is one random
 * finite difference sample (Eq. rfd, Sec. 3.4), lm_div_m_rfd with the
 * solver's call counter (0, 1, 2, ...) as seed and delta = 1e-4 a (LM_FP64)
 * or 1e-2 a (LM_FP32C).
 */
lm_status lm_div_m(lm_solver *solver, void *lin_out, void *ang_out);

/*
 * lm_div_m_rfd -- one random finite difference sample of divM, Eq. (rfd) of
 * Sec. 3.4:
 *   [lin; ang] = (M(X + delta W / 2) [W; 0] - M(X - delta W / 2) [W; 0]) / delta,
 * W = 3N standard normals from Philox-4x32-10 with key seed and stream
 * 0x524644 (element e = normal e mod 4 of counter block e / 4).  Its mean over
 * W is divM up to O(delta^2).  Only positions are displaced: the mobility of
 * spheres does not depend on their orientation.  delta > 0 (a length).
 * lin_out, ang_out as in lm_mdot.  For the open geometry the result is zero.
 * Allocates its scratch on the first call (four vectors of 3N or 6N doubles
 * and a packed copy of the positions).
 */
lm_status lm_div_m_rfd(lm_solver *solver, uint64_t seed, double delta, void *lin_out, void *ang_out);

/*
 * lm_set_wall_height -- setParameters(wallHeight) of Sec. 3.2 for a
 * single-wall solver: the no-slip wall lies at z = height (default 0).  All
 * heights (wall corrections, damping, the steric wall term) are measured from
 * it; positions already set are re-packed.  Other solvers give
 * LM_ERR_INVALID_ARG.
 */
lm_status lm_set_wall_height(lm_solver *solver, double height);

/*
 * lm_langevin_velocities -- LangevinVelocities of Sec. 3.2: the three terms
 * of Eq. (bdhi) divided by dt, i.e. the velocities of one Euler-Maruyama
 * step,
 *   [lin; ang] = M [F; T] + sqrt(2 kT / dt) M^{1/2} W + kT divM,
 * with the square root by the Lanczos method (lm_sqrt_mdot with tol,
 * max_iter, seed; W NULL draws Philox normals keyed by seed) and divM one
 * random finite difference sample keyed by seed (zero in the open
 * geometry).  kT = 0 gives M [F; T].  forces, torques: N x 3 (NULL = zero;
 * torques only with angular blocks); lin_out, ang_out as in lm_mdot.
 * Returns the status of the Lanczos step.  Synchronises the stream.
 */
lm_status lm_langevin_velocities(lm_solver *solver, const void *forces, const void *torques, const double *W,
                                 uint64_t seed, double kT, double dt, double tol, int max_iter,
                                 void *lin_out, void *ang_out, int *iters_out);

/*
 * lm_soft_repulsion -- forces of the soft steric potential of the roller
 * example, Eq. (soft_potential) of Sec. 5.1,
 *   U(r) = U0 (1 + (d - r)/b) for r < d,   U0 exp((d - r)/b) for r >= d,
 * summed over every particle pair (d = d_pair, r = centre distance) and,
 * for a single-wall solver, every particle-wall pair (d = d_wall, r = the
 * height of the centre above the wall).  forces_out (N x 3, overwritten) = -dU/dX at the
 * positions last set; a coincident pair (r = 0) exerts no force.  b > 0;
 * U0, d_pair, d_wall finite.  Direct O(N^2) sum on the GPU.
 */
lm_status lm_soft_repulsion(lm_solver *solver, double U0, double b, double d_pair, double d_wall,
                            void *forces_out);

/*
 * lm_ab_step -- one step of the stochastic Adams-Bashforth scheme of
 * Sec. 5.1 for the positions X (Eq. bdhi discretised):
 *   X' = X + dt [(3/2) u^n - (1/2) u^{n-1} + kT ((3/2) d^n - (1/2) d^{n-1})]
 *          + sqrt(2 kT dt) (M^{1/2} W)_lin,
 * u^n = (M [F; T])_lin at the current positions, d^n = one random finite
 * difference sample of divM (lm_div_m_rfd with key seed and the default
 * delta; zero in the open geometry or at kT = 0), and the square root by
 * the Lanczos method (lm_sqrt_mdot with tol, max_iter, seed).
 *   forces, torques: F^n, T^n (N x 3, solver precision, host or device;
 *     NULL = zero; torques only with angular blocks).
 *   W: 3N (6N with angular blocks) normals, host or device, or NULL to draw
 *     them from Philox with key seed (as lm_sqrt_mdot).
 *   history: device array of 6N doubles, [u^{n-1} (3N); d^{n-1} (3N)], owned
 *     by the caller; read unless first != 0, always overwritten with
 *     (u^n, d^n).  first != 0 gives the Euler-Maruyama step (previous terms
 *     equal to the current ones).
 *   pos_out: N x 3 new positions (host or device); the solver's positions
 *     are set to them as well (lm_set_positions).
 *   iters_out: optional Lanczos iteration count.
 * Returns the status of the Lanczos step (LM_ERR_NOT_CONVERGED with the
 * positions updated from the last iterate).  Synchronises the stream.
 */
lm_status lm_ab_step(lm_solver *solver, const void *forces, const void *torques, const double *W,
                     uint64_t seed, double kT, double dt, double tol, int max_iter, double *history,
                     int first, void *pos_out, int *iters_out);

/*
 * lm_mdot_backward -- adjoint of Mdot (not in the paper; the differentiable
 * form of the product).  For the scalar L = sum_i G_i . lin_i + H_i . ang_i
 * with [lin; ang] = M(X) [F; T] it writes
 *   dX = dL/dX (N x 3), dF = dL/dF = (M [G; H])_lin, dT = dL/dT = (M [G; H])_ang,
 * in one fused pass that recomputes the pair terms (no N^2 storage).
 *   forces (required), torques (NULL = zero, angular only), grad_lin (G,
 *   required), grad_ang (H, NULL = zero, angular only).
 *   dX and dF may be NULL to skip them; dT must be NULL unless angular.
 *   The gradient of a pair term at r = 0 (coincident particles) is taken
 *   as zero.  Open geometry only: a single-wall solver gives
 *   LM_ERR_UNSUPPORTED_GEOMETRY.
 *   For LM_FP64 and for angular blocks the default kernel is a symmetric
 *   one, whose two sides meet in FP64 atomic adds: the last bits of the
 *   results can vary from run to run.  lm_set_adjoint_config with packed 0
 *   selects the one-sided kernel, which is bitwise reproducible.
 */
lm_status lm_mdot_backward(lm_solver *solver, const void *forces, const void *torques,
                           const void *grad_lin, const void *grad_ang, void *dX, void *dF,
                           void *dT);

/*
 * Pair-kernel launch configuration (chosen by the autotuner or set by hand).
 *   threads: CTA size (128 or 256); ilp: i-particles per thread (1, 2, 4, 8
 *   for LM_FP32C; 1, 2 for LM_FP64); splits: number of j-range splits
 *   (>= 1; 0 = automatic; split k of s holds j-tiles [k T/s, (k+1) T/s) of
 *   the T tiles of `threads` particles, at most T splits are launched);
 *   packed: 0 the scalar form; 1 the packed FP32 form, which evaluates two
 *   i-particles per f32x2 instruction (LM_FP32C with ilp 2, 4 or 8); 2 and 4
 *   the packed form with two or four j-particles per overlap vote (open
 *   geometry only; 4 needs ilp >= 4).
 *   Single-wall solvers: threads 128 or 256, ilp 1, 2, 4 (scalar) or 2, 4
 *   (packed = 1); FP64 ilp 1.  All forms give results within the FP32
 *   tolerance of the FP64 product; they differ in rounding order only.
 */
/* Launch configuration of the pair kernels (no paper counterpart):
 *   threads: CTA size and j-tile length (128 or 256);
 *   ilp: i-particles per thread (FP32: 1, 2, 4, 8; FP64: 1, 2);
 *   splits: j-range chunks per i-block, >= 1 (0 in lm_set_pair_config: the
 *     library's model chooses); several splits add FP64 partial sums in a
 *     second kernel;
 *   packed: 0 the scalar kernel; FP32 only, with even ilp: 1, 2 or 4 the
 *     packed f32x2 kernel evaluating 1, 2 or 4 j-particles per overlap vote
 *     (4 needs ilp >= 4). */
typedef struct {
    int threads;
    int ilp;
    int splits;
    int packed;
} lm_pair_config;

/* lm_get_pair_config / lm_set_pair_config -- read or force the launch
 * configuration used for the solver's current N.  Setting an unsupported
 * combination gives LM_ERR_INVALID_ARG. */
lm_status lm_get_pair_config(lm_solver *solver, lm_pair_config *cfg);
lm_status lm_set_pair_config(lm_solver *solver, const lm_pair_config *cfg);

/* lm_get_adjoint_config / lm_set_adjoint_config -- launch configuration of
 * lm_mdot_backward for the current N.  LM_FP32C without angular blocks (the
 * packed kernels): threads 128 or 256, ilp 2 or 4, and packed
 *   1 or 2: the one-sided kernel, j-particles per overlap vote; splits =
 *     j-range chunks per i-block;
 *   3: the symmetric kernel: each unordered pair is evaluated once and added
 *     to both particles (the gradient of a pair term is odd in x_i - x_j and
 *     the tt block even), about 18% faster at N = 65536; splits = tiles per
 *     work item (0: chosen from N).  Its two sides meet in FP64 atomic adds,
 *     so the last bits of an FP64 sum, and rarely the last bit of an FP32
 *     output, can differ from run to run;
 * otherwise (LM_FP64, or angular blocks) threads 128 and packed
 *   3: the symmetric scalar kernel (the LM_FP64 default): each unordered
 *     pair once, its gradient added to one particle and subtracted from the
 *     other, the mobility parts of both directions from the same
 *     coefficients; ilp 1 (LM_FP64) or 2, 4 (LM_FP32C); 1.5x faster than
 *     packed 0 at N = 16384 (FP64, angular);
 *   4: the same in packed f32x2 form, two i-particles per instruction
 *     (LM_FP32C with angular blocks, ilp 2 or 4; the default there with
 *     ilp 4): 1.7x faster than packed 0 at N = 65536;
 *     for 3 and 4, splits = tiles per work item (0: chosen from N), and the
 *     FP64 atomic adds make the last bits of the results vary from run to
 *     run, as above;
 *   0: the one-sided scalar kernel, ilp 1 (LM_FP64) or 2 (LM_FP32C);
 *     splits = j-range chunks per i-block.
 * splits 0 = automatic.  Unsupported combinations give LM_ERR_INVALID_ARG. */
lm_status lm_get_adjoint_config(lm_solver *solver, lm_pair_config *cfg);
lm_status lm_set_adjoint_config(lm_solver *solver, const lm_pair_config *cfg);

/*
 * lm_autotune -- time every supported pair-kernel configuration for the
 * solver's precision, angular flag and current N (positions must be set),
 * keep the fastest, and return it in *best (nullable).  reps >= 1 timed
 * launches per candidate (after one warm-up launch); the three fastest are
 * then timed three more times each, interleaved, and the best of their four
 * timings decides.  For an LM_FP32C open solver without angular blocks it
 * also times the configurations of the adjoint kernel the same way and
 * keeps the fastest (lm_get_adjoint_config).  The choice is also recorded
 * for the process under (device, precision, angular flag, geometry,
 * floor(log2 N)): a solver without a configuration of its own (none set or
 * tuned) whose N falls in a recorded bucket starts from that choice, with
 * the split count recomputed for its N.  For FP32 products large enough
 * that one launch takes more than about 20 ms (N^2 x flops per pair above
 * 1e12), the sweep keeps only the packed forms with at least 512 particles
 * per i-block and the split counts of the model and of whole waves, and
 * candidates after the first are timed without a warm-up launch of their
 * own.  Synchronises the stream.
 */
lm_status lm_autotune(lm_solver *solver, int reps, lm_pair_config *best);

/* Statistics of the last lm_sqrt_mdot call on this solver. */
typedef struct {
    int iterations;       /* Lanczos iterations */
    int converged;        /* 1 if the tolerance or a breakdown stopped it */
    double rel_change;    /* last relative change of successive iterates */
    double norm_w;        /* |W| */
    int clamped_eigs;     /* tridiagonal eigenvalues clamped from < 0 to 0 */
} lm_lanczos_stats;

lm_status lm_get_lanczos_stats(lm_solver *solver, lm_lanczos_stats *stats);

/*
 * Device-time profile of the forward pair kernel and of the Lanczos vector
 * kernels.  While enabled, the solver records a CUDA event pair on its stream
 * around every pair-kernel launch (the split reduction is not included) and
 * around the vector kernels of every Lanczos iteration that follow its
 * product (alpha, the three-term update, the Gram-Schmidt passes and beta).
 * The bytes of an iteration are the algorithmic FP64 vector traffic, in
 * vectors of n = 3N or 6N doubles: 2 + 4 (3 at k = 0) + (2k + 5) per
 * Gram-Schmidt pass at 0-based iteration k, the second pass counted only
 * where it ran.  Iterations of an lm_sqrt_mdot call that returned an error
 * are left out.  lm_profile_read synchronises the stream, returns the totals
 * since the last reset, and resets them if reset is nonzero.
 */
typedef struct {
    int64_t pair_launches;    /* pair-kernel launches recorded */
    double pair_ms;           /* their summed device time, milliseconds */
    double pair_interactions; /* ordered pairs evaluated, N^2 per launch */
    double pair_flops;        /* algorithmic flops: 35 per pair (forces only) or 86 (all blocks);
                                 single wall: 131 or 299 */
    int64_t vector_iterations; /* Lanczos iterations whose vector kernels were timed */
    double vector_ms;          /* their summed device time, milliseconds */
    double vector_bytes;       /* their algorithmic bytes (see above) */
} lm_profile;

lm_status lm_profile_enable(lm_solver *solver, int enable);
lm_status lm_profile_read(lm_solver *solver, lm_profile *out, int reset);

/* Number of GPU kernel launches the library has issued in this process, over
 * all solvers (monotone counter; the argument is ignored and may be NULL). */
int64_t lm_launch_count(lm_solver *solver);

/*
 * lm_tridiag_sqrt_e1 -- host-only helper (no GPU needed): out = T^{1/2} e1
 * for the m x m symmetric tridiagonal T with diagonal alpha[0..m-1] and
 * off-diagonal beta[0..m-2], the last step of the Lanczos square root
 * (Sec. 3.3).  Eigenvalues below zero from round-off are clamped to zero.
 * Returns 0, -1 if the QR iteration did not converge, -2 on bad arguments.
 */
int lm_tridiag_sqrt_e1(int m, const double *alpha, const double *beta, double *out);

/*
 * ---------------------------------------------------------------------------
 * Batches of independent open-boundary suspensions (uneven sizes).
 * The Brownian dynamics of Eq. (bdhi) with the default Euler-Maruyama step
 * (Sec. 3.2, LangevinVelocities) for many small systems at once: every call
 * below runs as ONE persistent cooperative kernel launch over all systems
 * (the thermal drift is zero in the open geometry, Sec. 2).  Pairs in FP32
 * with compensated sums, Lanczos vectors in FP64, translational blocks only.
 * Systems are concatenated: system s owns particles [offsets[s],
 * offsets[s+1]) of every N_total x 3 array.
 * ---------------------------------------------------------------------------
 */
typedef struct lm_batch lm_batch;

/*
 * lm_batch_create -- 1 <= S <= 2^20 systems (the solve requests encode the
 * system in 21 bits); offsets: host array of S+1 int64 with
 * offsets[0] = 0 and offsets[s+1] - offsets[s] in [1, 65536].
 * max_iter (1..128): Lanczos iteration cap per system and step; it sizes the
 * Krylov storage, max_iter x 3 N_total doubles.
 */
lm_status lm_batch_create(lm_batch **out, int64_t S, const int64_t *offsets, double viscosity,
                          double hydrodynamic_radius, int max_iter, void *cuda_stream);
lm_status lm_batch_destroy(lm_batch *batch);

/* Positions of all systems, N_total x 3 float (host or device); copied. */
lm_status lm_batch_set_positions(lm_batch *batch, const float *pos);
/* Current positions (after lm_batch_bd_run), N_total x 3 float. */
lm_status lm_batch_get_positions(lm_batch *batch, float *pos_out);

/* lin = M_s F_s for every system s (Mdot per system), N_total x 3 float. */
lm_status lm_batch_mdot(lm_batch *batch, const float *forces, float *lin_out);

/*
 * lm_batch_sqrt_mdot -- lin = prefactor * M_s^{1/2} W_s for every system, by
 * the Lanczos method of Sec. 3.3 with the stopping rule of lm_sqrt_mdot,
 * applied per system.  W: 3 N_total doubles (host or device), or NULL to
 * draw system s's noise from Philox-4x32-10 with key seed and stream s
 * (element e of the system is normal e mod 4 of counter block e / 4).
 * iters_out: optional host array of S ints (iterations per system).
 * Returns LM_ERR_NOT_CONVERGED if some system reached max_iter.
 */
lm_status lm_batch_sqrt_mdot(lm_batch *batch, const double *W, uint64_t seed, double prefactor,
                             double tol, float *lin_out, int *iters_out);

/*
 * lm_batch_bd_run -- nsteps Euler-Maruyama steps of Eq. (bdhi) for every
 * system, with harmonic confining forces F = -k_trap x (trap centre at the
 * origin, no torques):
 *   x <- x + dt M F + sqrt(2 kT dt) M^{1/2} W,
 * W of system s at step t from Philox-4x32-10 with key seed and stream
 * (t << 32) | s, t counted from step0 (so that runs can be continued).
 * All steps run in one persistent cooperative launch; with use_graph != 0
 * that launch is captured into a CUDA graph and the graph is launched.
 * The stopping rule is that of lm_sqrt_mdot per system, except that the
 * relative-change test is first made one iteration before the count the
 * system needed in its previous step (its tridiagonal solves start one
 * iteration earlier still): counts change little from step to step, and each
 * test costs an FP64 eigen-solve.
 * Breakdown and max_iter are tested at every iteration.
 * Positions stay on the device (lm_batch_get_positions reads them).
 * iters_out: optional host array of S ints (total Lanczos iterations per
 * system over the run).  Device-side waits are bounded; if one expires the
 * call returns LM_ERR_TIMEOUT.  Synchronises the stream.
 */
lm_status lm_batch_bd_run(lm_batch *batch, double kT, double dt, double k_trap, int nsteps,
                          int64_t step0, uint64_t seed, double tol, int use_graph, int *iters_out);

/*
 * Pair tiling of the batched launches: threads per CTA (64 or 128) and
 * i-particles per thread (1 or 2); picked by lm_batch_autotune (timing a
 * batched square root, Philox noise at tol 1e-4, over all systems: the
 * products, vector phases and tridiagonal solves of a Brownian step; the
 * systems' warm-start iteration counts are kept) or set by hand.
 */
lm_status lm_batch_set_tiling(lm_batch *batch, int threads, int ilp);
lm_status lm_batch_set_reorthogonalization(lm_batch *batch, int mode);
lm_status lm_batch_autotune(lm_batch *batch, int *threads_out, int *ilp_out);

/*
 * Phase timeline of a batched run (profiling).  While enabled, the
 * persistent kernel records the device global timer (ns) at the start of the
 * last step of the run and after every phase of that step: [start, A1, A2, then per
 * Lanczos iteration B, C2, C3, C4, C5, then the wait for the last
 * tridiagonal results, then D].  C3 includes each system's end of iteration
 * (beta, solve request, stopping rule); C4 is empty unless some system takes
 * the second Gram-Schmidt pass; C5 is an empty stamp kept for the layout.  lm_batch_profile_read copies
 * up to n stamps of the last run into out and the number recorded into
 * *count.  lm_batch_profile_pairs gives the pair evaluations of the last
 * profiled run, all steps and systems: the particle pairs of every product
 * work item, including the iterations a system runs past its stopping point
 * while its tridiagonal results are pending (synchronises the stream).
 */
lm_status lm_batch_profile_enable(lm_batch *batch, int enable);
lm_status lm_batch_profile_read(lm_batch *batch, uint64_t *out, int n, int *count);
lm_status lm_batch_profile_pairs(lm_batch *batch, uint64_t *pairs);

/*
 * lm_tridiag_sqrt_e1_device -- the device form of the tridiagonal step
 * (Sec. 3.3) that the batched kernel runs, one warp per system, exposed for
 * testing and timing: for each of `count` systems c, out[c m .. c m + m) =
 * sqrt(T_c) e1 with T_c = tridiag(beta_c, alpha_c, beta_c), alpha_c =
 * alpha[c m ..] (m entries), beta_c = beta[c m ..] (m - 1 entries used).
 * alpha, beta, out: device memory, count x m doubles each; 1 <= m <= 128.
 * A T that FP32 Sturm counts certify positive definite (smallest eigenvalue
 * above about 1e-5 of its largest entry) is solved by a trapezoid-rule
 * quadrature of (2/pi) int_0^inf T (T + t^2 I)^{-1} e1 dt over log t (about
 * 200 nodes, relative error about 1e-13, one tridiagonal solve per node, the
 * nodes shared among the warp's lanes); any other T by the implicit QR
 * iteration in double-float on one lane, which clamps negative eigenvalues to
 * zero.  Allocates its scratch, runs on cuda_stream and waits for it.
 * Returns LM_ERR_CUDA if a system's QR iteration failed or T has a
 * non-finite entry.  lm_tridiag_sqrt_e1_device_paths also writes, when
 * paths (host memory, count ints) is not NULL, 0 for each system the
 * quadrature solved and 1 for each the QR form solved.
 */
lm_status lm_tridiag_sqrt_e1_device(int count, int m, const double *alpha, const double *beta, double *out,
                                    void *cuda_stream);
lm_status lm_tridiag_sqrt_e1_device_paths(int count, int m, const double *alpha, const double *beta, double *out,
                                          int *paths, void *cuda_stream);

/*
 * Tridiagonal solve requests of the last batched run (profiling): *posted
 * receives the number of f(T_k) e1 solves the iterating CTAs requested,
 * *solved the number the solver CTAs finished (stale requests of an earlier
 * step included; they are dropped unsolved).
 */
lm_status lm_batch_solve_counts(lm_batch *batch, int64_t *posted, int64_t *solved);

/*
 * lm_batch_timeout_selftest -- check of the bounded device-side waits (no
 * paper counterpart): launches a kernel whose grid barrier waits for one CTA
 * more than it has, so every wait runs out after about spin_cycles clock
 * cycles (1e3..1e8).  Returns LM_ERR_TIMEOUT when the timeout path works.
 */
lm_status lm_batch_timeout_selftest(long long spin_cycles);

/*
 * lm_philox_normals -- the library's noise generator on the device: n
 * standard normals, element e = normal (e mod 4) of Philox-4x32-10 counter
 * block (e/4 low, e/4 high, stream low, stream high) with key (seed low,
 * seed high), Box-Muller in FP64.  out: n doubles, device memory.
 */
lm_status lm_philox_normals(uint64_t seed, uint64_t stream, double *out, int64_t n, void *cuda_stream);

/*
 * lm_philox4x32_10 -- the raw words of the device generator behind
 * lm_philox_normals, the Lanczos noise, the RFD displacements and the
 * batched Brownian noise: Philox-4x32 with 10 rounds (Salmon, Moraes, Dror &
 * Shaw, SC'11), so that it can be checked against the generator's published
 * known-answer vectors.  The paper has no counterpart (it only requires
 * Gaussian W, Eq. fdt).
 *   counters: count x 4 uint32 (c0..c3), keys: count x 2 uint32 (k0, k1),
 *   out: count x 4 uint32; all device memory, owned by the caller.
 *   count >= 0; host pointers give LM_ERR_INVALID_ARG.  Stream-ordered on
 *   cuda_stream (NULL = legacy default stream).
 */
lm_status lm_philox4x32_10(const uint32_t *counters, const uint32_t *keys, uint32_t *out, int64_t count,
                           void *cuda_stream);

/*
 * lm_mdot_noalloc -- the FP32 (compensated) mobility product for callers that
 * cannot let a library allocate device memory.  The paper has no counterpart:
 * its solvers own their buffers.  Such callers are applications whose
 * device memory all belongs to their own pool or caching allocator (where a
 * foreign cudaMalloc can fail or fragment it), latency-critical loops that
 * cannot take the implicit device synchronisation of cudaMalloc / cudaFree,
 * and hosts that forbid allocation inside plugins.
 *
 * It computes what lm_mdot computes for an LM_FP32C solver with the given
 * viscosity, radius and angular flag, with no solver object: no cudaMalloc,
 * cudaFree, pinned or library allocation, and no stream synchronisation.
 *   pos, forces, torques, lin_out, ang_out: device arrays, N x 3 float, with
 *     the lm_mdot conventions (forces / torques NULL = zero; torques and
 *     ang_out only with include_angular, ang_out then required).  Host arrays
 *     are rejected with LM_ERR_INVALID_ARG (copying them would need buffers).
 *   1 <= N <= LM_NOALLOC_MAX_N, else LM_ERR_INVALID_ARG.
 *   Positions are not checked for NaN/Inf (the check needs a read-back).
 *   cuda_stream: the stream to run on (NULL = legacy default stream).
 * Scratch: a fixed device array of LM_NOALLOC_SCRATCH_BYTES inside the
 * library (packed positions and split partial sums), held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls
 * share the array: calls whose GPU work overlaps (e.g. on unordered streams)
 * race on it and give wrong results.
 */
#define LM_NOALLOC_MAX_N 32768
#define LM_NOALLOC_SCRATCH_BYTES (16u << 20)
lm_status lm_mdot_noalloc(const float *pos, const float *forces, const float *torques, int64_t N,
                          double viscosity, double hydrodynamic_radius, int include_angular,
                          float *lin_out, float *ang_out, void *cuda_stream);

/*
 * lm_fp32_probe -- measured FP32 FMA throughput of the current GPU, the
 * ceiling of the pair kernels (no paper counterpart: a calibration of the
 * roofline the pair kernels are reported against).  Runs `iters` outer
 * iterations of independent FMA chains on every SM (one full wave of CTAs)
 * on cuda_stream (NULL = legacy default stream), twice, and returns the
 * second launch's rate in *tflops (2 flops per FMA lane).
 *   mode 0: scalar FMA chains x = x a + b;
 *   mode 1: packed f32x2 FMA chains of the same form (the instruction form of
 *           the packed pair kernels);
 *   mode 2: packed f32x2 FMAs on 12 independent accumulators, each reading
 *           two loop-invariant register pairs of its own (three distinct
 *           register pairs per instruction);
 *   mode 3: packed f32x2 FMAs in rotating dependent chains whose operands are
 *           values produced a few instructions earlier (the data flow of the
 *           pair formulas);
 *   mode 4: FP64 FMA chains x = x a + b (the ceiling of the Lanczos
 *           Gram-Schmidt kernels, one FP64 FMA per basis element; the FP64
 *           pipe runs at a small fraction of the FP32 rate, so about 2^8
 *           iterations give a launch of tens of milliseconds).
 *   1 <= iters <= 2^24 (about 2^14 gives an FP32 launch of tens of
 *   milliseconds).
 * Allocates and frees a small output buffer; synchronises the stream.
 */
lm_status lm_fp32_probe(int mode, int64_t iters, double *tflops, void *cuda_stream);

/*
 * Debug bounds checks (no paper counterpart; the stand-in for a memory
 * sanitizer).  A build with -DLM_DEBUG_BOUNDS checks the indices of the
 * kernels' main loads and stores against their buffers (j < N in every pair
 * tile, partial-sum and output indices, basis rows < m in the Lanczos
 * passes, particle indices < N_total in the batched kernel).  A failed check
 * records its code and index in a device word, the first failure wins, and
 * the access is skipped: a check never faults the GPU.
 * lm_debug_bounds returns 1 for such a build, else 0.
 * lm_debug_check synchronises the current device, reads and clears every
 * check word and returns LM_OK if no check failed, LM_ERR_CUDA with the check
 * and index in lm_last_error otherwise.  In other builds it returns LM_OK
 * without touching the GPU.
 */
int lm_debug_bounds(void);
lm_status lm_debug_check(void);

/*
 * Environment switches read by the library (no paper counterpart):
 *   LM_METRICS_JSONL=<path>  lm_mdot, lm_sqrt_mdot, lm_mdot_backward and the
 *     batch calls synchronise their stream at the end and append one JSON
 *     object per call to <path>: call, status, milliseconds, N, precision,
 *     blocks, geometry, products, pair interactions, flops per pair,
 *     iterations and relative change (square roots), GPU name, SM count and
 *     its nominal FP32 peak.  Every call records an NVTX range either way.
 *   LM_AUTOTUNE_CACHE=<path>  lm_autotune appends its choice to <path> (JSON
 *     lines keyed by GPU name, SM count, precision, angular flag, geometry and
 *     floor(log2 N)); a solver without a configuration of its own starts from
 *     the last entry for its key, in this or a later process.
 *   LM_AUTOTUNE=1  such a solver with no recorded entry runs lm_autotune the
 *     first time it needs a configuration at a new N bucket.
 */

/* Thread-local message for the last non-OK status ("" if none). */
const char *lm_last_error(void);

/* Library version string. */
const char *lm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LM_GB300_H */
