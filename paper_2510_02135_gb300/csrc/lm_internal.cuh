// Internal interfaces between the library's translation units.
// Kernels live in pair_kernels.cu, adjoint_kernels.cu, lanczos_kernels.cu and
// batch_kernels.cu; the C ABI and the solver state live in lm_api.cu.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>

namespace lmk {

// Packed FP64 position / vector slot (x, y, z, pad), 32-byte aligned.
struct __align__(32) dvec4 {
    double x, y, z, w;
};

// Kernel launches issued by the library (all solvers, all threads).
void count_launches(int n);

// ---------------------------------------------------------------------------
// Device bounds checks (a build with -DLM_DEBUG_BOUNDS; the stand-in for a
// memory sanitizer).  LM_INBOUNDS(cond, code, index) is true in other builds;
// in a checked build a false condition records (code, index) in the
// translation unit's check word (the first failure wins) and the caller skips
// the access, so a failed check never faults the GPU.  lm_debug_check reads
// and clears the words of every unit.
// ---------------------------------------------------------------------------
using BoundsReadFn = cudaError_t (*)(unsigned long long*);
void register_bounds_reader(BoundsReadFn fn, const char* unit);

}  // namespace lmk

#ifdef LM_DEBUG_BOUNDS
namespace {
__device__ unsigned long long g_lm_bounds_word;

__device__ __forceinline__ bool lm_bounds_ok(bool ok, unsigned code, long long idx) {
    if (!ok)
        atomicCAS(&g_lm_bounds_word, 0ull,
                  ((unsigned long long)code << 48) | ((unsigned long long)idx & 0xffffffffffffull));
    return ok;
}

cudaError_t lm_bounds_read_and_clear(unsigned long long* w) {
    cudaError_t e = cudaMemcpyFromSymbol(w, g_lm_bounds_word, sizeof(*w));
    const unsigned long long zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_lm_bounds_word, &zero, sizeof(zero));
    return e;
}

struct LmBoundsRegistrar {
    explicit LmBoundsRegistrar(const char* unit) { lmk::register_bounds_reader(&lm_bounds_read_and_clear, unit); }
};
const LmBoundsRegistrar g_lm_bounds_registrar(__FILE__);
}  // namespace
#define LM_INBOUNDS(cond, code, idx) lm_bounds_ok((cond), (unsigned)(code), (long long)(idx))
#else
#define LM_INBOUNDS(cond, code, idx) (true)
#endif

namespace lmk {

// Raises the dynamic shared-memory limit of kernel `fn` to `bytes` on the
// current device, once per device.  The attribute belongs to the device
// context, so a process that drives several GPUs sets it on each of them;
// `devs` (one per kernel instantiation) records the devices done, bit d for
// device d (devices 64 and above set it on every launch).
template <typename K>
inline cudaError_t smem_attr_once(std::atomic<unsigned long long>& devs, K fn, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (devs.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) devs.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}
// Message returned by lm_last_error() on the calling thread.
void set_last_error(const char* msg);

// Algorithmic work per ordered pair (far-field formula, FMA = 2 flops),
// frozen for the roofline figures: translation only, and all four blocks.
constexpr double kFlopsPerPairTT = 35.0;
constexpr double kFlopsPerPair6N = 86.0;
// Above a single wall: the free-space pair plus the wall part, counted from
// the formulas as wall_kernels.cu evaluates them.
constexpr double kFlopsPerPairWallTT = 131.0;
constexpr double kFlopsPerPairWall6N = 299.0;

// Constants of the RPY pair blocks for radius a, in units of 1/(8 pi eta).
// Far field (r >= 2a), d = x_i - x_j, F the force and T the torque on j:
//   u_i += A F + B (d.F) d + g (T x d)
//   w_i += g (F x d) + ar T + br (d.T) d
//   A = 1/r + K1/r^3, B = 1/r^3 - K2/r^5, g = 1/r^3, ar = -1/(2 r^3), br = 3/(2 r^5)
// Overlap (r < 2a), s = r / a:
//   A = (4/(3a)) (1 - 9 s / 32),        B = 1 / (8 a^2 r)
//   g = (1/(2 a^3)) (1 - 3 s / 8),
//   ar = (1/a^3) (1 - 27 s/32 + 5 s^3/64),  br = (1/a^3) (9/(32 a r) - 3 r/(64 a^3))
// The results are multiplied by 1/(8 pi eta) once per particle.
template <typename R>
struct RpyConst {
    R four_a2;  // (2a)^2
    R K1;       // 2a^2/3
    R K2;       // 2a^2
    R nA0;      // 4/(3a)
    R nA1;      // 3/(8a^2)
    R nB;       // 1/(8a^2)
    R ng0;      // 1/(2a^3)
    R ng1;      // 3/(16a^4)
    R inv_a3;   // 1/a^3
    R rr1;      // 27/(32a)
    R rr3;      // 5/(64a^3)
    R rrb0;     // 9/(32a)
    R rrb1;     // 3/(64a^3)
};

template <typename R>
inline RpyConst<R> make_rpy_const(double a) {
    RpyConst<R> k;
    k.four_a2 = (R)(4.0 * a * a);
    k.K1 = (R)(2.0 * a * a / 3.0);
    k.K2 = (R)(2.0 * a * a);
    k.nA0 = (R)(4.0 / (3.0 * a));
    k.nA1 = (R)(3.0 / (8.0 * a * a));
    k.nB = (R)(1.0 / (8.0 * a * a));
    k.ng0 = (R)(1.0 / (2.0 * a * a * a));
    k.ng1 = (R)(3.0 / (16.0 * a * a * a * a));
    k.inv_a3 = (R)(1.0 / (a * a * a));
    k.rr1 = (R)(27.0 / (32.0 * a));
    k.rr3 = (R)(5.0 / (64.0 * a * a * a));
    k.rrb0 = (R)(9.0 / (32.0 * a));
    k.rrb1 = (R)(3.0 / (64.0 * a * a * a));
    return k;
}

// Positions are packed as (x, y, z, 0) float4 (FP32C) or double4 (FP64).
// Padding coordinate for unused tile slots: far from any admissible particle.
constexpr double kPadCoord = 1.0e18;
constexpr double kMaxAbsCoord = 1.0e15;

// One mobility product on the packed positions.
struct MdotArgs {
    int fp64;              // 0: FP32 pairs with compensated sums, 1: FP64
    int angular;           // 0: 3N (forces only), 1: 6N
    int64_t N;
    const void* pos4;      // packed positions
    const void* F;         // N x 3 (nullable = zero)
    const void* T;         // N x 3 (nullable = zero; ignored without angular)
    int in_f64;            // element type of F, T
    void* lin;             // N x 3
    void* ang;             // N x 3 (angular only)
    int out_f64;           // element type of lin, ang
    double a, eta;
    int threads, ilp, splits;
    int packed = 0;        // 1: packed f32x2 form (FP32, even ilp)
    double* partials;      // splits * (3 or 6) * N doubles when splits > 1
    cudaEvent_t ev_begin = nullptr;   // recorded right before / after the pair
    cudaEvent_t ev_end = nullptr;     // kernel when non-null (profiling)
};

// Backward (adjoint) product.
struct AdjointArgs {
    int fp64;
    int angular;
    int64_t N;
    const void* pos4;
    const void* F; const void* T;     // forward inputs
    const void* G; const void* H;     // cotangents of lin, ang
    void* dX; void* dF; void* dT;     // outputs (nullable dX / dF)
    double a, eta;
    int threads, splits;
    int ilp = 4;                      // i-particles per thread (packed FP32 translation form: 2 or 4)
    int uj = 1;                       // j-particles per overlap vote (packed form: 1 or 2); 3: symmetric
                                      // form (packed for FP32 translation, scalar otherwise); 4: symmetric
                                      // packed form with angular blocks (FP32)
    double* partials;                 // splits * (3 + 3 or 6) * N doubles when splits > 1
    // symmetric forms (uj >= 3): work items (int4: i-block, first tile, end tile, 0) and the
    // FP64 accumulators acc[N][C], C = 6 or 9 with angular blocks (zeroed by the launcher)
    const void* sym_items = nullptr;
    int64_t n_sym_items = 0;
    double* sym_acc = nullptr;
};

// Launch-configuration tables (pair_kernels.cu / adjoint_kernels.cu).
bool mdot_config_supported(int fp64, int angular, int threads, int ilp, int packed = 0);
int mdot_ctas_per_sm(int fp64, int angular, int threads, int ilp, int packed = 0);
// Default j-split count for `slots` concurrently resident CTAs (lm_api.cu);
// every split holds at least min_tps j-tiles.
int auto_splits(int64_t N, int threads, int ilp, int slots, int min_tps = 4);
// Number of j-splits actually launched for a requested split count.
int64_t mdot_effective_splits(int64_t N, int threads, int splits);
int mdot_partial_components(int angular);
cudaError_t launch_mdot(const MdotArgs& a, cudaStream_t s);
// Single-wall geometry (wall_kernels.cu): the same arguments, positions packed
// by launch_pack_wall_positions.
bool wall_config_supported(int fp64, int threads, int ilp, int packed);
int wall_ctas_per_sm(int fp64, int angular, int threads, int ilp, int packed);
cudaError_t launch_wall_mdot(const MdotArgs& a, cudaStream_t s);
cudaError_t launch_adjoint(const AdjointArgs& a, cudaStream_t s);
int adjoint_partial_components(int angular);
int adjoint_ilp(int fp64, int angular);
bool adjoint_config_supported(int fp64, int angular, int threads, int ilp, int uj);
int adjoint_ctas_per_sm(int fp64, int angular, int threads, int ilp, int uj);

// Pack N x 3 positions into (x, y, z, 0) and flag non-finite or too large
// coordinates in *bad (device int, set to 1).
cudaError_t launch_pack_positions(const void* pos, int in_f64, int64_t N, void* pos4, int out_f64,
                                  int* bad, cudaStream_t s);
// Wall geometry (wall at z = z0): (x, y, max(z - z0, a), f) with the damping
// factor f = clamp((z - z0) / a, 0, 1).
cudaError_t launch_pack_wall_positions(const void* pos, int in_f64, int64_t N, double a, double z0, void* pos4,
                                       int out_f64, int* bad, cudaStream_t s);
// Random finite differences (wall geometry): pack x + scale W (W: 3N doubles),
// and write (P - Q) * inv_delta (FP64 grand vectors) to lin / ang.
cudaError_t launch_displace_pack_wall(const void* pos, int in_f64, const double* W, double scale, int64_t N,
                                      double a, double z0, void* pos4, int out_f64, cudaStream_t s);
cudaError_t launch_rfd_difference(const double* P, const double* Q, double inv_delta, int64_t N, int angular,
                                  void* lin, void* ang, int out_f64, cudaStream_t s);
// Jacobi preconditioner of the Lanczos square root (wall_kernels.cu):
// p = diag(M)^{-1/2}, q = diag(M)^{1/2} from the packed positions (3N or 6N
// doubles each), and y = a * x elementwise.
cudaError_t launch_mobility_diag(const void* pos4, int fp64, int64_t N, double a, double eta, int angular, int wall,
                                 double* p, double* q, cudaStream_t s);
cudaError_t launch_vmul(const double* a, const double* x, double* y, int64_t n, cudaStream_t s);
// Roller-example time stepping (integrator_kernels.cu): soft steric forces
// (N x 3 positions in, N x 3 forces out, element type by f64) and the
// stochastic Adams-Bashforth update of the positions.
cudaError_t launch_soft_repulsion(const void* pos, int f64, int64_t N, double U0, double b, double d_pair,
                                  double d_wall, int wall, double z_wall, void* out, cudaStream_t s);
// out (lin / ang, element type by out_f64) = u + kT d + y over the 3N (6N)
// entries: u, d FP64 grand vectors (d nullable = 0), y in the out precision.
cudaError_t launch_langevin_combine(const double* u, const double* d, const void* y, double kT, int64_t N,
                                    int angular, void* lin, void* ang, int out_f64, cudaStream_t s);
cudaError_t launch_ab_update(const void* pos, int f64, const double* u, const double* d, const void* y,
                             double* hist, int first, double kT, double dt, int64_t N, void* out, cudaStream_t s);

// Lanczos vector kernels (lanczos_kernels.cu).  All vectors are FP64 of
// length n; the basis V is row-major (row j = v_j, stride n).  Reductions are
// deterministic: blocks write partials and the last block to finish (a device
// counter that must start at 0 and is reset by that block) adds them in a
// fixed order.  `red` is scratch of lz_red_doubles(n, m) doubles and `ctr`
// holds lz_ctr_count(m) counters for bases of up to m rows.
size_t lz_red_doubles(int64_t n, int m);
size_t lz_ctr_count(int m);
// out[0] = |x|, out[1] = |x|^2 (two launches, no counter)
cudaError_t lz_norm(const double* x, int64_t n, double* red, double* out, cudaStream_t s);
// mode 0: out[0] = x.y; mode 1: out[0] = |x|, out[1] = |x|^2
cudaError_t lz_dot1(const double* x, const double* y, int64_t n, double* red, unsigned* ctr, double* out,
                    int mode, cudaStream_t s);
// w -= alpha[0] vk + beta[0] vkm1 (vkm1 / beta nullable), then out = (|w|, |w|^2)
cudaError_t lz_axpy2_norm(double* w, const double* vk, const double* alpha, const double* vkm1, const double* beta,
                          int64_t n, double* red, unsigned* ctr, double* out, cudaStream_t s);
// c[j] = v_j . w for j < m.  With cond = [h0, h0^2, h1, h1^2] (device) the
// kernel does nothing unless h1 < h0 / sqrt(2) (DGKS second-pass test).
cudaError_t lz_multidot1(const double* V, int m, const double* w, int64_t n, double* red, unsigned* ctr, double* c,
                         cudaStream_t s, const double* cond = nullptr);
// w -= sum_j c[j] v_j (same optional condition), then out = (|w|, |w|^2);
// a skipped pass copies (cond[2], cond[3]) into out.
cudaError_t lz_sub_vc_norm(const double* V, int m, const double* c, double* w, int64_t n, double* red,
                           unsigned* ctr, double* out, cudaStream_t s, const double* cond = nullptr);
// y = x / nrm[0]
cudaError_t lz_scale(const double* x, const double* nrm, double* y, int64_t n, cudaStream_t s);
// y = sum_j z[j] v_j
cudaError_t lz_combine(const double* V, int m, const double* z, double* y, int64_t n, cudaStream_t s);
// lin / ang (float or double) = scale * y, lin from y[0, 3N), ang from y[3N, 6N)
cudaError_t lz_store(const double* y, double scale, int64_t N, int angular, void* lin, void* ang, int out_f64,
                     cudaStream_t s);
// W from Philox-4x32-10: element e is normal number (e % 4) of block q = e / 4,
// counter (q low, q high, stream low, stream high), key (seed low, seed high),
// two Box-Muller pairs from the words (0, 1) and (2, 3).
cudaError_t lz_philox_normals(uint64_t seed, uint64_t stream, double* W, int64_t n, cudaStream_t s);
cudaError_t lz_philox_words(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t count,
                            cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched persistent kernel (batch_kernels.cu) over S concatenated systems.
// ---------------------------------------------------------------------------
enum BatchMode { kBatchBD = 0, kBatchMdot = 1, kBatchSqrt = 2 };
enum BatchError { kBatchOk = 0, kBatchTimeout = 1, kBatchTridiag = 2 };
// Elements per vector-phase work unit.  A unit's time is set by the basis
// rows it walks (serialised DRAM rounds), not by its length, and the phase
// lasts as many units as the busiest CTA holds: 384 leaves two units per CTA
// for the benchmark batch (256 left a third one for a few CTAs; 512 lengthens
// the dot loop of every unit).  A multiple of both CTA widths (64, 128).
constexpr int kBatchChunk = 384;
constexpr int kBatchJPart = 1024;      // j-range of one product work item
// Grid barrier of the persistent kernel: bar[0] counts arrived groups,
// bar[1] is the generation, and group g of kBarGroup consecutive main CTAs
// counts its arrivals at bar[kBarStride * (1 + g)] (one 128-byte line each).
constexpr int kBarGroup = 32;
constexpr int kBarStride = 32;
constexpr int kBarMaxGroups = 256;
constexpr size_t kBarWords = (size_t)kBarStride * (1 + kBarMaxGroups);
constexpr int kSolverWarps = 64;       // solver warps of a batched launch (one request each at a time)

// Scratch of the warp form of the tridiagonal step f(T) e1 in doubles, for
// T of at most m_max rows: d, b, b^2, u as double-float (4 m_max), z (m_max),
// the lanes' reciprocal pivots and partial sums (2 x 32 m_max double-float,
// lane-interleaved).  The QR fallback uses the pivot region for its d, e, r.
__host__ __device__ constexpr size_t tridiag_warp_scratch_doubles(int m_max) {
    return (size_t)69 * (size_t)m_max;
}

struct BatchParams {
    int S, m_max, mode, nsteps;
    int64_t Ntot;                      // particles over all systems
    int64_t step0;
    const int64_t* off;                // S + 1 particle offsets
    float4* pos4;                      // Ntot packed FP32 positions for the pair kernel
    double* x64;                       // 3 Ntot FP64 positions (the BD state)
    float* Fbuf;                       // 3 Ntot forces of the step
    double* u;                         // 3 Ntot drift product M F
    double* w0;                        // 3 Ntot Lanczos residual, even iterations
    double* w1;                        // 3 Ntot Lanczos residual, odd iterations
    double* V;                         // Krylov bases: system s at V + m_max * 3 off[s], row j stride 3 N_s
    double* alpha;                     // S x m_max
    double* amax;                      // S: max |alpha_i| so far in the step (breakdown test)
    double* beta;                      // S x m_max
    double* z;                         // S x m_max: |W| f(T_k) e1 of the latest iteration
    double* zprev;                     // S x m_max
    double* normW;                     // S
    double* rel;                       // S: last relative change
    int* active;                       // S: 1 while iterating in the current step
    int* msys;                         // S: iterations used in the current step
    int* itsum;                        // S: iterations summed over the call
    int* notconv;                      // S: 1 if max_iter was reached in some step
    int* kprev;                        // S: iterations of the previous BD step (0 = none)
    int warm_start;                    // 1: start the stopping test near kprev (BD mode)
    int reorth;                        // 1: always run the second Gram-Schmidt pass
    int* nact;                         // m_max + 1 counters of systems still active
    int* pass2;                        // m_max + 1 flags: some system needs the second Gram-Schmidt pass at k
    int* sys_cnt;                      // S arrival counters of the chunks of the current pass
    double* wsplit;                    // per-system j-part partial products of w (or F for mdot)
    double* usplit;                    // per-system j-part partial products of u = M F
    const int64_t* woff;               // S: offset of system s in wsplit / usplit (parts x 3 N_s)
    const int* items;                  // n_items x (system, first particle, j-part)
    int n_items;
    const int* item_range;             // S x (first item, end item)
    const int* chunks;                 // n_chunks x (system, first element)
    int n_chunks;
    const int* chunk_range;            // S x (first chunk, end chunk)
    double* part_item;                 // n_items partial dots
    double* part_chunk;                // 2 x n_chunks x (m_max + 1) partial dots
    // Asynchronous tridiagonal solves.  CTAs [n_main, gridDim.x) are solver
    // CTAs: each of their warps serves one request at a time with all its
    // lanes (tridiag_sqrt_e1_warp; the QR form on lane 0 where that declines).
    int n_main;                        // CTAs that run the phases and the grid barrier
    double* sv_w;                      // per solver warp: tridiag_warp_scratch_doubles(m_max) doubles
    int* trk;                          // per solver warp: max_rot rotation indices (QR fallback)
    double* trc;                       // per solver warp: max_rot rotation cosines (double-float)
    double* trs;                       // per solver warp: max_rot rotation sines (double-float)
    int max_rot;
    long long* q_req;                  // request ring: (step << 28) | (system << 7) | k
    unsigned long long* q_seq;         // ticket + 1 once the slot holds that ticket's request
    unsigned long long* q_ack;         // ticket + 1 once a solver has read that ticket's request
    unsigned long long* q_ctr;         // [0] next ticket to take, [1] next ticket to post, [2] requests done
    int q_cap;
    int* inflight;                     // [step parity]: requests posted and not yet done
    double* zres;                      // S x 2 (step parity) x R x m_max results |W| f(T_k) e1
    unsigned long long* zdone;         // S x 2 x R tags: step * 128 + k + 1
    int R;
    int* state;                        // S: 1 iterating, 2 / 3 waiting for the last result
                                       //    (max_iter / breakdown), 0 done
    int* next_check;                   // S: next iteration whose stopping test is due
    int* last_k;                       // S: last iteration (states 2, 3)
    int* k0s;                          // S: first iteration with a solve in this step
    int* posted;                       // S: last iteration whose solve was requested
    int* main_done;                    // set when no more requests can come
    long long* cur_step;               // step the main CTAs are in (solvers drop older requests)
    unsigned* bar;                     // grid barrier: count, generation
    unsigned long long* ticket;        // dynamic work counter
    int* err;                          // BatchError
    long long spin_limit;              // clock cycles a barrier may wait
    RpyConst<float> k;
    double c8;                         // 1 / (8 pi eta)
    double kT, dt, k_trap, tol, brk_rel, prefactor;
    uint64_t seed;
    const float* F_in;                 // kBatchMdot input
    float* lin_out;                    // kBatchMdot / kBatchSqrt output
    const double* W_in;                // kBatchSqrt noise (nullable: Philox)
    unsigned long long* pair_count;    // nullable: pair evaluations of the run (profiling)
    unsigned long long* timeline;      // nullable: phase end times (ns) of the first step
    int timeline_len;
};

// Launch the persistent kernel (cooperative) with `threads` x `ilp` tiling.
cudaError_t launch_batch(const BatchParams& p, int threads, int ilp, int grid, cudaStream_t s);
// CTAs of the persistent kernel that can be co-resident per SM.
int batch_ctas_per_sm(int threads, int ilp);
bool batch_tiling_supported(int threads, int ilp);
// Pack N x 3 float positions into pos4 and x64.
cudaError_t launch_batch_pack(const float* pos, int64_t N, float4* pos4, double* x64, int* bad, cudaStream_t s);
// out (N x 3 float) = x64
cudaError_t launch_batch_unpack(const double* x64, int64_t N, float* out, cudaStream_t s);
// A kernel whose barrier waits for one CTA more than it launches: every
// wait runs out after spin_limit cycles and *err becomes kBatchTimeout.
cudaError_t launch_tridiag_dev(int count, int m, const double* alpha, const double* beta, double* scratch, int* rk,
                               double* rc, double* rs, int max_rot, double* out, int* status, int* path,
                               cudaStream_t s);
cudaError_t launch_batch_timeout_probe(unsigned* bar, int* err, long long spin_limit, int grid,
                                       cudaStream_t s);

}  // namespace lmk
