// C ABI of the library (include/lm.h): solver state, argument validation,
// host/device staging of arrays, launch-configuration choice, the Lanczos
// driver of lm_sqrt_mdot and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/lm.h"
#include "lm_internal.cuh"
#include "lm_runtime.cuh"
#include "tridiag.cuh"

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

lm_status fail(lm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

lm_status cuda_fail(cudaError_t e, const char* where) {
    cudaGetLastError();  // clear a sticky launch error where possible
    if (e == cudaErrorMemoryAllocation) return fail(LM_ERR_OOM, "%s: out of device memory", where);
    return fail(LM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define LM_CUDA(call, where)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

struct DBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p != nullptr) return cudaSuccess;
        release();
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) { p = nullptr; cap = 0; return e; }
        cap = bytes;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = (cudaSetDevice(dev) == cudaSuccess);
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct LanczosHost {
    std::vector<double> alpha, beta, z, zprev, d, e, rc, rs;
    std::vector<int> rk;
    int solve(int m, double normW, int* clamped) {
        z.assign(m, 0.0);
        d.resize(m);
        e.resize(m);
        size_t max_rot = (size_t)4 * m * m + 64;
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (rk.size() < max_rot) { rk.resize(max_rot); rc.resize(max_rot); rs.resize(max_rot); }
            const int r = lmk::tridiag_sqrt_e1(m, alpha.data(), beta.data(), d.data(), e.data(), rk.data(),
                                               rc.data(), rs.data(), (int)max_rot, z.data(), clamped);
            if (r != -2) {
                for (double& v : z) v *= normW;
                return r;
            }
            max_rot = (size_t)30 * m * m + 64;
        }
        return -2;
    }
};

}  // namespace

namespace {
// Random finite differences (Sec. 3.4): Philox stream of the noise, and the
// default step relative to the radius (FP64 pairs / FP32 pairs).
constexpr uint64_t kRfdStream = 0x524644ull;   // "RFD"
constexpr double kRfdDeltaFP64 = 1e-4;
constexpr double kRfdDeltaFP32 = 1e-2;
}  // namespace

namespace lmk {
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace lmk

struct lm_solver {
    int angular = 0;
    int fp64 = 0;
    int wall = 0;          // 1: no-slip wall at z = z_wall ("single_wall" in z)
    double z_wall = 0.0;   // wall height (setParameters(wallHeight) of Sec. 3.2)
    double eta = 1.0, a = 1.0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 1;

    int64_t N = 0;
    bool has_pos = false;

    DBuf pos4;
    DBuf partials;
    DBuf in_stage[4];
    DBuf out_stage[3];
    DBuf flag;
    DBuf tune_in, tune_out;
    // the caller's positions (N x 3, solver precision) and RFD scratch
    DBuf pos_raw, rfd_pos4, rfd_W, rfd_P, rfd_Q;
    // Adams-Bashforth step scratch: M [F; T] and the scaled square root (6N doubles / 6N values), new positions
    DBuf ab_u, ab_d, ab_y, ab_x;
    // Jacobi preconditioner of the Lanczos square root: p = diag(M)^{-1/2}, q = diag(M)^{1/2}, scratch
    int precond = 0;
    DBuf pc_p, pc_q, pc_t;
    // device counter of the single-launch reductions (zero between launches)
    DBuf lzctr;
    uint64_t rfd_calls = 0;

    // Lanczos state
    DBuf V, w, y, red, scal, zbuf, cbuf, Wbuf;
    // symmetric adjoint: work-item table (for sym_key) and FP64 accumulators
    DBuf sym_items, sym_acc;
    std::array<int64_t, 4> sym_key{{-1, 0, 0, 0}};
    int64_t sym_n_items = 0;
    double* pinned = nullptr;  // host scalar read-back
    size_t pinned_doubles = 0;

    lm_pair_config cfg{128, 4, 1, 0};
    bool cfg_forced = false;
    int64_t cfg_N = -1;
    lm_pair_config adj_cfg{128, 1, 1, 0};
    int64_t adj_cfg_N = -1;

    lm_lanczos_stats stats{0, 0, 0.0, 0.0, 0};

    int reorth = 0;   // 0: DGKS-adaptive second Gram-Schmidt pass, 1: always two passes
    // Lanczos host state and per-iteration events
    LanczosHost lz_host;
    std::vector<cudaEvent_t> lz_ev;

    // profiling of the pair kernel
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;   // pairs (begin, end)
    size_t prof_used = 0;               // event pairs in use
    double prof_pairs = 0.0;
    // profiling of the Lanczos vector kernels: one event pair per iteration
    // around the kernels that follow the product (alpha, three-term update,
    // Gram-Schmidt passes, beta); bytes are counted once the iteration's
    // scalars (and so whether the second pass ran) are on the host
    std::vector<cudaEvent_t> vprof_ev;
    std::vector<double> vprof_bytes;    // per event pair; < 0 while unknown
    std::vector<std::pair<size_t, int>> vprof_pending;   // (event pair, iteration) of the running call
    size_t vprof_used = 0;

    ~lm_solver() {
        DBuf* all[] = {&pos4, &partials, &in_stage[0], &in_stage[1], &in_stage[2], &in_stage[3],
                       &out_stage[0], &out_stage[1], &out_stage[2], &flag, &tune_in, &tune_out,
                       &pos_raw, &rfd_pos4, &rfd_W, &rfd_P, &rfd_Q, &ab_u, &ab_d, &ab_y, &ab_x, &pc_p, &pc_q, &pc_t, &lzctr,
                       &V, &w, &y, &red, &scal, &zbuf, &cbuf, &Wbuf, &sym_items, &sym_acc};
        for (DBuf* b : all) b->release();
        if (pinned) cudaFreeHost(pinned);
        for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
        for (cudaEvent_t e : vprof_ev) cudaEventDestroy(e);
        for (cudaEvent_t e : lz_ev) cudaEventDestroy(e);
    }
};

namespace {

size_t elem_size(const lm_solver* s) { return s->fp64 ? sizeof(double) : sizeof(float); }

// Device view of an input array: device pointers pass through, host arrays
// are copied into a staging buffer on the solver's stream.
lm_status stage_in(lm_solver* s, const void* p, size_t bytes, int slot, const void** out) {
    *out = nullptr;
    if (p == nullptr) return LM_OK;
    if (is_device_ptr(p)) { *out = p; return LM_OK; }
    LM_CUDA(s->in_stage[slot].ensure(bytes), "staging input");
    LM_CUDA(cudaMemcpyAsync(s->in_stage[slot].p, p, bytes, cudaMemcpyHostToDevice, s->stream), "copy input to device");
    *out = s->in_stage[slot].p;
    return LM_OK;
}

struct OutView {
    void* user = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool host = false;
};

lm_status stage_out(lm_solver* s, void* p, size_t bytes, int slot, OutView* v) {
    v->user = p;
    v->bytes = bytes;
    v->dev = nullptr;
    v->host = false;
    if (p == nullptr) return LM_OK;
    if (is_device_ptr(p)) { v->dev = p; return LM_OK; }
    LM_CUDA(s->out_stage[slot].ensure(bytes), "staging output");
    v->dev = s->out_stage[slot].p;
    v->host = true;
    return LM_OK;
}

lm_status finish_out(lm_solver* s, OutView* views, int nv) {
    bool any = false;
    for (int k = 0; k < nv; ++k) {
        if (views[k].host && views[k].user) {
            LM_CUDA(cudaMemcpyAsync(views[k].user, views[k].dev, views[k].bytes, cudaMemcpyDeviceToHost, s->stream),
                    "copy output to host");
            any = true;
        }
    }
    if (any) LM_CUDA(cudaStreamSynchronize(s->stream), "synchronise outputs");
    return LM_OK;
}

}  // namespace

// Split count minimising (waves x tiles per CTA): keeps all SMs busy when N
// is small and limits the tail wave when N is large.  Split k of s holds
// tiles [k T / s, (k + 1) T / s), so a CTA holds at most ceil(T / s) tiles.
int lmk::auto_splits(int64_t N, int threads, int ilp, int slots, int min_tps) {
    const int64_t nblk = (N + (int64_t)threads * ilp - 1) / ((int64_t)threads * ilp);
    const int64_t ntiles = (N + threads - 1) / threads;
    int best = 1;
    double best_cost = 1e300;
    for (int s = 1; s <= 64 && s <= ntiles; ++s) {
        const int64_t tps = (ntiles + s - 1) / s;
        if (s > 1 && tps < min_tps) break;
        const int64_t items = nblk * s;
        const int64_t waves = (items + slots - 1) / std::max(1, slots);
        const double cost = (double)waves * (double)tps * (1.0 + 0.002 * (double)s);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = s; }
    }
    return best;
}

namespace {
using lmk::auto_splits;

bool pair_config_supported(const lm_solver* s, int threads, int ilp, int packed) {
    return s->wall ? lmk::wall_config_supported(s->fp64, threads, ilp, packed)
                   : lmk::mdot_config_supported(s->fp64, s->angular, threads, ilp, packed);
}

int pair_ctas_per_sm(const lm_solver* s, int threads, int ilp, int packed) {
    return s->wall ? lmk::wall_ctas_per_sm(s->fp64, s->angular, threads, ilp, packed)
                   : lmk::mdot_ctas_per_sm(s->fp64, s->angular, threads, ilp, packed);
}

// Split counts the autotuner times for one tiling: the model's choice, half,
// one and a half and twice it, and the counts that make the CTA count a whole
// number (1..4) of waves of `slots` resident CTAs.  `model_and_waves` keeps
// only the model's choice and the whole-wave counts.
std::vector<int> split_candidates(int64_t N, int threads, int ilp, int slots, bool model_and_waves = false) {
    const int64_t nblk = (N + (int64_t)threads * ilp - 1) / ((int64_t)threads * ilp);
    const int64_t ntiles = (N + threads - 1) / threads;
    const int sa = auto_splits(N, threads, ilp, slots);
    std::vector<int> c = {sa};
    if (!model_and_waves) {
        c.push_back(std::max(1, sa / 2));
        c.push_back(std::max(1, (3 * sa) / 2));
        c.push_back(sa * 2);
        c.push_back(auto_splits(N, threads, ilp, slots, 1));
    }
    for (int w = 1; w <= 4; ++w) {
        const int64_t sp = ((int64_t)w * slots) / std::max<int64_t>(1, nblk);
        if (sp >= 1 && sp <= ntiles && sp <= 256 && sp * nblk == (int64_t)w * slots) c.push_back((int)sp);
    }
    // many i-blocks: the smallest split count of at least the model's choice
    // that makes the CTA count a whole number of waves (nblk x s a multiple of
    // slots), e.g. 19 splits of 256 i-blocks on 152 slots
    if (nblk > 0 && slots > 0) {
        const int64_t step = slots / std::gcd<int64_t>(nblk, slots);
        const int64_t sp = ((std::max<int64_t>(sa, 1) + step - 1) / step) * step;
        if (sp <= ntiles && sp <= 64) c.push_back((int)sp);
    }
    std::vector<int> out;
    for (int v : c)
        if (std::find(out.begin(), out.end(), v) == out.end()) out.push_back(v);
    return out;
}

lm_pair_config default_config(const lm_solver* s, int64_t N) {
    lm_pair_config c;
    // FP32: the packed form (fastest measured on GB300: 256 x 4 with angular
    // blocks, 128 x 8 without); FP64: the scalar form.
    c.threads = (!s->fp64 && s->angular) ? 256 : 128;
    c.ilp = s->fp64 ? (s->angular ? 1 : 2) : (s->angular ? 4 : 8);
    c.packed = s->fp64 ? 0 : 1;
    if (s->wall) {
        // single wall: FP32 packed 256 x 4 (translation) / 256 x 2 (all blocks), FP64 scalar 128 x 1
        c.threads = s->fp64 ? 128 : 256;
        c.ilp = s->fp64 ? 1 : (s->angular ? 2 : 4);
        c.packed = s->fp64 ? 0 : 1;
    }
    int occ = std::max(1, pair_ctas_per_sm(s, c.threads, c.ilp, c.packed));
    c.splits = auto_splits(N, c.threads, c.ilp, occ * s->sm_count);
    const int64_t nblk = (N + (int64_t)c.threads * c.ilp - 1) / ((int64_t)c.threads * c.ilp);
    if (nblk * lmk::mdot_effective_splits(N, c.threads, c.splits) < (int64_t)occ * s->sm_count) {
        // too few CTAs to fill the GPU: the smallest i-blocks, and splits of down
        // to one j-tile each
        c.threads = 128;
        c.ilp = s->fp64 ? 1 : 2;
        c.packed = s->fp64 ? 0 : 1;
        occ = std::max(1, pair_ctas_per_sm(s, c.threads, c.ilp, c.packed));
        c.splits = auto_splits(N, c.threads, c.ilp, occ * s->sm_count, 1);
    }
    return c;
}

// Tuned launch configurations shared by the solvers of this process:
// lm_autotune records its choice under (device, precision, angular blocks,
// geometry, N bucket = floor(log2 N)), and a solver without a configuration
// of its own takes the one recorded for its bucket, with the split count
// recomputed when its N is not the tuned N.
struct TunedEntry {
    lm_pair_config cfg;
    lm_pair_config adj;
    bool has_adj = false;
    int64_t N = 0;
};
std::mutex g_tuned_mu;
std::map<std::array<int, 5>, TunedEntry> g_tuned;

std::array<int, 5> tuned_key(const lm_solver* s, int64_t N) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << (b + 1)) <= N) ++b;
    return {s->device, s->fp64 ? 1 : 0, s->angular ? 1 : 0, s->wall ? 1 : 0, b};
}

// The process's record, else the persistent cache (LM_AUTOTUNE_CACHE).
bool lookup_tuned(const lm_solver* s, int64_t N, TunedEntry* e) {
    const std::array<int, 5> key = tuned_key(s, N);
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *e = it->second;
            return true;
        }
    }
    lmk::TuneCacheKey ck;
    long long n = 0;
    bool has_adj = false;
    if (!lmk::tune_cache_key(s->device, key[1], key[2], key[3], key[4], &ck) ||
        !lmk::tune_cache_lookup(ck, &n, &e->cfg, &e->adj, &has_adj))
        return false;
    if (!pair_config_supported(s, e->cfg.threads, e->cfg.ilp, e->cfg.packed) || e->cfg.splits < 1) return false;
    e->N = n;
    e->has_adj = has_adj && lmk::adjoint_config_supported(s->fp64, s->angular, e->adj.threads, e->adj.ilp,
                                                          e->adj.packed);
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned[key] = *e;
    return true;
}

lm_status autotune_impl(lm_solver* s, int reps, lm_pair_config* best);

void ensure_config(lm_solver* s) {
    if (s->cfg_N == s->N) return;
    if (!s->cfg_forced) {
        s->cfg = default_config(s, s->N);
        TunedEntry e;
        bool found = lookup_tuned(s, s->N, &e);
        if (!found && lmk::autotune_on_first_use()) {
            // LM_AUTOTUNE=1: tune this N bucket now (recorded for the process and
            // in the persistent cache); on failure keep the model's choice
            lm_pair_config best;
            if (autotune_impl(s, 2, &best) == LM_OK) return;
        }
        if (found) {
            s->cfg = e.cfg;
            if (e.N != s->N) {
                const int occ = std::max(1, pair_ctas_per_sm(s, e.cfg.threads, e.cfg.ilp, e.cfg.packed));
                s->cfg.splits = auto_splits(s->N, e.cfg.threads, e.cfg.ilp, occ * s->sm_count);
            }
        }
    }
    s->cfg_N = s->N;
}

lm_status run_mdot(lm_solver* s, const void* F, const void* T, int in_f64, void* lin, void* ang, int out_f64,
                   const lm_pair_config& cfg, const void* pos4_override = nullptr) {
    lmk::MdotArgs a;
    a.fp64 = s->fp64;
    a.angular = s->angular;
    a.N = s->N;
    a.pos4 = pos4_override ? pos4_override : s->pos4.p;
    a.F = F;
    a.T = s->angular ? T : nullptr;
    a.in_f64 = in_f64;
    a.lin = lin;
    a.ang = s->angular ? ang : nullptr;
    a.out_f64 = out_f64;
    a.a = s->a;
    a.eta = s->eta;
    a.threads = cfg.threads;
    a.ilp = cfg.ilp;
    a.splits = cfg.splits;
    a.packed = cfg.packed;
    a.partials = nullptr;
    const int64_t se = lmk::mdot_effective_splits(s->N, cfg.threads, cfg.splits);
    if (se > 1) {
        const size_t bytes =
            (size_t)se * lmk::mdot_partial_components(s->angular) * (size_t)s->N * sizeof(double);
        LM_CUDA(s->partials.ensure(bytes), "allocating split partial sums");
        a.partials = s->partials.as<double>();
    }
    if (s->prof_on) {
        while (s->prof_ev.size() < 2 * (s->prof_used + 1)) {
            cudaEvent_t e;
            LM_CUDA(cudaEventCreate(&e), "profiling event");
            s->prof_ev.push_back(e);
        }
        a.ev_begin = s->prof_ev[2 * s->prof_used];
        a.ev_end = s->prof_ev[2 * s->prof_used + 1];
        s->prof_used += 1;
        s->prof_pairs += (double)s->N * (double)s->N;
    }
    if (s->wall)
        LM_CUDA(lmk::launch_wall_mdot(a, s->stream), "mobility product kernel (single wall)");
    else
        LM_CUDA(lmk::launch_mdot(a, s->stream), "mobility product kernel");
    return LM_OK;
}

lm_status check_solver(lm_solver* s, bool need_pos) {
    if (s == nullptr) return fail(LM_ERR_INVALID_ARG, "solver is NULL");
    if (need_pos && !s->has_pos) return fail(LM_ERR_STATE, "positions not set (call lm_set_positions first)");
    return LM_OK;
}

// One random finite difference sample of div M (Eq. rfd) into device
// buffers lin / ang (element type by out_f64), wall geometry.
lm_status rfd_sample(lm_solver* s, uint64_t seed, double delta, void* lin, void* ang, int out_f64);

bool valid_name(const char* p) {
    return p && (!strcmp(p, "open") || !strcmp(p, "periodic") || !strcmp(p, "single_wall") ||
                 !strcmp(p, "two_walls"));
}

}  // namespace

namespace {
// Adjoint launch configuration (item sizes chosen at launch).  FP32 with
// angular blocks: the symmetric packed form (packed = 4, ilp 4), 1.7x faster
// than the one-sided scalar kernel at N = 65536; FP64: the symmetric scalar
// form (packed = 3), 1.5x faster at N = 16384.  FP32 translation: the packed
// one-sided kernel, packed = j-particles per overlap vote (the autotuner also
// times the symmetric form).
lm_pair_config default_adjoint_config(const lm_solver* s) {
    if (s->fp64) return lm_pair_config{128, 1, 0, 3};
    if (s->angular) return lm_pair_config{128, 4, 0, 4};
    lm_pair_config c{128, lmk::adjoint_ilp(0, 0), 1, 1};
    int occ = std::max(1, lmk::adjoint_ctas_per_sm(0, 0, c.threads, c.ilp, c.packed));
    c.splits = auto_splits(s->N, c.threads, c.ilp, occ * s->sm_count);
    const int64_t nblk = (s->N + (int64_t)c.threads * c.ilp - 1) / ((int64_t)c.threads * c.ilp);
    if (nblk * lmk::mdot_effective_splits(s->N, c.threads, c.splits) < (int64_t)occ * s->sm_count) {
        // too few CTAs to fill the GPU: the smaller i-blocks and splits of down to one j-tile
        c.ilp = 2;
        occ = std::max(1, lmk::adjoint_ctas_per_sm(0, 0, c.threads, c.ilp, c.packed));
        c.splits = auto_splits(s->N, c.threads, c.ilp, occ * s->sm_count, 1);
    }
    return c;
}

void ensure_adjoint_config(lm_solver* s) {
    if (s->adj_cfg_N == s->N) return;
    s->adj_cfg = default_adjoint_config(s);
    TunedEntry e;
    if (lookup_tuned(s, s->N, &e) && e.has_adj) {
        s->adj_cfg = e.adj;
        if (e.N != s->N && e.adj.packed >= 3) {
            s->adj_cfg.splits = 0;   // item size recomputed for this N
        } else if (e.N != s->N) {
            const int occ = std::max(1, lmk::adjoint_ctas_per_sm(s->fp64, s->angular, e.adj.threads, e.adj.ilp,
                                                                  e.adj.packed));
            s->adj_cfg.splits = auto_splits(s->N, e.adj.threads, e.adj.ilp, occ * s->sm_count);
        }
    }
    s->adj_cfg_N = s->N;
}

// Tiles per work item of the symmetric adjoint when the configuration leaves
// it open: about six items per resident CTA slot over the block-triangle of
// (i-block, tile) units, and for the heavier angular and FP64 pairs at most
// four tiles (4 against 8-19 was 2-3% faster at N = 65536 and 16384).
int64_t sym_auto_chunk(const lm_solver* s, int threads, int ilp, int packed) {
    const int64_t BI = (int64_t)threads * ilp;
    const int64_t nblk = (s->N + BI - 1) / BI;
    const int64_t T = (s->N + threads - 1) / threads;
    const int occ = std::max(1, lmk::adjoint_ctas_per_sm(s->fp64, s->angular, threads, ilp, packed));
    const double total = (double)nblk * (double)T - (double)ilp * (double)nblk * (double)(nblk - 1) / 2.0;
    const int64_t chunk = std::max<int64_t>(1, (int64_t)std::ceil(total / (6.0 * occ * s->sm_count)));
    return (s->fp64 || s->angular) ? std::min<int64_t>(chunk, 4) : chunk;
}

lm_status run_adjoint(lm_solver* s, const void* F, const void* T, const void* G, const void* H, void* dX, void* dF,
                      void* dT, const lm_pair_config& cfg) {
    lmk::AdjointArgs a;
    a.fp64 = s->fp64;
    a.angular = s->angular;
    a.N = s->N;
    a.pos4 = s->pos4.p;
    a.F = F; a.T = T; a.G = G; a.H = H;
    a.dX = dX; a.dF = dF; a.dT = dT;
    a.a = s->a;
    a.eta = s->eta;
    a.threads = cfg.threads;
    a.ilp = cfg.ilp;
    a.uj = cfg.packed > 0 ? cfg.packed : 1;
    a.splits = cfg.splits;
    a.partials = nullptr;
    if (a.uj >= 3) {
        // symmetric form: items (i-block b, tiles [t0, t1)) over each block's
        // tiles from its own range onward, at most `chunk` tiles each, longest first
        const int64_t BI = (int64_t)cfg.threads * cfg.ilp;
        const int64_t nblk = (s->N + BI - 1) / BI;
        const int64_t T = (s->N + cfg.threads - 1) / cfg.threads;
        const int64_t chunk = cfg.splits >= 1 ? cfg.splits : sym_auto_chunk(s, cfg.threads, cfg.ilp, a.uj);
        const std::array<int64_t, 4> key{{s->N, cfg.threads, cfg.ilp, chunk}};
        if (s->sym_key != key) {
            std::vector<int4> items;
            for (int64_t b = 0; b < nblk; ++b)
                for (int64_t t0 = b * cfg.ilp; t0 < T; t0 += chunk)
                    items.push_back(make_int4((int)b, (int)t0, (int)std::min(T, t0 + chunk), 0));
            std::stable_sort(items.begin(), items.end(),
                             [](const int4& x, const int4& y) { return (x.z - x.y) > (y.z - y.y); });
            LM_CUDA(s->sym_items.ensure(items.size() * sizeof(int4)), "allocating adjoint work items");
            LM_CUDA(cudaMemcpyAsync(s->sym_items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    s->stream),
                    "adjoint work items");
            LM_CUDA(cudaStreamSynchronize(s->stream), "adjoint work items");
            s->sym_key = key;
            s->sym_n_items = (int64_t)items.size();
        }
        LM_CUDA(s->sym_acc.ensure((size_t)lmk::adjoint_partial_components(s->angular) * s->N * sizeof(double)),
                "allocating adjoint accumulators");
        a.sym_items = s->sym_items.p;
        a.n_sym_items = s->sym_n_items;
        a.sym_acc = s->sym_acc.as<double>();
        LM_CUDA(lmk::launch_adjoint(a, s->stream), "adjoint kernel");
        return LM_OK;
    }
    const int64_t se = lmk::mdot_effective_splits(s->N, a.threads, a.splits);
    if (se > 1) {
        const size_t pb = (size_t)se * lmk::adjoint_partial_components(s->angular) * (size_t)s->N * sizeof(double);
        LM_CUDA(s->partials.ensure(pb), "allocating split partial sums");
        a.partials = s->partials.as<double>();
    }
    LM_CUDA(lmk::launch_adjoint(a, s->stream), "adjoint kernel");
    return LM_OK;
}
}  // namespace

namespace {
lm_status rfd_sample(lm_solver* s, uint64_t seed, double delta, void* lin, void* ang, int out_f64) {
    const int64_t N = s->N;
    const size_t nvec = (size_t)(s->angular ? 6 : 3) * N;
    LM_CUDA(s->rfd_W.ensure(nvec * sizeof(double)), "allocating RFD scratch");
    LM_CUDA(s->rfd_P.ensure(nvec * sizeof(double)), "allocating RFD scratch");
    LM_CUDA(s->rfd_Q.ensure(nvec * sizeof(double)), "allocating RFD scratch");
    LM_CUDA(s->rfd_pos4.ensure((size_t)N * (s->fp64 ? sizeof(lmk::dvec4) : sizeof(float4))), "allocating RFD scratch");
    double* W = s->rfd_W.as<double>();
    // W: 3N normals (translational part); the torque part stays zero, since
    // the mobility of spheres does not depend on their orientation.
    LM_CUDA(cudaMemsetAsync(W, 0, nvec * sizeof(double), s->stream), "RFD noise");
    LM_CUDA(lmk::lz_philox_normals(seed, kRfdStream, W, 3 * N, s->stream), "RFD noise");
    ensure_config(s);
    for (int side = 0; side < 2; ++side) {
        const double scale = side == 0 ? 0.5 * delta : -0.5 * delta;
        LM_CUDA(lmk::launch_displace_pack_wall(s->pos_raw.p, s->fp64, W, scale, N, s->a, s->z_wall, s->rfd_pos4.p,
                                               s->fp64, s->stream),
                "RFD positions");
        double* out = side == 0 ? s->rfd_P.as<double>() : s->rfd_Q.as<double>();
        if (lm_status st = run_mdot(s, W, s->angular ? W + 3 * N : nullptr, 1, out, s->angular ? out + 3 * N : nullptr,
                                    1, s->cfg, s->rfd_pos4.p))
            return st;
    }
    LM_CUDA(lmk::launch_rfd_difference(s->rfd_P.as<double>(), s->rfd_Q.as<double>(), 1.0 / delta, N, s->angular,
                                       lin, ang, out_f64, s->stream),
            "RFD difference");
    return LM_OK;
}
}  // namespace

namespace {
// One ABI call: an NVTX range for its duration and, with LM_METRICS_JSONL
// set, one JSON line written after the call's stream has been synchronised
// (the metrics mode makes every logged call synchronous).
struct CallScope {
    lmk::TraceRange range;
    const char* name;
    std::chrono::steady_clock::time_point t0;
    explicit CallScope(const char* n) : range(n), name(n), t0(std::chrono::steady_clock::now()) {}
};

lm_status log_call(const CallScope& c, cudaStream_t stream, int device, lm_status st, const char* fields) {
    if (!lmk::metrics_enabled()) return st;
    {
        DeviceGuard g(device);
        cudaStreamSynchronize(stream);
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c.t0).count();
    char buf[1024];
    std::snprintf(buf, sizeof(buf), "\"call\":\"%s\",\"status\":%d,\"ms\":%.6f,%s,%s", c.name, (int)st, ms, fields,
                  lmk::metrics_device_fields(device).c_str());
    lmk::metrics_write(buf);
    return st;
}

double solver_flops_per_pair(const lm_solver* s) {
    return s->wall ? (s->angular ? lmk::kFlopsPerPairWall6N : lmk::kFlopsPerPairWallTT)
                   : (s->angular ? lmk::kFlopsPerPair6N : lmk::kFlopsPerPairTT);
}

// Fields of a solver call: N, precision, blocks, geometry and the pair
// interactions of its products (N^2 per product); extra starts with a comma.
lm_status log_solver_call(const CallScope& c, lm_solver* s, lm_status st, double products, double flops_per_pair,
                          const char* extra = "") {
    if (!lmk::metrics_enabled() || s == nullptr) return st;
    char buf[512];
    std::snprintf(buf, sizeof(buf),
                  "\"N\":%lld,\"precision\":\"%s\",\"angular\":%d,\"geometry\":\"%s\",\"products\":%.0f,"
                  "\"pair_interactions\":%.6e,\"flops_per_pair\":%.0f%s",
                  (long long)s->N, s->fp64 ? "fp64" : "fp32c", s->angular, s->wall ? "single_wall" : "open", products,
                  products * (double)s->N * (double)s->N, flops_per_pair, extra);
    return log_call(c, s->stream, s->device, st, buf);
}
}  // namespace

extern "C" {

const char* lm_last_error(void) { return g_err.c_str(); }

const char* lm_version(void) { return "lm-gb300 0.1 (sm_103a)"; }

int64_t lm_launch_count(lm_solver* solver) {
    (void)solver;
    return g_launches.load(std::memory_order_relaxed);
}

lm_status lm_create(lm_solver** out, const char* px, const char* py, const char* pz, double viscosity,
                    double hydrodynamic_radius, int include_angular, lm_precision precision, void* cuda_stream) {
    lmk::TraceRange trace_("lm_create");
    g_err.clear();
    if (out == nullptr) return fail(LM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_name(px) || !valid_name(py) || !valid_name(pz))
        return fail(LM_ERR_INVALID_ARG, "periodicity must be one of open, periodic, single_wall, two_walls");
    if (strcmp(px, "open") || strcmp(py, "open") || (strcmp(pz, "open") && strcmp(pz, "single_wall")))
        return fail(LM_ERR_UNSUPPORTED_GEOMETRY,
                    "supported geometries: x and y \"open\", z \"open\" or \"single_wall\"");
    if (!(viscosity > 0.0) || !std::isfinite(viscosity)) return fail(LM_ERR_INVALID_ARG, "viscosity must be > 0");
    if (!(hydrodynamic_radius > 0.0) || !std::isfinite(hydrodynamic_radius))
        return fail(LM_ERR_INVALID_ARG, "hydrodynamic radius must be > 0");
    if (precision != LM_FP32C && precision != LM_FP64) return fail(LM_ERR_INVALID_ARG, "unknown precision");
    lm_solver* s = new (std::nothrow) lm_solver();
    if (!s) return fail(LM_ERR_OOM, "host allocation failed");
    s->angular = include_angular ? 1 : 0;
    s->fp64 = precision == LM_FP64 ? 1 : 0;
    s->wall = strcmp(pz, "single_wall") == 0 ? 1 : 0;
    s->eta = viscosity;
    s->a = hydrodynamic_radius;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = s->flag.ensure(64);
    if (e == cudaSuccess) {
        s->pinned_doubles = 64;
        e = cudaMallocHost(reinterpret_cast<void**>(&s->pinned), s->pinned_doubles * sizeof(double));
    }
    if (e != cudaSuccess) {
        lm_status st = cuda_fail(e, "lm_create");
        delete s;
        return st;
    }
    *out = s;
    return LM_OK;
}

lm_status lm_destroy(lm_solver* solver) {
    lmk::TraceRange trace_("lm_destroy");
    if (solver == nullptr) return LM_OK;
    DeviceGuard g(solver->device);
    cudaStreamSynchronize(solver->stream);
    delete solver;
    return LM_OK;
}

lm_status lm_set_stream(lm_solver* solver, void* cuda_stream) {
    if (lm_status st = check_solver(solver, false)) return st;
    solver->stream = static_cast<cudaStream_t>(cuda_stream);
    return LM_OK;
}

lm_status lm_set_positions(lm_solver* s, const void* pos, int64_t N) {
    lmk::TraceRange trace_("lm_set_positions");
    if (lm_status st = check_solver(s, false)) return st;
    if (pos == nullptr) return fail(LM_ERR_INVALID_ARG, "pos is NULL");
    if (N < 1) return fail(LM_ERR_INVALID_ARG, "N must be >= 1 (got %lld)", (long long)N);
    if (N > (int64_t)1 << 31) return fail(LM_ERR_INVALID_ARG, "N too large");
    DeviceGuard g(s->device);
    s->has_pos = false;
    const size_t bytes = (size_t)N * 3 * elem_size(s);
    const void* dpos = nullptr;
    if (lm_status st = stage_in(s, pos, bytes, 0, &dpos)) return st;
    LM_CUDA(s->pos4.ensure((size_t)N * (s->fp64 ? sizeof(lmk::dvec4) : sizeof(float4))), "allocating positions");
    LM_CUDA(cudaMemsetAsync(s->flag.p, 0, sizeof(int), s->stream), "clearing flag");
    if (s->wall)
        LM_CUDA(lmk::launch_pack_wall_positions(dpos, s->fp64, N, s->a, s->z_wall, s->pos4.p, s->fp64,
                                                s->flag.as<int>(), s->stream),
                "packing positions");
    else
        LM_CUDA(lmk::launch_pack_positions(dpos, s->fp64, N, s->pos4.p, s->fp64, s->flag.as<int>(), s->stream),
                "packing positions");
    int bad = 0;
    LM_CUDA(cudaMemcpyAsync(&s->pinned[0], s->flag.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream),
            "reading flag");
    LM_CUDA(cudaStreamSynchronize(s->stream), "set_positions");
    memcpy(&bad, &s->pinned[0], sizeof(int));
    if (bad) return fail(LM_ERR_NONFINITE, "positions contain NaN/Inf or |x| > 1e15");
    // the caller's positions as given (random finite differences, steric forces, time steps)
    LM_CUDA(s->pos_raw.ensure(bytes), "allocating positions");
    LM_CUDA(cudaMemcpyAsync(s->pos_raw.p, dpos, bytes, cudaMemcpyDeviceToDevice, s->stream), "copying positions");
    s->N = N;
    s->has_pos = true;
    return LM_OK;
}

static lm_status mdot_body(lm_solver* s, const void* forces, const void* torques, void* lin_out, void* ang_out) {
    if (lm_status st = check_solver(s, true)) return st;
    if (lin_out == nullptr) return fail(LM_ERR_INVALID_ARG, "lin_out is NULL");
    if (s->angular && ang_out == nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out is required with angular blocks");
    if (!s->angular && ang_out != nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out given but include_angular is 0");
    if (!s->angular && torques != nullptr) return fail(LM_ERR_INVALID_ARG, "torques given but include_angular is 0");
    DeviceGuard g(s->device);
    const size_t bytes = (size_t)s->N * 3 * elem_size(s);
    const void *dF = nullptr, *dT = nullptr;
    if (lm_status st = stage_in(s, forces, bytes, 1, &dF)) return st;
    if (lm_status st = stage_in(s, torques, bytes, 2, &dT)) return st;
    OutView ov[2];
    if (lm_status st = stage_out(s, lin_out, bytes, 0, &ov[0])) return st;
    if (lm_status st = stage_out(s, ang_out, bytes, 1, &ov[1])) return st;
    if (dF == nullptr && dT == nullptr) {
        LM_CUDA(cudaMemsetAsync(ov[0].dev, 0, bytes, s->stream), "zero output");
        if (s->angular) LM_CUDA(cudaMemsetAsync(ov[1].dev, 0, bytes, s->stream), "zero output");
    } else {
        ensure_config(s);
        if (lm_status st = run_mdot(s, dF, dT, s->fp64, ov[0].dev, ov[1].dev, s->fp64, s->cfg)) return st;
    }
    return finish_out(s, ov, 2);
}
lm_status lm_mdot(lm_solver* s, const void* forces, const void* torques, void* lin_out, void* ang_out) {
    CallScope cs("lm_mdot");
    const lm_status st = mdot_body(s, forces, torques, lin_out, ang_out);
    return log_solver_call(cs, s, st, (forces || torques) ? 1.0 : 0.0, s ? solver_flops_per_pair(s) : 0.0);
}

lm_status lm_div_m_rfd(lm_solver* s, uint64_t seed, double delta, void* lin_out, void* ang_out) {
    lmk::TraceRange trace_("lm_div_m_rfd");
    if (lm_status st = check_solver(s, true)) return st;
    if (lin_out == nullptr) return fail(LM_ERR_INVALID_ARG, "lin_out is NULL");
    if (s->angular && ang_out == nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out is required with angular blocks");
    if (!s->angular && ang_out != nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out given but include_angular is 0");
    if (!(delta > 0.0) || !std::isfinite(delta)) return fail(LM_ERR_INVALID_ARG, "delta must be > 0");
    if (!s->wall) return lm_div_m(s, lin_out, ang_out);   // open geometry: exactly zero
    DeviceGuard g(s->device);
    const size_t bytes = (size_t)s->N * 3 * elem_size(s);
    OutView ov[2];
    if (lm_status st = stage_out(s, lin_out, bytes, 0, &ov[0])) return st;
    if (lm_status st = stage_out(s, ang_out, bytes, 1, &ov[1])) return st;
    if (lm_status st = rfd_sample(s, seed, delta, ov[0].dev, ov[1].dev, s->fp64)) return st;
    return finish_out(s, ov, 2);
}

lm_status lm_div_m(lm_solver* s, void* lin_out, void* ang_out) {
    lmk::TraceRange trace_("lm_div_m");
    if (lm_status st = check_solver(s, true)) return st;
    if (lin_out == nullptr) return fail(LM_ERR_INVALID_ARG, "lin_out is NULL");
    if (s->angular && ang_out == nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out is required with angular blocks");
    if (!s->angular && ang_out != nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out given but include_angular is 0");
    if (s->wall) {
        // one random-finite-difference sample per call, seeds 0, 1, 2, ... per solver
        const double delta = (s->fp64 ? kRfdDeltaFP64 : kRfdDeltaFP32) * s->a;
        return lm_div_m_rfd(s, s->rfd_calls++, delta, lin_out, ang_out);
    }
    DeviceGuard g(s->device);
    const size_t bytes = (size_t)s->N * 3 * elem_size(s);
    OutView ov[2];
    if (lm_status st = stage_out(s, lin_out, bytes, 0, &ov[0])) return st;
    if (lm_status st = stage_out(s, ang_out, bytes, 1, &ov[1])) return st;
    LM_CUDA(cudaMemsetAsync(ov[0].dev, 0, bytes, s->stream), "zero output");
    if (s->angular) LM_CUDA(cudaMemsetAsync(ov[1].dev, 0, bytes, s->stream), "zero output");
    return finish_out(s, ov, 2);
}

lm_status lm_soft_repulsion(lm_solver* s, double U0, double b, double d_pair, double d_wall, void* forces_out) {
    lmk::TraceRange trace_("lm_soft_repulsion");
    if (lm_status st = check_solver(s, true)) return st;
    if (forces_out == nullptr) return fail(LM_ERR_INVALID_ARG, "forces_out is NULL");
    if (!std::isfinite(U0) || !(b > 0.0) || !std::isfinite(b) || !std::isfinite(d_pair) || !std::isfinite(d_wall))
        return fail(LM_ERR_INVALID_ARG, "U0, d_pair, d_wall must be finite and b > 0");
    DeviceGuard g(s->device);
    const size_t bytes = (size_t)s->N * 3 * elem_size(s);
    OutView ov[1];
    if (lm_status st = stage_out(s, forces_out, bytes, 0, &ov[0])) return st;
    LM_CUDA(lmk::launch_soft_repulsion(s->pos_raw.p, s->fp64, s->N, U0, b, d_pair, d_wall, s->wall, s->z_wall,
                                       ov[0].dev, s->stream),
            "soft repulsion kernel");
    return finish_out(s, ov, 1);
}

lm_status lm_set_wall_height(lm_solver* s, double height) {
    if (lm_status st = check_solver(s, false)) return st;
    if (!s->wall) return fail(LM_ERR_INVALID_ARG, "the wall height applies to single_wall solvers only");
    if (!std::isfinite(height) || std::fabs(height) > lmk::kMaxAbsCoord)
        return fail(LM_ERR_INVALID_ARG, "wall height must be finite");
    s->z_wall = height;
    if (s->has_pos) {   // re-pack the positions relative to the new wall
        DeviceGuard g(s->device);
        LM_CUDA(cudaMemsetAsync(s->flag.p, 0, sizeof(int), s->stream), "clearing flag");
        LM_CUDA(lmk::launch_pack_wall_positions(s->pos_raw.p, s->fp64, s->N, s->a, s->z_wall, s->pos4.p, s->fp64,
                                                s->flag.as<int>(), s->stream),
                "packing positions");
    }
    return LM_OK;
}

lm_status lm_langevin_velocities(lm_solver* s, const void* forces, const void* torques, const double* W,
                                 uint64_t seed, double kT, double dt, double tol, int max_iter, void* lin_out,
                                 void* ang_out, int* iters_out) {
    lmk::TraceRange trace_("lm_langevin_velocities");
    if (lm_status st = check_solver(s, true)) return st;
    if (lin_out == nullptr) return fail(LM_ERR_INVALID_ARG, "lin_out is NULL");
    if (s->angular && ang_out == nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out is required with angular blocks");
    if (!s->angular && (ang_out != nullptr || torques != nullptr))
        return fail(LM_ERR_INVALID_ARG, "torques or ang_out given but include_angular is 0");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return fail(LM_ERR_INVALID_ARG, "kT must be finite and >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(LM_ERR_INVALID_ARG, "dt must be > 0");
    DeviceGuard g(s->device);
    if (iters_out) *iters_out = 0;
    const int64_t N = s->N;
    const size_t n3 = (size_t)3 * N;
    const size_t bytes = n3 * elem_size(s);
    const void *dF = nullptr, *dT = nullptr;
    if (lm_status st = stage_in(s, forces, bytes, 1, &dF)) return st;
    if (lm_status st = stage_in(s, torques, bytes, 2, &dT)) return st;
    OutView ov[2];
    if (lm_status st = stage_out(s, lin_out, bytes, 0, &ov[0])) return st;
    if (lm_status st = stage_out(s, ang_out, bytes, 1, &ov[1])) return st;
    LM_CUDA(s->ab_u.ensure(2 * n3 * sizeof(double)), "allocating scratch");
    LM_CUDA(s->ab_d.ensure(2 * n3 * sizeof(double)), "allocating scratch");
    LM_CUDA(s->ab_y.ensure(2 * n3 * sizeof(double)), "allocating scratch");
    double* u = s->ab_u.as<double>();
    double* d = s->ab_d.as<double>();
    if (dF == nullptr && dT == nullptr) {
        LM_CUDA(cudaMemsetAsync(u, 0, 2 * n3 * sizeof(double), s->stream), "zero velocities");
    } else {
        ensure_config(s);
        if (lm_status st = run_mdot(s, dF, dT, s->fp64, u, s->angular ? u + n3 : nullptr, 1, s->cfg)) return st;
    }
    const bool drift = s->wall && kT > 0.0;
    if (drift) {
        const double delta = (s->fp64 ? kRfdDeltaFP64 : kRfdDeltaFP32) * s->a;
        if (lm_status st = rfd_sample(s, seed, delta, d, s->angular ? d + n3 : nullptr, 1)) return st;
    }
    void* y = s->ab_y.p;
    if (kT > 0.0) {
        int its = 0;
        lm_status st = lm_sqrt_mdot(s, W, seed, std::sqrt(2.0 * kT / dt), tol, max_iter, y,
                                    s->angular ? static_cast<char*>(y) + bytes : nullptr, &its);
        if (iters_out) *iters_out = its;
        if (st != LM_OK) return st;
    } else {
        LM_CUDA(cudaMemsetAsync(y, 0, 2 * bytes, s->stream), "zero noise");
    }
    LM_CUDA(lmk::launch_langevin_combine(u, drift ? d : nullptr, y, kT, N, s->angular, ov[0].dev, ov[1].dev, s->fp64,
                                         s->stream),
            "Langevin velocities");
    return finish_out(s, ov, 2);
}

lm_status lm_ab_step(lm_solver* s, const void* forces, const void* torques, const double* W, uint64_t seed,
                     double kT, double dt, double tol, int max_iter, double* history, int first, void* pos_out,
                     int* iters_out) {
    lmk::TraceRange trace_("lm_ab_step");
    if (lm_status st = check_solver(s, true)) return st;
    if (pos_out == nullptr) return fail(LM_ERR_INVALID_ARG, "pos_out is NULL");
    if (history == nullptr || !is_device_ptr(history))
        return fail(LM_ERR_INVALID_ARG, "history must be a device array of 6N doubles");
    if (!s->angular && torques != nullptr) return fail(LM_ERR_INVALID_ARG, "torques given but include_angular is 0");
    if (!(kT >= 0.0) || !std::isfinite(kT)) return fail(LM_ERR_INVALID_ARG, "kT must be finite and >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(LM_ERR_INVALID_ARG, "dt must be > 0");
    DeviceGuard g(s->device);
    if (iters_out) *iters_out = 0;
    const int64_t N = s->N;
    const size_t n3 = (size_t)3 * N;
    const size_t bytes = n3 * elem_size(s);
    const void *dF = nullptr, *dT = nullptr;
    if (lm_status st = stage_in(s, forces, bytes, 1, &dF)) return st;
    if (lm_status st = stage_in(s, torques, bytes, 2, &dT)) return st;
    LM_CUDA(s->ab_u.ensure(2 * n3 * sizeof(double)), "allocating step scratch");
    LM_CUDA(s->ab_d.ensure(2 * n3 * sizeof(double)), "allocating step scratch");
    LM_CUDA(s->ab_y.ensure(2 * n3 * sizeof(double)), "allocating step scratch");
    LM_CUDA(s->ab_x.ensure(bytes), "allocating step scratch");
    double* u = s->ab_u.as<double>();
    double* d = s->ab_d.as<double>();
    // u = (M [F; T])_lin (FP64)
    if (dF == nullptr && dT == nullptr) {
        LM_CUDA(cudaMemsetAsync(u, 0, 2 * n3 * sizeof(double), s->stream), "zero velocities");
    } else {
        ensure_config(s);
        if (lm_status st = run_mdot(s, dF, dT, s->fp64, u, s->angular ? u + n3 : nullptr, 1, s->cfg)) return st;
    }
    // d = one RFD sample of div M (single wall, kT > 0; zero otherwise)
    const bool drift = s->wall && kT > 0.0;
    if (drift) {
        const double delta = (s->fp64 ? kRfdDeltaFP64 : kRfdDeltaFP32) * s->a;
        if (lm_status st = rfd_sample(s, seed, delta, d, s->angular ? d + n3 : nullptr, 1)) return st;
    }
    // y = sqrt(2 kT dt) (M^{1/2} W)_lin in the solver precision
    void* y = s->ab_y.p;
    if (kT > 0.0) {
        int its = 0;
        lm_status st = lm_sqrt_mdot(s, W, seed, std::sqrt(2.0 * kT * dt), tol, max_iter, y,
                                    s->angular ? static_cast<char*>(y) + bytes : nullptr, &its);
        if (iters_out) *iters_out = its;
        if (st != LM_OK) return st;
    } else {
        LM_CUDA(cudaMemsetAsync(y, 0, bytes, s->stream), "zero noise");
    }
    LM_CUDA(lmk::launch_ab_update(s->pos_raw.p, s->fp64, u, drift ? d : nullptr, y, history, first ? 1 : 0, kT, dt,
                                  N, s->ab_x.p, s->stream),
            "Adams-Bashforth update");
    if (lm_status st = lm_set_positions(s, s->ab_x.p, N)) return st;
    if (is_device_ptr(pos_out)) {
        LM_CUDA(cudaMemcpyAsync(pos_out, s->ab_x.p, bytes, cudaMemcpyDeviceToDevice, s->stream), "copying positions");
    } else {
        LM_CUDA(cudaMemcpyAsync(pos_out, s->ab_x.p, bytes, cudaMemcpyDeviceToHost, s->stream), "copying positions");
        LM_CUDA(cudaStreamSynchronize(s->stream), "copying positions");
    }
    return LM_OK;
}

// ---------------------------------------------------------------------------
// Lanczos square root (Sec. 3.3).  Per iteration k (v_k = row k of V):
//   w = M v_k;  alpha_k = v_k . w;  w -= alpha_k v_k + beta_{k-1} v_{k-1};
//   h0 = |w|; w -= V_k (V_k^T w); h1 = |w|; if h1 < h0 / sqrt(2): again (DGKS);
//   beta_k = |w|;
//   z_k = |W| f(T_k) e1 (host);  stop if k >= 1 and
//   |z_k - [z_{k-1}; 0]| / |z_k| < tol, or on breakdown, or at max_iter;
//   v_{k+1} = w / beta_k.
// Result: y = V_m z_m, scaled by the prefactor.
// The GPU runs one iteration ahead of the host: iteration k+1 is enqueued
// (it needs only device data) before the host reads alpha_k, beta_k and
// decides whether to stop at k, so the read-back and the tridiagonal step
// overlap the next product.  The speculative iteration is skipped when the
// geometric trend of the relative changes predicts a stop at k.
// ---------------------------------------------------------------------------
namespace {

// Device scalars per iteration k at scal + kScal * k:
//   [alpha, beta, beta^2, -, h0, h0^2, h1, h1^2]
constexpr int kScal = 8;

lm_status enqueue_lanczos_iteration(lm_solver* s, int k, int64_t n, double* V, double* w, double* scal, double* red,
                                    double* cb, cudaEvent_t ev) {
    const int64_t N = s->N;
    double* vk = V + (int64_t)k * n;
    double* sk = scal + kScal * k;
    if (k > 0) LM_CUDA(lmk::lz_scale(w, sk - kScal + 1, vk, n, s->stream), "next basis vector");
    if (s->precond) {
        // w = P M P v_k, P = diag(M)^{-1/2}
        double* t = s->pc_t.as<double>();
        const double* p = s->pc_p.as<double>();
        LM_CUDA(lmk::launch_vmul(p, vk, t, n, s->stream), "preconditioner");
        if (lm_status st = run_mdot(s, t, t + 3 * N, 1, w, w + 3 * N, 1, s->cfg)) return st;
        LM_CUDA(lmk::launch_vmul(p, w, w, n, s->stream), "preconditioner");
    } else {
        if (lm_status st = run_mdot(s, vk, vk + 3 * N, 1, w, w + 3 * N, 1, s->cfg)) return st;
    }
    unsigned* ctr = s->lzctr.as<unsigned>();
    cudaEvent_t vend = nullptr;
    if (s->prof_on) {
        while (s->vprof_ev.size() < 2 * (s->vprof_used + 1)) {
            cudaEvent_t e;
            LM_CUDA(cudaEventCreate(&e), "profiling event");
            s->vprof_ev.push_back(e);
        }
        s->vprof_bytes.resize(s->vprof_used + 1);
        s->vprof_bytes[s->vprof_used] = -1.0;
        s->vprof_pending.emplace_back(s->vprof_used, k);
        LM_CUDA(cudaEventRecord(s->vprof_ev[2 * s->vprof_used], s->stream), "profiling event");
        vend = s->vprof_ev[2 * s->vprof_used + 1];
        s->vprof_used += 1;
    }
    LM_CUDA(lmk::lz_dot1(vk, w, n, red, ctr, sk, 0, s->stream), "alpha");
    // three-term update and |w| before the Gram-Schmidt pass
    LM_CUDA(lmk::lz_axpy2_norm(w, vk, sk, k > 0 ? vk - n : nullptr, k > 0 ? sk - kScal + 1 : nullptr, n, red, ctr,
                               sk + 4, s->stream),
            "three-term update");
    // full reorthogonalisation: one Gram-Schmidt pass (|w| after it), a second
    // one only after cancellation (DGKS); beta = |w| at the end
    LM_CUDA(lmk::lz_multidot1(V, k + 1, w, n, red, ctr, cb, s->stream), "reorthogonalisation");
    LM_CUDA(lmk::lz_sub_vc_norm(V, k + 1, cb, w, n, red, ctr, sk + 6, s->stream), "reorthogonalisation");
    const double* cond = s->reorth ? nullptr : sk + 4;   // nullptr: the second pass always runs
    LM_CUDA(lmk::lz_multidot1(V, k + 1, w, n, red, ctr, cb, s->stream, cond), "reorthogonalisation");
    LM_CUDA(lmk::lz_sub_vc_norm(V, k + 1, cb, w, n, red, ctr, sk + 1, s->stream, cond), "beta");
    if (vend) LM_CUDA(cudaEventRecord(vend, s->stream), "profiling event");
    LM_CUDA(cudaMemcpyAsync(s->pinned + kScal * k, sk, kScal * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
            "read alpha, beta");
    LM_CUDA(cudaEventRecord(ev, s->stream), "iteration event");
    return LM_OK;
}

// Algorithmic bytes of the vector kernels of iteration k (those inside the
// profiling events), in units of one FP64 vector of length n: alpha reads v_k
// and w (2); the three-term update reads w, v_k, v_{k-1} and writes w (4, or
// 3 at k = 0); a Gram-Schmidt pass reads the k + 1 basis vectors and w for
// the dots (k + 2), then the basis, w and writes w (k + 3).
double lanczos_vector_bytes(int k, int64_t n, bool second_pass) {
    const double pass = (double)(k + 2) + (double)(k + 3);
    const double units = 2.0 + (k > 0 ? 4.0 : 3.0) + pass * (second_pass ? 2.0 : 1.0);
    return units * 8.0 * (double)n;
}

// Counts the bytes of the profiled iterations of the finished lm_sqrt_mdot
// call (its scalars are on the host after the final synchronisation).
void settle_vector_profile(lm_solver* s, int64_t n) {
    for (const auto& pk : s->vprof_pending) {
        const double* sc = s->pinned + kScal * pk.second;
        const bool second = s->reorth != 0 || sc[6] < sc[4] * 0.70710678118654752440;   // the kernels' DGKS test
        if (pk.first < s->vprof_bytes.size()) s->vprof_bytes[pk.first] = lanczos_vector_bytes(pk.second, n, second);
    }
    s->vprof_pending.clear();
}

}  // namespace

static lm_status sqrt_mdot_body(lm_solver* s, const double* W, uint64_t seed, double prefactor, double tol, int max_iter,
                       void* lin_out, void* ang_out, int* iters_out) {
    if (lm_status st = check_solver(s, true)) return st;
    if (lin_out == nullptr) return fail(LM_ERR_INVALID_ARG, "lin_out is NULL");
    if (s->angular && ang_out == nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out is required with angular blocks");
    if (!s->angular && ang_out != nullptr) return fail(LM_ERR_INVALID_ARG, "ang_out given but include_angular is 0");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(LM_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (max_iter < 1) return fail(LM_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (!std::isfinite(prefactor)) return fail(LM_ERR_INVALID_ARG, "prefactor must be finite");
    DeviceGuard g(s->device);
    if (iters_out) *iters_out = 0;
    s->stats = lm_lanczos_stats{0, 0, 0.0, 0.0, 0};
    s->vprof_pending.clear();

    const int64_t N = s->N;
    const int64_t n = (s->angular ? 6 : 3) * N;
    const int m_max = (int)std::min<int64_t>(max_iter, n);
    const size_t out_bytes = (size_t)N * 3 * elem_size(s);
    OutView ov[2];
    if (lm_status st = stage_out(s, lin_out, out_bytes, 0, &ov[0])) return st;
    if (lm_status st = stage_out(s, ang_out, out_bytes, 1, &ov[1])) return st;

    ensure_config(s);
    // one spare basis row for the speculative iteration
    LM_CUDA(s->V.ensure((size_t)(m_max + 1) * n * sizeof(double)), "allocating Krylov basis");
    LM_CUDA(s->w.ensure((size_t)n * sizeof(double)), "allocating Lanczos vector");
    LM_CUDA(s->y.ensure((size_t)n * sizeof(double)), "allocating Lanczos vector");
    LM_CUDA(s->red.ensure(lmk::lz_red_doubles(n, m_max + 1) * sizeof(double)), "allocating reduction scratch");
    LM_CUDA(s->scal.ensure((size_t)(kScal * (m_max + 3)) * sizeof(double)), "allocating scalars");
    LM_CUDA(s->zbuf.ensure((size_t)m_max * sizeof(double)), "allocating coefficients");
    LM_CUDA(s->cbuf.ensure((size_t)(m_max + 1) * sizeof(double)), "allocating coefficients");
    const size_t ctr_bytes = std::max<size_t>(64, lmk::lz_ctr_count(m_max + 1) * sizeof(unsigned));
    if (s->lzctr.p == nullptr || s->lzctr.cap < ctr_bytes) {
        // the counters must start at zero; the kernels reset them after use
        LM_CUDA(s->lzctr.ensure(ctr_bytes), "allocating counters");
        LM_CUDA(cudaMemsetAsync(s->lzctr.p, 0, s->lzctr.cap, s->stream), "allocating counters");
    }
    if (s->pinned_doubles < (size_t)(kScal * (m_max + 3))) {
        cudaFreeHost(s->pinned);
        s->pinned = nullptr;
        s->pinned_doubles = 0;
        LM_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s->pinned), (size_t)(kScal * (m_max + 3)) * sizeof(double)),
                "allocating pinned scalars");
        s->pinned_doubles = (size_t)(kScal * (m_max + 3));
    }
    while (s->lz_ev.size() < (size_t)(m_max + 1)) {
        cudaEvent_t e;
        LM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "lanczos event");
        s->lz_ev.push_back(e);
    }
    double* V = s->V.as<double>();
    double* w = s->w.as<double>();
    double* scal = s->scal.as<double>();
    double* red = s->red.as<double>();
    double* cb = s->cbuf.as<double>();
    double* wn = scal + kScal * (m_max + 2);  // |W|, |W|^2
    if (s->precond) {
        LM_CUDA(s->pc_p.ensure((size_t)n * sizeof(double)), "allocating preconditioner");
        LM_CUDA(s->pc_q.ensure((size_t)n * sizeof(double)), "allocating preconditioner");
        LM_CUDA(s->pc_t.ensure((size_t)n * sizeof(double)), "allocating preconditioner");
        LM_CUDA(lmk::launch_mobility_diag(s->pos4.p, s->fp64, N, s->a, s->eta, s->angular, s->wall,
                                          s->pc_p.as<double>(), s->pc_q.as<double>(), s->stream),
                "preconditioner");
    }

    // W: user array (host or device) or Philox normals
    const double* dW = nullptr;
    if (W == nullptr) {
        LM_CUDA(s->Wbuf.ensure((size_t)n * sizeof(double)), "allocating noise");
        LM_CUDA(lmk::lz_philox_normals(seed, 0, s->Wbuf.as<double>(), n, s->stream), "noise generator");
        dW = s->Wbuf.as<double>();
    } else {
        const void* p = nullptr;
        if (lm_status st = stage_in(s, W, (size_t)n * sizeof(double), 3, &p)) return st;
        dW = static_cast<const double*>(p);
    }
    LM_CUDA(lmk::lz_norm(dW, n, red, wn, s->stream), "norm of W");
    LM_CUDA(lmk::lz_scale(dW, wn, V, n, s->stream), "normalise W");
    LM_CUDA(cudaMemcpyAsync(s->pinned + kScal * (m_max + 2), wn, sizeof(double), cudaMemcpyDeviceToHost, s->stream),
            "read |W|");
    if (lm_status st = enqueue_lanczos_iteration(s, 0, n, V, w, scal, red, cb, s->lz_ev[0])) return st;
    LM_CUDA(cudaEventSynchronize(s->lz_ev[0]), "lanczos");
    const double normW = s->pinned[kScal * (m_max + 2)];
    s->stats.norm_w = normW;
    if (!std::isfinite(normW)) return fail(LM_ERR_INVALID_ARG, "W contains NaN or Inf");
    if (normW == 0.0) {
        LM_CUDA(cudaMemsetAsync(ov[0].dev, 0, out_bytes, s->stream), "zero output");
        if (s->angular) LM_CUDA(cudaMemsetAsync(ov[1].dev, 0, out_bytes, s->stream), "zero output");
        s->stats.converged = 1;
        return finish_out(s, ov, 2);
    }

    LanczosHost& H = s->lz_host;
    H.alpha.clear();
    H.beta.clear();
    H.zprev.clear();
    const double brk_rel = s->fp64 ? 1e-13 : 1e-7;
    bool converged = false;
    double rel = 0.0, rel_prev = 0.0;
    int clamped = 0;
    int k = 0;
    for (k = 0; k < m_max; ++k) {
        // speculative enqueue of iteration k+1 unless a stop at k is predicted
        bool predicted_stop = false;
        if (k >= 2 && rel_prev > 0.0 && rel > 0.0) predicted_stop = (rel * rel / rel_prev) < 2.0 * tol;
        if (k + 1 < m_max && !predicted_stop && k > 0) {
            if (lm_status st = enqueue_lanczos_iteration(s, k + 1, n, V, w, scal, red, cb, s->lz_ev[k + 1])) return st;
        }
        LM_CUDA(cudaEventSynchronize(s->lz_ev[k]), "lanczos iteration");
        const double a_k = s->pinned[kScal * k];
        const double b_k = s->pinned[kScal * k + 1];
        if (!std::isfinite(a_k) || !std::isfinite(b_k))
            return fail(LM_ERR_CUDA, "Lanczos produced a non-finite coefficient at iteration %d", k + 1);
        H.alpha.push_back(a_k);
        const int m = k + 1;
        int ncl = 0;
        if (H.solve(m, normW, &ncl) != 0) return fail(LM_ERR_NOT_CONVERGED, "tridiagonal eigensolver did not converge");
        clamped = ncl;
        bool stop = false;
        if (k >= 1) {
            double dn = 0.0, zn = 0.0;
            for (int i = 0; i < m; ++i) {
                const double dd = H.z[i] - (i < m - 1 ? H.zprev[i] : 0.0);
                dn += dd * dd;
                zn += H.z[i] * H.z[i];
            }
            rel_prev = rel;
            rel = (zn > 0.0) ? std::sqrt(dn / zn) : 0.0;
            if (rel < tol) { converged = true; stop = true; }
        }
        if (!stop) {
            double amax = 0.0;
            for (double v : H.alpha) amax = std::max(amax, std::fabs(v));
            if (b_k <= brk_rel * amax) { converged = true; stop = true; }
        }
        if (!stop && k + 1 == m_max) stop = true;
        if (stop) break;
        H.beta.push_back(b_k);
        H.zprev = H.z;
        // iteration k+1 not enqueued yet (first iteration, or a predicted stop that did not happen)
        if (k == 0 || predicted_stop) {
            if (lm_status st = enqueue_lanczos_iteration(s, k + 1, n, V, w, scal, red, cb, s->lz_ev[k + 1])) return st;
        }
    }
    const int m = std::min(k + 1, m_max);
    LM_CUDA(cudaMemcpyAsync(s->zbuf.p, H.z.data(), (size_t)m * sizeof(double), cudaMemcpyHostToDevice, s->stream),
            "coefficients to device");
    LM_CUDA(lmk::lz_combine(V, m, s->zbuf.as<double>(), s->y.as<double>(), n, s->stream), "combine basis");
    if (s->precond)   // y = P^{-1} (P M P)^{1/2} W
        LM_CUDA(lmk::launch_vmul(s->pc_q.as<double>(), s->y.as<double>(), s->y.as<double>(), n, s->stream),
                "preconditioner");
    LM_CUDA(lmk::lz_store(s->y.as<double>(), prefactor, N, s->angular, ov[0].dev, ov[1].dev, s->fp64, s->stream),
            "store result");
    // z lives in host memory read by the copy above: wait before it changes
    LM_CUDA(cudaStreamSynchronize(s->stream), "lanczos result");
    settle_vector_profile(s, n);
    s->stats.iterations = m;
    s->stats.converged = converged ? 1 : 0;
    s->stats.rel_change = rel;
    s->stats.clamped_eigs = clamped;
    if (iters_out) *iters_out = m;
    if (lm_status st = finish_out(s, ov, 2)) return st;
    if (!converged)
        return fail(LM_ERR_NOT_CONVERGED, "Lanczos did not reach tol %.3g in %d iterations (last change %.3g)", tol,
                    m, rel);
    return LM_OK;
}
lm_status lm_sqrt_mdot(lm_solver* s, const double* W, uint64_t seed, double prefactor, double tol, int max_iter,
                       void* lin_out, void* ang_out, int* iters_out) {
    CallScope cs("lm_sqrt_mdot");
    int it = 0;
    const lm_status st = sqrt_mdot_body(s, W, seed, prefactor, tol, max_iter, lin_out, ang_out, &it);
    if (iters_out) *iters_out = it;
    if (!lmk::metrics_enabled() || s == nullptr) return st;
    char extra[160];
    std::snprintf(extra, sizeof(extra), ",\"iterations\":%d,\"tol\":%.3e,\"rel_change\":%.6e,\"converged\":%d", it,
                  tol, s->stats.rel_change, s->stats.converged);
    return log_solver_call(cs, s, st, (double)it, solver_flops_per_pair(s), extra);
}

lm_status lm_get_lanczos_stats(lm_solver* s, lm_lanczos_stats* stats) {
    if (lm_status st = check_solver(s, false)) return st;
    if (stats == nullptr) return fail(LM_ERR_INVALID_ARG, "stats is NULL");
    *stats = s->stats;
    return LM_OK;
}

static lm_status mdot_backward_body(lm_solver* s, const void* forces, const void* torques, const void* grad_lin,
                           const void* grad_ang, void* dX, void* dF, void* dT) {
    if (lm_status st = check_solver(s, true)) return st;
    if (s->wall)
        return fail(LM_ERR_UNSUPPORTED_GEOMETRY, "the adjoint is implemented for the open geometry only");
    if (forces == nullptr || grad_lin == nullptr) return fail(LM_ERR_INVALID_ARG, "forces and grad_lin are required");
    if (!s->angular && (torques != nullptr || grad_ang != nullptr || dT != nullptr))
        return fail(LM_ERR_INVALID_ARG, "torque arguments given but include_angular is 0");
    DeviceGuard g(s->device);
    const size_t bytes = (size_t)s->N * 3 * elem_size(s);
    const void *pF = nullptr, *pT = nullptr, *pG = nullptr, *pH = nullptr;
    if (lm_status st = stage_in(s, forces, bytes, 0, &pF)) return st;
    if (lm_status st = stage_in(s, torques, bytes, 1, &pT)) return st;
    if (lm_status st = stage_in(s, grad_lin, bytes, 2, &pG)) return st;
    if (lm_status st = stage_in(s, grad_ang, bytes, 3, &pH)) return st;
    OutView ov[3];
    if (lm_status st = stage_out(s, dX, bytes, 0, &ov[0])) return st;
    if (lm_status st = stage_out(s, dF, bytes, 1, &ov[1])) return st;
    if (lm_status st = stage_out(s, dT, bytes, 2, &ov[2])) return st;
    if (dX == nullptr && dF == nullptr && dT == nullptr) return LM_OK;
    ensure_adjoint_config(s);
    if (lm_status st = run_adjoint(s, pF, pT, pG, pH, ov[0].dev, ov[1].dev, ov[2].dev, s->adj_cfg)) return st;
    return finish_out(s, ov, 3);
}

lm_status lm_mdot_backward(lm_solver* s, const void* forces, const void* torques, const void* grad_lin,
                           const void* grad_ang, void* dX, void* dF, void* dT) {
    CallScope cs("lm_mdot_backward");
    const lm_status st = mdot_backward_body(s, forces, torques, grad_lin, grad_ang, dX, dF, dT);
    return log_solver_call(cs, s, st, 1.0, 0.0, ",\"note\":\"fused dL/dX and dL/dF pass\"");
}

lm_status lm_set_sqrt_preconditioner(lm_solver* s, int kind) {
    if (lm_status st = check_solver(s, false)) return st;
    if (kind != 0 && kind != 1) return fail(LM_ERR_INVALID_ARG, "preconditioner kind must be 0 (none) or 1 (Jacobi)");
    s->precond = kind;
    return LM_OK;
}

lm_status lm_set_reorthogonalization(lm_solver* s, int mode) {
    if (lm_status st = check_solver(s, false)) return st;
    if (mode != 0 && mode != 1) return fail(LM_ERR_INVALID_ARG, "reorthogonalization mode must be 0 (DGKS) or 1 (two passes)");
    s->reorth = mode;
    return LM_OK;
}

lm_status lm_get_adjoint_config(lm_solver* s, lm_pair_config* cfg) {
    if (lm_status st = check_solver(s, true)) return st;
    if (cfg == nullptr) return fail(LM_ERR_INVALID_ARG, "cfg is NULL");
    ensure_adjoint_config(s);
    *cfg = s->adj_cfg;
    return LM_OK;
}

lm_status lm_set_adjoint_config(lm_solver* s, const lm_pair_config* cfg) {
    if (lm_status st = check_solver(s, true)) return st;
    if (cfg == nullptr) return fail(LM_ERR_INVALID_ARG, "cfg is NULL");
    if (!lmk::adjoint_config_supported(s->fp64, s->angular, cfg->threads, cfg->ilp, cfg->packed) || cfg->splits < 0 ||
        (!s->fp64 && !s->angular && cfg->packed < 1))
        return fail(LM_ERR_INVALID_ARG, "unsupported adjoint configuration (threads %d, ilp %d, splits %d, packed %d)",
                    cfg->threads, cfg->ilp, cfg->splits, cfg->packed);
    lm_pair_config c = *cfg;
    if (c.splits == 0 && c.packed < 3) {   // the symmetric forms choose their item size at launch
        const int occ = std::max(1, lmk::adjoint_ctas_per_sm(s->fp64, s->angular, c.threads, c.ilp, c.packed));
        c.splits = auto_splits(s->N, c.threads, c.ilp, occ * s->sm_count);
    }
    s->adj_cfg = c;
    s->adj_cfg_N = s->N;
    return LM_OK;
}

lm_status lm_get_pair_config(lm_solver* s, lm_pair_config* cfg) {
    if (lm_status st = check_solver(s, true)) return st;
    if (cfg == nullptr) return fail(LM_ERR_INVALID_ARG, "cfg is NULL");
    ensure_config(s);
    *cfg = s->cfg;
    return LM_OK;
}

lm_status lm_set_pair_config(lm_solver* s, const lm_pair_config* cfg) {
    if (lm_status st = check_solver(s, false)) return st;
    if (cfg == nullptr) return fail(LM_ERR_INVALID_ARG, "cfg is NULL");
    if (!pair_config_supported(s, cfg->threads, cfg->ilp, cfg->packed) || cfg->splits < 0)
        return fail(LM_ERR_INVALID_ARG, "unsupported pair configuration (threads %d, ilp %d, splits %d, packed %d)",
                    cfg->threads, cfg->ilp, cfg->splits, cfg->packed);
    s->cfg = *cfg;
    if (s->cfg.splits == 0) {
        int occ = std::max(1, pair_ctas_per_sm(s, cfg->threads, cfg->ilp, cfg->packed));
        s->cfg.splits = s->has_pos ? auto_splits(s->N, cfg->threads, cfg->ilp, occ * s->sm_count) : 1;
    }
    s->cfg_forced = true;
    s->cfg_N = s->has_pos ? s->N : -1;
    return LM_OK;
}

}  // extern "C"

namespace {
lm_status autotune_impl(lm_solver* s, int reps, lm_pair_config* best) {
    if (lm_status st = check_solver(s, true)) return st;
    if (reps < 1) return fail(LM_ERR_INVALID_ARG, "reps must be >= 1");
    DeviceGuard g(s->device);
    const int64_t N = s->N;
    const size_t bytes = (size_t)N * 3 * elem_size(s);
    LM_CUDA(s->tune_in.ensure(2 * bytes), "autotune buffers");
    LM_CUDA(s->tune_out.ensure(2 * bytes), "autotune buffers");
    LM_CUDA(cudaMemsetAsync(s->tune_in.p, 0, 2 * bytes, s->stream), "autotune buffers");
    char* fin = s->tune_in.as<char>();
    char* fout = s->tune_out.as<char>();
    std::vector<lm_pair_config> cands;
    const int threads_opts[2] = {128, 256};
    const int ilp_opts[4] = {1, 2, 4, 8};
    // Large products (an FP32 launch of more than about 20 ms at the measured
    // 50 TFLOP/s): the sweep keeps the packed FP32 forms with i-blocks of at
    // least 512 particles and the split counts of whole waves, and times each
    // candidate without its own warm-up launch.  The scalar form and small
    // i-blocks lost at every size above 2^17 where they were timed, and a full
    // sweep would take minutes there.
    const double flops_pp = s->wall ? (s->angular ? lmk::kFlopsPerPairWall6N : lmk::kFlopsPerPairWallTT)
                                    : (s->angular ? lmk::kFlopsPerPair6N : lmk::kFlopsPerPairTT);
    const bool large = !s->fp64 && (double)N * (double)N * flops_pp > 20e-3 * 50e12;
    for (int pk : {0, 1, 2, 4}) {
        if (large && pk == 0) continue;
        for (int t : threads_opts) {
            for (int il : ilp_opts) {
                if (large && t * il < 512) continue;
                if (!pair_config_supported(s, t, il, pk)) continue;
                const int occ = pair_ctas_per_sm(s, t, il, pk);
                if (occ < 1) continue;
                for (int sp : split_candidates(N, t, il, occ * s->sm_count, large))
                    cands.push_back(lm_pair_config{t, il, sp, pk});
            }
        }
    }
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0), "autotune events");
    LM_CUDA(cudaEventCreate(&e1), "autotune events");
    // Times `reps` launches of one candidate (after one warm-up launch).
    bool warm = false;
    auto time_one = [&](auto&& launch, const lm_pair_config& c, float* ms) -> lm_status {
        if (!large || !warm) {
            if (lm_status st = launch(c)) return st;
            warm = true;
        }
        cudaEventRecord(e0, s->stream);
        for (int r = 0; r < reps; ++r)
            if (lm_status st = launch(c)) return st;
        cudaEventRecord(e1, s->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return cuda_fail(e, "autotune");
        cudaEventElapsedTime(ms, e0, e1);
        return LM_OK;
    };
    // One timing of every candidate, then the three fastest again in three
    // interleaved rounds (the minimum of the four timings decides), so that
    // clock and scheduling noise of a single timing does not pick the winner.
    auto pick = [&](auto&& launch, const std::vector<lm_pair_config>& cs, lm_pair_config* out) -> lm_status {
        std::vector<std::pair<float, size_t>> t;
        for (size_t i = 0; i < cs.size(); ++i) {
            float ms = 0.f;
            if (lm_status st = time_one(launch, cs[i], &ms)) return st;
            t.emplace_back(ms, i);
        }
        if (t.empty()) return LM_OK;
        std::sort(t.begin(), t.end());
        const size_t top = std::min<size_t>(3, t.size());
        for (int round = 0; round < 3; ++round) {
            for (size_t q = 0; q < top; ++q) {
                float ms = 0.f;
                if (lm_status st = time_one(launch, cs[t[q].second], &ms)) return st;
                t[q].first = std::min(t[q].first, ms);
            }
        }
        size_t best_q = 0;
        for (size_t q = 1; q < top; ++q)
            if (t[q].first < t[best_q].first) best_q = q;
        *out = cs[t[best_q].second];
        return LM_OK;
    };
    lm_pair_config best_cfg = default_config(s, N);
    lm_status result = pick(
        [&](const lm_pair_config& c) { return run_mdot(s, fin, fin + bytes, s->fp64, fout, fout + bytes, s->fp64, c); },
        cands, &best_cfg);
    // the packed translation adjoint (open geometry): threads x ilp x j per vote x splits
    if (result == LM_OK && !s->fp64 && !s->angular && !s->wall) {
        std::vector<lm_pair_config> acands;
        for (int uj = 1; uj <= 3; ++uj) {
            for (int t : threads_opts) {
                for (int il = 2; il <= 4; il += 2) {
                    const int occ = lmk::adjoint_ctas_per_sm(0, 0, t, il, uj);
                    if (occ < 1) continue;
                    if (uj == 3) {
                        // symmetric form: the item size (tiles) of the model, half and twice it
                        const int64_t ch = sym_auto_chunk(s, t, il, 3);
                        for (int64_t c : {ch, std::max<int64_t>(1, ch / 2), 2 * ch})
                            acands.push_back(lm_pair_config{t, il, (int)std::min<int64_t>(c, 1 << 20), 3});
                        continue;
                    }
                    for (int sp : split_candidates(N, t, il, occ * s->sm_count))
                        acands.push_back(lm_pair_config{t, il, sp, uj});
                }
            }
        }
        // inputs F = G = 0 (the timing does not depend on the values); outputs dX, dF
        lm_pair_config best_a = default_adjoint_config(s);
        result = pick(
            [&](const lm_pair_config& c) {
                return run_adjoint(s, fin, nullptr, fin, nullptr, fout, fout + bytes, nullptr, c);
            },
            acands, &best_a);
        if (result == LM_OK) {
            s->adj_cfg = best_a;
            s->adj_cfg_N = N;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != LM_OK) return result;
    s->cfg = best_cfg;
    s->cfg_forced = true;
    s->cfg_N = N;
    {
        TunedEntry e;
        e.cfg = best_cfg;
        e.N = N;
        e.has_adj = (s->adj_cfg_N == N) && !s->fp64 && !s->angular && !s->wall;
        if (e.has_adj) e.adj = s->adj_cfg;
        const std::array<int, 5> key = tuned_key(s, N);
        {
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            g_tuned[key] = e;
        }
        lmk::TuneCacheKey ck;
        if (lmk::tune_cache_key(s->device, key[1], key[2], key[3], key[4], &ck))
            lmk::tune_cache_store(ck, N, best_cfg, e.has_adj ? &e.adj : nullptr);
    }
    if (best) *best = best_cfg;
    return LM_OK;
}
}  // namespace

extern "C" {

lm_status lm_autotune(lm_solver* s, int reps, lm_pair_config* best) {
    lmk::TraceRange tr("lm_autotune");
    return autotune_impl(s, reps, best);
}

lm_status lm_profile_enable(lm_solver* s, int enable) {
    if (lm_status st = check_solver(s, false)) return st;
    s->prof_on = enable != 0;
    return LM_OK;
}

lm_status lm_profile_read(lm_solver* s, lm_profile* out, int reset) {
    if (lm_status st = check_solver(s, false)) return st;
    if (out == nullptr) return fail(LM_ERR_INVALID_ARG, "out is NULL");
    DeviceGuard g(s->device);
    LM_CUDA(cudaStreamSynchronize(s->stream), "profile read");
    double ms = 0.0;
    for (size_t k = 0; k < s->prof_used; ++k) {
        float t = 0.f;
        LM_CUDA(cudaEventElapsedTime(&t, s->prof_ev[2 * k], s->prof_ev[2 * k + 1]), "profile read");
        ms += t;
    }
    out->pair_launches = (int64_t)s->prof_used;
    out->pair_ms = ms;
    out->pair_interactions = s->prof_pairs;
    out->pair_flops = s->prof_pairs * (s->wall ? (s->angular ? lmk::kFlopsPerPairWall6N : lmk::kFlopsPerPairWallTT)
                                                : (s->angular ? lmk::kFlopsPerPair6N : lmk::kFlopsPerPairTT));
    out->vector_iterations = 0;
    out->vector_ms = 0.0;
    out->vector_bytes = 0.0;
    for (size_t k = 0; k < s->vprof_used && k < s->vprof_bytes.size(); ++k) {
        if (s->vprof_bytes[k] < 0.0) continue;   // iteration of a call that did not finish
        float t = 0.f;
        LM_CUDA(cudaEventElapsedTime(&t, s->vprof_ev[2 * k], s->vprof_ev[2 * k + 1]), "profile read");
        out->vector_iterations += 1;
        out->vector_ms += t;
        out->vector_bytes += s->vprof_bytes[k];
    }
    if (reset) {
        s->prof_used = 0;
        s->prof_pairs = 0.0;
        s->vprof_used = 0;
        s->vprof_bytes.clear();
        s->vprof_pending.clear();
    }
    return LM_OK;
}

// Host-only helper exposed for testing the tridiagonal step on the CPU:
// out = f(T) e1, f = sqrt, for T = tridiag(beta, alpha, beta) of size m.
int lm_tridiag_sqrt_e1(int m, const double* alpha, const double* beta, double* out) {
    if (m < 1 || !alpha || !out || (m > 1 && !beta)) return -2;
    LanczosHost H;
    H.alpha.assign(alpha, alpha + m);
    H.beta.assign(beta ? beta : alpha, beta ? beta + (m - 1) : alpha);
    int cl = 0;
    const int r = H.solve(m, 1.0, &cl);
    if (r == 0)
        for (int i = 0; i < m; ++i) out[i] = H.z[i];
    return r == -2 ? -1 : r;
}

}  // extern "C"

// ===========================================================================
// Batched systems (lm_batch_*): host side of the persistent kernel.
// ===========================================================================
struct lm_batch {
    int S = 0;
    int64_t Ntot = 0;
    int m_max = 64;
    cudaStream_t stream = nullptr;
    cudaStream_t graph_stream = nullptr;
    int device = 0, sms = 1;
    double eta = 1.0, a = 1.0;
    std::vector<int64_t> off_h;
    DBuf off, pos4, x64, Fbuf, u, w0, w1, V, alpha, amax, beta, z, zprev, normW, rel, active, msys, itsum, notconv, nact;
    DBuf kprev, wsplit, usplit, woff;
    DBuf items, item_range, chunks, chunk_range, part_item, part_chunk, trk, trc, trs, bar, ticket, err, flag;
    DBuf in_stage, out_stage, W_stage;
    // asynchronous tridiagonal solves
    DBuf pass2, sys_cnt;
    DBuf sv_w, q_req, q_seq, q_ack, q_ctr, inflight, zres, zdone, state, next_check, last_k, k0s, posted, main_done,
        cur_step;
    int solver_lanes = 0, q_cap = 0, R = 32;
    int n_items = 0, n_chunks = 0, max_rot = 0;
    int threads = 128, ilp = 1;
    int reorth = 0;   // as lm_solver::reorth
    bool has_pos = false;
    int* pinned = nullptr;
    bool prof_on = false;
    DBuf timeline, pcount;
    int timeline_len = 0;
    ~lm_batch() {
        timeline.release();
        pcount.release();
        kprev.release();
        wsplit.release();
        usplit.release();
        woff.release();
        DBuf* all[] = {&off, &pos4, &x64, &Fbuf, &u, &w0, &w1, &V, &alpha, &amax, &beta, &z, &zprev, &normW, &rel,
                       &active, &msys, &itsum, &notconv, &nact, &items, &item_range, &chunks, &chunk_range,
                       &part_item, &part_chunk, &trk, &trc, &trs, &bar, &ticket, &err, &flag, &in_stage,
                       &out_stage, &W_stage, &pass2, &sys_cnt, &sv_w, &q_req, &q_seq, &q_ack, &q_ctr, &inflight, &zres, &zdone,
                       &state, &next_check, &last_k, &k0s, &posted, &main_done, &cur_step};
        for (DBuf* b : all) b->release();
        if (pinned) cudaFreeHost(pinned);
        if (graph_stream) cudaStreamDestroy(graph_stream);
    }
};

namespace {

// Work items: systems in decreasing size, each cut into blocks of
// threads * ilp particles.
lm_status batch_build_items(lm_batch* b) {
    const int per = b->threads * b->ilp;
    std::vector<int> order(b->S);
    for (int s = 0; s < b->S; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (b->off_h[x + 1] - b->off_h[x]) > (b->off_h[y + 1] - b->off_h[y]);
    });
    std::vector<int> items, range(2 * b->S);
    for (int s : order) {
        const int64_t n = b->off_h[s + 1] - b->off_h[s];
        range[2 * s] = (int)(items.size() / 3);
        for (int64_t jp = 0; jp * lmk::kBatchJPart < n; ++jp)
            for (int64_t i0 = 0; i0 < n; i0 += per) {
                items.push_back(s);
                items.push_back((int)i0);
                items.push_back((int)jp);
            }
        range[2 * s + 1] = (int)(items.size() / 3);
    }
    b->n_items = (int)(items.size() / 3);
    LM_CUDA(b->items.ensure(items.size() * sizeof(int)), "batch items");
    LM_CUDA(b->item_range.ensure(range.size() * sizeof(int)), "batch items");
    LM_CUDA(b->part_item.ensure((size_t)b->n_items * sizeof(double)), "batch items");
    LM_CUDA(cudaMemcpy(b->items.p, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice), "batch items");
    LM_CUDA(cudaMemcpy(b->item_range.p, range.data(), range.size() * sizeof(int), cudaMemcpyHostToDevice),
            "batch items");
    return LM_OK;
}

int batch_grid(const lm_batch* b) {
    const int occ = lmk::batch_ctas_per_sm(b->threads, b->ilp);
    return std::max(1, occ) * b->sms;
}

// Solver CTAs at the end of the cooperative grid: kSolverWarps warps.
int batch_solver_ctas(const lm_batch* b) { return (lmk::kSolverWarps * 32 + b->threads - 1) / b->threads; }

lmk::BatchParams batch_params(lm_batch* b, int mode) {
    lmk::BatchParams p = {};
    p.S = b->S;
    p.m_max = b->m_max;
    p.mode = mode;
    p.nsteps = 1;
    p.Ntot = b->Ntot;
    p.off = b->off.as<int64_t>();
    p.pos4 = b->pos4.as<float4>();
    p.x64 = b->x64.as<double>();
    p.Fbuf = b->Fbuf.as<float>();
    p.u = b->u.as<double>();
    p.w0 = b->w0.as<double>();
    p.w1 = b->w1.as<double>();
    p.V = b->V.as<double>();
    p.alpha = b->alpha.as<double>();
    p.amax = b->amax.as<double>();
    p.beta = b->beta.as<double>();
    p.z = b->z.as<double>();
    p.zprev = b->zprev.as<double>();
    p.normW = b->normW.as<double>();
    p.rel = b->rel.as<double>();
    p.active = b->active.as<int>();
    p.msys = b->msys.as<int>();
    p.itsum = b->itsum.as<int>();
    p.notconv = b->notconv.as<int>();
    p.kprev = b->kprev.as<int>();
    p.wsplit = b->wsplit.as<double>();
    p.usplit = b->usplit.as<double>();
    p.woff = b->woff.as<int64_t>();
    p.warm_start = (mode == lmk::kBatchBD) ? 1 : 0;
    p.reorth = b->reorth;
    p.nact = b->nact.as<int>();
    p.pass2 = b->pass2.as<int>();
    p.sys_cnt = b->sys_cnt.as<int>();
    p.items = b->items.as<int>();
    p.n_items = b->n_items;
    p.item_range = b->item_range.as<int>();
    p.chunks = b->chunks.as<int>();
    p.n_chunks = b->n_chunks;
    p.chunk_range = b->chunk_range.as<int>();
    p.part_item = b->part_item.as<double>();
    p.part_chunk = b->part_chunk.as<double>();
    p.n_main = batch_grid(b) - batch_solver_ctas(b);
    p.sv_w = b->sv_w.as<double>();
    p.trk = b->trk.as<int>();
    p.trc = b->trc.as<double>();
    p.trs = b->trs.as<double>();
    p.max_rot = b->max_rot;
    p.q_req = b->q_req.as<long long>();
    p.q_seq = b->q_seq.as<unsigned long long>();
    p.q_ack = b->q_ack.as<unsigned long long>();
    p.q_ctr = b->q_ctr.as<unsigned long long>();
    p.q_cap = b->q_cap;
    p.inflight = b->inflight.as<int>();
    p.zres = b->zres.as<double>();
    p.zdone = b->zdone.as<unsigned long long>();
    p.R = b->R;
    p.state = b->state.as<int>();
    p.next_check = b->next_check.as<int>();
    p.last_k = b->last_k.as<int>();
    p.k0s = b->k0s.as<int>();
    p.posted = b->posted.as<int>();
    p.main_done = b->main_done.as<int>();
    p.cur_step = b->cur_step.as<long long>();
    p.bar = b->bar.as<unsigned>();
    p.ticket = b->ticket.as<unsigned long long>();
    p.err = b->err.as<int>();
    p.spin_limit = 4000000000LL;  // ~2 s at 2 GHz: far above any phase
    p.k = lmk::make_rpy_const<float>(b->a);
    p.c8 = 1.0 / (8.0 * 3.14159265358979323846 * b->eta);
    p.brk_rel = 1e-7;
    p.prefactor = 1.0;
    if (b->prof_on && b->timeline.p) {
        p.timeline = b->timeline.as<unsigned long long>();
        p.timeline_len = b->timeline_len;
        p.pair_count = b->pcount.as<unsigned long long>();
    }
    return p;
}

// Reset the per-call device state and run the persistent kernel (directly or
// captured in a CUDA graph on the batch's own stream); waits for it.
lm_status batch_run(lm_batch* b, const lmk::BatchParams& p, bool use_graph) {
    const int grid = batch_grid(b);
    cudaStream_t st = b->stream;
    if (use_graph) {
        LM_CUDA(cudaStreamSynchronize(b->stream), "batch run");
        if (!b->graph_stream)
            LM_CUDA(cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking), "batch graph stream");
        st = b->graph_stream;
        LM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "batch graph capture");
    }
    if (p.n_main < 1) return fail(LM_ERR_CUDA, "cooperative grid of %d CTAs leaves no main CTA", grid);
    if (p.n_main > lmk::kBarGroup * lmk::kBarMaxGroups)
        return fail(LM_ERR_CUDA, "cooperative grid of %d CTAs exceeds the grid barrier's capacity", grid);
    // every level of the grid barrier starts at zero (a run that ended on an
    // error may have left counts behind)
    cudaError_t e = cudaMemsetAsync(b->bar.p, 0, lmk::kBarWords * sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ticket.p, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && p.pair_count) e = cudaMemsetAsync(p.pair_count, 0, sizeof(unsigned long long), st);
    // request ring, counters and result tags start empty in every launch
    const size_t S_ = (size_t)b->S;
    if (e == cudaSuccess) e = cudaMemsetAsync(b->q_seq.p, 0, (size_t)b->q_cap * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->q_ack.p, 0, (size_t)b->q_cap * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->q_ctr.p, 0, 4 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->inflight.p, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->zdone.p, 0, S_ * 2 * b->R * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->state.p, 0, S_ * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->main_done.p, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->cur_step.p, 0xff, sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->err.p, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->itsum.p, 0, (size_t)b->S * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->notconv.p, 0, (size_t)b->S * sizeof(int), st);
    if (e == cudaSuccess) e = lmk::launch_batch(p, b->threads, b->ilp, grid, st);
    if (use_graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st, &g);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(ex, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
    } else if (e == cudaSuccess) {
        e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched kernel");
    int errv = 0;
    LM_CUDA(cudaMemcpy(&errv, b->err.p, sizeof(int), cudaMemcpyDeviceToHost), "batched kernel status");
    if (errv == lmk::kBatchTimeout) return fail(LM_ERR_TIMEOUT, "a device-side barrier wait expired");
    if (errv == lmk::kBatchTridiag) return fail(LM_ERR_CUDA, "tridiagonal eigensolver failed on the device");
    return LM_OK;
}

lm_status check_batch(lm_batch* b, bool need_pos) {
    if (b == nullptr) return fail(LM_ERR_INVALID_ARG, "batch is NULL");
    if (need_pos && !b->has_pos) return fail(LM_ERR_STATE, "positions not set (call lm_batch_set_positions first)");
    return LM_OK;
}

lm_status batch_stage_in(lm_batch* b, const void* p, size_t bytes, DBuf& buf, const void** out) {
    *out = nullptr;
    if (!p) return LM_OK;
    if (is_device_ptr(p)) { *out = p; return LM_OK; }
    LM_CUDA(buf.ensure(bytes), "staging input");
    LM_CUDA(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, b->stream), "copy input");
    *out = buf.p;
    return LM_OK;
}

}  // namespace

extern "C" {

lm_status lm_batch_create(lm_batch** out, int64_t S, const int64_t* offsets, double viscosity,
                          double hydrodynamic_radius, int max_iter, void* cuda_stream) {
    lmk::TraceRange trace_("lm_batch_create");
    g_err.clear();
    if (!out) return fail(LM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (S < 1 || S > (1 << 20)) return fail(LM_ERR_INVALID_ARG, "S must be in [1, 2^20]");
    if (!offsets) return fail(LM_ERR_INVALID_ARG, "offsets is NULL");
    if (offsets[0] != 0) return fail(LM_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int64_t s = 0; s < S; ++s) {
        const int64_t n = offsets[s + 1] - offsets[s];
        if (n < 1 || n > 65536) return fail(LM_ERR_INVALID_ARG, "system %lld has %lld particles (1..65536 allowed)",
                                            (long long)s, (long long)n);
    }
    if (!(viscosity > 0.0) || !(hydrodynamic_radius > 0.0))
        return fail(LM_ERR_INVALID_ARG, "viscosity and radius must be > 0");
    if (max_iter < 1 || max_iter > 128) return fail(LM_ERR_INVALID_ARG, "max_iter must be in [1, 128]");
    lm_batch* b = new (std::nothrow) lm_batch();
    if (!b) return fail(LM_ERR_OOM, "host allocation failed");
    std::unique_ptr<lm_batch> guard(b);
    b->S = (int)S;
    b->off_h.assign(offsets, offsets + S + 1);
    b->Ntot = offsets[S];
    b->m_max = max_iter;
    b->eta = viscosity;
    b->a = hydrodynamic_radius;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    LM_CUDA(cudaGetDevice(&b->device), "lm_batch_create");
    LM_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device), "lm_batch_create");
    int coop = 0;
    LM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device), "lm_batch_create");
    if (!coop) return fail(LM_ERR_CUDA, "device does not support cooperative launches");
    const int64_t n3 = 3 * b->Ntot;
    const size_t S_ = (size_t)S, M = (size_t)b->m_max;
    // chunks
    std::vector<int> chunks, crange(2 * S_);
    for (int64_t s = 0; s < S; ++s) {
        const int64_t ns = 3 * (offsets[s + 1] - offsets[s]);
        crange[2 * s] = (int)(chunks.size() / 2);
        for (int64_t e0 = 0; e0 < ns; e0 += lmk::kBatchChunk) { chunks.push_back((int)s); chunks.push_back((int)e0); }
        crange[2 * s + 1] = (int)(chunks.size() / 2);
    }
    b->n_chunks = (int)(chunks.size() / 2);
    std::vector<int64_t> woff(S_);
    int64_t wtot = 0;
    for (int64_t s = 0; s < S; ++s) {
        const int64_t n = offsets[s + 1] - offsets[s];
        woff[s] = wtot;
        wtot += ((n + lmk::kBatchJPart - 1) / lmk::kBatchJPart) * 3 * n;
    }
    b->max_rot = (int)(4 * M * M + 64);
    // one solver slot per solver warp (CTAs of 64 or 128 threads hold whole
    // warps: kSolverWarps is a multiple of 4)
    const size_t lanes = (size_t)lmk::kSolverWarps;
    b->solver_lanes = (int)lanes;
    b->q_cap = 16384;
    struct { DBuf* buf; size_t bytes; } allocs[] = {
        {&b->off, (S_ + 1) * sizeof(int64_t)}, {&b->pos4, (size_t)b->Ntot * sizeof(float4)},
        {&b->x64, (size_t)n3 * sizeof(double)}, {&b->Fbuf, (size_t)n3 * sizeof(float)},
        {&b->u, (size_t)n3 * sizeof(double)}, {&b->w0, (size_t)n3 * sizeof(double)},
        {&b->w1, (size_t)n3 * sizeof(double)}, {&b->V, M * (size_t)n3 * sizeof(double)},
        {&b->alpha, S_ * M * sizeof(double)}, {&b->amax, S_ * sizeof(double)}, {&b->beta, S_ * M * sizeof(double)},
        {&b->z, S_ * M * sizeof(double)}, {&b->zprev, S_ * M * sizeof(double)},
        {&b->normW, S_ * sizeof(double)}, {&b->rel, S_ * sizeof(double)}, {&b->active, S_ * sizeof(int)},
        {&b->msys, S_ * sizeof(int)}, {&b->itsum, S_ * sizeof(int)}, {&b->notconv, S_ * sizeof(int)},
        {&b->nact, (M + 1) * sizeof(int)}, {&b->pass2, (M + 1) * sizeof(int)}, {&b->sys_cnt, S_ * sizeof(int)},
        {&b->chunks, chunks.size() * sizeof(int)},
        {&b->chunk_range, crange.size() * sizeof(int)},
        {&b->part_chunk, 2 * (size_t)b->n_chunks * (M + 1) * sizeof(double)},
        {&b->sv_w, lanes * lmk::tridiag_warp_scratch_doubles((int)M) * sizeof(double)}, {&b->trk, lanes * (size_t)b->max_rot * sizeof(int)},
        {&b->trc, lanes * (size_t)b->max_rot * sizeof(double)}, {&b->trs, lanes * (size_t)b->max_rot * sizeof(double)},
        {&b->q_req, (size_t)b->q_cap * sizeof(long long)}, {&b->q_seq, (size_t)b->q_cap * sizeof(unsigned long long)},
        {&b->q_ack, (size_t)b->q_cap * sizeof(unsigned long long)}, {&b->q_ctr, 4 * sizeof(unsigned long long)},
        {&b->inflight, 2 * sizeof(int)}, {&b->zres, S_ * 2 * (size_t)b->R * M * sizeof(double)},
        {&b->zdone, S_ * 2 * (size_t)b->R * sizeof(unsigned long long)}, {&b->state, S_ * sizeof(int)},
        {&b->next_check, S_ * sizeof(int)}, {&b->last_k, S_ * sizeof(int)}, {&b->k0s, S_ * sizeof(int)}, {&b->posted, S_ * sizeof(int)},
        {&b->main_done, sizeof(int)}, {&b->cur_step, sizeof(long long)},
        {&b->bar, lmk::kBarWords * sizeof(unsigned)}, {&b->ticket, sizeof(unsigned long long)}, {&b->err, sizeof(int)},
        {&b->flag, sizeof(int)}, {&b->kprev, S_ * sizeof(int)}, {&b->woff, S_ * sizeof(int64_t)},
        {&b->wsplit, (size_t)wtot * sizeof(double)}, {&b->usplit, (size_t)wtot * sizeof(double)}};
    for (auto& al : allocs) LM_CUDA(al.buf->ensure(al.bytes), "allocating batch buffers");
    LM_CUDA(cudaMemcpy(b->off.p, offsets, (S_ + 1) * sizeof(int64_t), cudaMemcpyHostToDevice), "batch offsets");
    LM_CUDA(cudaMemcpy(b->chunks.p, chunks.data(), chunks.size() * sizeof(int), cudaMemcpyHostToDevice), "chunks");
    LM_CUDA(cudaMemcpy(b->chunk_range.p, crange.data(), crange.size() * sizeof(int), cudaMemcpyHostToDevice),
            "chunks");
    LM_CUDA(cudaMemset(b->bar.p, 0, lmk::kBarWords * sizeof(unsigned)), "batch barrier");
    LM_CUDA(cudaMemset(b->kprev.p, 0, S_ * sizeof(int)), "batch history");
    LM_CUDA(cudaMemset(b->sys_cnt.p, 0, S_ * sizeof(int)), "batch counters");
    LM_CUDA(cudaMemset(b->pass2.p, 0, (M + 1) * sizeof(int)), "batch counters");
    LM_CUDA(cudaMemcpy(b->woff.p, woff.data(), S_ * sizeof(int64_t), cudaMemcpyHostToDevice), "batch offsets");
    if (lm_status st = batch_build_items(b)) return st;
    LM_CUDA(cudaMallocHost(reinterpret_cast<void**>(&b->pinned), 2 * S_ * sizeof(int)), "batch pinned");
    *out = guard.release();
    return LM_OK;
}

lm_status lm_batch_destroy(lm_batch* b) {
    if (!b) return LM_OK;
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    delete b;
    return LM_OK;
}

lm_status lm_batch_set_positions(lm_batch* b, const float* pos) {
    lmk::TraceRange trace_("lm_batch_set_positions");
    if (lm_status st = check_batch(b, false)) return st;
    if (!pos) return fail(LM_ERR_INVALID_ARG, "pos is NULL");
    DeviceGuard g(b->device);
    b->has_pos = false;
    const void* d = nullptr;
    if (lm_status st = batch_stage_in(b, pos, (size_t)b->Ntot * 3 * sizeof(float), b->in_stage, &d)) return st;
    LM_CUDA(cudaMemsetAsync(b->flag.p, 0, sizeof(int), b->stream), "batch positions");
    LM_CUDA(lmk::launch_batch_pack(static_cast<const float*>(d), b->Ntot, b->pos4.as<float4>(), b->x64.as<double>(),
                                   b->flag.as<int>(), b->stream),
            "batch positions");
    LM_CUDA(cudaMemcpyAsync(b->pinned, b->flag.p, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "batch positions");
    LM_CUDA(cudaStreamSynchronize(b->stream), "batch positions");
    if (b->pinned[0]) return fail(LM_ERR_NONFINITE, "positions contain NaN/Inf or |x| > 1e15");
    b->has_pos = true;
    return LM_OK;
}

lm_status lm_batch_get_positions(lm_batch* b, float* pos_out) {
    if (lm_status st = check_batch(b, true)) return st;
    if (!pos_out) return fail(LM_ERR_INVALID_ARG, "pos_out is NULL");
    DeviceGuard g(b->device);
    const size_t bytes = (size_t)b->Ntot * 3 * sizeof(float);
    const bool host = !is_device_ptr(pos_out);
    float* d = pos_out;
    if (host) {
        LM_CUDA(b->out_stage.ensure(bytes), "staging output");
        d = b->out_stage.as<float>();
    }
    LM_CUDA(lmk::launch_batch_unpack(b->x64.as<double>(), b->Ntot, d, b->stream), "batch positions");
    if (host) LM_CUDA(cudaMemcpyAsync(pos_out, d, bytes, cudaMemcpyDeviceToHost, b->stream), "batch positions");
    LM_CUDA(cudaStreamSynchronize(b->stream), "batch positions");
    return LM_OK;
}

static lm_status batch_mdot_body(lm_batch* b, const float* forces, float* lin_out) {
    if (lm_status st = check_batch(b, true)) return st;
    if (!forces || !lin_out) return fail(LM_ERR_INVALID_ARG, "forces and lin_out are required");
    DeviceGuard g(b->device);
    const size_t bytes = (size_t)b->Ntot * 3 * sizeof(float);
    const void* dF = nullptr;
    if (lm_status st = batch_stage_in(b, forces, bytes, b->in_stage, &dF)) return st;
    const bool host = !is_device_ptr(lin_out);
    float* dout = lin_out;
    if (host) {
        LM_CUDA(b->out_stage.ensure(bytes), "staging output");
        dout = b->out_stage.as<float>();
    }
    lmk::BatchParams p = batch_params(b, lmk::kBatchMdot);
    p.F_in = static_cast<const float*>(dF);
    p.lin_out = dout;
    if (lm_status st = batch_run(b, p, false)) return st;
    if (host) LM_CUDA(cudaMemcpy(lin_out, dout, bytes, cudaMemcpyDeviceToHost), "copy output");
    return LM_OK;
}

lm_status lm_batch_mdot(lm_batch* b, const float* forces, float* lin_out) {
    CallScope cs("lm_batch_mdot");
    const lm_status st = batch_mdot_body(b, forces, lin_out);
    if (!lmk::metrics_enabled() || b == nullptr) return st;
    char f[128];
    std::snprintf(f, sizeof(f), "\"systems\":%d,\"N_total\":%lld", b->S, (long long)b->Ntot);
    return log_call(cs, b->stream, b->device, st, f);
}

static lm_status batch_sqrt_mdot_body(lm_batch* b, const double* W, uint64_t seed, double prefactor, double tol,
                             float* lin_out, int* iters_out) {
    if (lm_status st = check_batch(b, true)) return st;
    if (!lin_out) return fail(LM_ERR_INVALID_ARG, "lin_out is NULL");
    if (!(tol >= 0.0) || !std::isfinite(prefactor)) return fail(LM_ERR_INVALID_ARG, "bad tol or prefactor");
    DeviceGuard g(b->device);
    const size_t bytes = (size_t)b->Ntot * 3 * sizeof(float);
    const void* dW = nullptr;
    if (lm_status st = batch_stage_in(b, W, (size_t)b->Ntot * 3 * sizeof(double), b->W_stage, &dW)) return st;
    const bool host = !is_device_ptr(lin_out);
    float* dout = lin_out;
    if (host) {
        LM_CUDA(b->out_stage.ensure(bytes), "staging output");
        dout = b->out_stage.as<float>();
    }
    lmk::BatchParams p = batch_params(b, lmk::kBatchSqrt);
    p.W_in = static_cast<const double*>(dW);
    p.seed = seed;
    p.tol = tol;
    p.prefactor = prefactor;
    p.lin_out = dout;
    if (lm_status st = batch_run(b, p, false)) return st;
    if (host) LM_CUDA(cudaMemcpy(lin_out, dout, bytes, cudaMemcpyDeviceToHost), "copy output");
    std::vector<int> nc(b->S), its(b->S);
    LM_CUDA(cudaMemcpy(its.data(), b->itsum.p, b->S * sizeof(int), cudaMemcpyDeviceToHost), "iterations");
    LM_CUDA(cudaMemcpy(nc.data(), b->notconv.p, b->S * sizeof(int), cudaMemcpyDeviceToHost), "iterations");
    if (iters_out) std::copy(its.begin(), its.end(), iters_out);
    for (int v : nc)
        if (v) return fail(LM_ERR_NOT_CONVERGED, "some systems reached max_iter before tol %.3g", tol);
    return LM_OK;
}

lm_status lm_batch_sqrt_mdot(lm_batch* b, const double* W, uint64_t seed, double prefactor, double tol,
                             float* lin_out, int* iters_out) {
    CallScope cs("lm_batch_sqrt_mdot");
    const lm_status st = batch_sqrt_mdot_body(b, W, seed, prefactor, tol, lin_out, iters_out);
    if (!lmk::metrics_enabled() || b == nullptr) return st;
    char f[256];
    std::snprintf(f, sizeof(f), "\"systems\":%d,\"N_total\":%lld,\"tol\":%.3e", b->S, (long long)b->Ntot, tol);
    return log_call(cs, b->stream, b->device, st, f);
}

static lm_status batch_bd_run_body(lm_batch* b, double kT, double dt, double k_trap, int nsteps, int64_t step0,
                          uint64_t seed, double tol, int use_graph, int* iters_out) {
    if (lm_status st = check_batch(b, true)) return st;
    if (nsteps < 1 || !(kT >= 0.0) || !(dt >= 0.0) || !std::isfinite(k_trap) || !(tol >= 0.0) || step0 < 0)
        return fail(LM_ERR_INVALID_ARG, "bad Brownian-dynamics parameters");
    DeviceGuard g(b->device);
    lmk::BatchParams p = batch_params(b, lmk::kBatchBD);
    p.nsteps = nsteps;
    p.step0 = step0;
    p.kT = kT;
    p.dt = dt;
    p.k_trap = k_trap;
    p.tol = tol;
    p.seed = seed;
    if (lm_status st = batch_run(b, p, use_graph != 0)) return st;
    if (iters_out)
        LM_CUDA(cudaMemcpy(iters_out, b->itsum.p, b->S * sizeof(int), cudaMemcpyDeviceToHost), "iterations");
    std::vector<int> nc(b->S);
    LM_CUDA(cudaMemcpy(nc.data(), b->notconv.p, b->S * sizeof(int), cudaMemcpyDeviceToHost), "iterations");
    for (int v : nc)
        if (v) return fail(LM_ERR_NOT_CONVERGED, "some systems reached max_iter before tol %.3g", tol);
    return LM_OK;
}

lm_status lm_batch_bd_run(lm_batch* b, double kT, double dt, double k_trap, int nsteps, int64_t step0,
                          uint64_t seed, double tol, int use_graph, int* iters_out) {
    CallScope cs("lm_batch_bd_run");
    const lm_status st = batch_bd_run_body(b, kT, dt, k_trap, nsteps, step0, seed, tol, use_graph, iters_out);
    if (!lmk::metrics_enabled() || b == nullptr) return st;
    char f[256];
    std::snprintf(f, sizeof(f), "\"systems\":%d,\"N_total\":%lld,\"steps\":%d,\"tol\":%.3e,\"graph\":%d", b->S,
                  (long long)b->Ntot, nsteps, tol, use_graph);
    return log_call(cs, b->stream, b->device, st, f);
}

lm_status lm_batch_set_reorthogonalization(lm_batch* b, int mode) {
    if (lm_status st = check_batch(b, false)) return st;
    if (mode != 0 && mode != 1) return fail(LM_ERR_INVALID_ARG, "reorthogonalization mode must be 0 (DGKS) or 1 (two passes)");
    b->reorth = mode;
    return LM_OK;
}

lm_status lm_batch_set_tiling(lm_batch* b, int threads, int ilp) {
    if (lm_status st = check_batch(b, false)) return st;
    if (!lmk::batch_tiling_supported(threads, ilp))
        return fail(LM_ERR_INVALID_ARG, "unsupported batch tiling (threads %d, ilp %d)", threads, ilp);
    DeviceGuard g(b->device);
    b->threads = threads;
    b->ilp = ilp;
    return batch_build_items(b);
}

lm_status lm_batch_autotune(lm_batch* b, int* threads_out, int* ilp_out) {
    lmk::TraceRange trace_("lm_batch_autotune");
    if (lm_status st = check_batch(b, true)) return st;
    DeviceGuard g(b->device);
    const size_t bytes = (size_t)b->Ntot * 3 * sizeof(float);
    LM_CUDA(b->out_stage.ensure(bytes), "autotune buffers");
    const int opts[4][2] = {{64, 1}, {64, 2}, {128, 1}, {128, 2}};
    float best = 1e30f;
    int bt = b->threads, bi = b->ilp;
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0), "autotune");
    LM_CUDA(cudaEventCreate(&e1), "autotune");
    lm_status result = LM_OK;
    // each tiling times a batched square root (Philox noise, tol 1e-4): the
    // products, the vector phases and the solves of a Brownian step, whose
    // best tilings differ (the vector phases favour more, smaller CTAs).  The
    // solves overwrite the systems' warm-start counts: kept and put back.
    DBuf kprev_keep;
    LM_CUDA(kprev_keep.ensure((size_t)b->S * sizeof(int)), "autotune buffers");
    LM_CUDA(cudaMemcpyAsync(kprev_keep.p, b->kprev.p, (size_t)b->S * sizeof(int), cudaMemcpyDeviceToDevice,
                            b->stream),
            "autotune buffers");
    for (auto& o : opts) {
        if ((result = lm_batch_set_tiling(b, o[0], o[1])) != LM_OK) break;
        lmk::BatchParams p = batch_params(b, lmk::kBatchSqrt);
        p.W_in = nullptr;
        p.seed = 0x5eedull;
        p.tol = 1e-4;
        p.prefactor = 1.0;
        p.lin_out = b->out_stage.as<float>();
        if ((result = batch_run(b, p, false)) != LM_OK) break;  // warm-up
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < 3 && result == LM_OK; ++r) result = batch_run(b, p, false);
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (result == LM_OK && ms < best) { best = ms; bt = o[0]; bi = o[1]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LM_CUDA(cudaMemcpyAsync(b->kprev.p, kprev_keep.p, (size_t)b->S * sizeof(int), cudaMemcpyDeviceToDevice,
                            b->stream),
            "autotune buffers");
    LM_CUDA(cudaStreamSynchronize(b->stream), "autotune");
    if (result != LM_OK) return result;
    if (lm_status st = lm_batch_set_tiling(b, bt, bi)) return st;
    if (threads_out) *threads_out = bt;
    if (ilp_out) *ilp_out = bi;
    return LM_OK;
}

lm_status lm_batch_profile_enable(lm_batch* b, int enable) {
    if (lm_status st = check_batch(b, false)) return st;
    DeviceGuard g(b->device);
    b->prof_on = enable != 0;
    if (b->prof_on) {
        b->timeline_len = 5 + 5 * b->m_max;
        LM_CUDA(b->timeline.ensure((size_t)b->timeline_len * sizeof(unsigned long long)), "batch timeline");
        LM_CUDA(cudaMemset(b->timeline.p, 0, (size_t)b->timeline_len * sizeof(unsigned long long)), "timeline");
        LM_CUDA(b->pcount.ensure(sizeof(unsigned long long)), "batch pair counter");
        LM_CUDA(cudaMemset(b->pcount.p, 0, sizeof(unsigned long long)), "batch pair counter");
    }
    return LM_OK;
}

lm_status lm_batch_profile_pairs(lm_batch* b, uint64_t* pairs) {
    if (lm_status st = check_batch(b, false)) return st;
    if (pairs == nullptr) return fail(LM_ERR_INVALID_ARG, "pairs is NULL");
    DeviceGuard g(b->device);
    *pairs = 0;
    if (b->pcount.p == nullptr) return LM_OK;
    LM_CUDA(cudaStreamSynchronize(b->stream), "batch pair counter");
    unsigned long long v = 0;
    LM_CUDA(cudaMemcpy(&v, b->pcount.p, sizeof(v), cudaMemcpyDeviceToHost), "batch pair counter");
    *pairs = (uint64_t)v;
    return LM_OK;
}

lm_status lm_batch_profile_read(lm_batch* b, uint64_t* out, int n, int* count) {
    if (lm_status st = check_batch(b, false)) return st;
    if (!out || n < 0) return fail(LM_ERR_INVALID_ARG, "bad output array");
    DeviceGuard g(b->device);
    std::vector<unsigned long long> t(b->timeline_len);
    if (b->timeline.p && b->timeline_len)
        LM_CUDA(cudaMemcpy(t.data(), b->timeline.p, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost),
                "timeline");
    int c = 0;
    while (c < (int)t.size() && t[c] != 0) ++c;
    for (int i = 0; i < std::min(c, n); ++i) out[i] = t[i];
    if (count) *count = c;
    return LM_OK;
}

lm_status lm_tridiag_sqrt_e1_device_paths(int count, int m, const double* alpha, const double* beta, double* out,
                                          int* paths, void* cuda_stream) {
    g_err.clear();
    if (count < 0 || m < 1 || m > 128) return fail(LM_ERR_INVALID_ARG, "need count >= 0 and 1 <= m <= 128");
    if (count == 0) return LM_OK;
    if (!alpha || !beta || !out) return fail(LM_ERR_INVALID_ARG, "alpha, beta and out are required");
    if (!is_device_ptr(alpha) || !is_device_ptr(beta) || !is_device_ptr(out))
        return fail(LM_ERR_INVALID_ARG, "alpha, beta and out must be device memory");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int max_rot = 4 * m * m + 64;
    const size_t C = (size_t)count;
    DBuf scr, rk, rc, rs, status, path;
    LM_CUDA(scr.ensure(C * lmk::tridiag_warp_scratch_doubles(m) * sizeof(double)), "tridiagonal scratch");
    LM_CUDA(rk.ensure(C * max_rot * sizeof(int)), "tridiagonal scratch");
    LM_CUDA(rc.ensure(C * max_rot * sizeof(double)), "tridiagonal scratch");
    LM_CUDA(rs.ensure(C * max_rot * sizeof(double)), "tridiagonal scratch");
    LM_CUDA(status.ensure(sizeof(int)), "tridiagonal scratch");
    if (paths) LM_CUDA(path.ensure(C * sizeof(int)), "tridiagonal scratch");
    LM_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st), "tridiagonal status");
    LM_CUDA(lmk::launch_tridiag_dev(count, m, alpha, beta, scr.as<double>(), rk.as<int>(), rc.as<double>(),
                                    rs.as<double>(), max_rot, out, status.as<int>(),
                                    paths ? path.as<int>() : nullptr, st),
            "tridiagonal kernel");
    int h = 0;
    LM_CUDA(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "tridiagonal status");
    if (paths) LM_CUDA(cudaMemcpyAsync(paths, path.p, C * sizeof(int), cudaMemcpyDeviceToHost, st), "tridiagonal paths");
    LM_CUDA(cudaStreamSynchronize(st), "tridiagonal kernel");
    if (h != 0) return fail(LM_ERR_CUDA, "device tridiagonal step failed (code %d)", h);
    return LM_OK;
}

lm_status lm_tridiag_sqrt_e1_device(int count, int m, const double* alpha, const double* beta, double* out,
                                    void* cuda_stream) {
    return lm_tridiag_sqrt_e1_device_paths(count, m, alpha, beta, out, nullptr, cuda_stream);
}

lm_status lm_batch_solve_counts(lm_batch* b, int64_t* posted, int64_t* solved) {
    if (lm_status st = check_batch(b, false)) return st;
    if (!posted || !solved) return fail(LM_ERR_INVALID_ARG, "posted and solved are required");
    DeviceGuard g(b->device);
    unsigned long long c[4] = {0, 0, 0, 0};
    LM_CUDA(cudaStreamSynchronize(b->stream), "solve counts");
    LM_CUDA(cudaMemcpy(c, b->q_ctr.p, sizeof(c), cudaMemcpyDeviceToHost), "solve counts");
    *posted = (int64_t)c[1];
    *solved = (int64_t)c[2];
    return LM_OK;
}

lm_status lm_philox_normals(uint64_t seed, uint64_t stream, double* out, int64_t n, void* cuda_stream) {
    if (!out || n < 0) return fail(LM_ERR_INVALID_ARG, "out must be a device array and n >= 0");
    if (!is_device_ptr(out)) return fail(LM_ERR_INVALID_ARG, "out must be device memory");
    if (n == 0) return LM_OK;
    LM_CUDA(lmk::lz_philox_normals(seed, stream, out, n, static_cast<cudaStream_t>(cuda_stream)), "noise generator");
    return LM_OK;
}

lm_status lm_philox4x32_10(const uint32_t* counters, const uint32_t* keys, uint32_t* out, int64_t count,
                           void* cuda_stream) {
    if (count < 0) return fail(LM_ERR_INVALID_ARG, "count must be >= 0");
    if (count == 0) return LM_OK;
    if (!counters || !keys || !out) return fail(LM_ERR_INVALID_ARG, "counters, keys and out are required");
    if (!is_device_ptr(counters) || !is_device_ptr(keys) || !is_device_ptr(out))
        return fail(LM_ERR_INVALID_ARG, "counters, keys and out must be device memory");
    LM_CUDA(lmk::lz_philox_words(counters, keys, out, count, static_cast<cudaStream_t>(cuda_stream)),
            "Philox words");
    return LM_OK;
}

// Test hook for the bounded waits of the persistent kernel: a barrier that can
// never complete must end with LM_ERR_TIMEOUT after about spin_cycles cycles.
lm_status lm_batch_timeout_selftest(long long spin_cycles) {
    if (spin_cycles < 1000 || spin_cycles > 100000000LL)
        return fail(LM_ERR_INVALID_ARG, "spin_cycles must be in [1e3, 1e8]");
    DBuf bar, err;
    LM_CUDA(bar.ensure(4 * sizeof(unsigned)), "selftest");
    LM_CUDA(err.ensure(sizeof(int)), "selftest");
    LM_CUDA(cudaMemset(bar.p, 0, 4 * sizeof(unsigned)), "selftest");
    LM_CUDA(cudaMemset(err.p, 0, sizeof(int)), "selftest");
    LM_CUDA(lmk::launch_batch_timeout_probe(bar.as<unsigned>(), err.as<int>(), spin_cycles, 4, nullptr), "selftest");
    LM_CUDA(cudaDeviceSynchronize(), "selftest");
    int e = 0;
    LM_CUDA(cudaMemcpy(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost), "selftest");
    bar.release();
    err.release();
    if (e == lmk::kBatchTimeout) return fail(LM_ERR_TIMEOUT, "barrier wait expired as intended");
    return fail(LM_ERR_CUDA, "timeout probe did not report a timeout");
}

}  // extern "C"
