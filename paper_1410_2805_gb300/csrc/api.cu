// C-ABI entry points of the hacc library: context, validation, scratch pool
// and the composition of the binning, pair-force and PM kernels into the
// calls declared in include/hacc.h.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hacc_internal.cuh"

namespace hacc {

thread_local int64_t *tl_launches = nullptr;

hacc_status set_error(hacc_ctx *ctx, hacc_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

hacc_status check_cuda(hacc_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HACC_OK;
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(ctx, e == cudaErrorMemoryAllocation ? HACC_ENOMEM : HACC_ECUDA, msg);
}

// Grow-only scratch arena (allocated once per size class, reused across calls:
// the phase-scoped pool of Sec. 2.7 reduced to one region per context).
hacc_status ensure_scratch(hacc_ctx *ctx, size_t bytes, cudaStream_t stream) {
    if (bytes <= ctx->scratch.cap) return HACC_OK;
    size_t want = bytes + bytes / 8;
    if (ctx->budget && want > ctx->budget) want = bytes;
    if (ctx->budget && want > ctx->budget) {
        char msg[160];
        snprintf(msg, sizeof msg, "scratch of %zu bytes exceeds the context budget of %zu bytes", bytes, ctx->budget);
        return set_error(ctx, HACC_ENOMEM, msg);
    }
    if (ctx->scratch.base) {
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaStreamSynchronize");
        cudaFree(ctx->scratch.base);
        ctx->scratch.base = nullptr;
        ctx->scratch.cap = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, HACC_ENOMEM, std::string("cudaMalloc of scratch failed: ") + cudaGetErrorString(e));
    }
    ctx->scratch.base = static_cast<char *>(p);
    ctx->scratch.cap = want;
    return HACC_OK;
}

int32_t default_nc(double L, double r_cut) {
    if (!(L > 0) || !(r_cut > 0)) return -1;
    int64_t nc = (int64_t)std::floor(L / r_cut);
    if (nc >= 1 && L / (double)nc < r_cut * (1.0 + 1e-6)) --nc;
    if (nc < 3) return -1;
    if (nc > 1024) nc = 1024;
    return (int32_t)nc;
}

hacc_status make_geometry(hacc_ctx *ctx, const hacc_box *box, float r_cut, Geometry *g) {
    if (!box) return set_error(ctx, HACC_EINVAL, "box is NULL");
    const double L = box->L;
    if (!(L > 0) || !std::isfinite(L)) return set_error(ctx, HACC_EINVAL, "box side L must be finite and > 0");
    if ((double)(float)L != L) return set_error(ctx, HACC_EINVAL, "box side L must be exactly representable in FP32");
    if (!(r_cut > 0) || !std::isfinite(r_cut)) return set_error(ctx, HACC_EINVAL, "r_cut must be finite and > 0");
    int nc = box->nc;
    if (nc == 0) {
        nc = default_nc(L, r_cut);
        if (nc < 0) return set_error(ctx, HACC_EDOMAIN, "box holds fewer than 3 chaining-mesh cells of width >= r_cut");
    }
    if (nc < 3 || nc > 1024) return set_error(ctx, HACC_EDOMAIN, "nc must be in [3, 1024]");
    if (L / (double)nc < (double)r_cut)
        return set_error(ctx, HACC_EDOMAIN, "chaining-mesh cell width L/nc is below r_cut");
    g->Lf = (float)L;
    g->Ld = L;
    g->nc = nc;
    g->ncell = (int64_t)nc * nc * nc;
    g->inv_w = (float)((double)nc / L);
    return HACC_OK;
}

// Geometry of the single-box force paths: cells at least r_cut / R wide,
// searched over the (2R+1)^3 cells around each (R = the context's stencil).
hacc_status make_sr_geometry(hacc_ctx *ctx, const hacc_box *box, float r_cut, Geometry *g) {
    const int R = ctx->stencil;
    HACC_STATUS_RETURN(make_geometry(ctx, box, R == 2 ? 0.5f * r_cut : r_cut, g));
    if (g->nc < 2 * R + 1) return set_error(ctx, HACC_EDOMAIN, "a 125-cell stencil needs at least 5 cells per side");
    g->R = R;
    return HACC_OK;
}

// Geometry of the (cell, offset) paths: cells step by the FP32 width
// ci_step(g), the last one absorbs the remainder; both widths must reach r_cut.
hacc_status make_ci_geometry(hacc_ctx *ctx, const hacc_box *box, float r_cut, Geometry *g) {
    HACC_STATUS_RETURN(make_geometry(ctx, box, r_cut, g));
    const double W = ci_step(*g);
    if (W < (double)r_cut || W + ci_rem(*g) < (double)r_cut)
        return set_error(ctx, HACC_EDOMAIN, "FP32 cell width of the cell/offset mesh is below r_cut");
    return HACC_OK;
}

// Item caps the single-box tuner tries (0: cell-wide items of up to kItemMax).
const int kTuneCaps[] = {0, 16, 24, 32, 48};
constexpr int kTuneCapCount = 5;
constexpr int kTuneSettings = kTuneCapCount * 2 * kForceVariants;   // cap x queue order x variant
static_assert(kTuneSettings == HACC_TUNE_SETTINGS, "tuner table size");
static_assert(sizeof(hacc_ctx::io_ev) / sizeof(void *) >= 3 + kPmChunks, "one event per PM chunk");

static double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

hacc_status make_force_consts(hacc_ctx *ctx, const hacc_split *split, const Geometry &g, ForceConsts *fc) {
    (void)g;
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    if (!(split->r_cut > 0) || !(split->eps >= 0) || !std::isfinite(split->eps) || !std::isfinite(split->G))
        return set_error(ctx, HACC_EINVAL, "split needs r_cut > 0, eps >= 0 and a finite G");
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(split->poly[k])) return set_error(ctx, HACC_EINVAL, "split poly must be finite");
    const double eps = split->eps, rc = split->r_cut;
    fc->eps = split->eps;
    fc->T = (float)(rc * rc + eps);
    fc->G = split->G;
    // P5(s) with s = t - eps, expanded in powers of t
    for (int m = 0; m < 6; ++m) {
        double q = 0.0;
        for (int k = m; k < 6; ++k) q += split->poly[k] * binom(k, m) * std::pow(-eps, k - m);
        fc->q[m] = (float)q;
    }
    // U(s) = sum_k c_k s^(k+1) / (2(k+1)) = sum_j a_j s^j, j = 1..6; in powers of t
    double a[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 6; ++k) a[k + 1] = split->poly[k] / (2.0 * (k + 1));
    for (int m = 0; m < 7; ++m) {
        double u = 0.0;
        for (int j = m; j < 7; ++j) u += a[j] * binom(j, m) * std::pow(-eps, j - m);
        fc->u[m] = (float)u;
    }
    double s = rc * rc, Us = 0.0, sj = s;
    for (int j = 1; j < 7; ++j) { Us += a[j] * sj; sj *= s; }
    fc->phi0 = (float)(-1.0 / std::sqrt(s + eps) - Us);
    return HACC_OK;
}

}  // namespace hacc

using namespace hacc;

namespace {

// Device staging for the *_host entry points.
hacc_status ensure_io(hacc_ctx *ctx, size_t bytes, cudaStream_t s) {
    if (bytes <= ctx->io_cap) return HACC_OK;
    if (ctx->io_base) {
        cudaStreamSynchronize(s);
        cudaFree(ctx->io_base);
        ctx->io_base = nullptr;
        ctx->io_cap = 0;
    }
    if (cudaMalloc(&ctx->io_base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, HACC_ENOMEM, "cudaMalloc of host-copy staging failed");
    }
    ctx->io_cap = bytes;
    return HACC_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

hacc_status hacc::hacc_enter(hacc_ctx *ctx) {
    if (!ctx) return HACC_EINVAL;
    ctx->last_error.clear();
    tl_launches = &ctx->launches;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return check_cuda(ctx, e, "cudaSetDevice");
    return HACC_OK;
}

namespace {

hacc_status enter(hacc_ctx *ctx) { return hacc_enter(ctx); }

#define HACC_TRY(x)                      \
    do {                                 \
        hacc_status st__ = (x);          \
        if (st__ != HACC_OK) return st__; \
    } while (0)
#define HACC_CUDA(x, what) HACC_TRY(check_cuda(ctx, (x), what))

// Sorted working set of one box for the force and sub-cycle paths.
struct Work {
    float4 *P, *V, *Ps, *Vs;
    int32_t *ID, *IDs;
    int *counter;
    unsigned long long *within;
    float *phi;
    double *diag;
    int4 *ml_items;     // multi-level: work items of an event (at most one per particle)
    int *present;       // multi-level: kick counts that occur
    // multi-level: binned reference positions, a second velocity buffer and
    // input rows (two buffers)
    float4 *R, *V2;
    int32_t *I1, *I2;
    BinBuffers b;
};

size_t carve_work(char *base, int64_t n, int64_t ncell, bool dyn, Work *w, bool ml = false) {
    Carver c(base);
    w->R = ml ? c.take<float4>(n) : nullptr;
    w->V2 = ml ? c.take<float4>(n) : nullptr;
    w->I1 = ml ? c.take<int32_t>(n) : nullptr;
    w->I2 = ml ? c.take<int32_t>(n) : nullptr;
    w->P = c.take<float4>(n);
    w->Ps = c.take<float4>(n);
    w->V = dyn ? c.take<float4>(n) : nullptr;
    w->Vs = dyn ? c.take<float4>(n) : nullptr;
    w->ID = dyn ? c.take<int32_t>(n) : nullptr;
    w->IDs = dyn ? c.take<int32_t>(n) : nullptr;
    w->counter = c.take<int>(1);
    w->within = c.take<unsigned long long>(1);
    w->phi = c.take<float>(n);
    w->diag = c.take<double>(5);
    w->ml_items = ml ? c.take<int4>(n + 1) : nullptr;
    w->present = c.take<int>(kMaxLevels + 3);
    carve_bin(c, n, ncell, &w->b);
    return c.off + 256;
}

hacc_status prepare_work(hacc_ctx *ctx, int64_t n, const Geometry &g, bool dyn, cudaStream_t s, Work *w,
                         bool ml = false) {
    size_t need = carve_work(nullptr, n, g.ncell, dyn, w, ml);
    HACC_TRY(ensure_scratch(ctx, need, s));
    carve_work(ctx->scratch.base, n, g.ncell, dyn, w, ml);
    return HACC_OK;
}

hacc_status check_particles(hacc_ctx *ctx, int64_t n, const void *a, const void *b) {
    if (n < 0) return set_error(ctx, HACC_EINVAL, "n must be >= 0");
    if (n >= (int64_t)1 << 31) return set_error(ctx, HACC_EINVAL, "n must be below 2^31");
    if (n > 0 && (!a || !aligned16(a))) return set_error(ctx, HACC_EINVAL, "particle array NULL or not 16-byte aligned");
    if (n > 0 && b && !aligned16(b)) return set_error(ctx, HACC_EINVAL, "particle array not 16-byte aligned");
    return HACC_OK;
}

hacc_status launch_force(hacc_ctx *ctx, const Geometry &g, const ForceConsts &fc, const ForceLaunch &fl, bool counted,
                         cudaStream_t s);

// The short-range force on sorted positions (w->Ps, cell starts and items in w->b).
hacc_status run_sorted_force(hacc_ctx *ctx, const Geometry &g, const ForceConsts &fc, Work *w, int mode,
                             float4 *out, const int32_t *perm, float4 *vel, float4 *pos_next, float hk, float hd,
                             unsigned long long *within, cudaStream_t s, int64_t n = 0) {
    ForceLaunch fl;
    if (ctx->queue_order && n >= kHeavyFirstMinN) {
        HACC_CUDA(items_heavy_first(w->b, max_items(n, g.ncell), s), "item order");
        fl.order = w->b.order;
    }
    fl.pos = w->Ps;
    fl.items = w->b.items;
    fl.n_items = w->b.n_items;
    fl.cell_start = w->b.cell_start;
    fl.work_counter = w->counter;
    fl.mode = mode;
    fl.out = out;
    fl.perm = perm;
    fl.vel = vel;
    fl.pos_next = pos_next;
    fl.h_kick = hk;
    fl.h_drift = hd;
    fl.phi_out = w->phi;
    fl.within = within;
    fl.mass_flag = w->b.mass_flag;
    fl.variant = ctx->variant;
    if (ctx->counting && mode != kModePotential && !within) {
        HACC_CUDA(candidate_count(g, w->b.cell_start, ctx->d_pairs, s), "candidate count");
        fl.within = ctx->d_pairs + 1;
    }
    if (ctx->counting && fl.within) fl.evaluated = ctx->d_pairs + 2;
    return launch_force(ctx, g, fc, fl, mode != kModePotential, s);
}

// Event pair around a stretch of work on s (statistics timing): begin takes
// a pair from the free list and records its first event; end records the
// second and files the pair under `kind` (0 pair force, 1 chaining-mesh build).
hacc_status timing_begin(hacc_ctx *ctx, cudaStream_t s, std::pair<cudaEvent_t, cudaEvent_t> *ev) {
    *ev = {nullptr, nullptr};
    if (!ctx->timing) return HACC_OK;
    if (ctx->ev_free.empty()) {
        cudaEvent_t a, b;
        HACC_CUDA(cudaEventCreate(&a), "cudaEventCreate");
        HACC_CUDA(cudaEventCreate(&b), "cudaEventCreate");
        ctx->ev_free.emplace_back(a, b);
    }
    *ev = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    HACC_CUDA(cudaEventRecord(ev->first, s), "cudaEventRecord");
    return HACC_OK;
}

hacc_status timing_end(hacc_ctx *ctx, cudaStream_t s, const std::pair<cudaEvent_t, cudaEvent_t> &ev, int kind) {
    if (!ev.first) return HACC_OK;
    HACC_CUDA(cudaEventRecord(ev.second, s), "cudaEventRecord");
    ctx->ev_used.push_back(ev);
    ctx->ev_kind.push_back(kind);
    if (kind == 1) ctx->builds++;
    return HACC_OK;
}

// One pair-kernel launch; timed with an event pair when timing is on.
hacc_status launch_force(hacc_ctx *ctx, const Geometry &g, const ForceConsts &fc, const ForceLaunch &fl, bool counted,
                         cudaStream_t s) {
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (counted) HACC_TRY(timing_begin(ctx, s, &ev));
    HACC_CUDA(sr_force_launch(g, fc, fl, ctx->num_sms, s), "short-range force launch");
    if (counted) ctx->force_launches++;
    return timing_end(ctx, s, ev, 0);
}

}  // namespace

// One counted pair-kernel launch, timed when statistics timing is on (for
// the batched path; not while the stream is being captured).
hacc_status hacc::timed_force_launch(hacc_ctx *ctx, const Geometry &g, const ForceConsts &fc, const ForceLaunch &fl,
                                     cudaStream_t s) {
    return launch_force(ctx, g, fc, fl, true, s);
}


extern "C" {

hacc_status hacc_ctx_create(hacc_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return HACC_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HACC_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return HACC_ECUDA;
    hacc_ctx *ctx = new hacc_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_flags, 4 * sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_flags, 0, 4 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pairs, 5 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->d_pairs, 0, 5 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return HACC_ENOMEM;
    }
    *out = ctx;
    return HACC_OK;
}

void hacc_ctx_destroy(hacc_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    pm_destroy(ctx);
    batch_destroy(ctx);
    if (ctx->scratch.base) cudaFree(ctx->scratch.base);
    if (ctx->io_base) cudaFree(ctx->io_base);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    if (ctx->d_pairs) cudaFree(ctx->d_pairs);
    if (ctx->ml_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(ctx->ml_exec));
    if (ctx->cap_stream) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->cap_stream));
    if (ctx->cap_stream2) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->cap_stream2));
    if (ctx->io_stream) cudaStreamDestroy(static_cast<cudaStream_t>(ctx->io_stream));
    for (void *e : ctx->io_ev)
        if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
    for (auto &e : ctx->ev_used) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (auto &e : ctx->ev_free) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    if (tl_launches == &ctx->launches) tl_launches = nullptr;
    delete ctx;
}

const char *hacc_last_error(const hacc_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

size_t hacc_ctx_scratch_bytes(const hacc_ctx *ctx) {
    if (!ctx) return 0;
    return ctx->scratch.cap + ctx->io_cap;
}

hacc_status hacc_ctx_sync(hacc_ctx *ctx, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    HACC_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    HACC_CUDA(cudaGetLastError(), "pending CUDA error");
    int flags[4] = {0, 0, 0, 0};
    HACC_CUDA(cudaMemcpy(flags, ctx->d_flags, sizeof flags, cudaMemcpyDeviceToHost), "reading device flags");
    HACC_CUDA(cudaMemset(ctx->d_flags, 0, sizeof flags), "clearing device flags");
    if (flags[0] & kFlagItems) return set_error(ctx, HACC_ECUDA, "internal: a work-item list ran out of room");
    if (flags[0] & kFlagDomain)
        return set_error(ctx, HACC_EDOMAIN, "a coordinate was outside [-L, 2L) or not finite");
    return HACC_OK;
}

int32_t hacc_mesh_cells(double L, float r_cut) { return default_nc(L, r_cut); }

int32_t hacc_ml_mesh_cells(double L, float r_cut, float skin) {
    const int32_t nc = default_nc(L, r_cut);
    if (nc < 0 || !(skin > 0) || !std::isfinite(skin)) return nc;
    const int32_t nc2 = default_nc(L, (double)r_cut * (1.0 + (double)skin));
    return (nc2 >= 3 && nc2 < nc) ? nc2 : nc;
}

hacc_status hacc_set_stencil(hacc_ctx *ctx, int32_t cells_per_rcut) {
    HACC_TRY(enter(ctx));
    if (cells_per_rcut != 1 && cells_per_rcut != 2) return set_error(ctx, HACC_EINVAL, "stencil must be 1 or 2");
    ctx->stencil = cells_per_rcut;
    return HACC_OK;
}

hacc_status hacc_set_item_cap(hacc_ctx *ctx, int32_t cap, int32_t split_max) {
    HACC_TRY(enter(ctx));
    if (cap != -1 && cap != 0 && (cap < kItemCapMin || cap > kItemMax))
        return set_error(ctx, HACC_EINVAL, "item cap must be -1, 0 or in [16, 160]");
    if (split_max < 0) return set_error(ctx, HACC_EINVAL, "split_max must be >= 0");
    ctx->item_cap = cap;
    ctx->split_max = split_max ? split_max : kDefaultSplitMax;
    return HACC_OK;
}

hacc_status hacc_set_queue_order(hacc_ctx *ctx, int32_t heavy_first) {
    HACC_TRY(enter(ctx));
    if (heavy_first != 0 && heavy_first != 1) return set_error(ctx, HACC_EINVAL, "heavy_first must be 0 or 1");
    ctx->queue_order = heavy_first;
    return HACC_OK;
}

hacc_status hacc_set_variant(hacc_ctx *ctx, int32_t variant) {
    HACC_TRY(enter(ctx));
    if (variant < 0 || variant >= kForceVariants) return set_error(ctx, HACC_EINVAL, "variant out of range");
    ctx->variant = variant;
    return HACC_OK;
}

hacc_status hacc_tune(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n, const float *pos_m,
                      int32_t reps, double *times_ms, int32_t *chosen, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    if (reps < 1) return set_error(ctx, HACC_EINVAL, "reps must be >= 1");
    Geometry g;
    HACC_TRY(make_sr_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, pos_m, nullptr));
    if (n == 0) return HACC_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the working set of a sub-cycle, plus zero velocities for it (the kick and
    // stream then cost what they cost in a sub-cycle).  As in the sub-cycle
    // loop, each timed sub-cycle bins the positions the previous one left in
    // cell order (a warm-up sub-cycle from pos_m starts each setting); with
    // zero velocities and a step of 1e-3 they move by ~1e-6.
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, true, s, &w));
    HACC_CUDA(cudaMemsetAsync(w.V, 0, sizeof(float4) * (size_t)n, s), "clearing tuner velocities");
    cudaEvent_t e0, e1;
    HACC_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    HACC_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    const int saved_v = ctx->variant, saved_cap = ctx->item_cap, saved_order = ctx->queue_order;
    const bool saved_timing = ctx->timing, saved_counting = ctx->counting;
    ctx->timing = ctx->counting = false;
    double best = 1e300;
    int best_k = 0;
    hacc_status st = HACC_OK;
    const float4 *src = reinterpret_cast<const float4 *>(pos_m);
    const float h = 1e-3f;
    // one sub-cycle's chaining-mesh build and pair-kernel launch (kick + stream)
    auto subcycle_work = [&](int cap, bool first) -> hacc_status {
        HACC_CUDA(bin_build(g, n, first ? src : w.P, nullptr, 0.0f, w.P, w.b, ctx->d_flags, true, s, cap,
                            ctx->split_max, nullptr, !first),
                  "tuner binning");
        HACC_CUDA(gather_sorted(n, w.b.perm, w.P, w.Ps, w.V, w.Vs, nullptr, w.IDs, s), "tuner gather");
        return run_sorted_force(ctx, g, fc, &w, kModeKickDrift, nullptr, nullptr, w.Vs, w.P, h, h, nullptr, s, n);
    };
    for (int k = 0; k < kTuneSettings && st == HACC_OK; ++k) {
        const int cap = kTuneCaps[k / (2 * kForceVariants)];
        ctx->queue_order = (k / kForceVariants) % 2;
        ctx->variant = k % kForceVariants;
        st = subcycle_work(cap, true);   // warm-up, from pos_m
        if (st != HACC_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == HACC_OK; ++r) st = subcycle_work(cap, false);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = check_cuda(ctx, e, "cudaEventSynchronize");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = (double)ms / reps;
        if (times_ms) times_ms[k] = per;
        if (per < best) {
            best = per;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = saved_timing;
    ctx->counting = saved_counting;
    if (st == HACC_OK) {
        ctx->variant = best_k % kForceVariants;
        ctx->queue_order = (best_k / kForceVariants) % 2;
        ctx->item_cap = kTuneCaps[best_k / (2 * kForceVariants)];
    } else {
        ctx->variant = saved_v;
        ctx->queue_order = saved_order;
        ctx->item_cap = saved_cap;
    }
    if (chosen) *chosen = best_k;
    return st;
}

hacc_status hacc_stats_enable(hacc_ctx *ctx, int timing, int counting) {
    HACC_TRY(enter(ctx));
    ctx->timing = timing != 0;
    ctx->counting = counting != 0;
    return HACC_OK;
}

hacc_status hacc_stats_read(hacc_ctx *ctx, hacc_stats *out, int reset) {
    HACC_TRY(enter(ctx));
    if (!out) return set_error(ctx, HACC_EINVAL, "out is NULL");
    HACC_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    for (size_t k = 0; k < ctx->ev_used.size(); ++k) {
        auto &e = ctx->ev_used[k];
        float ms = 0.f;
        HACC_CUDA(cudaEventElapsedTime(&ms, e.first, e.second), "cudaEventElapsedTime");
        (ctx->ev_kind[k] == 1 ? ctx->build_ms : ctx->force_ms) += ms;
        ctx->ev_free.push_back(e);
    }
    ctx->ev_used.clear();
    ctx->ev_kind.clear();
    // candidates, inside the cutoff, evaluated; multi-level graph rebinnings and their kernel launches
    unsigned long long pairs[5] = {0, 0, 0, 0, 0};
    HACC_CUDA(cudaMemcpy(pairs, ctx->d_pairs, sizeof pairs, cudaMemcpyDeviceToHost), "reading pair counts");
    out->kernel_launches = ctx->launches + (int64_t)pairs[4];
    out->force_launches = ctx->force_launches;
    out->force_ms = ctx->force_ms;
    out->candidate_pairs = pairs[0];
    out->within_pairs = pairs[1];
    out->evaluated_pairs = pairs[2];
    out->ml_rebins = ctx->ml_rebins + (int64_t)pairs[3];
    out->build_ms = ctx->build_ms;
    out->builds = ctx->builds;
    if (reset) {
        ctx->ml_rebins = 0;
        ctx->launches = 0;
        ctx->force_launches = 0;
        ctx->force_ms = 0.0;
        ctx->build_ms = 0.0;
        ctx->builds = 0;
        HACC_CUDA(cudaMemset(ctx->d_pairs, 0, sizeof pairs), "clearing pair counts");
    }
    return HACC_OK;
}

hacc_status hacc_bin(hacc_ctx *ctx, const hacc_box *box, float r_cut, int64_t n, float *pos_m, int32_t *cell_id,
                     int32_t *cell_start, int32_t *perm, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    Geometry g;
    HACC_TRY(make_geometry(ctx, box, r_cut, &g));
    HACC_TRY(check_particles(ctx, n, pos_m, nullptr));
    if (!cell_start || (n > 0 && (!cell_id || !perm))) return set_error(ctx, HACC_EINVAL, "output array is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // scratch: everything of BinBuffers except the caller-owned outputs
    auto carve = [&](char *base, BinBuffers *b) {
        Carver c(base);
        carve_bin(c, n, g.ncell, b, false);
        return c.off + 256;
    };
    BinBuffers b;
    HACC_TRY(ensure_scratch(ctx, carve(nullptr, &b), s));
    carve(ctx->scratch.base, &b);
    b.key = cell_id;
    b.cell_start = cell_start;
    b.perm = perm;
    float4 *p = reinterpret_cast<float4 *>(pos_m);
    HACC_CUDA(bin_build(g, n, p, nullptr, 0.0f, p, b, ctx->d_flags, false, s), "binning");
    return HACC_OK;
}

hacc_status hacc_sr_force(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                          const float *pos_m, float *acc, uint64_t *pair_counts, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    Geometry g;
    HACC_TRY(make_sr_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, pos_m, acc));
    if (n > 0 && !acc) return set_error(ctx, HACC_EINVAL, "acc is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, false, s, &w));
    const float4 *src = reinterpret_cast<const float4 *>(pos_m);
    HACC_CUDA(bin_build(g, n, src, nullptr, 0.0f, w.P, w.b, ctx->d_flags, true, s, item_cap_for(ctx, n),
                        ctx->split_max),
              "binning");
    HACC_CUDA(gather_sorted(n, w.b.perm, w.P, w.Ps, nullptr, nullptr, nullptr, nullptr, s), "gather");
    unsigned long long *within = nullptr;
    if (pair_counts) {
        unsigned long long *pc = reinterpret_cast<unsigned long long *>(pair_counts);
        HACC_CUDA(cudaMemsetAsync(pc, 0, 2 * sizeof(unsigned long long), s), "clearing pair counts");
        HACC_CUDA(candidate_count(g, w.b.cell_start, pc, s), "candidate count");
        within = pc + 1;
    }
    if (n > 0)
        HACC_TRY(run_sorted_force(ctx, g, fc, &w, kModeForce, reinterpret_cast<float4 *>(acc), w.b.perm, nullptr,
                                  nullptr, 0.f, 0.f, within, s, n));
    return HACC_OK;
}

hacc_status hacc_subcycle(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n, float *pos_m,
                          float *vel, double dt, int32_t n_sub, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    if (n_sub < 1) return set_error(ctx, HACC_EINVAL, "n_sub must be >= 1");
    if (!std::isfinite(dt)) return set_error(ctx, HACC_EINVAL, "dt must be finite");
    Geometry g;
    HACC_TRY(make_sr_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, pos_m, vel));
    if (n > 0 && !vel) return set_error(ctx, HACC_EINVAL, "vel is NULL");
    if (n == 0) return HACC_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, true, s, &w));
    const float h = (float)(dt / n_sub);
    const float h2 = (float)(0.5 * dt / n_sub);
    float4 *pos_in = reinterpret_cast<float4 *>(pos_m);
    float4 *vel_in = reinterpret_cast<float4 *>(vel);
    for (int k = 0; k < n_sub; ++k) {
        const bool first = k == 0, last = k == n_sub - 1;
        // stream h/2 (first sub-cycle only; later ones were fused into the
        // previous kick) + wrap + rebin
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        HACC_TRY(timing_begin(ctx, s, &ev));
        HACC_CUDA(bin_build(g, n, first ? pos_in : w.P, first ? vel_in : nullptr, h2, w.P, w.b, ctx->d_flags, true,
                            s, item_cap_for(ctx, n), ctx->split_max, nullptr, !first),
                  "binning");
        HACC_CUDA(gather_sorted(n, w.b.perm, w.P, w.Ps, first ? vel_in : w.V, w.Vs, first ? nullptr : w.ID, w.IDs,
                                s),
                  "gather");
        HACC_TRY(timing_end(ctx, s, ev, 1));
        // kick h, then stream h (fused halves) or h/2 (closing the last sub-cycle);
        // positions of this sub-cycle's sorted order go to w.P
        HACC_TRY(run_sorted_force(ctx, g, fc, &w, kModeKickDrift, nullptr, nullptr, w.Vs, w.P, h, last ? h2 : h,
                                  nullptr, s, n));
        std::swap(w.V, w.Vs);
        std::swap(w.ID, w.IDs);
    }
    // wrap the final positions and return rows to input order
    HACC_CUDA(scatter_rows(n, w.ID, w.P, pos_in, w.V, vel_in, g.Lf, ctx->d_flags, s), "scatter");
    return HACC_OK;
}

hacc_status hacc_ci_from_f64(hacc_ctx *ctx, const hacc_box *box, float r_cut, int64_t n, const double *pos64,
                             const float *mass, int32_t *cell, float *off_m, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    Geometry g;
    HACC_TRY(make_ci_geometry(ctx, box, r_cut, &g));
    HACC_TRY(check_particles(ctx, n, off_m, nullptr));
    if (n > 0 && (!pos64 || !cell)) return set_error(ctx, HACC_EINVAL, "pos64 or cell is NULL");
    HACC_CUDA(ci_from_f64(g, n, pos64, mass, cell, reinterpret_cast<float4 *>(off_m), ctx->d_flags,
                          reinterpret_cast<cudaStream_t>(stream)),
              "cell/offset split");
    return HACC_OK;
}

hacc_status hacc_ci_to_f64(hacc_ctx *ctx, const hacc_box *box, float r_cut, int64_t n, const int32_t *cell,
                           const float *off_m, double *pos64, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    Geometry g;
    HACC_TRY(make_ci_geometry(ctx, box, r_cut, &g));
    HACC_TRY(check_particles(ctx, n, off_m, nullptr));
    if (n > 0 && (!pos64 || !cell)) return set_error(ctx, HACC_EINVAL, "pos64 or cell is NULL");
    HACC_CUDA(ci_to_f64(g, n, cell, reinterpret_cast<const float4 *>(off_m), pos64,
                        reinterpret_cast<cudaStream_t>(stream)),
              "cell/offset join");
    return HACC_OK;
}

namespace {
hacc_status ci_force(hacc_ctx *ctx, const Geometry &g, const ForceConsts &fc, Work *w, int mode, float4 *out,
                     float4 *vel, float hk, cudaStream_t s) {
    ForceLaunch fl;
    fl.pos = w->Ps;
    fl.items = w->b.items;
    fl.n_items = w->b.n_items;
    fl.cell_start = w->b.cell_start;
    fl.work_counter = w->counter;
    fl.mode = mode;
    fl.out = out;
    fl.perm = w->b.perm;
    fl.vel = w->Vs;
    fl.pos_next = nullptr;
    fl.h_kick = hk;
    fl.h_drift = 0.f;
    fl.phi_out = nullptr;
    fl.within = nullptr;
    fl.mass_flag = w->b.mass_flag;
    fl.ids = w->b.perm;
    fl.vel_pool = vel;
    fl.flags = ctx->d_flags;
    fl.cell_offset = true;
    fl.w = (float)ci_step(g);
    fl.delta = (float)ci_rem(g);
    HACC_CUDA(sr_force_launch(g, fc, fl, ctx->num_sms, s), "short-range force launch (cell/offset)");
    ctx->force_launches++;
    return HACC_OK;
}
}  // namespace

hacc_status hacc_sr_force_ci(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                             const int32_t *cell, const float *off_m, float *acc, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    Geometry g;
    HACC_TRY(make_ci_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, off_m, acc));
    if (n > 0 && (!cell || !acc)) return set_error(ctx, HACC_EINVAL, "cell or acc is NULL");
    if (n == 0) return HACC_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, false, s, &w));
    // no stream: the cell ids are the keys as stored (cell and off_m are not written)
    HACC_CUDA(bin_build_ci(g, n, const_cast<int32_t *>(cell), reinterpret_cast<float4 *>(const_cast<float *>(off_m)),
                           nullptr, 0.0, w.P, w.b, ctx->d_flags, s),
              "binning");
    HACC_CUDA(gather_sorted(n, w.b.perm, w.P, w.Ps, nullptr, nullptr, nullptr, nullptr, s), "gather");
    return ci_force(ctx, g, fc, &w, kModeForce, reinterpret_cast<float4 *>(acc), nullptr, 0.f, s);
}

hacc_status hacc_diagnostics_ci(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                                const int32_t *cell, const float *off_m, const float *vel, double *out,
                                hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split || !out) return set_error(ctx, HACC_EINVAL, "split or out is NULL");
    Geometry g;
    HACC_TRY(make_ci_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, off_m, vel));
    if (n > 0 && (!cell || !vel)) return set_error(ctx, HACC_EINVAL, "cell or vel is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    HACC_CUDA(cudaMemsetAsync(out, 0, 8 * sizeof(double), s), "clearing diagnostics");
    if (n == 0) return HACC_OK;
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, true, s, &w));
    HACC_CUDA(bin_build_ci(g, n, const_cast<int32_t *>(cell), reinterpret_cast<float4 *>(const_cast<float *>(off_m)),
                           nullptr, 0.0, w.P, w.b, ctx->d_flags, s),
              "binning");
    HACC_CUDA(gather_sorted(n, w.b.perm, w.P, w.Ps, reinterpret_cast<const float4 *>(vel), w.Vs, nullptr, nullptr, s),
              "gather");
    ForceLaunch fl;
    fl.pos = w.Ps;
    fl.items = w.b.items;
    fl.n_items = w.b.n_items;
    fl.cell_start = w.b.cell_start;
    fl.work_counter = w.counter;
    fl.mode = kModePotential;
    fl.out = nullptr;
    fl.perm = nullptr;
    fl.vel = nullptr;
    fl.pos_next = nullptr;
    fl.h_kick = 0.f;
    fl.h_drift = 0.f;
    fl.phi_out = w.phi;
    fl.within = nullptr;
    fl.mass_flag = w.b.mass_flag;
    fl.flags = ctx->d_flags;
    fl.cell_offset = true;
    fl.w = (float)ci_step(g);
    fl.delta = (float)ci_rem(g);
    HACC_CUDA(sr_force_launch(g, fc, fl, ctx->num_sms, s), "pair potential (cell/offset)");
    HACC_CUDA(diag_reduce(n, w.Ps, w.Vs, w.phi, out, s), "diagnostics");
    HACC_CUDA(diag_mass_moment_ci(n, cell, reinterpret_cast<const float4 *>(off_m), g.nc, ci_step(g), out + 5, s),
              "mass moment");
    return HACC_OK;
}

hacc_status hacc_subcycle_ci(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n, int32_t *cell,
                             float *off_m, float *vel, double dt, int32_t n_sub, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    if (n_sub < 1 || !std::isfinite(dt)) return set_error(ctx, HACC_EINVAL, "n_sub >= 1 and finite dt required");
    Geometry g;
    HACC_TRY(make_ci_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, off_m, vel));
    if (n > 0 && (!cell || !vel)) return set_error(ctx, HACC_EINVAL, "cell or vel is NULL");
    if (n == 0) return HACC_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, true, s, &w));
    float4 *off = reinterpret_cast<float4 *>(off_m);
    float4 *v = reinterpret_cast<float4 *>(vel);
    const double h = dt / n_sub;
    for (int k = 0; k < n_sub; ++k) {
        // stream (FP64 on the global position: h/2 opening, then h fusing two halves), rebin
        HACC_CUDA(bin_build_ci(g, n, cell, off, v, k == 0 ? 0.5 * h : h, w.P, w.b, ctx->d_flags, s), "binning");
        HACC_CUDA(gather_sorted(n, w.b.perm, w.P, w.Ps, v, w.Vs, nullptr, nullptr, s), "gather");
        // kick h (FP32), velocities back to input order
        HACC_TRY(ci_force(ctx, g, fc, &w, kModeKick, nullptr, v, (float)h, s));
    }
    HACC_CUDA(drift_ci(g, n, cell, off, v, 0.5 * h, ctx->d_flags, s), "closing stream");
    return HACC_OK;
}

namespace {

// One event of the multi-level step: its time and the kick of each count.
struct MlEvent {
    double t;
    KickTable kt;
};

// Events (2k+1)/(2l) dt, k < l, over the kick counts l that occur, in time
// order with duplicates merged (exact reduced fractions).
std::vector<MlEvent> ml_schedule(const int *present, int lmax, double dt) {
    std::vector<std::pair<int64_t, int64_t>> ev;
    for (int l = 1; l <= lmax; ++l) {
        if (!present[l]) continue;
        for (int k = 0; k < l; ++k) {
            int64_t a = 2 * k + 1, b = 2 * l, x = a, y = b;
            while (y) { int64_t t = x % y; x = y; y = t; }
            a /= x;
            b /= x;
            bool dup = false;
            for (auto &e : ev) dup |= (e.first == a && e.second == b);
            if (!dup) ev.emplace_back(a, b);
        }
    }
    std::sort(ev.begin(), ev.end(), [](const std::pair<int64_t, int64_t> &p, const std::pair<int64_t, int64_t> &q) {
        return p.first * q.second < q.first * p.second;
    });
    std::vector<MlEvent> out;
    for (auto &e : ev) {
        MlEvent m;
        m.t = dt * (double)e.first / (double)e.second;
        for (int l = 0; l <= kMaxLevels; ++l) {
            m.kt.h[l] = 0.0f;
            if (l >= 1 && l <= lmax && present[l] && (2 * l * e.first) % e.second == 0 &&
                ((2 * l * e.first) / e.second) % 2 == 1)
                m.kt.h[l] = (float)(dt / l);
        }
        out.push_back(m);
    }
    return out;
}

uint64_t mixk(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}

uint32_t fbits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
}

// Buffers of the multi-level event loop, fixed for one call.
struct MlLoop {
    int64_t n;
    float4 *Ps, *Vs, *Vt, *Ref, *pos_in, *V;
    int32_t *lev_s, *lev_t, *id_s, *id_t;
    unsigned *disp_bits;
    float half_lim;
};

ForceLaunch ml_force(hacc_ctx *ctx, Work &w, const MlLoop &m, const KickTable &kt) {
    ForceLaunch fl;
    fl.pos = m.Ps;
    fl.items = w.ml_items;
    fl.n_items = w.b.n_items;
    fl.cell_start = w.b.cell_start;
    fl.work_counter = w.counter;
    fl.mode = kModeKickLevels;
    fl.out = nullptr;
    fl.perm = nullptr;
    fl.vel = m.Vs;   // kicked in place, sorted order
    fl.pos_next = nullptr;
    fl.h_kick = 0.f;
    fl.h_drift = 0.f;
    fl.phi_out = nullptr;
    fl.within = ctx->counting ? ctx->d_pairs + 1 : nullptr;
    fl.evaluated = ctx->counting ? ctx->d_pairs + 2 : nullptr;
    fl.mass_flag = w.b.mass_flag;
    fl.variant = ctx->variant;
    fl.ids = nullptr;
    fl.vel_pool = nullptr;
    fl.levels = m.lev_s;
    fl.kick = kt;
    fl.flags = ctx->d_flags;
    return fl;
}

// Capture the event loop (streams, drift checks, rebinnings as conditional
// graph nodes, work items, pair-kernel launches, closing stream and scatter)
// as one CUDA graph.  Recorded on the context's own capture streams; nothing
// runs here.
cudaError_t ml_capture(hacc_ctx *ctx, const Geometry &g, const ForceConsts &fc, Work &w, const MlLoop &m,
                       const std::vector<MlEvent> &ev, const std::vector<int> &caps, double dt, cudaGraphExec_t *out,
                       int64_t *launches, int64_t *forces) {
    cudaError_t e;
    if (!ctx->cap_stream) {
        cudaStream_t a = nullptr, b = nullptr;
        if ((e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking)) != cudaSuccess) {
            cudaStreamDestroy(a);
            return e;
        }
        ctx->cap_stream = a;
        ctx->cap_stream2 = b;
    }
    cudaStream_t cs = static_cast<cudaStream_t>(ctx->cap_stream), cs2 = static_cast<cudaStream_t>(ctx->cap_stream2);
    const int64_t l0 = ctx->launches, f0 = ctx->force_launches;
    int64_t body = 0;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    double t_prev = 0.0;
    for (size_t k = 0; k < ev.size() && e == cudaSuccess; ++k) {
        if ((e = stream_sorted(m.n, m.Ps, m.Vs, (float)(ev[k].t - t_prev), m.Ref, m.disp_bits, cs)) != cudaSuccess) break;
        t_prev = ev[k].t;
        cudaStreamCaptureStatus st;
        cudaGraph_t graph = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        if ((e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &graph, &deps, nullptr, &nd)) != cudaSuccess) break;
        cudaGraphConditionalHandle h;
        if ((e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess) break;
        if ((e = ml_decide(m.disp_bits, m.half_lim, h, ctx->d_pairs + 3, ctx->d_flags, cs)) != cudaSuccess) break;
        if ((e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &graph, &deps, nullptr, &nd)) != cudaSuccess) break;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        if ((e = cudaGraphAddNode(&cn, graph, deps, nullptr, nd, &cp)) != cudaSuccess) break;
        if ((e = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            break;
        // the rebinning body: bin the streamed positions, gather everything
        // into the second buffers, move them back
        cudaGraph_t bg = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(cs2, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            break;
        const int64_t b0 = ctx->launches;
        cudaError_t eb = bin_build(g, m.n, m.Ps, nullptr, 0.0f, w.P, w.b, ctx->d_flags, false, cs2,
                                   item_cap_for(ctx, m.n), ctx->split_max, m.lev_s);
        if (eb == cudaSuccess)
            eb = gather_ml(m.n, w.b.perm, w.P, m.Ps, m.Ref, m.Vs, m.Vt, m.lev_s, m.lev_t, m.id_s, m.id_t, cs2);
        body = ctx->launches - b0 + 1;
        if (eb == cudaSuccess)
            eb = ml_commit(m.n, m.Vt, m.Vs, m.lev_t, m.lev_s, m.id_t, m.id_s, m.disp_bits, (unsigned)body,
                           ctx->d_pairs + 4, cs2);
        e = cudaStreamEndCapture(cs2, &bg);
        if (eb != cudaSuccess) e = eb;
        if (e != cudaSuccess) break;
        if ((e = items_kicked(g.ncell, w.b, m.lev_s, ev[k].kt, caps[k], w.ml_items, (int32_t)(m.n + 1),
                              ctx->d_flags, cs)) != cudaSuccess)
            break;
        if ((e = sr_force_launch(g, fc, ml_force(ctx, w, m, ev[k].kt), ctx->num_sms, cs)) != cudaSuccess) break;
        ctx->force_launches++;
    }
    if (e == cudaSuccess) e = stream_sorted(m.n, m.Ps, m.Vs, (float)(dt - t_prev), nullptr, nullptr, cs);
    if (e == cudaSuccess) e = scatter_rows(m.n, m.id_s, m.Ps, m.pos_in, m.Vs, m.V, g.Lf, ctx->d_flags, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    // kernels of the rebinning bodies are counted on the device when they run
    *launches = ctx->launches - l0 - (int64_t)ev.size() * body;
    *forces = ctx->force_launches - f0;
    ctx->launches = l0;
    ctx->force_launches = f0;
    cudaGetLastError();
    return e;
}

}  // namespace

hacc_status hacc_subcycle_ml(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n, float *pos_m,
                             float *vel, double dt, int32_t d, int32_t lmin, int32_t lmax, float skin,
                             int32_t *level_out, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    if (lmax < 1 || lmax > kMaxLevels) return set_error(ctx, HACC_EINVAL, "lmax must be in [1, 16]");
    if (lmin < 1 || lmin > lmax) return set_error(ctx, HACC_EINVAL, "lmin must be in [1, lmax]");
    if (!std::isfinite(dt)) return set_error(ctx, HACC_EINVAL, "dt must be finite");
    if (!(skin >= 0) || !std::isfinite(skin)) return set_error(ctx, HACC_EINVAL, "skin must be finite and >= 0");
    Geometry g;
    HACC_TRY(make_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, pos_m, vel));
    if (n > 0 && !vel) return set_error(ctx, HACC_EINVAL, "vel is NULL");
    if (n == 0) return HACC_OK;
    // the step's mesh: cells at least r_cut (1 + skin) wide where the box allows
    if (box->nc == 0) {
        const int32_t nc = hacc_ml_mesh_cells(g.Ld, split->r_cut, skin);
        g.nc = nc;
        g.ncell = (int64_t)nc * nc * nc;
        g.inv_w = (float)((double)nc / g.Ld);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, true, s, &w, true));
    float4 *pos_in = reinterpret_cast<float4 *>(pos_m);
    float4 *V = reinterpret_cast<float4 *>(vel);
    unsigned *disp_bits = reinterpret_cast<unsigned *>(w.present + kMaxLevels + 1);

    // The mesh is kept while the particles move: as long as none has drifted
    // more than `half` along an axis from where it was binned, every pair
    // within r_cut is still in neighbouring cells (the paper keeps its tree
    // for the whole sub-cycle in the same way, Sec. 3.1).  Between events the
    // sorted arrays are only streamed in place; the largest drift is read at
    // every event and the particles are rebinned only when it passed `half`.
    const double half = 0.5 * (g.Ld / g.nc - (double)split->r_cut);
    float4 *Ps = w.Ps, *Vs = w.Vs, *Vt = w.V2, *Ref = w.R;
    int32_t *lev_s = w.IDs, *lev_t = w.ID, *id_s = w.I1, *id_t = w.I2;   // kick counts start in lev_s, input order
    const int icap = item_cap_for(ctx, n);
    // bin src (wrapped into w.P), then gather every array into its other buffer and swap the two
    auto rebin = [&](const float4 *src, bool first) -> hacc_status {
        if (!first)
            HACC_CUDA(bin_build(g, n, src, nullptr, 0.0f, w.P, w.b, ctx->d_flags, false, s, icap, ctx->split_max,
                                lev_s),
                      "binning");
        HACC_CUDA(gather_ml(n, w.b.perm, w.P, Ps, Ref, first ? V : Vs, Vt, lev_s, lev_t, first ? nullptr : id_s, id_t,
                            s),
                  "gather");
        std::swap(Vs, Vt);
        std::swap(lev_s, lev_t);
        std::swap(id_s, id_t);
        HACC_CUDA(cudaMemsetAsync(disp_bits, 0, sizeof(unsigned), s), "memset");
        return HACC_OK;
    };
    // kick counts from the cell densities at the start of the step
    HACC_CUDA(bin_build(g, n, pos_in, nullptr, 0.0f, w.P, w.b, ctx->d_flags, false, s, icap, ctx->split_max),
              "binning");
    HACC_CUDA(cudaMemsetAsync(w.present, 0, sizeof(int) * (kMaxLevels + 1), s), "memset");
    HACC_CUDA(ml_levels(g, n, w.b, d, lmin, lmax, lev_s, w.present, s), "kick counts");
    if (level_out)
        HACC_CUDA(cudaMemcpyAsync(level_out, lev_s, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s), "levels out");
    HACC_TRY(rebin(pos_in, true));
    int present[kMaxLevels + 1];
    HACC_CUDA(cudaMemcpyAsync(present, w.present, sizeof present, cudaMemcpyDeviceToHost, s), "levels present");
    HACC_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const std::vector<MlEvent> ev = ml_schedule(present, lmax, dt);
    const float half_lim = (float)(half * (1.0 - 1e-5));
    // particles kicked at each event; a small launch splits its cells into
    // smaller items (down to one lane per particle) so that enough warps share it
    std::vector<int> caps(ev.size());
    for (size_t k = 0; k < ev.size(); ++k) {
        int64_t kicked = 0;
        for (int l = 1; l <= lmax; ++l)
            if (ev[k].kt.h[l] != 0.0f) kicked += present[l];
        const int64_t per_item = kicked / ((int64_t)ctx->num_sms * 64);
        caps[k] = (int)std::max<int64_t>(kItemMin, std::min<int64_t>(kItemMax, per_item / 32 * 32));
        if (icap) caps[k] = std::min(caps[k], icap);
    }

    // Without timing or counting the event loop runs as one cached CUDA graph
    // whose rebinnings are conditional nodes set by the drift check on the
    // device: no host round trip per event.
    if (!ctx->timing && !ctx->counting && !ctx->ml_graph_off) {
        const MlLoop m{n, Ps, Vs, Vt, Ref, pos_in, V, lev_s, lev_t, id_s, id_t, disp_bits, half_lim};
        uint64_t key = 0x6d6c67ull;
        key = mixk(key, (uint64_t)n);
        key = mixk(key, (uint64_t)g.nc);
        key = mixk(key, fbits(g.Lf));
        key = mixk(key, fbits(half_lim));
        for (size_t k = 0; k < ev.size(); ++k) {
            uint64_t tb;
            std::memcpy(&tb, &ev[k].t, 8);
            key = mixk(key, tb);
            for (int l = 0; l <= kMaxLevels; ++l) key = mixk(key, fbits(ev[k].kt.h[l]));
            key = mixk(key, (uint64_t)caps[k]);
        }
        key = mixk(key, (uint64_t)ctx->item_cap);
        key = mixk(key, (uint64_t)ctx->split_max);
        uint64_t db;
        std::memcpy(&db, &dt, 8);
        key = mixk(key, db);
        uint32_t fcb[sizeof(ForceConsts) / 4];
        std::memcpy(fcb, &fc, sizeof fcb);
        for (uint32_t v : fcb) key = mixk(key, v);
        for (const void *p : {(const void *)pos_in, (const void *)V, (const void *)ctx->scratch.base, (const void *)Ps,
                              (const void *)Vs, (const void *)Vt, (const void *)lev_s, (const void *)id_s})
            key = mixk(key, (uint64_t)(uintptr_t)p);
        key = mixk(key, (uint64_t)ctx->variant);
        if (!ctx->ml_exec || ctx->ml_key != key) {
            if (ctx->ml_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(ctx->ml_exec));
            ctx->ml_exec = nullptr;
            cudaGraphExec_t exec = nullptr;
            int64_t gl = 0, gf = 0;
            if (ml_capture(ctx, g, fc, w, m, ev, caps, dt, &exec, &gl, &gf) == cudaSuccess) {
                ctx->ml_exec = exec;
                ctx->ml_key = key;
                ctx->ml_launches = gl;
                ctx->ml_forces = gf;
            } else {
                if (exec) cudaGraphExecDestroy(exec);
                ctx->ml_graph_off = true;   // run the loop from the host from now on
            }
        }
        if (ctx->ml_exec) {
            HACC_CUDA(cudaGraphLaunch(static_cast<cudaGraphExec_t>(ctx->ml_exec), s), "cudaGraphLaunch");
            ctx->launches += ctx->ml_launches;
            ctx->force_launches += ctx->ml_forces;
            return HACC_OK;
        }
    }

    // the same loop from the host: one synchronisation per event reads the drift
    double t_prev = 0.0;
    for (size_t k = 0; k < ev.size(); ++k) {
        const MlEvent &e = ev[k];
        HACC_CUDA(stream_sorted(n, Ps, Vs, (float)(e.t - t_prev), Ref, disp_bits, s), "stream");
        t_prev = e.t;
        unsigned bits = 0;
        HACC_CUDA(cudaMemcpyAsync(&bits, disp_bits, sizeof bits, cudaMemcpyDeviceToHost, s), "largest drift");
        HACC_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        float drift;
        std::memcpy(&drift, &bits, sizeof drift);
        if (!std::isfinite(drift)) return set_error(ctx, HACC_EDOMAIN, "non-finite position in the multi-level step");
        if (drift > half_lim) {
            HACC_TRY(rebin(Ps, false));
            ctx->ml_rebins++;
        }
        HACC_CUDA(items_kicked(g.ncell, w.b, lev_s, e.kt, caps[k], w.ml_items, (int32_t)(n + 1), ctx->d_flags, s),
                  "work items");
        const MlLoop m{n, Ps, Vs, Vt, Ref, pos_in, V, lev_s, lev_t, id_s, id_t, disp_bits, half_lim};
        HACC_TRY(launch_force(ctx, g, fc, ml_force(ctx, w, m, e.kt), true, s));
    }
    // last stream, then wrapped positions and velocities back to input order
    HACC_CUDA(stream_sorted(n, Ps, Vs, (float)(dt - t_prev), nullptr, nullptr, s), "closing stream");
    HACC_CUDA(scatter_rows(n, id_s, Ps, pos_in, Vs, V, g.Lf, ctx->d_flags, s), "scatter");
    return HACC_OK;
}

hacc_status hacc_diagnostics(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                             const float *pos_m, const float *vel, double *out, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (!split || !out) return set_error(ctx, HACC_EINVAL, "split or out is NULL");
    Geometry g;
    HACC_TRY(make_sr_geometry(ctx, box, split->r_cut, &g));
    ForceConsts fc;
    HACC_TRY(make_force_consts(ctx, split, g, &fc));
    HACC_TRY(check_particles(ctx, n, pos_m, vel));
    if (n > 0 && !vel) return set_error(ctx, HACC_EINVAL, "vel is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Work w;
    HACC_TRY(prepare_work(ctx, n, g, true, s, &w));
    if (n == 0) {
        HACC_CUDA(cudaMemsetAsync(out, 0, 5 * sizeof(double), s), "clearing diagnostics");
        return HACC_OK;
    }
    const float4 *src = reinterpret_cast<const float4 *>(pos_m);
    HACC_CUDA(bin_build(g, n, src, nullptr, 0.0f, w.P, w.b, ctx->d_flags, true, s, item_cap_for(ctx, n),
                        ctx->split_max),
              "binning");
    HACC_CUDA(gather_sorted(n, w.b.perm, w.P, w.Ps, reinterpret_cast<const float4 *>(vel), w.Vs, nullptr, nullptr, s),
              "gather");
    HACC_TRY(run_sorted_force(ctx, g, fc, &w, kModePotential, nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, nullptr,
                              s));
    HACC_CUDA(diag_reduce(n, w.Ps, w.Vs, w.phi, out, s), "diagnostics");
    return HACC_OK;
}

hacc_status hacc_pm_force(hacc_ctx *ctx, const hacc_box *box, const hacc_pm *pm, int64_t n, const float *pos_m,
                          float *acc, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    HACC_TRY(check_particles(ctx, n, pos_m, acc));
    if (n > 0 && !acc) return set_error(ctx, HACC_EINVAL, "acc is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return pm_accel(ctx, box, pm, 1.0, n, reinterpret_cast<const float4 *>(pos_m), reinterpret_cast<float4 *>(acc),
                    nullptr, 0.0f, s);
}

// The full step (Eq. tstep); open_io / close_io (nullable): host copies
// overlapped with the opening and the closing PM half kick (PmHostIO).
static hacc_status step_impl(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, const hacc_pm *pm,
                             int64_t n, float *pos_m, float *vel, double dt, int32_t n_c, hacc_stream_t stream,
                             const PmHostIO *open_io, const PmHostIO *close_io) {
    if (n_c < 1) return set_error(ctx, HACC_EINVAL, "n_c must be >= 1");
    HACC_TRY(check_particles(ctx, n, pos_m, vel));
    if (n > 0 && !vel) return set_error(ctx, HACC_EINVAL, "vel is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float4 *p = reinterpret_cast<float4 *>(pos_m);
    float4 *v = reinterpret_cast<float4 *>(vel);
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    // M_lr(dt/2): kick by the long-range force
    HACC_TRY(pm_accel(ctx, box, pm, split->G, n, p, nullptr, v, (float)(0.5 * dt), s, nullptr, open_io));
    HACC_TRY(hacc_subcycle(ctx, box, split, n, pos_m, vel, dt, n_c, stream));
    HACC_TRY(pm_accel(ctx, box, pm, split->G, n, p, nullptr, v, (float)(0.5 * dt), s, nullptr, close_io));
    return HACC_OK;
}

hacc_status hacc_step(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, const hacc_pm *pm, int64_t n,
                      float *pos_m, float *vel, double dt, int32_t n_c, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    return step_impl(ctx, box, split, pm, n, pos_m, vel, dt, n_c, stream, nullptr, nullptr);
}

hacc_status hacc_sr_force_host(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                               const float *pos_m, float *acc, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (n < 0 || (n > 0 && (!pos_m || !acc))) return set_error(ctx, HACC_EINVAL, "bad host arrays");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t bytes = (size_t)n * 16;
    HACC_TRY(ensure_io(ctx, 2 * bytes + 512, s));
    char *base = static_cast<char *>(ctx->io_base);
    float *dp = reinterpret_cast<float *>(base);
    float *da = reinterpret_cast<float *>(base + ((bytes + 255) & ~size_t(255)));
    HACC_CUDA(cudaMemcpyAsync(dp, pos_m, bytes, cudaMemcpyHostToDevice, s), "H2D copy");
    HACC_TRY(hacc_sr_force(ctx, box, split, n, dp, da, nullptr, stream));
    HACC_CUDA(cudaMemcpyAsync(acc, da, bytes, cudaMemcpyDeviceToHost, s), "D2H copy");
    return hacc_ctx_sync(ctx, stream);
}

hacc_status hacc_subcycle_host(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n, float *pos_m,
                               float *vel, double dt, int32_t n_sub, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (n < 0 || (n > 0 && (!pos_m || !vel))) return set_error(ctx, HACC_EINVAL, "bad host arrays");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t bytes = (size_t)n * 16;
    HACC_TRY(ensure_io(ctx, 2 * bytes + 512, s));
    char *base = static_cast<char *>(ctx->io_base);
    float *dp = reinterpret_cast<float *>(base);
    float *dv = reinterpret_cast<float *>(base + ((bytes + 255) & ~size_t(255)));
    HACC_CUDA(cudaMemcpyAsync(dp, pos_m, bytes, cudaMemcpyHostToDevice, s), "H2D copy");
    HACC_CUDA(cudaMemcpyAsync(dv, vel, bytes, cudaMemcpyHostToDevice, s), "H2D copy");
    HACC_TRY(hacc_subcycle(ctx, box, split, n, dp, dv, dt, n_sub, stream));
    HACC_CUDA(cudaMemcpyAsync(pos_m, dp, bytes, cudaMemcpyDeviceToHost, s), "D2H copy");
    HACC_CUDA(cudaMemcpyAsync(vel, dv, bytes, cudaMemcpyDeviceToHost, s), "D2H copy");
    return hacc_ctx_sync(ctx, stream);
}

hacc_status hacc_step_host(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, const hacc_pm *pm,
                           int64_t n, float *pos_m, float *vel, double dt, int32_t n_c, hacc_stream_t stream) {
    HACC_TRY(enter(ctx));
    if (n < 0 || (n > 0 && (!pos_m || !vel))) return set_error(ctx, HACC_EINVAL, "bad host arrays");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    size_t bytes = (size_t)n * 16;
    HACC_TRY(ensure_io(ctx, 2 * bytes + 512, s));
    char *base = static_cast<char *>(ctx->io_base);
    float *dp = reinterpret_cast<float *>(base);
    float *dv = reinterpret_cast<float *>(base + ((bytes + 255) & ~size_t(255)));
    // a second stream carries the copies, overlapped with the PM stages: the
    // positions go up chunk by chunk, each chunk deposited as it lands, then
    // the velocities; at the end the positions come down while the closing
    // field is solved and the velocities chunk by chunk as they are kicked
    if (!ctx->io_stream) {
        cudaStream_t a = nullptr;
        HACC_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking), "cudaStreamCreate");
        ctx->io_stream = a;
        for (auto &ev : ctx->io_ev) {
            cudaEvent_t e = nullptr;
            HACC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
            ev = e;
        }
    }
    cudaStream_t aux = static_cast<cudaStream_t>(ctx->io_stream);
    cudaEvent_t ev_start = static_cast<cudaEvent_t>(ctx->io_ev[0]);
    PmHostIO open_io, close_io;
    open_io.copy = close_io.copy = aux;
    for (int c = 0; c < kPmChunks; ++c) open_io.ev[c] = close_io.ev[c] = static_cast<cudaEvent_t>(ctx->io_ev[3 + c]);
    open_io.pos_up = reinterpret_cast<const float4 *>(pos_m);
    open_io.vel_up = reinterpret_cast<const float4 *>(vel);
    close_io.pos_down = reinterpret_cast<float4 *>(pos_m);
    close_io.vel_down = reinterpret_cast<float4 *>(vel);
    // the copy stream starts after the work already queued on the stream
    HACC_CUDA(cudaEventRecord(ev_start, s), "cudaEventRecord");
    HACC_CUDA(cudaStreamWaitEvent(aux, ev_start, 0), "cudaStreamWaitEvent");
    HACC_TRY(step_impl(ctx, box, split, pm, n, dp, dv, dt, n_c, stream, n > 0 ? &open_io : nullptr,
                       n > 0 ? &close_io : nullptr));
    HACC_CUDA(cudaEventRecord(ev_start, aux), "cudaEventRecord");
    HACC_CUDA(cudaStreamWaitEvent(s, ev_start, 0), "cudaStreamWaitEvent");
    return hacc_ctx_sync(ctx, stream);
}

}  // extern "C"
