// Batches of independent boxes in one pass (the serving / batching mode).
//
// Every box of a batch is advanced by the same short-range SKS sub-cycle as
// hacc_subcycle (Sec. 2.5), but all boxes share one binning pass (global cell
// ids = the box's cell base + its local id, so one counting sort covers them
// all) and ONE persistent pair-kernel launch whose warps take work items of
// every box from a single atomic queue (the work queue of Sec. 3.1, one item
// per cell or 128-particle slice of a cell).  The pair kernel writes kicked
// and streamed particles straight back to their pool rows, wrapped.
//
// Within a cell the particles are ordered by pool row, and a box's items only
// read its own cells, so each box's result is bitwise the same whether it runs
// alone or in any mix (and whatever warp takes which item).
//
// hacc_batch_subcycle can capture its n_sub ticks as one CUDA graph; the per-tick
// box tables live in device memory that the graph reads at replay, so a replay
// with new step sizes needs no re-capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hacc_internal.cuh"

namespace hacc {
namespace {

struct BatchWork {
    float4 *P, *Ps, *Vs;
    int32_t *ID, *IDs;
    int *counter;
    BoxDev *tables;  // n_tables x nbox
    BinBuffers b;
};

size_t carve_batch(char *base, int64_t n, int64_t ncell, int64_t table_entries, BatchWork *w) {
    Carver c(base);
    w->P = c.take<float4>(n);
    w->Ps = c.take<float4>(n);
    w->Vs = c.take<float4>(n);
    w->ID = c.take<int32_t>(n);
    w->IDs = c.take<int32_t>(n);
    w->counter = c.take<int>(1);
    w->tables = c.take<BoxDev>(table_entries);
    carve_bin(c, n, ncell, &w->b);
    return c.off + 256;
}

struct Plan {
    int nbox = 0;                 // non-empty boxes
    int64_t n_total = 0, ncell_total = 0;
    std::vector<BoxDev> base;     // geometry and offsets (h, pre, post filled per tick)
};

hacc_status make_plan(hacc_ctx *ctx, const hacc_split *split, int32_t nbox, const hacc_batch_box *boxes, Plan *pl) {
    if (nbox < 0 || (nbox > 0 && !boxes)) return set_error(ctx, HACC_EINVAL, "bad box list");
    pl->base.clear();
    int64_t n_total = 0, ncell_total = 0;
    for (int b = 0; b < nbox; ++b) {
        const hacc_batch_box &bb = boxes[b];
        if (bb.n < 0 || bb.offset < 0) return set_error(ctx, HACC_EINVAL, "box with negative size or offset");
        if (bb.n == 0) continue;
        hacc_box hb{bb.L, bb.nc, 0};
        Geometry g;
        HACC_STATUS_RETURN(make_geometry(ctx, &hb, split->r_cut, &g));
        BoxDev d;
        std::memset(&d, 0, sizeof d);
        d.L = g.Lf;
        d.inv_w = g.inv_w;
        d.Ld = g.Ld;
        d.nc = g.nc;
        d.cell_base = (int)ncell_total;
        d.part_base = (int)n_total;
        d.n = (int)bb.n;
        d.row_off = bb.offset;
        d.orig = b;
        n_total += bb.n;
        ncell_total += g.ncell;
        if (n_total >= ((int64_t)1 << 31) || ncell_total >= ((int64_t)1 << 31) || bb.offset + bb.n >= ((int64_t)1 << 31))
            return set_error(ctx, HACC_EINVAL, "batch too large (2^31 particles, cells or rows)");
        pl->base.push_back(d);
    }
    pl->nbox = (int)pl->base.size();
    pl->n_total = n_total;
    pl->ncell_total = ncell_total;
    if (pl->nbox >= (1 << 23)) return set_error(ctx, HACC_EINVAL, "too many boxes");
    return HACC_OK;
}

hacc_status ensure_staging(hacc_ctx *ctx, size_t bytes) {
    if (ctx->stage_cap >= bytes) {
        if (ctx->stage_event) cudaEventSynchronize(ctx->stage_event);  // last upload done reading it
        return HACC_OK;
    }
    if (ctx->stage_event) cudaEventSynchronize(ctx->stage_event);
    if (ctx->stage) cudaFreeHost(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_cap = 0;
    if (cudaHostAlloc(&ctx->stage, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, HACC_ENOMEM, "cudaHostAlloc of the box-table staging failed");
    }
    ctx->stage_cap = bytes;
    if (!ctx->stage_event && cudaEventCreateWithFlags(&ctx->stage_event, cudaEventDisableTiming) != cudaSuccess)
        return set_error(ctx, HACC_ECUDA, "cudaEventCreate failed");
    return HACC_OK;
}

uint64_t mix(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}

// Geometry of a batch as the tuner keys it: every box's side, cells and size.
uint64_t plan_key(const Plan &pl) {
    uint64_t key = 0x7475ull;
    key = mix(key, (uint64_t)pl.nbox);
    for (const BoxDev &d : pl.base) {
        uint32_t lb;
        std::memcpy(&lb, &d.L, 4);
        key = mix(key, lb);
        key = mix(key, (uint64_t)d.nc);
        key = mix(key, (uint64_t)d.n);
    }
    return key;
}

// Launch shape of a batched pass: the tuned one for this batch geometry, else
// the context's variant and item cap.
struct Shape {
    int variant, cap, order;
};

Shape batch_shape(const hacc_ctx *ctx, const Plan &pl) {
    if (ctx->btune_key && ctx->btune_key == plan_key(pl))
        return Shape{ctx->btune_variant, ctx->btune_cap, ctx->btune_order};
    return Shape{ctx->variant, item_cap_for(ctx, pl.n_total), ctx->queue_order};
}

// One tick on the device tables `tab` (nbox entries).
hacc_status run_tick(hacc_ctx *ctx, const ForceConsts &fc, const Plan &pl, const BoxDev *tab, float4 *pos_pool,
                     float4 *vel_pool, const BatchWork &w, cudaStream_t s) {
    const Shape sh = batch_shape(ctx, pl);
    HACC_CUDA_RETURN(bin_build_batch(pl.nbox, tab, pl.n_total, pl.ncell_total, pos_pool, vel_pool, w.P, w.ID, w.b,
                                     ctx->d_flags, s, sh.cap, ctx->split_max),
                     "batched binning");
    HACC_CUDA_RETURN(gather_sorted(pl.n_total, w.b.perm, w.P, w.Ps, nullptr, nullptr, w.ID, w.IDs, s), "gather");
    HACC_CUDA_RETURN(gather_sorted(pl.n_total, w.IDs, vel_pool, w.Vs, nullptr, nullptr, nullptr, nullptr, s),
                     "gather velocities");
    ForceLaunch fl;
    fl.pos = w.Ps;
    fl.items = w.b.items;
    fl.n_items = w.b.n_items;
    fl.cell_start = w.b.cell_start;
    fl.work_counter = w.counter;
    fl.mode = kModeBatch;
    fl.out = nullptr;
    fl.perm = nullptr;
    fl.vel = w.Vs;
    fl.pos_next = nullptr;
    fl.h_kick = 0.f;
    fl.h_drift = 0.f;
    fl.phi_out = nullptr;
    fl.within = ctx->counting ? ctx->d_pairs + 1 : nullptr;
    fl.evaluated = ctx->counting ? ctx->d_pairs + 2 : nullptr;
    fl.mass_flag = w.b.mass_flag;
    fl.variant = sh.variant;
    if (sh.order && pl.n_total >= kHeavyFirstMinN) {
        HACC_CUDA_RETURN(items_heavy_first(w.b, max_items(pl.n_total, pl.ncell_total), s), "item order");
        fl.order = w.b.order;
    }
    fl.boxes = tab;
    fl.ids = w.IDs;
    fl.pos_pool = pos_pool;
    fl.vel_pool = vel_pool;
    fl.flags = ctx->d_flags;
    Geometry g;  // unused by the batched kernel (per-item geometry comes from the table)
    g.Lf = 1.f;
    g.Ld = 1.0;
    g.nc = 3;
    g.ncell = 27;
    g.inv_w = 3.f;
    if (ctx->counting)
        HACC_CUDA_RETURN(candidate_count_batch(pl.ncell_total, tab, pl.nbox, w.b.cell_start, ctx->d_pairs, s),
                         "batched candidate count");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    HACC_CUDA_RETURN(cudaStreamIsCapturing(s, &cap), "cudaStreamIsCapturing");
    if (cap == cudaStreamCaptureStatusNone) return timed_force_launch(ctx, g, fc, fl, s);
    HACC_CUDA_RETURN(sr_force_launch(g, fc, fl, ctx->num_sms, s), "batched pair force");
    ctx->force_launches++;
    return HACC_OK;
}

}  // namespace

size_t batch_tick_scratch_bytes(int64_t n_total, int64_t ncell_total, int64_t nbox) {
    BatchWork w;
    return carve_batch(nullptr, n_total, ncell_total, nbox, &w);
}

void batch_destroy(hacc_ctx *ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(ctx->graph_exec));
    ctx->graph_exec = nullptr;
    if (ctx->stage_event) cudaEventSynchronize(ctx->stage_event);
    if (ctx->stage) cudaFreeHost(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_cap = 0;
    if (ctx->stage_event) cudaEventDestroy(ctx->stage_event);
    ctx->stage_event = nullptr;
}

}  // namespace hacc

using namespace hacc;

extern "C" size_t hacc_batch_scratch_bytes(const hacc_split *split, int32_t nbox, const hacc_batch_box *boxes) {
    if (!split) return 0;
    Plan pl;
    if (make_plan(nullptr, split, nbox, boxes, &pl) != HACC_OK || pl.nbox == 0) return 0;
    return batch_tick_scratch_bytes(pl.n_total, pl.ncell_total, pl.nbox);
}

extern "C" hacc_status hacc_batch_tick(hacc_ctx *ctx, const hacc_split *split, int32_t nbox,
                                       const hacc_batch_box *boxes, float *pos_pool, float *vel_pool,
                                       hacc_stream_t stream) {
    HACC_STATUS_RETURN(hacc_enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    Plan pl;
    HACC_STATUS_RETURN(make_plan(ctx, split, nbox, boxes, &pl));
    if (pl.nbox == 0) return HACC_OK;
    if (!pos_pool || !vel_pool || ((uintptr_t)pos_pool & 15u) || ((uintptr_t)vel_pool & 15u))
        return set_error(ctx, HACC_EINVAL, "pool arrays NULL or not 16-byte aligned");
    Geometry g0;  // the force constants do not depend on the box
    g0.Lf = pl.base[0].L;
    g0.Ld = pl.base[0].Ld;
    g0.nc = pl.base[0].nc;
    g0.ncell = (int64_t)g0.nc * g0.nc * g0.nc;
    g0.inv_w = pl.base[0].inv_w;
    ForceConsts fc;
    HACC_STATUS_RETURN(make_force_consts(ctx, split, g0, &fc));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BatchWork w;
    size_t need = carve_batch(nullptr, pl.n_total, pl.ncell_total, pl.nbox, &w);
    HACC_STATUS_RETURN(ensure_scratch(ctx, need, s));
    carve_batch(ctx->scratch.base, pl.n_total, pl.ncell_total, pl.nbox, &w);
    HACC_STATUS_RETURN(ensure_staging(ctx, sizeof(BoxDev) * pl.nbox));
    BoxDev *st = static_cast<BoxDev *>(ctx->stage);
    for (int b = 0, k = 0; b < nbox; ++b) {
        if (boxes[b].n == 0) continue;
        BoxDev d = pl.base[k];
        const float h = (float)boxes[b].dt;
        d.h = h;
        d.pre = (boxes[b].flags & HACC_TICK_FIRST) ? 0.5f * h : 0.0f;
        d.post = (boxes[b].flags & HACC_TICK_LAST) ? 0.5f * h : h;
        st[k++] = d;
    }
    HACC_CUDA_RETURN(cudaMemcpyAsync(w.tables, st, sizeof(BoxDev) * pl.nbox, cudaMemcpyHostToDevice, s),
                     "box table upload");
    HACC_CUDA_RETURN(cudaEventRecord(ctx->stage_event, s), "cudaEventRecord");
    return run_tick(ctx, fc, pl, w.tables, reinterpret_cast<float4 *>(pos_pool), reinterpret_cast<float4 *>(vel_pool),
                    w, s);
}

// Item caps the batched tuner tries (0: cell-wide items of up to kItemMax);
// setting k = (cap index * 2 + queue order) * kForceVariants + variant.
static const int kTuneCaps[] = {0, 32, 64, 96, 128, 160};
static constexpr int kTuneSettings = (int)(sizeof(kTuneCaps) / sizeof(kTuneCaps[0])) * 2 * kForceVariants;
static_assert(kTuneSettings == HACC_BATCH_TUNE_SETTINGS, "tuner table size");

extern "C" hacc_status hacc_batch_tune(hacc_ctx *ctx, const hacc_split *split, int32_t nbox,
                                       const hacc_batch_box *boxes, const float *pos_pool, const float *vel_pool,
                                       int32_t reps, double *times_ms, int32_t *chosen, hacc_stream_t stream) {
    HACC_STATUS_RETURN(hacc_enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    if (reps < 1) return set_error(ctx, HACC_EINVAL, "reps must be >= 1");
    Plan pl;
    HACC_STATUS_RETURN(make_plan(ctx, split, nbox, boxes, &pl));
    if (pl.nbox == 0) return HACC_OK;
    if (!pos_pool || !vel_pool || ((uintptr_t)pos_pool & 15u) || ((uintptr_t)vel_pool & 15u))
        return set_error(ctx, HACC_EINVAL, "pool arrays NULL or not 16-byte aligned");
    for (int b = 0; b < nbox; ++b)
        if (!std::isfinite(boxes[b].dt)) return set_error(ctx, HACC_EINVAL, "dt must be finite");
    Geometry g0;
    g0.Lf = pl.base[0].L;
    g0.Ld = pl.base[0].Ld;
    g0.nc = pl.base[0].nc;
    g0.ncell = (int64_t)g0.nc * g0.nc * g0.nc;
    g0.inv_w = pl.base[0].inv_w;
    ForceConsts fc;
    HACC_STATUS_RETURN(make_force_consts(ctx, split, g0, &fc));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the batched tick as it runs, on scratch copies of the pools (the tick
    // writes its results back to the pool rows)
    int64_t rows = 0;
    for (const BoxDev &d : pl.base) rows = std::max<int64_t>(rows, d.row_off + d.n);
    BatchWork w;
    auto carve = [&](char *base, float4 **pc, float4 **vc) {
        Carver c(base);
        c.off = carve_batch(base, pl.n_total, pl.ncell_total, pl.nbox, &w);
        *pc = c.take<float4>(rows);
        *vc = c.take<float4>(rows);
        return c.off + 256;
    };
    float4 *pc = nullptr, *vc = nullptr;
    HACC_STATUS_RETURN(ensure_scratch(ctx, carve(nullptr, &pc, &vc), s));
    carve(ctx->scratch.base, &pc, &vc);
    HACC_STATUS_RETURN(ensure_staging(ctx, sizeof(BoxDev) * pl.nbox));
    BoxDev *st = static_cast<BoxDev *>(ctx->stage);
    for (int b = 0, q = 0; b < nbox; ++b) {
        if (boxes[b].n == 0) continue;
        BoxDev d = pl.base[q];
        const float h = (float)boxes[b].dt;   // one whole sub-cycle of step dt
        d.h = h;
        d.pre = 0.5f * h;
        d.post = 0.5f * h;
        st[q++] = d;
    }
    HACC_CUDA_RETURN(cudaMemcpyAsync(w.tables, st, sizeof(BoxDev) * pl.nbox, cudaMemcpyHostToDevice, s),
                     "box table upload");
    HACC_CUDA_RETURN(cudaEventRecord(ctx->stage_event, s), "cudaEventRecord");
    cudaEvent_t e0, e1;
    HACC_CUDA_RETURN(cudaEventCreate(&e0), "cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(ctx, HACC_ECUDA, "cudaEventCreate failed");
    }
    const uint64_t key = plan_key(pl);
    const uint64_t saved_key = ctx->btune_key;
    const int saved_v = ctx->btune_variant, saved_cap = ctx->btune_cap, saved_order = ctx->btune_order;
    const bool saved_timing = ctx->timing, saved_counting = ctx->counting;
    ctx->timing = ctx->counting = false;
    hacc_status res = HACC_OK;
    double best = 1e300;
    int best_k = -1;
    const size_t bytes = sizeof(float4) * (size_t)rows;
    for (int k = 0; k < kTuneSettings && res == HACC_OK; ++k) {
        ctx->btune_key = key;   // run_tick takes the shape under test
        ctx->btune_cap = kTuneCaps[k / (2 * kForceVariants)];
        ctx->btune_order = (k / kForceVariants) % 2;
        ctx->btune_variant = k % kForceVariants;
        double total = 0.0;
        for (int r = 0; r <= reps && res == HACC_OK; ++r) {   // r = 0: warm-up
            cudaError_t e = cudaMemcpyAsync(pc, pos_pool, bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(vc, vel_pool, bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e != cudaSuccess) {
                res = check_cuda(ctx, e, "tuner pool copy");
                break;
            }
            res = run_tick(ctx, fc, pl, w.tables, pc, vc, w, s);
            if (res != HACC_OK) break;
            e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                res = check_cuda(ctx, e, "tuner timing");
                break;
            }
            if (r > 0) total += ms;
        }
        if (res != HACC_OK) break;
        const double per = total / reps;
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
    if (res != HACC_OK) {
        ctx->btune_key = saved_key;
        ctx->btune_variant = saved_v;
        ctx->btune_cap = saved_cap;
        ctx->btune_order = saved_order;
        return res;
    }
    ctx->btune_key = key;
    ctx->btune_cap = kTuneCaps[best_k / (2 * kForceVariants)];
    ctx->btune_order = (best_k / kForceVariants) % 2;
    ctx->btune_variant = best_k % kForceVariants;
    if (chosen) *chosen = best_k;
    return HACC_OK;
}

extern "C" hacc_status hacc_batch_diagnostics(hacc_ctx *ctx, const hacc_split *split, int32_t nbox,
                                              const hacc_batch_box *boxes, const float *pos_pool,
                                              const float *vel_pool, double *out, hacc_stream_t stream) {
    HACC_STATUS_RETURN(hacc_enter(ctx));
    if (!split || (nbox > 0 && !out)) return set_error(ctx, HACC_EINVAL, "split or out is NULL");
    Plan pl;
    HACC_STATUS_RETURN(make_plan(ctx, split, nbox, boxes, &pl));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (nbox > 0) HACC_CUDA_RETURN(cudaMemsetAsync(out, 0, sizeof(double) * 5 * nbox, s), "clearing diagnostics");
    if (pl.nbox == 0) return HACC_OK;
    if (!pos_pool || !vel_pool || ((uintptr_t)pos_pool & 15u) || ((uintptr_t)vel_pool & 15u))
        return set_error(ctx, HACC_EINVAL, "pool arrays NULL or not 16-byte aligned");
    Geometry g0;
    g0.Lf = pl.base[0].L;
    g0.Ld = pl.base[0].Ld;
    g0.nc = pl.base[0].nc;
    g0.ncell = (int64_t)g0.nc * g0.nc * g0.nc;
    g0.inv_w = pl.base[0].inv_w;
    ForceConsts fc;
    HACC_STATUS_RETURN(make_force_consts(ctx, split, g0, &fc));
    // scratch: the batched tick's buffers, then the potentials and the partial sums
    BatchWork w;
    auto carve = [&](char *base, float **phi, double **partial) {
        Carver c(base);
        c.off = carve_batch(base, pl.n_total, pl.ncell_total, pl.nbox, &w);
        *phi = c.take<float>(pl.n_total);
        *partial = c.take<double>((size_t)pl.nbox * kDiagParts * 5);
        return c.off + 256;
    };
    float *phi = nullptr;
    double *partial = nullptr;
    HACC_STATUS_RETURN(ensure_scratch(ctx, carve(nullptr, &phi, &partial), s));
    carve(ctx->scratch.base, &phi, &partial);
    HACC_STATUS_RETURN(ensure_staging(ctx, sizeof(BoxDev) * pl.nbox));
    BoxDev *st = static_cast<BoxDev *>(ctx->stage);
    for (int q = 0; q < pl.nbox; ++q) st[q] = pl.base[q];   // no stream, no kick
    HACC_CUDA_RETURN(cudaMemcpyAsync(w.tables, st, sizeof(BoxDev) * pl.nbox, cudaMemcpyHostToDevice, s),
                     "box table upload");
    HACC_CUDA_RETURN(cudaEventRecord(ctx->stage_event, s), "cudaEventRecord");
    float4 *pp = const_cast<float4 *>(reinterpret_cast<const float4 *>(pos_pool));
    float4 *vp = const_cast<float4 *>(reinterpret_cast<const float4 *>(vel_pool));
    // the pools are only read: the binning writes wrapped copies to scratch
    HACC_CUDA_RETURN(bin_build_batch(pl.nbox, w.tables, pl.n_total, pl.ncell_total, pp, vp, w.P, w.ID, w.b,
                                     ctx->d_flags, s, item_cap_for(ctx, pl.n_total), ctx->split_max),
                     "batched binning");
    HACC_CUDA_RETURN(gather_sorted(pl.n_total, w.b.perm, w.P, w.Ps, nullptr, nullptr, w.ID, w.IDs, s), "gather");
    HACC_CUDA_RETURN(gather_sorted(pl.n_total, w.IDs, vp, w.Vs, nullptr, nullptr, nullptr, nullptr, s),
                     "gather velocities");
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
    fl.phi_out = phi;
    fl.within = nullptr;
    fl.mass_flag = w.b.mass_flag;
    fl.variant = ctx->variant;
    fl.boxes = w.tables;
    fl.ids = w.IDs;
    fl.flags = ctx->d_flags;
    HACC_CUDA_RETURN(sr_force_launch(g0, fc, fl, ctx->num_sms, s), "batched pair potential");
    HACC_CUDA_RETURN(diag_reduce_batch(pl.nbox, w.tables, w.b.cell_start, w.Ps, w.Vs, phi, partial, out, s),
                     "batched diagnostics");
    return HACC_OK;
}

extern "C" hacc_status hacc_batch_subcycle(hacc_ctx *ctx, const hacc_split *split, int32_t nbox,
                                           const hacc_batch_box *boxes, float *pos_pool, float *vel_pool,
                                           int32_t n_sub, int32_t use_graph, hacc_stream_t stream) {
    HACC_STATUS_RETURN(hacc_enter(ctx));
    if (!split) return set_error(ctx, HACC_EINVAL, "split is NULL");
    if (n_sub < 1) return set_error(ctx, HACC_EINVAL, "n_sub must be >= 1");
    Plan pl;
    HACC_STATUS_RETURN(make_plan(ctx, split, nbox, boxes, &pl));
    if (pl.nbox == 0) return HACC_OK;
    if (!pos_pool || !vel_pool || ((uintptr_t)pos_pool & 15u) || ((uintptr_t)vel_pool & 15u))
        return set_error(ctx, HACC_EINVAL, "pool arrays NULL or not 16-byte aligned");
    for (int b = 0; b < nbox; ++b)
        if (!std::isfinite(boxes[b].dt)) return set_error(ctx, HACC_EINVAL, "dt must be finite");
    Geometry g0;  // the force constants do not depend on the box
    g0.Lf = pl.base[0].L;
    g0.Ld = pl.base[0].Ld;
    g0.nc = pl.base[0].nc;
    g0.ncell = (int64_t)g0.nc * g0.nc * g0.nc;
    g0.inv_w = pl.base[0].inv_w;
    ForceConsts fc;
    HACC_STATUS_RETURN(make_force_consts(ctx, split, g0, &fc));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t entries = (int64_t)pl.nbox * n_sub;
    BatchWork w;
    size_t need = carve_batch(nullptr, pl.n_total, pl.ncell_total, entries, &w);
    HACC_STATUS_RETURN(ensure_scratch(ctx, need, s));
    carve_batch(ctx->scratch.base, pl.n_total, pl.ncell_total, entries, &w);
    // per-tick tables: SKS with the outer half streams fused into the binning
    // of the first tick and the epilogue of the last
    HACC_STATUS_RETURN(ensure_staging(ctx, sizeof(BoxDev) * entries));
    BoxDev *st = static_cast<BoxDev *>(ctx->stage);
    for (int k = 0; k < n_sub; ++k)
        for (int b = 0, q = 0; b < nbox; ++b) {
            if (boxes[b].n == 0) continue;
            BoxDev d = pl.base[q];
            const float h = (float)(boxes[b].dt / n_sub);
            d.h = h;
            d.pre = k == 0 ? 0.5f * h : 0.0f;
            d.post = k == n_sub - 1 ? 0.5f * h : h;
            st[(int64_t)k * pl.nbox + q++] = d;
        }
    HACC_CUDA_RETURN(cudaMemcpyAsync(w.tables, st, sizeof(BoxDev) * entries, cudaMemcpyHostToDevice, s),
                     "box table upload");
    HACC_CUDA_RETURN(cudaEventRecord(ctx->stage_event, s), "cudaEventRecord");
    float4 *pp = reinterpret_cast<float4 *>(pos_pool);
    float4 *vp = reinterpret_cast<float4 *>(vel_pool);
    // the legacy default stream cannot be captured: run directly there
    if (!use_graph || s == nullptr) {
        for (int k = 0; k < n_sub; ++k)
            HACC_STATUS_RETURN(run_tick(ctx, fc, pl, w.tables + (int64_t)k * pl.nbox, pp, vp, w, s));
        return HACC_OK;
    }
    uint64_t key = 0x51ed27ull;
    key = mix(key, (uint64_t)pl.nbox);
    key = mix(key, (uint64_t)n_sub);
    for (const BoxDev &d : pl.base) {
        uint32_t lb;
        std::memcpy(&lb, &d.L, 4);
        key = mix(key, lb);
        key = mix(key, (uint64_t)d.nc);
        key = mix(key, (uint64_t)d.n);
        key = mix(key, (uint64_t)d.row_off);
    }
    uint32_t fcb[sizeof(ForceConsts) / 4];
    std::memcpy(fcb, &fc, sizeof fcb);
    for (uint32_t v : fcb) key = mix(key, v);
    key = mix(key, (uint64_t)(uintptr_t)pp);
    key = mix(key, (uint64_t)(uintptr_t)vp);
    key = mix(key, (uint64_t)(uintptr_t)ctx->scratch.base);
    const Shape sh = batch_shape(ctx, pl);
    key = mix(key, (uint64_t)sh.variant);
    key = mix(key, (uint64_t)ctx->counting);
    key = mix(key, (uint64_t)sh.cap);
    key = mix(key, (uint64_t)ctx->split_max);
    key = mix(key, (uint64_t)sh.order);
    key = mix(key, (uint64_t)(uintptr_t)s);
    if (!ctx->graph_exec || ctx->graph_key != key) {
        if (ctx->graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(ctx->graph_exec));
        ctx->graph_exec = nullptr;
        const int64_t launches0 = ctx->launches, forces0 = ctx->force_launches;
        HACC_CUDA_RETURN(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        hacc_status r = HACC_OK;
        for (int k = 0; k < n_sub && r == HACC_OK; ++k)
            r = run_tick(ctx, fc, pl, w.tables + (int64_t)k * pl.nbox, pp, vp, w, s);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (r != HACC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (ce != cudaSuccess) return check_cuda(ctx, ce, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return check_cuda(ctx, ce, "cudaGraphInstantiate");
        ctx->graph_exec = exec;
        ctx->graph_key = key;
        ctx->graph_launches = ctx->launches - launches0;
        ctx->graph_forces = ctx->force_launches - forces0;
        ctx->launches = launches0;
        ctx->force_launches = forces0;
    }
    HACC_CUDA_RETURN(cudaGraphLaunch(static_cast<cudaGraphExec_t>(ctx->graph_exec), s), "cudaGraphLaunch");
    ctx->launches += ctx->graph_launches;
    ctx->force_launches += ctx->graph_forces;
    return HACC_OK;
}
