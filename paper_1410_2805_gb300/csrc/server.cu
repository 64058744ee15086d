// Serving runtime: continuous batching of short-range runs on one GPU.
//
// Requests (a periodic box of n particles, a sub-cycle step h and a number of
// sub-cycles) queue on the host.  Each tick:
//   1. admits queued runs in arrival order while they fit: their rows come
//      from one device pool (first-fit over a free list of row ranges,
//      coalesced on release -- a long-lived form of the phase-scoped pool of
//      Sec. 2.7), the particles advanced per tick stay within an optional cap,
//      and, when the context has an HBM budget, the row pool plus the scratch
//      that the batched tick of the resident runs will take from the context
//      stay within it;
//   2. advances EVERY resident run by one SKS sub-cycle in one batched pass
//      (hacc_batch_tick: one binning pass, one persistent pair-kernel launch
//      over all boxes), so runs that arrive while others are on the GPU join
//      at the next tick and their work overlaps with the others';
//   3. while that pass runs, admits more queued runs for the next tick and
//      uploads their inputs on a second stream (their rows are not touched by
//      the running pass);
//   4. retires runs whose last sub-cycle ran: copies their rows back to the
//      caller's host arrays and releases the rows.
// The tick waits for the device before returning, so results of retired runs
// are in host memory when it returns.  A run's result does not depend on what
// else was resident (batched results are bitwise the same alone or mixed).
#include <cuda_runtime.h>
#include <stdint.h>

#include <deque>
#include <map>
#include <string>
#include <vector>

#include "hacc_internal.cuh"

struct hacc_server {
    hacc_ctx *ctx = nullptr;
    hacc_split split{};
    float4 *pos = nullptr, *vel = nullptr;   // pool, `rows` rows each
    int64_t rows = 0;
    size_t pool_bytes = 0;
    int64_t max_active = 0;                  // 0: no cap
    std::map<int64_t, int64_t> free_rows;    // offset -> length
    struct Run {
        int64_t id;
        double L;
        int64_t n, ncell;
        float *pos_host, *vel_host;
        double h;
        int32_t steps, done;
        int64_t offset;
    };
    std::deque<Run> queue;
    std::vector<Run> active;                 // resident: done < steps advance, done == steps await retirement
    cudaStream_t copy = nullptr;             // admission uploads and retirement downloads
    cudaEvent_t ev_up = nullptr;             // the last admission upload
    cudaEvent_t ev_tick = nullptr;           // the end of the last batched pass
    bool up_pending = false;
};

namespace {

bool alloc_rows(hacc_server *sv, int64_t n, int64_t *off) {
    for (auto it = sv->free_rows.begin(); it != sv->free_rows.end(); ++it) {
        if (it->second >= n) {
            *off = it->first;
            int64_t rest = it->second - n, start = it->first + n;
            sv->free_rows.erase(it);
            if (rest > 0) sv->free_rows[start] = rest;
            return true;
        }
    }
    return false;
}

void free_rows(hacc_server *sv, int64_t off, int64_t n) {
    auto it = sv->free_rows.emplace(off, n).first;
    auto next = std::next(it);
    if (next != sv->free_rows.end() && it->first + it->second == next->first) {
        it->second += next->second;
        sv->free_rows.erase(next);
    }
    if (it != sv->free_rows.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            sv->free_rows.erase(it);
        }
    }
}

// Particles, cells and boxes of the runs that the next batched pass advances.
struct Load {
    int64_t n = 0, ncell = 0, nbox = 0;
    void add(const hacc_server::Run &r) {
        n += r.n;
        ncell += r.ncell;
        ++nbox;
    }
};

// Whether a run fits next to `load` (the runs of the same pass): the
// per-tick particle cap and, with a context budget, the row pool plus the
// context's scratch for that pass (its arena only grows, so the larger of the
// arena held now and the pass's need).
bool fits(const hacc_server *sv, const Load &load, const hacc_server::Run &r) {
    if (sv->max_active && load.n + r.n > sv->max_active) return false;
    const size_t budget = sv->ctx->budget;
    if (!budget) return true;
    size_t need = hacc::batch_tick_scratch_bytes(load.n + r.n, load.ncell + r.ncell, load.nbox + 1);
    if (need < sv->ctx->scratch.cap) need = sv->ctx->scratch.cap;
    return sv->pool_bytes + need + sv->ctx->io_cap <= budget;
}

// Admit queued runs in arrival order while they fit next to `load`; their
// inputs go up on the copy stream.  On a failed copy the run goes back to
// the front of the queue with its rows released.
hacc_status admit(hacc_server *sv, Load &load, int32_t *admitted) {
    hacc_ctx *ctx = sv->ctx;
    while (!sv->queue.empty()) {
        hacc_server::Run r = sv->queue.front();
        if (!fits(sv, load, r)) break;
        int64_t off;
        if (!alloc_rows(sv, r.n, &off)) break;
        r.offset = off;
        cudaError_t e = cudaMemcpyAsync(sv->pos + off, r.pos_host, (size_t)r.n * 16, cudaMemcpyHostToDevice, sv->copy);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sv->vel + off, r.vel_host, (size_t)r.n * 16, cudaMemcpyHostToDevice, sv->copy);
        if (e != cudaSuccess) {
            free_rows(sv, off, r.n);
            return hacc::check_cuda(ctx, e, "admission copy");
        }
        sv->queue.pop_front();
        sv->active.push_back(r);
        load.add(r);
        sv->up_pending = true;
        ++*admitted;
    }
    if (sv->up_pending) HACC_CUDA_RETURN(cudaEventRecord(sv->ev_up, sv->copy), "cudaEventRecord");
    return HACC_OK;
}

}  // namespace

extern "C" {

hacc_status hacc_server_create(hacc_server **out, hacc_ctx *ctx, const hacc_split *split, size_t pool_bytes,
                               int64_t max_active_particles) {
    if (!out) return HACC_EINVAL;
    *out = nullptr;
    HACC_STATUS_RETURN(hacc::hacc_enter(ctx));
    if (!split || max_active_particles < 0) return hacc::set_error(ctx, HACC_EINVAL, "bad server arguments");
    const int64_t rows = (int64_t)(pool_bytes / 32);
    if (rows < 1) return hacc::set_error(ctx, HACC_EINVAL, "pool too small");
    if (ctx->budget && pool_bytes > ctx->budget)
        return hacc::set_error(ctx, HACC_ENOMEM, "server pool exceeds the context budget");
    hacc_server *sv = new hacc_server();
    sv->ctx = ctx;
    sv->split = *split;
    sv->rows = rows;
    sv->pool_bytes = (size_t)rows * 32;
    sv->max_active = max_active_particles;
    if (cudaMalloc(&sv->pos, (size_t)rows * 16) != cudaSuccess || cudaMalloc(&sv->vel, (size_t)rows * 16) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sv->pos);
        delete sv;
        return hacc::set_error(ctx, HACC_ENOMEM, "cudaMalloc of the server pool failed");
    }
    if (cudaStreamCreateWithFlags(&sv->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->ev_up, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->ev_tick, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        hacc_server_destroy(sv);
        return hacc::set_error(ctx, HACC_ECUDA, "stream or event creation of the server failed");
    }
    sv->free_rows[0] = rows;
    *out = sv;
    return HACC_OK;
}

void hacc_server_destroy(hacc_server *sv) {
    if (!sv) return;
    cudaSetDevice(sv->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(sv->pos);
    cudaFree(sv->vel);
    if (sv->ev_up) cudaEventDestroy(sv->ev_up);
    if (sv->ev_tick) cudaEventDestroy(sv->ev_tick);
    if (sv->copy) cudaStreamDestroy(sv->copy);
    delete sv;
}

hacc_status hacc_server_submit(hacc_server *sv, int64_t id, double L, int64_t n, float *pos_host, float *vel_host,
                               double h, int32_t steps) {
    if (!sv) return HACC_EINVAL;
    hacc_ctx *ctx = sv->ctx;
    HACC_STATUS_RETURN(hacc::hacc_enter(ctx));
    if (n < 1 || steps < 1 || !pos_host || !vel_host || !(h == h))
        return hacc::set_error(ctx, HACC_EINVAL, "bad run (n >= 1, steps >= 1, host arrays, finite h)");
    hacc_box hb{L, 0, 0};
    hacc::Geometry g;
    HACC_STATUS_RETURN(hacc::make_geometry(ctx, &hb, sv->split.r_cut, &g));
    hacc_server::Run r{id, L, n, g.ncell, pos_host, vel_host, h, steps, 0, -1};
    if (n > sv->rows || (sv->max_active && n > sv->max_active) || !fits(sv, Load{}, r))
        return hacc::set_error(ctx, HACC_ENOMEM,
                               "run larger than the server pool, the per-tick cap or the HBM budget");
    sv->queue.push_back(r);
    return HACC_OK;
}

hacc_status hacc_server_tick(hacc_server *sv, hacc_stream_t stream, hacc_server_tick_info *info,
                             int64_t *finished_ids, int32_t finished_cap) {
    if (!sv) return HACC_EINVAL;
    hacc_ctx *ctx = sv->ctx;
    HACC_STATUS_RETURN(hacc::hacc_enter(ctx));
    if (finished_cap < 0) return hacc::set_error(ctx, HACC_EINVAL, "finished_cap must be >= 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t admitted = 0;
    // 1. admission for this tick, next to the runs admitted ahead of it
    Load load;
    for (const auto &r : sv->active)
        if (r.done < r.steps) load.add(r);
    HACC_STATUS_RETURN(admit(sv, load, &admitted));
    if (sv->up_pending) {
        HACC_CUDA_RETURN(cudaStreamWaitEvent(s, sv->ev_up, 0), "cudaStreamWaitEvent");
        sv->up_pending = false;
    }
    // 2. one sub-cycle of every resident run that has sub-cycles left
    std::vector<hacc_batch_box> boxes;
    boxes.reserve(sv->active.size());
    for (const auto &r : sv->active) {
        if (r.done >= r.steps) continue;
        hacc_batch_box b;
        b.L = r.L;
        b.nc = 0;
        b.flags = (r.done == 0 ? HACC_TICK_FIRST : 0) | (r.done == r.steps - 1 ? HACC_TICK_LAST : 0);
        b.offset = r.offset;
        b.n = r.n;
        b.dt = r.h;
        boxes.push_back(b);
    }
    const int64_t particles = load.n;
    if (!boxes.empty())
        HACC_STATUS_RETURN(hacc_batch_tick(ctx, &sv->split, (int32_t)boxes.size(), boxes.data(),
                                           reinterpret_cast<float *>(sv->pos), reinterpret_cast<float *>(sv->vel),
                                           stream));
    HACC_CUDA_RETURN(cudaEventRecord(sv->ev_tick, s), "cudaEventRecord");
    // 3. runs for the next tick: those that keep going plus newly admitted ones,
    //    uploaded while this pass runs (into rows the pass does not touch)
    Load next;
    for (const auto &r : sv->active)
        if (r.done + 1 < r.steps) next.add(r);
    const size_t n_before = sv->active.size();
    HACC_STATUS_RETURN(admit(sv, next, &admitted));
    // 4. retirement: runs whose last sub-cycle ran now or earlier, up to
    //    finished_cap of them (the others stay resident for the next tick)
    const int32_t cap = finished_ids ? finished_cap : INT32_MAX;
    std::vector<size_t> retire;
    for (size_t k = 0; k < n_before; ++k) {
        const auto &r = sv->active[k];
        const bool finished = r.done >= r.steps || (r.done + 1 == r.steps);
        if (finished && (int32_t)retire.size() < cap) retire.push_back(k);
    }
    if (!retire.empty()) HACC_CUDA_RETURN(cudaStreamWaitEvent(sv->copy, sv->ev_tick, 0), "cudaStreamWaitEvent");
    for (size_t k : retire) {
        const auto &r = sv->active[k];
        HACC_CUDA_RETURN(cudaMemcpyAsync(r.pos_host, sv->pos + r.offset, (size_t)r.n * 16, cudaMemcpyDeviceToHost,
                                         sv->copy),
                         "retire copy");
        HACC_CUDA_RETURN(cudaMemcpyAsync(r.vel_host, sv->vel + r.offset, (size_t)r.n * 16, cudaMemcpyDeviceToHost,
                                         sv->copy),
                         "retire copy");
    }
    HACC_CUDA_RETURN(cudaStreamSynchronize(s), "tick synchronize");
    HACC_CUDA_RETURN(cudaStreamSynchronize(sv->copy), "tick synchronize");
    // every copy and the pass are done: only now change the server's state
    for (size_t k = 0; k < n_before; ++k)
        if (sv->active[k].done < sv->active[k].steps) sv->active[k].done++;
    std::vector<hacc_server::Run> keep;
    keep.reserve(sv->active.size());
    int32_t finished = 0;
    for (size_t k = 0, q = 0; k < sv->active.size(); ++k) {
        if (q < retire.size() && retire[q] == k) {
            const auto &r = sv->active[k];
            free_rows(sv, r.offset, r.n);
            if (finished_ids) finished_ids[finished] = r.id;
            ++finished;
            ++q;
            continue;
        }
        keep.push_back(sv->active[k]);
    }
    sv->active.swap(keep);
    if (info) {
        info->admitted = admitted;
        info->finished = finished;
        info->active = (int32_t)boxes.size();
        info->queued = (int32_t)sv->queue.size();
        info->particles = particles;
        info->free_rows = 0;
        for (auto &f : sv->free_rows) info->free_rows += f.second;
    }
    return HACC_OK;
}

}  // extern "C"
