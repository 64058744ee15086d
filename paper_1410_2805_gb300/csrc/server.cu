// Serving runtime: continuous batching of short-range runs on one GPU.
//
// Requests (a periodic box of n particles, a sub-cycle step h and a number of
// sub-cycles) queue on the host.  Each tick:
//   1. admits queued runs in arrival order while they fit: their rows come
//      from one device pool (first-fit over a free list of row ranges,
//      coalesced on release -- a long-lived form of the phase-scoped pool of
//      Sec. 2.7) and, optionally, a cap on the particles advanced per tick;
//      admitted inputs are copied host -> device into their rows;
//   2. advances EVERY resident run by one SKS sub-cycle in one batched pass
//      (hacc_batch_tick: one binning pass, one persistent pair-kernel launch
//      over all boxes), so runs that arrive while others are on the GPU join
//      at the next tick and their work overlaps with the others';
//   3. retires runs whose last sub-cycle ran: copies their rows back to the
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
    int64_t max_active = 0;                  // 0: no cap
    std::map<int64_t, int64_t> free_rows;    // offset -> length
    struct Run {
        int64_t id;
        double L;
        int64_t n;
        float *pos_host, *vel_host;
        double h;
        int32_t steps, done;
        int64_t offset;
    };
    std::deque<Run> queue;
    std::vector<Run> active;
    int64_t active_particles = 0;
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
    sv->max_active = max_active_particles;
    if (cudaMalloc(&sv->pos, (size_t)rows * 16) != cudaSuccess || cudaMalloc(&sv->vel, (size_t)rows * 16) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sv->pos);
        delete sv;
        return hacc::set_error(ctx, HACC_ENOMEM, "cudaMalloc of the server pool failed");
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
    delete sv;
}

hacc_status hacc_server_submit(hacc_server *sv, int64_t id, double L, int64_t n, float *pos_host, float *vel_host,
                               double h, int32_t steps) {
    if (!sv) return HACC_EINVAL;
    hacc_ctx *ctx = sv->ctx;
    HACC_STATUS_RETURN(hacc::hacc_enter(ctx));
    if (n < 1 || steps < 1 || !pos_host || !vel_host || !(h == h))
        return hacc::set_error(ctx, HACC_EINVAL, "bad run (n >= 1, steps >= 1, host arrays, finite h)");
    if (n > sv->rows || (sv->max_active && n > sv->max_active))
        return hacc::set_error(ctx, HACC_ENOMEM, "run larger than the server pool or the per-tick cap");
    hacc_box hb{L, 0, 0};
    hacc::Geometry g;
    HACC_STATUS_RETURN(hacc::make_geometry(ctx, &hb, sv->split.r_cut, &g));
    sv->queue.push_back({id, L, n, pos_host, vel_host, h, steps, 0, -1});
    return HACC_OK;
}

hacc_status hacc_server_tick(hacc_server *sv, hacc_stream_t stream, hacc_server_tick_info *info,
                             int64_t *finished_ids, int32_t finished_cap) {
    if (!sv) return HACC_EINVAL;
    hacc_ctx *ctx = sv->ctx;
    HACC_STATUS_RETURN(hacc::hacc_enter(ctx));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t admitted = 0;
    // 1. admission, in arrival order
    while (!sv->queue.empty()) {
        hacc_server::Run r = sv->queue.front();
        if (sv->max_active && sv->active_particles + r.n > sv->max_active) break;
        int64_t off;
        if (!alloc_rows(sv, r.n, &off)) break;
        r.offset = off;
        HACC_CUDA_RETURN(cudaMemcpyAsync(sv->pos + off, r.pos_host, (size_t)r.n * 16, cudaMemcpyHostToDevice, s),
                         "admission copy");
        HACC_CUDA_RETURN(cudaMemcpyAsync(sv->vel + off, r.vel_host, (size_t)r.n * 16, cudaMemcpyHostToDevice, s),
                         "admission copy");
        sv->active.push_back(r);
        sv->active_particles += r.n;
        sv->queue.pop_front();
        ++admitted;
    }
    // 2. one sub-cycle of every resident run
    std::vector<hacc_batch_box> boxes;
    boxes.reserve(sv->active.size());
    for (const auto &r : sv->active) {
        hacc_batch_box b;
        b.L = r.L;
        b.nc = 0;
        b.flags = (r.done == 0 ? HACC_TICK_FIRST : 0) | (r.done == r.steps - 1 ? HACC_TICK_LAST : 0);
        b.offset = r.offset;
        b.n = r.n;
        b.dt = r.h;
        boxes.push_back(b);
    }
    int64_t particles = sv->active_particles;
    if (!boxes.empty())
        HACC_STATUS_RETURN(hacc_batch_tick(ctx, &sv->split, (int32_t)boxes.size(), boxes.data(),
                                           reinterpret_cast<float *>(sv->pos), reinterpret_cast<float *>(sv->vel),
                                           stream));
    // 3. retire finished runs
    int32_t finished = 0;
    std::vector<hacc_server::Run> keep;
    keep.reserve(sv->active.size());
    std::vector<std::pair<int64_t, int64_t>> released;
    for (auto &r : sv->active) {
        r.done++;
        if (r.done < r.steps) {
            keep.push_back(r);
            continue;
        }
        HACC_CUDA_RETURN(cudaMemcpyAsync(r.pos_host, sv->pos + r.offset, (size_t)r.n * 16, cudaMemcpyDeviceToHost, s),
                         "retire copy");
        HACC_CUDA_RETURN(cudaMemcpyAsync(r.vel_host, sv->vel + r.offset, (size_t)r.n * 16, cudaMemcpyDeviceToHost, s),
                         "retire copy");
        released.emplace_back(r.offset, r.n);
        sv->active_particles -= r.n;
        if (finished_ids && finished < finished_cap) finished_ids[finished] = r.id;
        ++finished;
    }
    sv->active.swap(keep);
    HACC_CUDA_RETURN(cudaStreamSynchronize(s), "tick synchronize");
    for (auto &fr : released) free_rows(sv, fr.first, fr.second);
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
