// Chaining-mesh build on the GPU (Sec. 2.4 / Sec. 3.3: Hockney's chaining
// mesh controls the number of particle-particle interactions; Sec. 2.7: the
// particle arrays are reordered out of place through a permutation).
//
// Pipeline (all HBM-bound, one pass each):
//   k_key     wrap (after an optional drift), exact cell id, per-cell count
//             and arrival slot (atomic), [sub-cell]        read 16-32 B, write 8-25 B
//             (in place without a drift only moved particles are written back)
//   scan      exclusive scan of (count, work-item count) packed in 64 bits
//   k_place   perm_tmp[start[c] + slot] = i, [its sub-cell] read 12-13 B, write 4-5 B
//   k_order   within each cell, sort perm by input row (stable order) or by
//             (sub-cell, input row)
//   k_items   cell starts and force work items
//   gather    sorted copies of positions / velocities / ids
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hacc_internal.cuh"

namespace hacc {
namespace {

constexpr int kBlock = 256;

// Largest k with k*L <= x*nc, for x in [0, L).  The FP32 product is within
// 2e-4 of the exact quotient for nc <= 1024, so away from a cell face its
// floor is exact; near a face the decision is made with exact FP64 products
// (x has 24 significant bits, nc < 2^11, L is an FP32 value).
__device__ __forceinline__ int cell1(float x, float inv_w, double Ld, int nc) {
    float f = x * inv_w;
    int k = (int)f;
    k = k < 0 ? 0 : (k > nc - 1 ? nc - 1 : k);
    float fr = f - (float)k;
    if (fr < 1e-3f || fr > 0.999f) {
        double xn = (double)x * (double)nc;
        if (k > 0 && (double)k * Ld > xn) --k;
        else if (k < nc - 1 && (double)(k + 1) * Ld <= xn) ++k;
    }
    return k;
}

// Morton index of the 4x4x4 sub-cell of a particle from its in-cell
// fractions (z, y, x bits of the halves, then of the quarters), used only to
// order particles within a cell.
__device__ __forceinline__ uint8_t sub_cell(float fx, float fy, float fz) {
    const int qx = min(max((int)(fx * 4.0f), 0), 3);
    const int qy = min(max((int)(fy * 4.0f), 0), 3);
    const int qz = min(max((int)(fz * 4.0f), 0), 3);
    return (uint8_t)(((qz >> 1) << 5) | ((qy >> 1) << 4) | ((qx >> 1) << 3) | ((qz & 1) << 2) | ((qy & 1) << 1) |
                     (qx & 1));
}

// Arrival slot of each lane's particle in its cell (count[c] counts the
// cell's particles).  Lanes whose cell equals the previous lane's form a run
// (input rows next to each other often share a cell); the first lane of a
// run claims the run's slots with one atomic and the others take the slots
// that follow, in lane order.  Lanes without a particle pass c < 0.  All
// lanes of the warp must call it.  (One atomic per distinct cell of the warp,
// found with a match, measured slower.)
__device__ __forceinline__ uint32_t claim_slot(uint32_t *__restrict__ count, int32_t c) {
    const int lane = threadIdx.x & 31;
    const int32_t prev = __shfl_up_sync(0xffffffffu, c, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != c || c < 0);
    const unsigned le = 0xffffffffu >> (31 - lane);              // lanes <= this lane
    const int head = 31 - __clz(heads & le);                     // first lane of this lane's run
    const unsigned after = heads & ~le;
    const int next = after ? __ffs(after) - 1 : 32;              // first lane of the next run
    uint32_t base = 0;
    if (head == lane && c >= 0) base = atomicAdd(&count[c], (uint32_t)(next - lane));
    base = __shfl_sync(0xffffffffu, base, head);
    return base + (uint32_t)(lane - head);
}

__global__ void __launch_bounds__(kBlock) k_key(int64_t n, const float4 *__restrict__ src,
                                                 const float4 *__restrict__ vel, float drift,
                                                 float4 *dst, float Lf, float inv_w, double Ld, int nc,
                                                 int32_t *__restrict__ key, int32_t *__restrict__ rank,
                                                 uint32_t *__restrict__ count, int *flags, int *mass_flag,
                                                 uint8_t *__restrict__ sub, const int32_t *__restrict__ sub_level) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t c = -1;
    if (i < n) {
        float4 p = src[i];
        if (p.w != src[0].w) atomicOr(mass_flag, 1);
        if (vel) {
            float4 v = vel[i];
            p.x = __fmaf_rn(drift, v.x, p.x);
            p.y = __fmaf_rn(drift, v.y, p.y);
            p.z = __fmaf_rn(drift, v.z, p.z);
        }
        // wrap1 leaves a coordinate in [0, L) bit for bit as it is, so an
        // in-place call (no drift) writes back only the particles it moved
        const bool inside = p.x >= 0.0f && p.x < Lf && p.y >= 0.0f && p.y < Lf && p.z >= 0.0f && p.z < Lf;
        bool ok = wrap1(p.x, Lf);
        ok &= wrap1(p.y, Lf);
        ok &= wrap1(p.z, Lf);
        if (!ok) atomicOr(flags, kFlagDomain);
        int cx = cell1(p.x, inv_w, Ld, nc), cy = cell1(p.y, inv_w, Ld, nc), cz = cell1(p.z, inv_w, Ld, nc);
        c = (int32_t)(((int64_t)cz * nc + cy) * nc + cx);
        if (!(inside && !vel && dst == src)) dst[i] = p;
        key[i] = c;
        if (sub) {
            const uint8_t m = sub_cell(p.x * inv_w - (float)cx, p.y * inv_w - (float)cy, p.z * inv_w - (float)cz);
            // with kick counts: (kick count, octant), else the 4x4x4 Morton sub-cell
            sub[i] = sub_level ? (uint8_t)((min(sub_level[i], 31) << 3) | (m >> 3)) : m;
        }
    }
    const uint32_t slot = claim_slot(count, c);
    if (i < n) rank[i] = (int32_t)slot;
}

// Lane layout of a work item of n <= 128 particles: 2^lg groups of 32 >> lg
// lanes, K particles per lane; the smallest slot count (32 >> lg) * K >= n,
// preferring larger K.  Encoded as (lg << 4) | K.
__device__ __forceinline__ int item_shape(uint32_t n) {
    if (n <= 4) return (3 << 4) | 1;
    if (n <= 8) return (3 << 4) | 2;
    if (n <= 12) return (3 << 4) | 3;
    if (n <= 16) return (3 << 4) | 4;
    if (n <= 20) return (3 << 4) | 5;
    if (n <= 24) return (2 << 4) | 3;
    if (n <= 32) return (2 << 4) | 4;
    if (n <= 40) return (2 << 4) | 5;
    if (n <= 48) return (1 << 4) | 3;
    if (n <= 64) return (1 << 4) | 4;
    if (n <= 80) return (1 << 4) | 5;
    if (n <= 96) return 3;
    if (n <= 128) return 4;
    return 5;
}

// How cells are cut into work items: a cell of cnt particles becomes
// ceil(cnt / cap) items, or ceil(cnt / kItemMax) when cnt > split_max (dense
// cells: their particles crowd into a few sub-cells, so smaller items would
// not shrink the bounds, only repeat the staging of the neighbours).
struct ItemRule {
    uint32_t cap, split_max;
};

__device__ __forceinline__ uint32_t items_of(uint32_t cnt, ItemRule r) {
    const uint32_t cap = cnt > r.split_max ? (uint32_t)kItemMax : r.cap;
    return cnt == 0 ? 0u : (cnt <= cap ? 1u : (cnt + cap - 1) / cap);
}

__global__ void __launch_bounds__(kBlock) k_pack(int64_t ncell, const uint32_t *__restrict__ count,
                                                  unsigned long long *__restrict__ packed, ItemRule cap) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    uint32_t k = count[c];
    const uint32_t it = items_of(k, cap);
    packed[c] = (unsigned long long)k | ((unsigned long long)it << 32);
}

// ---- exclusive scan of uint64, reduce-then-scan, 2048 values per block ----
constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

__device__ __forceinline__ unsigned long long block_exclusive(unsigned long long v, unsigned long long *total) {
    __shared__ unsigned long long warp_sums[kBlock / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < kBlock / 32 ? warp_sums[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kBlock / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    unsigned long long before = w ? warp_sums[w - 1] : 0ull;
    if (total) *total = warp_sums[kBlock / 32 - 1];
    unsigned long long r = before + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBlock) k_scan_reduce(int64_t len, const unsigned long long *__restrict__ in,
                                                         unsigned long long *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < len) s += in[base + j];
    unsigned long long total;
    block_exclusive(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kBlock) k_scan_down(int64_t len, unsigned long long *data,
                                                       const unsigned long long *__restrict__ offsets) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    unsigned long long v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < len ? data[base + j] : 0ull;
        s += v[j];
    }
    unsigned long long run = block_exclusive(s, nullptr) + (offsets ? offsets[blockIdx.x] : 0ull);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < len) data[base + j] = run;
        run += v[j];
    }
}

// Exclusive scan of data[0..len) in place; tmp holds the per-level block sums.
cudaError_t scan_exclusive(unsigned long long *data, int64_t len, unsigned long long *tmp, cudaStream_t s) {
    if (len <= 0) return cudaSuccess;
    int64_t nb = (len + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_down<<<1, kBlock, 0, s>>>(len, data, nullptr);
        note_launch();
        return cudaGetLastError();
    }
    unsigned long long *sums = tmp;
    k_scan_reduce<<<(unsigned)nb, kBlock, 0, s>>>(len, data, sums);
    note_launch();
    cudaError_t e = scan_exclusive(sums, nb, tmp + nb, s);
    if (e != cudaSuccess) return e;
    k_scan_down<<<(unsigned)nb, kBlock, 0, s>>>(len, data, sums);
    note_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_place(int64_t n, const int32_t *__restrict__ key,
                                                   const int32_t *__restrict__ rank,
                                                   const unsigned long long *__restrict__ packed,
                                                   int32_t *__restrict__ perm_tmp, const uint8_t *__restrict__ sub,
                                                   unsigned long long *__restrict__ order_tmp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = key[i];
    uint32_t start = (uint32_t)(packed[c] & 0xffffffffull);
    const uint32_t at = start + (uint32_t)rank[i];
    // with sub-cells the row and its sub-cell go out as one 8-byte word (one
    // scattered write, as for the row alone)
    if (sub) order_tmp[at] = ((unsigned long long)sub[i] << 32) | (uint32_t)i;
    else perm_tmp[at] = (int32_t)i;
}

// The arrival order from the atomics is arbitrary, so each element's final
// slot is the number of smaller keys in its cell.  The key is the input row
// (distinct), which gives ascending input row within the cell, or the pair
// (Morton sub-cell, input row), which groups the cell's particles by sub-cell.
// k_order_rows serves calls of up to 2^24 rows (the pair as one 32-bit key,
// code << 24 | row); k_order_sub, one warp per cell, larger ones: a cell that
// becomes one work item by row, the others by the pair with the row taken
// relative to the cell's smallest row (one 32-bit key when the cell's rows
// span less than 2^24, else 64-bit keys; codes are below 2^8), cells of up to
// 256 keys through the register networks above, larger ones by counting.
// Cells of more than kBigCell particles go to a list sorted by input row by
// k_order_big.
constexpr uint32_t kBigCell = 512;

// Bitonic sort of N = 32 KPL keys held KPL per lane (key of slot e = lane +
// 32 q in x[q]), in the form without directions: merging sorted runs of k/2
// into runs of k first compares slot e with e ^ (k - 1) (the second run
// reversed), then with e ^ j for j = k/4 .. 1; in every compare the lower slot
// keeps the minimum.  Pairs across lanes (j < 32) exchange keys with shuffles,
// the others compare two registers of the same lane.  Afterwards x[q] holds
// the key of sorted slot lane + 32 q.
template <int KPL>
__device__ __forceinline__ void bitonic_lanes(uint32_t (&x)[KPL], int lane) {
    constexpr int N = 32 * KPL;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
        if (k <= 32) {
            const bool low = (lane & (k >> 1)) == 0;
#pragma unroll
            for (int q = 0; q < KPL; ++q) {
                const uint32_t y = __shfl_xor_sync(0xffffffffu, x[q], k - 1);
                x[q] = low ? min(x[q], y) : max(x[q], y);
            }
        } else {
            // slot (lane, q) meets (lane ^ 31, q ^ m): the one with the lower q is lower
            const int m = (k >> 5) - 1;
#pragma unroll
            for (int q = 0; q < KPL; ++q) {
                if (q & (k >> 6)) continue;
                const int qq = q ^ m;
                const uint32_t yb = __shfl_xor_sync(0xffffffffu, x[qq], 31);
                const uint32_t ya = __shfl_xor_sync(0xffffffffu, x[q], 31);
                x[q] = min(x[q], yb);
                x[qq] = max(x[qq], ya);
            }
        }
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
            if (j >= 32) {
                const int qj = j >> 5;
#pragma unroll
                for (int q = 0; q < KPL; ++q) {
                    if (q & qj) continue;
                    const uint32_t a = x[q], b = x[q | qj];
                    x[q] = min(a, b);
                    x[q | qj] = max(a, b);
                }
            } else {
                const bool low = (lane & j) == 0;
#pragma unroll
                for (int q = 0; q < KPL; ++q) {
                    const uint32_t y = __shfl_xor_sync(0xffffffffu, x[q], j);
                    x[q] = low ? min(x[q], y) : max(x[q], y);
                }
            }
        }
    }
}

// The cell's cnt <= 32 KPL keys sorted by bitonic_lanes (slots past the cell
// hold the largest key); out[slot] = rowf(the slot's key).
template <int KPL, class Seg, class RowF>
__device__ __forceinline__ void sort_cell_f(const Seg &seg, uint32_t cnt, int lane, int32_t *out, const RowF &rowf) {
    uint32_t x[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) x[q] = (uint32_t)(lane + 32 * q) < cnt ? seg(lane + 32 * q) : 0xffffffffu;
    bitonic_lanes<KPL>(x, lane);
#pragma unroll
    for (int q = 0; q < KPL; ++q)
        if ((uint32_t)(lane + 32 * q) < cnt) out[lane + 32 * q] = rowf(x[q]);
}

template <int KPL, class Seg>
__device__ __forceinline__ void sort_cell(const Seg &seg, uint32_t cnt, int lane, int32_t *out, uint32_t row_mask) {
    sort_cell_f<KPL>(seg, cnt, lane, out, [row_mask](uint32_t k) { return (int32_t)(k & row_mask); });
}

// A cell of cnt <= 256 keys through the smallest network that holds it.
template <class Seg, class RowF>
__device__ __forceinline__ void sort_small_cell(const Seg &seg, uint32_t cnt, int lane, int32_t *out, const RowF &rowf) {
    if (cnt <= 32) sort_cell_f<1>(seg, cnt, lane, out, rowf);
    else if (cnt <= 64) sort_cell_f<2>(seg, cnt, lane, out, rowf);
    else if (cnt <= 128) sort_cell_f<4>(seg, cnt, lane, out, rowf);
    else sort_cell_f<8>(seg, cnt, lane, out, rowf);
}

struct RowOf64 {
    __device__ int32_t operator()(unsigned long long k) const { return (int32_t)(uint32_t)k; }
};
struct RowOfPacked {
    uint32_t base;
    __device__ int32_t operator()(uint32_t k) const { return (int32_t)((k & 0xffffffu) + base); }
};

// Rank of each lane's key among the cell's cnt <= 32 keys (lanes >= cnt hold
// the largest key); out[rank] = its row.
template <class Key, class Row>
__device__ __forceinline__ void rank_warp(Key v, int cnt, int lane, int32_t *out, Row row) {
    int r = 0;
    for (int q = 0; q < cnt; ++q) {
        const Key u = __shfl_sync(0xffffffffu, v, q);
        r += (u < v);
    }
    if (lane < cnt) out[r] = row(v);
}

// The same for the cnt keys in the warp's shared array w.
template <class Key, class Row>
__device__ __forceinline__ void rank_shared(const Key *w, uint32_t cnt, int lane, int32_t *out, Row row) {
    __syncwarp();
    for (uint32_t e = lane; e < cnt; e += 32) {
        const Key v = w[e];
        uint32_t r = 0;
        for (uint32_t q = 0; q < cnt; ++q) r += (w[q] < v);
        out[r] = row(v);
    }
}

__global__ void __launch_bounds__(kBlock) k_order_sub(int64_t ncell, const uint32_t *__restrict__ count,
                                                       const unsigned long long *__restrict__ packed,
                                                       int32_t *__restrict__ perm_tmp,
                                                       int32_t *__restrict__ perm, int32_t *__restrict__ big_list,
                                                       int *__restrict__ big_count,
                                                       const unsigned long long *__restrict__ order_tmp,
                                                       uint32_t row_below) {
    int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= ncell) return;
    uint32_t cnt = count[c];
    if (cnt == 0) return;
    uint32_t s = (uint32_t)(packed[c] & 0xffffffffull);
    if (cnt > kBigCell) {
        // big cells are ordered by row alone, from perm_tmp
        for (uint32_t e = lane; e < cnt; e += 32) perm_tmp[s + e] = (int32_t)(uint32_t)order_tmp[s + e];
        if (lane == 0) big_list[atomicAdd(big_count, 1)] = (int32_t)c;
        return;
    }
    int32_t *out = perm + s;
    const unsigned long long *seg = order_tmp + s;
    if (cnt <= row_below) {
        // a cell that becomes one work item keeps row order (cnt <= 160)
        sort_small_cell([&](uint32_t e) { return (uint32_t)seg[e]; }, cnt, lane, out,
                        [](uint32_t k) { return (int32_t)k; });
        return;
    }
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (uint32_t e = lane; e < cnt; e += 32) {
        const uint32_t r = (uint32_t)seg[e];
        lo = min(lo, r);
        hi = max(hi, r);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    __shared__ unsigned long long keys[kBlock / 32][kBigCell];
    unsigned long long *w = keys[threadIdx.x >> 5];
    if (hi - lo < (1u << 24)) {
        const RowOfPacked row{lo};
        if (cnt <= 256) {
            sort_small_cell([&](uint32_t e) { return ((uint32_t)(seg[e] >> 32) << 24) | ((uint32_t)seg[e] - lo); },
                            cnt, lane, out, [lo](uint32_t k) { return (int32_t)((k & 0xffffffu) + lo); });
            return;
        }
        uint32_t *w32 = reinterpret_cast<uint32_t *>(w);
        for (uint32_t e = lane; e < cnt; e += 32) w32[e] = ((uint32_t)(seg[e] >> 32) << 24) | ((uint32_t)seg[e] - lo);
        rank_shared(w32, cnt, lane, out, row);
        return;
    }
    if (cnt <= 32) {
        rank_warp(lane < (int)cnt ? seg[lane] : ~0ull, (int)cnt, lane, out, RowOf64{});
        return;
    }
    for (uint32_t e = lane; e < cnt; e += 32) w[e] = seg[e];
    rank_shared(w, cnt, lane, out, RowOf64{});
}

// The in-cell order, a block per kOrdCells consecutive cells: their slots
// form one range of the placement array, which the block stages into shared
// memory with coalesced loads (when it holds at most kOrdCap entries; else
// the warps read their cells' keys from global memory).  Each warp then ranks
// one cell at a time; keys are distinct, and the slot of a key is the number
// of smaller keys of its cell.  A cell of up to 32 keys is ranked in registers
// by its stretches of consecutive keys when it has few (the key pass's runs),
// else by a bitonic sort across the warp; a larger row-ordered cell tries
// the stretch ranking in shared memory, and otherwise a cell of up to 256
// keys is sorted by a bitonic network over 2, 4 or 8 keys per lane, a larger
// one ranked by counting with 4 keys per lane on each pass over the cell (up
// to kBigCell).  The key is the input row (row order), or with SUB the pair
// (sub-cell code, input row) as one 32-bit key, code << 24 | row (codes below
// 2^8, rows below 2^24; larger calls take k_order_sub).  Cells above kBigCell
// are ordered by input row alone, by k_order_big (with SUB their rows are
// copied to perm_tmp first).
constexpr int kOrdCells = 64;
constexpr int kOrdCap = 6144;
constexpr int64_t kOrdSubMaxRows = (int64_t)1 << 24;

template <bool SUB>
__device__ __forceinline__ uint32_t order_key(const int32_t *perm_tmp, const unsigned long long *order_tmp,
                                              uint32_t e) {
    if (SUB) {
        const unsigned long long v = order_tmp[e];
        return ((uint32_t)(v >> 32) << 24) | (uint32_t)v;
    }
    return (uint32_t)perm_tmp[e];
}

// Ranks of the keys seg[e0 + lane + 32 k], k < J, among the cnt keys of the
// cell (one pass over the cell feeds J comparisons per load); writes each
// row to its slot.
template <int J, class Seg>
__device__ __forceinline__ void rank_lanes(const Seg &seg, uint32_t cnt, uint32_t e0, int lane, int32_t *out,
                                           uint32_t row_mask) {
    uint32_t v[J], r[J];
#pragma unroll
    for (int k = 0; k < J; ++k) {
        const uint32_t e = e0 + lane + 32 * k;
        v[k] = e < cnt ? seg(e) : 0xffffffffu;
        r[k] = 0;
    }
    for (uint32_t u = 0; u < cnt; ++u) {
        const uint32_t x = seg(u);
#pragma unroll
        for (int k = 0; k < J; ++k) r[k] += x < v[k] ? 1u : 0u;
    }
#pragma unroll
    for (int k = 0; k < J; ++k)
        if (e0 + lane + 32 * k < cnt) out[r[k]] = (int32_t)(v[k] & row_mask);
}

// Ranking by stretches.  The key pass gives each run of adjacent lanes with
// the same cell consecutive slots in input-row order, so a cell's slots hold
// stretches of consecutive keys (key + 1 follows key), and stretches are
// disjoint intervals of keys: sorting the stretch heads sorts the cell.  A
// key's slot is the rank of its stretch's head (the lengths of the stretches
// with smaller heads) plus its offset within the stretch.  Work O(cnt log R +
// R^2) for R stretches instead of O(cnt^2): R is small when the input rows
// follow the previous binning's cell order (the sub-cycle loop), and about a
// third of cnt for lattice-ordered input.  Returns false, doing nothing, when
// R is above cnt / 2 or kHeads (a shuffled input), where counting is cheaper.
constexpr int kHeads = 128;
// Cells of at most 32 keys rank by stretches in registers when they have at
// most kRegHeads stretches (else by counting); row-ordered cells up to
// kStretchTryMax keys try the shared-memory stretch ranking on any input.
constexpr int kRegHeads = 16;
constexpr uint32_t kStretchTryMax = 64;

template <class Seg>
__device__ __forceinline__ bool rank_stretches(const Seg &seg, uint32_t cnt, int lane, int32_t *out,
                                               uint32_t row_mask, uint32_t *hkey, uint32_t *hslot, uint32_t *hrank) {
    const unsigned lt = (1u << lane) - 1u;
    int R = 0;
    for (uint32_t e0 = 0; e0 < cnt; e0 += 32) {
        const uint32_t e = e0 + lane;
        bool head = false;
        uint32_t v = 0;
        if (e < cnt) {
            v = seg(e);
            head = e == 0 || v != seg(e - 1) + 1u;
        }
        const unsigned m = __ballot_sync(0xffffffffu, head);
        const int at = R + __popc(m & lt);
        if (head && at < kHeads) {
            hkey[at] = v;
            hslot[at] = e;
        }
        R += __popc(m);
    }
    if (R > kHeads || 2 * (uint32_t)R > cnt) return false;
    __syncwarp();
    // rank of each stretch head: the summed lengths of the stretches below it
    for (int t = lane; t < R; t += 32) {
        const uint32_t kt = hkey[t];
        uint32_t r = 0;
        for (int u = 0; u < R; ++u) {
            const uint32_t len = (u + 1 < R ? hslot[u + 1] : cnt) - hslot[u];
            r += hkey[u] < kt ? len : 0u;
        }
        hrank[t] = r;
    }
    __syncwarp();
    for (uint32_t e = lane; e < cnt; e += 32) {
        // the last stretch starting at or before slot e
        int lo = 0, hi = R - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (hslot[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        out[hrank[lo] + (e - hslot[lo])] = (int32_t)(seg(e) & row_mask);
    }
    __syncwarp();
    return true;
}

// row_below: with SUB, cells of at most row_below particles are ordered by
// row alone (the row is the key's low 24 bits); stretches: try the ranking
// by stretches for row-ordered cells (the input follows a previous cell
// order).
template <bool SUB>
__global__ void __launch_bounds__(kBlock, 5) k_order_rows(int64_t ncell, const uint32_t *__restrict__ count,
                                                        const unsigned long long *__restrict__ packed,
                                                        int32_t *__restrict__ perm_tmp,
                                                        int32_t *__restrict__ perm, int32_t *__restrict__ big_list,
                                                        int *__restrict__ big_count,
                                                        const unsigned long long *__restrict__ order_tmp,
                                                        uint32_t row_below, int stretches) {
    __shared__ uint32_t keys[kOrdCap];
    __shared__ uint32_t heads[kBlock / 32][3][kHeads];    // a warp's stretch heads: keys, slots, ranks
    __shared__ uint32_t cstart[kOrdCells], ccount[kOrdCells];
    __shared__ int next_cell;   // the warps take the block's cells in turn (cells differ widely in cost)
    const int64_t c0 = (int64_t)blockIdx.x * kOrdCells;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int ncb = ncell - c0 < kOrdCells ? (int)(ncell - c0) : kOrdCells;   // cells of this block (>= 1)
    if (t == 0) next_cell = 0;
    if (t < kOrdCells) {
        uint32_t cnt = 0, st = 0;
        if (t < ncb) {
            cnt = count[c0 + t];
            st = (uint32_t)(packed[c0 + t] & 0xffffffffull);
        }
        ccount[t] = cnt;
        cstart[t] = st;
    }
    __syncthreads();
    const uint32_t S0 = cstart[0], S1 = cstart[ncb - 1] + ccount[ncb - 1];
    const bool staged = S1 - S0 <= (uint32_t)kOrdCap;
    if (staged) {
        for (uint32_t e = t; e < S1 - S0; e += kBlock) keys[e] = order_key<SUB>(perm_tmp, order_tmp, S0 + e);
        __syncthreads();
    }
    const uint32_t row_mask = SUB ? (1u << 24) - 1u : 0xffffffffu;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(&next_cell, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= ncb) break;
        const uint32_t cnt = ccount[q];
        if (cnt == 0) continue;
        const uint32_t st = cstart[q];
        int32_t *out = perm + st;
        // the cell's keys in slot order, from the staged range or from global
        // memory; a cell ordered by row alone takes the row bits of the key
        // (big cells are ordered by row alone too)
        const uint32_t *sk = keys + (st - S0);
        const bool by_row = !SUB || cnt <= row_below || cnt > kBigCell;
        const uint32_t kmask = by_row ? row_mask : 0xffffffffu;
        auto seg = [&](uint32_t e) -> uint32_t {
            return (staged ? sk[e] : order_key<SUB>(perm_tmp, order_tmp, st + e)) & kmask;
        };
        if (cnt <= 32) {
            const uint32_t v = lane < (int)cnt ? seg(lane) : 0u;
            // the stretches of consecutive keys in slot order (disjoint key
            // intervals): a key's slot is the summed length of the stretches
            // with smaller heads plus its offset in its own stretch
            const uint32_t prev = __shfl_up_sync(0xffffffffu, v, 1);
            const unsigned hm = __ballot_sync(0xffffffffu, lane < (int)cnt && (lane == 0 || v != prev + 1u));
            if (__popc(hm) <= kRegHeads) {
                const int h = 31 - __clz(hm & (0xffffffffu >> (31 - lane)));   // this lane's stretch head
                const uint32_t hv = __shfl_sync(0xffffffffu, v, h < 0 ? 0 : h);
                uint32_t r = (uint32_t)(lane - h);
                for (unsigned m = hm; m;) {
                    const int a = __ffs(m) - 1;
                    m &= m - 1u;
                    const int b = m ? __ffs(m) - 1 : (int)cnt;
                    const uint32_t ka = __shfl_sync(0xffffffffu, v, a);
                    r += ka < hv ? (uint32_t)(b - a) : 0u;
                }
                if (lane < (int)cnt) out[r] = (int32_t)(v & row_mask);
            } else {
                sort_cell<1>(seg, cnt, lane, out, row_mask);
            }
            continue;
        }
        // (sub-cell keys rarely run on: a cell's particles spread over 64 sub-cells)
        if (by_row && (stretches || cnt <= kStretchTryMax) &&
            rank_stretches(seg, cnt, lane, out, row_mask, heads[w][0], heads[w][1], heads[w][2]))
            continue;
        if (cnt > kBigCell) {
            // to the big-cell sort by row, from perm_tmp
            if (SUB)
                for (uint32_t e = lane; e < cnt; e += 32) perm_tmp[st + e] = (int32_t)(uint32_t)order_tmp[st + e];
            if (lane == 0) big_list[atomicAdd(big_count, 1)] = (int32_t)(c0 + q);
            continue;
        }
        if (cnt <= 64) {
            sort_cell<2>(seg, cnt, lane, out, row_mask);
            continue;
        }
        if (cnt <= 128) {
            sort_cell<4>(seg, cnt, lane, out, row_mask);
            continue;
        }
        if (cnt <= 256) {
            sort_cell<8>(seg, cnt, lane, out, row_mask);
            continue;
        }
        for (uint32_t e0 = 0; e0 < cnt; e0 += 4 * 32) rank_lanes<4>(seg, cnt, e0, lane, out, row_mask);
    }
}

// Big cells, one block per cell (grid-stride over the list): sort chunks of
// kChunk input rows with a shared-memory bitonic network, then merge runs of
// doubling width between the two segment buffers, each output element placed
// by its merge-path co-rank.  O(m log^2 m) work per cell of m particles.
constexpr int kOrderThreads = 1024;
constexpr int kChunk = 2048;

__global__ void __launch_bounds__(kOrderThreads) k_order_big(const uint32_t *__restrict__ count,
                                                              const unsigned long long *__restrict__ packed,
                                                              int32_t *__restrict__ perm_tmp,
                                                              int32_t *__restrict__ perm,
                                                              const int32_t *__restrict__ big_list,
                                                              const int *__restrict__ big_count) {
    __shared__ int32_t sh[kChunk];
    const int nbig = *big_count;
    const int tid = threadIdx.x;
    for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
        const int32_t c = big_list[q];
        const int m = (int)count[c];
        const uint32_t s = (uint32_t)(packed[c] & 0xffffffffull);
        int32_t *A = perm_tmp + s, *B = perm + s;
        // 1. sorted chunks, in place in A
        for (int base = 0; base < m; base += kChunk) {
            for (int t = tid; t < kChunk; t += kOrderThreads) sh[t] = base + t < m ? A[base + t] : 0x7fffffff;
            __syncthreads();
            for (int k = 2; k <= kChunk; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int t = tid; t < kChunk; t += kOrderThreads) {
                        int o = t ^ j;
                        if (o > t) {
                            int32_t a = sh[t], b = sh[o];
                            if ((a > b) == ((t & k) == 0)) {
                                sh[t] = b;
                                sh[o] = a;
                            }
                        }
                    }
                    __syncthreads();
                }
            for (int t = tid; t < kChunk && base + t < m; t += kOrderThreads) A[base + t] = sh[t];
            __syncthreads();
        }
        // 2. merge passes, ping-pong A <-> B
        int32_t *src = A, *dst = B;
        for (int width = kChunk; width < m; width <<= 1) {
            for (int k = tid; k < m; k += kOrderThreads) {
                const int base = (k / (2 * width)) * (2 * width);
                const int lenA = min(width, m - base);
                const int lenB = max(0, min(width, m - base - width));
                const int32_t *a = src + base, *b = src + base + width;
                const int qk = k - base;
                int lo = max(0, qk - lenB), hi = min(qk, lenA);
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (a[mid] < b[qk - mid - 1]) lo = mid + 1;
                    else hi = mid;
                }
                const int i = lo, j = qk - lo;
                dst[k] = (i < lenA && (j >= lenB || a[i] < b[j])) ? a[i] : b[j];
            }
            __syncthreads();
            int32_t *tmp = src;
            src = dst;
            dst = tmp;
        }
        if (src != B)
            for (int t = tid; t < m; t += kOrderThreads) B[t] = src[t];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) k_items(int64_t ncell, int64_t n, const uint32_t *__restrict__ count,
                                                   const unsigned long long *__restrict__ packed,
                                                   int32_t *__restrict__ cell_start, int4 *__restrict__ items,
                                                   int32_t *__restrict__ n_items, int make_items,
                                                   const BoxDev *__restrict__ boxes, int nbox, ItemRule cap) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) {
        cell_start[ncell] = (int32_t)n;
        if (make_items) {
            unsigned long long last = packed[ncell - 1];
            *n_items = (int32_t)((last >> 32) + items_of(count[ncell - 1], cap));
        }
    }
    if (c >= ncell) return;
    unsigned long long p = packed[c];
    uint32_t s = (uint32_t)(p & 0xffffffffull);
    cell_start[c] = (int32_t)s;
    if (!make_items) return;
    uint32_t cnt = count[c];
    uint32_t it = (uint32_t)(p >> 32);
    if (cnt == 0) return;
    int box = 0;
    if (boxes) {  // last box whose first cell is <= c
        int lo = 0, hi = nbox - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (boxes[mid].cell_base <= c) lo = mid;
            else hi = mid - 1;
        }
        box = lo;
    }
    // m near-equal runs: run q is [cnt q / m, cnt (q+1) / m)
    uint32_t m = items_of(cnt, cap);
    for (uint32_t q = 0; q < m; ++q) {
        const uint32_t a = (uint32_t)((uint64_t)cnt * q / m), e = (uint32_t)((uint64_t)cnt * (q + 1) / m);
        items[it + q] = make_int4((int)c, (int)(s + a), (int)(e - a), (box << 8) | item_shape(e - a));
    }
}

// Batched key pass: box of scratch index t by binary search over part_base.
__global__ void __launch_bounds__(kBlock) k_bkey(int64_t n_total, int nbox, const BoxDev *__restrict__ boxes,
                                                  const float4 *__restrict__ pos_pool,
                                                  const float4 *__restrict__ vel_pool, float4 *__restrict__ dst,
                                                  int32_t *__restrict__ id, int32_t *__restrict__ key,
                                                  int32_t *__restrict__ rank, uint32_t *__restrict__ count, int *flags,
                                                  int *mass_flag, uint8_t *__restrict__ sub) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t c = -1;
    if (t < n_total) {
        int lo = 0, hi = nbox - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (boxes[mid].part_base <= t) lo = mid;
            else hi = mid - 1;
        }
        const BoxDev bx = boxes[lo];
        const long long row = bx.row_off + (t - bx.part_base);
        float4 p = pos_pool[row];
        if (bx.pre != 0.0f) {
            float4 v = vel_pool[row];
            p.x = __fmaf_rn(bx.pre, v.x, p.x);
            p.y = __fmaf_rn(bx.pre, v.y, p.y);
            p.z = __fmaf_rn(bx.pre, v.z, p.z);
        }
        bool ok = wrap1(p.x, bx.L);
        ok &= wrap1(p.y, bx.L);
        ok &= wrap1(p.z, bx.L);
        if (!ok) atomicOr(flags, kFlagDomain);
        if (p.w != pos_pool[boxes[0].row_off].w) atomicOr(mass_flag, 1);
        const int nc = bx.nc;
        int cx = cell1(p.x, bx.inv_w, bx.Ld, nc), cy = cell1(p.y, bx.inv_w, bx.Ld, nc),
            cz = cell1(p.z, bx.inv_w, bx.Ld, nc);
        c = bx.cell_base + (int32_t)(((int64_t)cz * nc + cy) * nc + cx);
        dst[t] = p;
        id[t] = (int32_t)row;
        key[t] = c;
        if (sub)
            sub[t] = sub_cell(p.x * bx.inv_w - (float)cx, p.y * bx.inv_w - (float)cy, p.z * bx.inv_w - (float)cz);
    }
    const uint32_t slot = claim_slot(count, c);
    if (t < n_total) rank[t] = (int32_t)slot;
}

__global__ void __launch_bounds__(kBlock) k_gather(int64_t n, const int32_t *__restrict__ perm,
                                                    const float4 *__restrict__ p_in, float4 *__restrict__ p_out,
                                                    const float4 *__restrict__ v_in, float4 *__restrict__ v_out,
                                                    const int32_t *__restrict__ id_in, int32_t *__restrict__ id_out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int32_t i = perm[k];
    p_out[k] = p_in[i];
    if (v_out) v_out[k] = v_in[i];
    if (id_out) id_out[k] = id_in ? id_in[i] : i;
}

// Multi-level rebinning: gather positions (and a copy, the binned reference),
// velocities, kick counts, input rows and cell ids into the new sorted order.
__global__ void __launch_bounds__(kBlock) k_gather_ml(int64_t n, const int32_t *__restrict__ perm,
                                                       const float4 *__restrict__ p_in, float4 *__restrict__ p_out,
                                                       float4 *__restrict__ ref_out, const float4 *__restrict__ v_in,
                                                       float4 *__restrict__ v_out, const int32_t *__restrict__ lev_in,
                                                       int32_t *__restrict__ lev_out, const int32_t *__restrict__ id_in,
                                                       int32_t *__restrict__ id_out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t i = perm[k];
    const float4 p = p_in[i];
    p_out[k] = p;
    ref_out[k] = p;
    v_out[k] = v_in[i];
    lev_out[k] = lev_in[i];
    id_out[k] = id_in ? id_in[i] : i;
}

__global__ void __launch_bounds__(kBlock) k_scatter(int64_t n, const int32_t *__restrict__ id,
                                                     const float4 *__restrict__ p_in, float4 *__restrict__ p_out,
                                                     const float4 *__restrict__ v_in, float4 *__restrict__ v_out,
                                                     float Lf, int *flags) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int32_t i = id[k];
    if (p_out) {
        float4 p = p_in[k];
        bool ok = wrap1(p.x, Lf);
        ok &= wrap1(p.y, Lf);
        ok &= wrap1(p.z, Lf);
        if (!ok) atomicOr(flags, kFlagDomain);
        p_out[i] = p;
    }
    if (v_out) {
        float4 v = v_in[k];
        v.w = 0.0f;
        v_out[i] = v;
    }
}

__global__ void __launch_bounds__(kBlock) k_candidates_batch(int64_t ncell_total, const BoxDev *__restrict__ boxes,
                                                              int nbox, const int32_t *__restrict__ cell_start,
                                                              unsigned long long *out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (c < ncell_total) {
        const int ni = cell_start[c + 1] - cell_start[c];
        if (ni) {
            int lo = 0, hi = nbox - 1;   // last box whose first cell is <= c
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (boxes[mid].cell_base <= c) lo = mid;
                else hi = mid - 1;
            }
            const int nc = boxes[lo].nc, base = boxes[lo].cell_base;
            const int64_t l = c - base;
            const int cx = (int)(l % nc), cy = (int)((l / nc) % nc), cz = (int)(l / ((int64_t)nc * nc));
            unsigned long long nb = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int jx = (cx + dx + nc) % nc, jy = (cy + dy + nc) % nc, jz = (cz + dz + nc) % nc;
                        const int64_t j = base + ((int64_t)jz * nc + jy) * nc + jx;
                        nb += (unsigned long long)(cell_start[j + 1] - cell_start[j]);
                    }
            v = (unsigned long long)ni * nb;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// Candidate pairs of the chaining mesh: sum_c n_c * sum_{nbr} n_nbr over the
// (2R+1)^3 neighbour cells (R = 1: the 27 cells).
__global__ void __launch_bounds__(kBlock) k_candidates(int nc, int R, const int32_t *__restrict__ cell_start,
                                                        unsigned long long *out) {
    int64_t ncell = (int64_t)nc * nc * nc;
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (c < ncell) {
        int ni = cell_start[c + 1] - cell_start[c];
        if (ni) {
            int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
            unsigned long long nb = 0;
            for (int dz = -R; dz <= R; ++dz)
                for (int dy = -R; dy <= R; ++dy)
                    for (int dx = -R; dx <= R; ++dx) {
                        int jx = (cx + dx + nc) % nc, jy = (cy + dy + nc) % nc, jz = (cz + dz + nc) % nc;
                        int64_t j = ((int64_t)jz * nc + jy) * nc + jx;
                        nb += (unsigned long long)(cell_start[j + 1] - cell_start[j]);
                    }
            v = (unsigned long long)ni * nb;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// ---- positions as (cell, in-cell offset): the precision variant ------------
// The cells step by W = fl32(L / nc), an FP32 value, so that moving an offset
// by one cell is exact for the close pairs that decide the force; cell c
// covers [c W, (c+1) W) and the last cell [(nc-1) W, L), i.e. it absorbs the
// remainder L - nc W (a few ulp of W, of either sign).  A position is
// (c + 1/2) W + off.
// Cell of a global FP64 coordinate x in [0, L) and its FP32 offset from the
// cell centre, x - (c + 1/2) W, in [-W/2, W/2] (last cell: up to W/2 + L - nc W).
__device__ __forceinline__ int ci_split(double x, double W, double iW, int nc, float &off) {
    int c = (int)floor(x * iW);
    c = c < 0 ? 0 : (c > nc - 1 ? nc - 1 : c);
    // the estimate may land one cell off next to a face: decide with exact
    // products (c W is exact in FP64: W has 24 bits, c fewer than 11)
    if (c > 0 && (double)c * W > x) --c;
    else if (c < nc - 1 && (double)(c + 1) * W <= x) ++c;
    off = (float)(x - ((double)c + 0.5) * W);
    return c;
}

__device__ __forceinline__ bool wrap64(double &x, double L) {
    if (!(x >= -L && x < 2.0 * L)) {
        x = 0.0;
        return false;
    }
    if (x < 0.0) x += L;
    else if (x >= L) x -= L;
    if (x >= L) x = 0.0;
    return true;
}

// Optional stream x += drift * v in FP64 on the global position
// ((c + 1/2) W + off), then re-split into (cell, offset) in place; with key !=
// null also the counting-sort keys (the cell) and the sorted-copy source
// dst = (off, m).
__global__ void __launch_bounds__(kBlock) k_key_ci(int64_t n, int32_t *__restrict__ cell, float4 *__restrict__ off,
                                                    const float4 *__restrict__ vel, double drift, int nc, double L,
                                                    double W, double iW, float4 *__restrict__ dst,
                                                    int32_t *__restrict__ key,
                                                    int32_t *__restrict__ rank, uint32_t *__restrict__ count,
                                                    int *flags, int *mass_flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = cell[i];
    float4 o = off[i];
    if (vel) {
        const float4 v = vel[i];
        int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
        double x = fma((double)cx + 0.5, W, (double)o.x), y = fma((double)cy + 0.5, W, (double)o.y),
               z = fma((double)cz + 0.5, W, (double)o.z);
        x = fma(drift, (double)v.x, x);
        y = fma(drift, (double)v.y, y);
        z = fma(drift, (double)v.z, z);
        bool ok = wrap64(x, L);
        ok &= wrap64(y, L);
        ok &= wrap64(z, L);
        if (!ok) atomicOr(flags, kFlagDomain);
        cx = ci_split(x, W, iW, nc, o.x);
        cy = ci_split(y, W, iW, nc, o.y);
        cz = ci_split(z, W, iW, nc, o.z);
        c = (int32_t)(((int64_t)cz * nc + cy) * nc + cx);
        cell[i] = c;
        off[i] = o;
    }
    if (!key) return;
    if (o.w != off[0].w) atomicOr(mass_flag, 1);
    dst[i] = o;
    key[i] = c;
    rank[i] = (int32_t)atomicAdd(&count[c], 1u);
}

__global__ void __launch_bounds__(kBlock) k_ci_from_f64(int64_t n, const double *__restrict__ x64,
                                                         const float *__restrict__ mass, int nc, double L, double W,
                                                         double iW, int32_t *__restrict__ cell,
                                                         float4 *__restrict__ off,
                                                         int *flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = x64[3 * i], y = x64[3 * i + 1], z = x64[3 * i + 2];
    bool ok = wrap64(x, L);
    ok &= wrap64(y, L);
    ok &= wrap64(z, L);
    if (!ok) atomicOr(flags, kFlagDomain);
    float4 o;
    int cx = ci_split(x, W, iW, nc, o.x), cy = ci_split(y, W, iW, nc, o.y), cz = ci_split(z, W, iW, nc, o.z);
    o.w = mass ? mass[i] : 1.0f;
    cell[i] = (int32_t)(((int64_t)cz * nc + cy) * nc + cx);
    off[i] = o;
}

__global__ void __launch_bounds__(kBlock) k_ci_to_f64(int64_t n, const int32_t *__restrict__ cell,
                                                       const float4 *__restrict__ off, int nc, double W,
                                                       double *__restrict__ x64) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t c = cell[i];
    const float4 o = off[i];
    x64[3 * i] = fma((double)(c % nc) + 0.5, W, (double)o.x);
    x64[3 * i + 1] = fma((double)((c / nc) % nc) + 0.5, W, (double)o.y);
    x64[3 * i + 2] = fma((double)(c / (nc * nc)) + 0.5, W, (double)o.z);
}

// ---- multi-level stepping ------------------------------------------------
// Kick count of every particle from its cell's density (Eq. (kicks)):
// l = floor(floor(count nc^3 / n) / d) + 1, clamped to [lmin, lmax] (d <= 0: lmax);
// present[l] = 1 for the counts that occur.
__global__ void __launch_bounds__(kBlock) k_levels(int64_t n, int64_t ncell, const int32_t *__restrict__ key,
                                                    const uint32_t *__restrict__ count, int d, int lmin, int lmax,
                                                    int32_t *__restrict__ level, int *__restrict__ present) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int l = 0;   // 0: no particle on this lane
    if (i < n) {
        int64_t q = lmax;
        if (d > 0) {
            const int64_t ratio = (int64_t)count[key[i]] * ncell / n;
            q = ratio / d + 1;
            if (q > lmax) q = lmax;
        }
        l = (int)(q < lmin ? lmin : q);
        level[i] = l;
    }
    // particles per kick count, one atomic per distinct count in the warp
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    if (l > 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&present[l], __popc(peers));
}

// Stream sorted positions in place, without wrapping (inside one multi-level
// step a particle stays near the cell it was binned in; the step's end wraps).
// With p0, also the largest per-axis distance from the binned position (as
// float bits) into *disp.
__global__ void __launch_bounds__(kBlock) k_stream(int64_t n, float4 *__restrict__ pos,
                                                    const float4 *__restrict__ vel, float drift,
                                                    const float4 *__restrict__ p0, unsigned *disp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.0f;
    if (i < n) {
        float4 p = pos[i];
        const float4 v = vel[i];
        p.x = __fmaf_rn(drift, v.x, p.x);
        p.y = __fmaf_rn(drift, v.y, p.y);
        p.z = __fmaf_rn(drift, v.z, p.z);
        pos[i] = p;
        if (p0) {
            const float4 q = p0[i];
            m = fmaxf(fabsf(p.x - q.x), fmaxf(fabsf(p.y - q.y), fabsf(p.z - q.z)));
        }
    }
    if (!p0) return;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(disp, __float_as_uint(m));
}

__global__ void k_ml_decide(const unsigned *disp_bits, float half_lim, cudaGraphConditionalHandle handle,
                            unsigned long long *rebins, int *flags) {
    const float d = __uint_as_float(*disp_bits);
    bool rebin = d > half_lim;
    if (!isfinite(d)) {
        atomicOr(flags, kFlagDomain);
        rebin = false;
    }
    cudaGraphSetConditional(handle, rebin ? 1u : 0u);
    if (rebin) *rebins += 1ull;
}

__global__ void __launch_bounds__(kBlock) k_ml_commit(int64_t n, const float4 *__restrict__ v_from,
                                                       float4 *__restrict__ v_to, const int32_t *__restrict__ lev_from,
                                                       int32_t *__restrict__ lev_to,
                                                       const int32_t *__restrict__ id_from,
                                                       int32_t *__restrict__ id_to, unsigned *disp_bits,
                                                       unsigned body_launches, unsigned long long *launches) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *disp_bits = 0u;
        *launches += body_launches;
    }
    if (i >= n) return;
    v_to[i] = v_from[i];
    lev_to[i] = lev_from[i];
    id_to[i] = id_from[i];
}

// Work items of one multi-level event, one warp per cell: the particles
// kicked now form runs of consecutive sorted particles (the binning orders
// each cell by kick count); the warp reads the cell 32 particles at a time,
// finds the runs in the ballot of kicked lanes, and cuts each run into
// ceil(run / cap) items of near-equal size.  Items are appended through
// n_items (their order only changes which warp takes which item, not any sum).
__device__ __forceinline__ void emit_run(int64_t c, int32_t lo, int32_t hi, uint32_t cap, int lane, int4 *items,
                                         int32_t *n_items, int32_t max_items, int *flags) {
    const uint32_t cnt = (uint32_t)(hi - lo);
    const uint32_t m = (cnt + cap - 1) / cap;
    int32_t it = 0;
    if (lane == 0) it = atomicAdd(n_items, (int32_t)m);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it + (int64_t)m > max_items) {   // cannot happen: every item holds a particle
        if (lane == 0) atomicOr(flags, kFlagItems);
        return;
    }
    for (uint32_t k = lane; k < m; k += 32) {
        const uint32_t a = (uint32_t)((uint64_t)cnt * k / m), e = (uint32_t)((uint64_t)cnt * (k + 1) / m);
        items[it + k] = make_int4((int)c, (int)(lo + a), (int)(e - a), item_shape(e - a));
    }
}

__global__ void __launch_bounds__(kBlock) k_items_kicked(int64_t ncell, const int32_t *__restrict__ cell_start,
                                                          const int32_t *__restrict__ level, KickTable kt,
                                                          uint32_t cap, int4 *__restrict__ items,
                                                          int32_t *__restrict__ n_items, int32_t max_items,
                                                          int *flags) {
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncell) return;
    const int32_t a = cell_start[c], b = cell_start[c + 1];
    int32_t open = -1;   // start of the run in progress
    for (int32_t base = a; base < b; base += 32) {
        const int32_t q = base + lane;
        const unsigned m = __ballot_sync(0xffffffffu, q < b && kt.h[level[q]] != 0.0f);
        const int len = min(32, b - base);
        int pos = 0;
        while (pos < len) {
            if (open < 0) {
                const unsigned rest = m >> pos;
                if (!rest) break;
                pos += __ffs(rest) - 1;
                open = base + pos;
            }
            const unsigned gap = ~m >> pos;   // lanes >= len are never kicked
            if (!gap) break;                  // the run goes on into the next 32
            pos += __ffs(gap) - 1;
            emit_run(c, open, base + pos, cap, lane, items, n_items, max_items, flags);
            open = -1;
        }
    }
    if (open >= 0) emit_run(c, open, b, cap, lane, items, n_items, max_items, flags);
}


inline unsigned blocks_for(int64_t n, int per = kBlock) { return (unsigned)((n + per - 1) / per); }

// Size class of an item, 0 for the largest: ni >= 150 -> 0, ni < 10 -> 15.
__device__ __forceinline__ int item_class(int ni) { return kItemClasses - 1 - min(ni / 10, kItemClasses - 1); }

__global__ void __launch_bounds__(kBlock) k_item_hist(const int4 *__restrict__ items, const int32_t *__restrict__ n_items,
                                                       uint32_t *__restrict__ cls) {
    __shared__ uint32_t h[kItemClasses];
    if (threadIdx.x < kItemClasses) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it < *n_items) atomicAdd(&h[item_class(items[it].z)], 1u);
    __syncthreads();
    if (threadIdx.x < kItemClasses && h[threadIdx.x]) atomicAdd(&cls[threadIdx.x], h[threadIdx.x]);
}

// Exclusive scan of the class counts into the class cursors (one warp).
__global__ void k_item_bases(uint32_t *cls) {
    const int lane = threadIdx.x;
    uint32_t v = lane < kItemClasses ? cls[lane] : 0u, x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane < kItemClasses) cls[kItemClasses + lane] = x - v;
}

// Each block ranks its items per class in shared memory, reserves one range
// per class from the cursors and writes the item indices there.
__global__ void __launch_bounds__(kBlock) k_item_place(const int4 *__restrict__ items,
                                                        const int32_t *__restrict__ n_items, uint32_t *__restrict__ cls,
                                                        int32_t *__restrict__ order) {
    __shared__ uint32_t h[kItemClasses], base[kItemClasses];
    if (threadIdx.x < kItemClasses) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = -1;
    uint32_t local = 0;
    if (it < *n_items) {
        c = item_class(items[it].z);
        local = atomicAdd(&h[c], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kItemClasses && h[threadIdx.x])
        base[threadIdx.x] = atomicAdd(&cls[kItemClasses + threadIdx.x], h[threadIdx.x]);
    __syncthreads();
    if (c >= 0) order[base[c] + local] = (int32_t)it;
}

}  // namespace

size_t scan_tmp_elems(int64_t len) {
    size_t total = 0;
    int64_t nb = (len + kScanTile - 1) / kScanTile;
    while (nb > 1) {
        total += (size_t)nb;
        nb = (nb + kScanTile - 1) / kScanTile;
    }
    return total + 1;
}

int64_t max_items(int64_t n, int64_t ncell) { return ncell + n / kItemCapMin + 1; }

cudaError_t items_heavy_first(const BinBuffers &b, int64_t max_items, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.item_cls, 0, sizeof(uint32_t) * 2 * kItemClasses, s);
    if (e != cudaSuccess) return e;
    k_item_hist<<<blocks_for(max_items), kBlock, 0, s>>>(b.items, b.n_items, b.item_cls);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_item_bases<<<1, 32, 0, s>>>(b.item_cls);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_item_place<<<blocks_for(max_items), kBlock, 0, s>>>(b.items, b.n_items, b.item_cls, b.order);
    note_launch();
    return cudaGetLastError();
}

void carve_bin(Carver &c, int64_t n, int64_t ncell, BinBuffers *b, bool sub_order) {
    b->key = c.take<int32_t>(n);
    b->rank = c.take<int32_t>(n);
    b->count = c.take<uint32_t>(ncell);
    b->packed = c.take<unsigned long long>(ncell);
    b->scan_tmp = c.take<unsigned long long>(scan_tmp_elems(ncell));
    b->cell_start = c.take<int32_t>(ncell + 1);
    b->item_start = nullptr;
    b->perm_tmp = c.take<int32_t>(n);
    b->perm = c.take<int32_t>(n);
    b->items = c.take<int4>(max_items(n, ncell));
    b->order = c.take<int32_t>(max_items(n, ncell));
    b->item_cls = c.take<uint32_t>(2 * kItemClasses);
    b->n_items = c.take<int32_t>(1);
    b->mass_flag = c.take<int>(1);
    b->big_list = c.take<int32_t>(n / (kBigCell + 1) + 1);
    b->big_count = c.take<int>(1);
    b->sub = sub_order ? c.take<uint8_t>(n) : nullptr;
    b->order_tmp = sub_order ? c.take<unsigned long long>(n) : nullptr;
}

namespace {
ItemRule item_rule(int item_cap, int split_max) {
    if (!item_cap) return ItemRule{(uint32_t)kItemMax, 0xffffffffu};
    return ItemRule{(uint32_t)item_cap, (uint32_t)split_max};
}

// Counting sort by key and work items, shared by the single-box and batched passes.
cudaError_t bin_sort(int64_t n, int64_t ncell, const BinBuffers &b, bool make_items, const BoxDev *boxes, int nbox,
                     cudaStream_t s, ItemRule cap = {kItemMax, 0xffffffffu}, const uint8_t *sub = nullptr,
                     uint32_t row_below = 0, bool stretches = false) {
    cudaError_t e;
    k_pack<<<blocks_for(ncell), kBlock, 0, s>>>(ncell, b.count, b.packed, cap);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(b.packed, ncell, b.scan_tmp, s)) != cudaSuccess) return e;
    if (n > 0) {
        k_place<<<blocks_for(n), kBlock, 0, s>>>(n, b.key, b.rank, b.packed, b.perm_tmp, sub, b.order_tmp);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(b.big_count, 0, sizeof(int), s)) != cudaSuccess) return e;
        if (sub && n > kOrdSubMaxRows)
            k_order_sub<<<blocks_for(ncell * 32), kBlock, 0, s>>>(ncell, b.count, b.packed, b.perm_tmp, b.perm,
                                                                  b.big_list, b.big_count, b.order_tmp, row_below);
        else if (sub)
            k_order_rows<true><<<blocks_for(ncell, kOrdCells), kBlock, 0, s>>>(
                ncell, b.count, b.packed, b.perm_tmp, b.perm, b.big_list, b.big_count, b.order_tmp, row_below,
                stretches ? 1 : 0);
        else
            k_order_rows<false><<<blocks_for(ncell, kOrdCells), kBlock, 0, s>>>(
                ncell, b.count, b.packed, b.perm_tmp, b.perm, b.big_list, b.big_count, nullptr, 0u,
                stretches ? 1 : 0);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (n > (int64_t)kBigCell) {
            k_order_big<<<256, kOrderThreads, 0, s>>>(b.count, b.packed, b.perm_tmp, b.perm, b.big_list, b.big_count);
            note_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    k_items<<<blocks_for(ncell), kBlock, 0, s>>>(ncell, n, b.count, b.packed, b.cell_start, b.items, b.n_items,
                                                 make_items ? 1 : 0, boxes, nbox, cap);
    note_launch();
    return cudaGetLastError();
}
}  // namespace

cudaError_t bin_build(const Geometry &g, int64_t n, const float4 *src, const float4 *vel, float drift,
                      float4 *dst, const BinBuffers &b, int *d_flags, bool make_items, cudaStream_t s,
                      int item_cap, int split_max, const int32_t *sub_level, bool sorted_input) {
    if (item_cap != 0 && (item_cap < kItemCapMin || item_cap > kItemMax)) return cudaErrorInvalidValue;
    if (split_max < 1 || ((item_cap || sub_level) && !b.sub)) return cudaErrorInvalidValue;
    uint8_t *sub = (item_cap || sub_level) ? b.sub : nullptr;
    cudaError_t e = cudaMemsetAsync(b.count, 0, sizeof(uint32_t) * g.ncell, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.mass_flag, 0, sizeof(int), s)) != cudaSuccess) return e;
    if (n > 0) {
        k_key<<<blocks_for(n), kBlock, 0, s>>>(n, src, vel, drift, dst, g.Lf, g.inv_w, g.Ld, g.nc, b.key,
                                               b.rank, b.count, d_flags, b.mass_flag, sub, sub_level);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // a cell that becomes one work item keeps row order (not with kick counts,
    // whose order an event's items rely on)
    const uint32_t row_below = (item_cap && !sub_level) ? (uint32_t)item_cap : 0u;
    return bin_sort(n, g.ncell, b, make_items, nullptr, 1, s, item_rule(item_cap, split_max), sub, row_below,
                    sorted_input);
}

cudaError_t ml_levels(const Geometry &g, int64_t n, const BinBuffers &b, int d, int lmin, int lmax, int32_t *level,
                      int *present, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_levels<<<blocks_for(n), kBlock, 0, s>>>(n, g.ncell, b.key, b.count, d, lmin, lmax, level, present);
    note_launch();
    return cudaGetLastError();
}

cudaError_t ml_decide(const unsigned *disp_bits, float half_lim, cudaGraphConditionalHandle handle,
                      unsigned long long *rebins, int *d_flags, cudaStream_t s) {
    k_ml_decide<<<1, 1, 0, s>>>(disp_bits, half_lim, handle, rebins, d_flags);
    note_launch();
    return cudaGetLastError();
}

cudaError_t ml_commit(int64_t n, const float4 *v_from, float4 *v_to, const int32_t *lev_from, int32_t *lev_to,
                      const int32_t *id_from, int32_t *id_to, unsigned *disp_bits, unsigned body_launches,
                      unsigned long long *launches, cudaStream_t s) {
    k_ml_commit<<<blocks_for(n > 0 ? n : 1), kBlock, 0, s>>>(n, v_from, v_to, lev_from, lev_to, id_from, id_to,
                                                             disp_bits, body_launches, launches);
    note_launch();
    return cudaGetLastError();
}

cudaError_t stream_sorted(int64_t n, float4 *pos, const float4 *vel, float drift, const float4 *p0, unsigned *disp,
                          cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_stream<<<blocks_for(n), kBlock, 0, s>>>(n, pos, vel, drift, p0, disp);
    note_launch();
    return cudaGetLastError();
}

// Work items of one multi-level event from the runs of kicked particles.
cudaError_t items_kicked(int64_t ncell, const BinBuffers &b, const int32_t *level, const KickTable &kt, int cap,
                         int4 *items, int32_t max_items, int *d_flags, cudaStream_t s) {
    if (cap < kItemCapMin || cap > kItemMax) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(b.n_items, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_items_kicked<<<blocks_for(ncell * 32), kBlock, 0, s>>>(ncell, b.cell_start, level, kt, (uint32_t)cap, items,
                                                             b.n_items, max_items, d_flags);
    note_launch();
    return cudaGetLastError();
}


cudaError_t bin_build_batch(int nbox, const BoxDev *boxes, int64_t n_total, int64_t ncell_total,
                            const float4 *pos_pool, const float4 *vel_pool, float4 *dst, int32_t *id,
                            const BinBuffers &b, int *d_flags, cudaStream_t s, int item_cap, int split_max) {
    if (item_cap != 0 && (item_cap < kItemCapMin || item_cap > kItemMax)) return cudaErrorInvalidValue;
    if (split_max < 1 || (item_cap && !b.sub)) return cudaErrorInvalidValue;
    uint8_t *sub = item_cap ? b.sub : nullptr;
    cudaError_t e = cudaMemsetAsync(b.count, 0, sizeof(uint32_t) * ncell_total, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.mass_flag, 0, sizeof(int), s)) != cudaSuccess) return e;
    if (n_total > 0) {
        k_bkey<<<blocks_for(n_total), kBlock, 0, s>>>(n_total, nbox, boxes, pos_pool, vel_pool, dst, id, b.key,
                                                      b.rank, b.count, d_flags, b.mass_flag, sub);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // as bin_build: a cell that becomes one work item keeps row order
    return bin_sort(n_total, ncell_total, b, true, boxes, nbox, s, item_rule(item_cap, split_max), sub,
                    item_cap ? (uint32_t)item_cap : 0u, false);
}

cudaError_t bin_build_ci(const Geometry &g, int64_t n, int32_t *cell, float4 *off, const float4 *vel, double drift,
                         float4 *dst, const BinBuffers &b, int *d_flags, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.count, 0, sizeof(uint32_t) * g.ncell, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.mass_flag, 0, sizeof(int), s)) != cudaSuccess) return e;
    if (n > 0) {
        k_key_ci<<<blocks_for(n), kBlock, 0, s>>>(n, cell, off, vel, drift, g.nc, g.Ld, ci_step(g), 1.0 / ci_step(g),
                                                  dst, b.key, b.rank, b.count, d_flags, b.mass_flag);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return bin_sort(n, g.ncell, b, true, nullptr, 1, s);
}

cudaError_t drift_ci(const Geometry &g, int64_t n, int32_t *cell, float4 *off, const float4 *vel, double drift,
                     int *d_flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_key_ci<<<blocks_for(n), kBlock, 0, s>>>(n, cell, off, vel, drift, g.nc, g.Ld, ci_step(g), 1.0 / ci_step(g),
                                              nullptr, nullptr, nullptr, nullptr, d_flags, nullptr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t ci_from_f64(const Geometry &g, int64_t n, const double *x64, const float *mass, int32_t *cell,
                        float4 *off, int *d_flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_ci_from_f64<<<blocks_for(n), kBlock, 0, s>>>(n, x64, mass, g.nc, g.Ld, ci_step(g), 1.0 / ci_step(g), cell, off,
                                                   d_flags);
    note_launch();
    return cudaGetLastError();
}

cudaError_t ci_to_f64(const Geometry &g, int64_t n, const int32_t *cell, const float4 *off, double *x64,
                      cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_ci_to_f64<<<blocks_for(n), kBlock, 0, s>>>(n, cell, off, g.nc, ci_step(g), x64);
    note_launch();
    return cudaGetLastError();
}

cudaError_t gather_sorted(int64_t n, const int32_t *perm, const float4 *p_in, float4 *p_out, const float4 *v_in,
                          float4 *v_out, const int32_t *id_in, int32_t *id_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gather<<<blocks_for(n), kBlock, 0, s>>>(n, perm, p_in, p_out, v_in, v_out, id_in, id_out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t gather_ml(int64_t n, const int32_t *perm, const float4 *p_in, float4 *p_out, float4 *ref_out,
                      const float4 *v_in, float4 *v_out, const int32_t *lev_in, int32_t *lev_out, const int32_t *id_in,
                      int32_t *id_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_gather_ml<<<blocks_for(n), kBlock, 0, s>>>(n, perm, p_in, p_out, ref_out, v_in, v_out, lev_in, lev_out, id_in,
                                                 id_out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scatter_rows(int64_t n, const int32_t *id, const float4 *p_in, float4 *p_out, const float4 *v_in,
                         float4 *v_out, float Lf, int *d_flags, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_scatter<<<blocks_for(n), kBlock, 0, s>>>(n, id, p_in, p_out, v_in, v_out, Lf, d_flags);
    note_launch();
    return cudaGetLastError();
}

cudaError_t candidate_count_batch(int64_t ncell_total, const BoxDev *boxes, int nbox, const int32_t *cell_start,
                                  unsigned long long *out, cudaStream_t s) {
    k_candidates_batch<<<blocks_for(ncell_total), kBlock, 0, s>>>(ncell_total, boxes, nbox, cell_start, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t candidate_count(const Geometry &g, const int32_t *cell_start, unsigned long long *out, cudaStream_t s) {
    k_candidates<<<blocks_for(g.ncell), kBlock, 0, s>>>(g.nc, g.R, cell_start, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace hacc
