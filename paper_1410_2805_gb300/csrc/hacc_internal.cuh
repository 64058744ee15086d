// Internal declarations of the hacc library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/hacc.h"

namespace hacc {

// Device-side status flags (one int each, OR-ed by kernels).
enum DeviceFlag : int {
    kFlagDomain = 1,   // a coordinate outside [-L, 2L) or not finite
    kFlagItems = 4,    // a work-item list ran out of room (an internal bound failed)
};

// Chunking of a chaining-mesh cell into force work items: a cell of n
// particles is one item when n <= cap, else ceil(n/cap) items of near-equal
// size; each item is processed by one warp (see item_shape in bin.cu).
constexpr int kItemMax = 160;   // particles per work item at most (5 per lane)
constexpr int kItemMin = 32;    // smallest per-event item cap of the multi-level step
constexpr int kItemCapMin = 16; // smallest item cap of any path (sizes the item arrays)
constexpr int kDefaultItemCap = 48;  // item cap of the automatic choice for small calls
constexpr int64_t kAutoItemCapMaxN = (int64_t)1 << 22;  // largest call that the automatic choice splits
constexpr int kDefaultSplitMax = INT32_MAX;  // cells above this keep items of up to kItemMax

struct Scratch {
    char *base = nullptr;
    size_t cap = 0;
};

}  // namespace hacc

struct hacc_ctx {
    int device = 0;
    size_t budget = 0;         // 0 = unbounded
    int num_sms = 0;
    hacc::Scratch scratch;
    int *d_flags = nullptr;    // device status word
    std::string last_error;
    hacc_status pending = HACC_OK;
    // device staging of the *_host entry points (apart from the scratch arena,
    // so that the device entry points they call may grow the arena)
    void *io_base = nullptr;
    size_t io_cap = 0;
    // cuFFT state for the PM stage (owned by pm.cu)
    void *pm_state = nullptr;
    // statistics (hacc_stats_*)
    bool timing = false, counting = false;
    int64_t launches = 0, force_launches = 0;
    int64_t ml_rebins = 0;
    int variant = 0;                          // pair-kernel variant (hacc_tune)
    int stencil = 1;                          // single-box force paths: 1 (27 cells) or 2 (125 cells of half width)
    int item_cap = -1;                        // work-item cap of the force paths (0: cell-wide items, -1: auto)
    int split_max = hacc::kDefaultSplitMax;   // cells above this many particles keep items of up to kItemMax
    int queue_order = 0;                      // 1: largest work items first (calls of 2^20 particles and more), 0: cell order
    double force_ms = 0.0;
    double build_ms = 0.0;                    // event-timed chaining-mesh builds (binning + sorted gather)
    int64_t builds = 0;
    unsigned long long *d_pairs = nullptr;   // [2] candidate, within (device)
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
    std::vector<int> ev_kind;                 // per ev_used entry: 0 pair-force launch, 1 chaining-mesh build
    // batches (batch.cu): pinned staging of box tables, cached CUDA graph
    void *stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t stage_event = nullptr;
    void *graph_exec = nullptr;
    uint64_t graph_key = 0;
    // batched launch shape chosen by hacc_batch_tune for one batch geometry
    uint64_t btune_key = 0;
    int btune_variant = 0, btune_cap = 0, btune_order = 0;
    int64_t graph_launches = 0, graph_forces = 0;
    // multi-level steps (api.cu): cached CUDA graph of the event loop, with a
    // conditional rebinning node per event; captured on a stream of its own
    void *ml_exec = nullptr;
    uint64_t ml_key = 0;
    int64_t ml_launches = 0, ml_forces = 0;
    void *cap_stream = nullptr, *cap_stream2 = nullptr;
    // host-buffer full steps (api.cu): a second stream and events that let the
    // velocity upload and the position download overlap the PM stages
    void *io_stream = nullptr;
    void *io_ev[3 + 16] = {};   // [0..2] step events, [3..] the PM stage's chunk events (kPmChunks)
    bool ml_graph_off = false;   // set when the device refused the graph once
};

namespace hacc {
// Item cap of a force call over n particles (hacc_set_item_cap): the set
// value, or automatically kDefaultItemCap up to kAutoItemCapMaxN particles
// (short launches, where the longest items of dense cells set the tail) and
// cell-wide items above.
inline int item_cap_for(const hacc_ctx *ctx, int64_t n) {
    if (ctx->item_cap >= 0) return ctx->item_cap;
    return n <= kAutoItemCapMaxN ? kDefaultItemCap : 0;
}
}  // namespace hacc

namespace hacc {

// Bump allocator over a scratch region; with base == nullptr it only sizes.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(char *b) : base(b) {}
    template <class T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (count ? count : 1);
        return p;
    }
};

// Kernel launches of the calling API function are counted into the context
// that entered it (set per call; the library is not re-entrant per context).
extern thread_local int64_t *tl_launches;
inline void note_launch(int k = 1) {
    if (tl_launches) *tl_launches += k;
}

hacc_status set_error(hacc_ctx *ctx, hacc_status st, const std::string &msg);

// Start of every entry point on a context: clear the message, make the
// context's device current, count kernel launches into the context.
hacc_status hacc_enter(hacc_ctx *ctx);

#define HACC_STATUS_RETURN(x)                 \
    do {                                      \
        hacc_status st_r_ = (x);              \
        if (st_r_ != HACC_OK) return st_r_;   \
    } while (0)
#define HACC_CUDA_RETURN(x, what) HACC_STATUS_RETURN(::hacc::check_cuda(ctx, (x), what))

void batch_destroy(hacc_ctx *ctx);
// Scratch bytes one batched tick (hacc_batch_tick) takes from the context's
// arena for n_total particles in ncell_total cells of nbox boxes (the carving
// the tick itself uses, plus its alignment slack).
size_t batch_tick_scratch_bytes(int64_t n_total, int64_t ncell_total, int64_t nbox);
int32_t default_nc(double L, double r_cut);
hacc_status check_cuda(hacc_ctx *ctx, cudaError_t e, const char *what);
hacc_status ensure_scratch(hacc_ctx *ctx, size_t bytes, cudaStream_t stream);

// Validated geometry of one box.
struct Geometry {
    float Lf;        // box side (FP32 value)
    double Ld;       // same value in FP64
    int nc;          // chaining-mesh cells per side
    int64_t ncell;   // nc^3
    float inv_w;     // fl(nc / L), first guess of the cell index
    int R = 1;       // neighbour cells per side searched: 1 (27 cells >= r_cut), 2 (125 cells >= r_cut/2)
};

hacc_status make_geometry(hacc_ctx *ctx, const hacc_box *box, float r_cut, Geometry *g);

// Cell step of the (cell, offset) precision variant: W = fl32(L / nc), an FP32
// value, so that whole cell steps added to an FP32 offset are exact where it
// matters (close pairs).  Cell c covers [c W, (c+1) W), the last cell
// [(nc-1) W, L): it absorbs the remainder L - nc W, which is exact in FP64 and
// an FP32 value (a multiple of ulp(W) below nc ulp(W)).
inline double ci_step(const Geometry &g) { return (double)(float)(g.Ld / g.nc); }
inline double ci_rem(const Geometry &g) { return g.Ld - (double)g.nc * ci_step(g); }

// Force constants in the form the kernel evaluates.
struct ForceConsts {
    float T;        // fl(r_cut^2 + eps): cutoff test on t = s + eps
    float eps;
    float q[6];     // P5(t - eps) = sum_k q[k] t^k
    float G;
    float u[7];     // potential: sum_k c_k (t-eps)^(k+1) / (2(k+1)) = sum_k u[k] t^k
    float phi0;     // phi(r_cut^2) before the shift
};

hacc_status make_force_consts(hacc_ctx *ctx, const hacc_split *split, const Geometry &g, ForceConsts *fc);

// Wrap one FP32 coordinate into [0, L): x<0 -> x+L, x>=L -> x-L, a sum that
// rounds to L becomes 0.  Returns false (and leaves 0) outside [-L, 2L).
__device__ __forceinline__ bool wrap1(float &x, float Lf) {
    float v = x;
    if (!(v >= -Lf && v < 2.0f * Lf)) {
        x = 0.0f;
        return false;
    }
    if (v < 0.0f) v = __fadd_rn(v, Lf);
    else if (v >= Lf) v = __fsub_rn(v, Lf);
    if (v >= Lf) v = 0.0f;
    x = v;
    return true;
}

// Kick factor per kick count l (index 1..kMaxLevels) at one event of a
// multi-level step: dt / l if particles with l kicks are kicked now, else 0.
constexpr int kMaxLevels = 16;
struct KickTable {
    float h[kMaxLevels + 1];
};

// ---- batches of boxes (batch.cu) -----------------------------------------
// One box of a batched tick, as the kernels see it.
struct BoxDev {
    float L;             // side (FP32 value)
    float inv_w;         // fl(nc / L)
    double Ld;           // side in FP64 (same value)
    int nc;              // chaining-mesh cells per side
    int cell_base;       // first global cell id of this box
    int part_base;       // first tick-scratch index of this box
    int n;               // particles
    long long row_off;   // first row of this box in the pool arrays
    float h;             // kick factor of this tick
    float pre;           // stream applied before binning (h/2 on a run's first sub-cycle, else 0)
    float post;          // stream after the kick (h, or h/2 on a run's last sub-cycle)
    int orig;            // index of the box in the caller's list
};

// ---- binning (bin.cu) ----------------------------------------------------
struct BinBuffers {
    int32_t *key;          // [n]
    int32_t *rank;         // [n]
    uint32_t *count;       // [ncell]
    unsigned long long *packed;  // [ncell] scan workspace
    unsigned long long *scan_tmp;
    int32_t *cell_start;   // [ncell + 1]
    int32_t *item_start;   // [ncell + 1]
    int32_t *perm_tmp;     // [n]
    int32_t *perm;         // [n]
    int4 *items;           // [max_items]
    int32_t *order;        // [max_items] work-queue order of the items (heavy_first), or unused
    uint32_t *item_cls;    // [2 kItemClasses] per-class counts and cursors of heavy_first
    int32_t *n_items;      // [1] device
    int *mass_flag;        // [1] device: nonzero if some mass differs from the first
    int32_t *big_list;     // cells too large for the warp-level ordering
    int *big_count;
    uint8_t *sub;                  // [n] Morton sub-cell of each input row (item_cap > 0), or null
    unsigned long long *order_tmp; // [n] (sub-cell << 32 | row) in the slots of perm_tmp, or null
};

size_t scan_tmp_elems(int64_t len);
// Work-queue order of the force items: largest items first (classes of item
// size, a counting sort of item indices into b.order), so that the heaviest
// items do not set the tail of a persistent launch.  Changes which warp takes
// which item, never a sum.  max_items bounds the device item count.
constexpr int kItemClasses = 16;
constexpr int64_t kHeavyFirstMinN = (int64_t)1 << 20;   // smaller calls keep the plain order
cudaError_t items_heavy_first(const BinBuffers &b, int64_t max_items, cudaStream_t s);
int64_t max_items(int64_t n, int64_t ncell);
// sub_order = false leaves out the sub-cell arrays (item_cap must then be 0).
void carve_bin(Carver &c, int64_t n, int64_t ncell, BinBuffers *b, bool sub_order = true);

// Wrap (optionally after a drift x += d v) src into dst and compute keys,
// counts, the permutation, cell starts and force work items.  vel may be
// null (no drift).  dst may equal src.  item_cap = 0: ascending input row
// within each cell (the stable counting sort) and items of up to kItemMax;
// item_cap in [kItemCapMin, kItemMax]: within each cell of up to kBigCell
// particles the rows are ordered by the particle's 4x4x4 sub-cell (Morton
// order, z bit first; ties by input row), and the work items are runs of at
// most item_cap particles of that order, so an item covers a compact part of
// its cell; cells of more than split_max particles get items of up to
// kItemMax.  sub_level (nullable, n kick counts aligned with src): order each
// cell by (kick count, octant, input row) instead, so that the particles of a
// kick count are consecutive.
// sorted_input: src is in the cell order of a previous binning of the same
// particles (the sub-cycle loop), which makes the in-cell ordering cheap.
// With an item cap (and no kick counts), a cell that becomes one work item
// keeps input-row order: the sub-cell order only shapes the items of cells
// that are cut into several.
cudaError_t bin_build(const Geometry &g, int64_t n, const float4 *src, const float4 *vel, float drift,
                      float4 *dst, const BinBuffers &b, int *d_flags, bool make_items, cudaStream_t s,
                      int item_cap = 0, int split_max = kDefaultSplitMax, const int32_t *sub_level = nullptr,
                      bool sorted_input = false);

// Batched binning of nbox boxes (table `boxes` on the device, ascending
// part_base and cell_base): for every tick-scratch index t the particle at
// pool row boxes[b].row_off + t - part_base is streamed by pre, wrapped,
// binned into global cell cell_base + local id; dst[t] = its position,
// id[t] = its pool row.  Work items carry the box in item.w >> 8.  item_cap
// as for bin_build (ties in the sub-cell order by scratch index).
cudaError_t bin_build_batch(int nbox, const BoxDev *boxes, int64_t n_total, int64_t ncell_total,
                            const float4 *pos_pool, const float4 *vel_pool, float4 *dst, int32_t *id,
                            const BinBuffers &b, int *d_flags, cudaStream_t s, int item_cap = 0,
                            int split_max = kDefaultSplitMax);

// Multi-level stepping: kick counts from the cell densities of the last
// binning (keys/counts in b; present[l] += particles with l kicks); in-place stream of
// sorted positions with the largest drift from the binned ones; the rebinning
// gather (positions, reference positions, velocities, kick counts, input
// rows); the work items of an event are built by items_kicked below.
cudaError_t ml_levels(const Geometry &g, int64_t n, const BinBuffers &b, int d, int lmin, int lmax, int32_t *level,
                      int *present, cudaStream_t s);
cudaError_t stream_sorted(int64_t n, float4 *pos, const float4 *vel, float drift, const float4 *p0, unsigned *disp,
                          cudaStream_t s);
cudaError_t gather_ml(int64_t n, const int32_t *perm, const float4 *p_in, float4 *p_out, float4 *ref_out,
                      const float4 *v_in, float4 *v_out, const int32_t *lev_in, int32_t *lev_out, const int32_t *id_in,
                      int32_t *id_out, cudaStream_t s);
// Graph form of the drift check: set the conditional node `handle` to
// whether the largest drift passed `half_lim` (and count the rebinning in
// *rebins); a non-finite drift raises the domain flag instead.  ml_commit
// (last node of the rebinning body) moves the gathered arrays back into
// place, clears the drift word and adds the body's kernel count to *launches.
cudaError_t ml_decide(const unsigned *disp_bits, float half_lim, cudaGraphConditionalHandle handle,
                      unsigned long long *rebins, int *d_flags, cudaStream_t s);
cudaError_t ml_commit(int64_t n, const float4 *v_from, float4 *v_to, const int32_t *lev_from, int32_t *lev_to,
                      const int32_t *id_from, int32_t *id_to, unsigned *disp_bits, unsigned body_launches,
                      unsigned long long *launches, cudaStream_t s);
// Work items of a multi-level event: the runs of particles kicked now (level:
// kick counts in sorted order; cells ordered by kick count), in items of at
// most cap particles written to items (room for max_items).
cudaError_t items_kicked(int64_t ncell, const BinBuffers &b, const int32_t *level, const KickTable &kt, int cap,
                         int4 *items, int32_t max_items, int *d_flags, cudaStream_t s);

// Precision variant: positions as (cell id, FP32 in-cell offset, mass).
// bin_build_ci optionally streams (FP64 on the global position) first.
cudaError_t bin_build_ci(const Geometry &g, int64_t n, int32_t *cell, float4 *off, const float4 *vel, double drift,
                         float4 *dst, const BinBuffers &b, int *d_flags, cudaStream_t s);
cudaError_t drift_ci(const Geometry &g, int64_t n, int32_t *cell, float4 *off, const float4 *vel, double drift,
                     int *d_flags, cudaStream_t s);
cudaError_t ci_from_f64(const Geometry &g, int64_t n, const double *x64, const float *mass, int32_t *cell,
                        float4 *off, int *d_flags, cudaStream_t s);
cudaError_t ci_to_f64(const Geometry &g, int64_t n, const int32_t *cell, const float4 *off, double *x64,
                      cudaStream_t s);

// Gather rows into sorted order: out[k] = in[perm[k]] for float4, int ids.
cudaError_t gather_sorted(int64_t n, const int32_t *perm, const float4 *p_in, float4 *p_out,
                          const float4 *v_in, float4 *v_out, const int32_t *id_in, int32_t *id_out,
                          cudaStream_t s);

// Scatter rows back to input order: out[id[k]] = in[k]; positions are
// wrapped into [0, L) on the way (flagging coordinates outside [-L, 2L)).
cudaError_t scatter_rows(int64_t n, const int32_t *id, const float4 *p_in, float4 *p_out,
                         const float4 *v_in, float4 *v_out, float Lf, int *d_flags, cudaStream_t s);

// Candidate pairs of a batch: each global cell against the 27 cells around
// it inside its own box (boxes sorted by cell_base).
cudaError_t candidate_count_batch(int64_t ncell_total, const BoxDev *boxes, int nbox, const int32_t *cell_start,
                                  unsigned long long *out, cudaStream_t s);
cudaError_t candidate_count(const Geometry &g, const int32_t *cell_start, unsigned long long *out,
                            cudaStream_t s);

// ---- pair force (sr_force.cu) -------------------------------------------
enum ForceMode : int {
    kModeForce = 0,      // store the force (out[perm[i]])
    kModeKickDrift = 1,  // kick + stream in sorted order
    kModePotential = 2,  // per-particle pair potential
    kModeBatch = 3,      // kick + stream, write back to pool rows (batches)
    kModeKick = 4,       // kick only, velocities back to ids[i]
    kModeKickLevels = 5  // kick by the table entry of the particle's kick count (multi-level)
};

struct ForceLaunch {
    const float4 *pos;          // sorted, wrapped
    const int4 *items;
    const int32_t *n_items;     // device count
    const int32_t *cell_start;
    int *work_counter;          // zeroed before launch
    int mode;
    // kModeForce: out[perm[i]] (perm null: out[i])
    float4 *out;
    const int32_t *perm;
    // kModeKickDrift
    float4 *vel;                // sorted, updated in place
    float4 *pos_next;           // sorted order of this sub-cycle
    float h_kick, h_drift;
    // kModePotential: phi_out[i] = G m_i/2 sum_j m_j phi(s_ij) (sorted order)
    float *phi_out;
    unsigned long long *within; // non-null: count pairs inside the cutoff
    unsigned long long *evaluated = nullptr;   // with within: count the pairs evaluated (after culling)
    const int *mass_flag;       // from the binning pass (null: masses differ)
    // kModeBatch: geometry and kick/stream factors per box, write-back to the pool
    const BoxDev *boxes = nullptr;
    const int32_t *ids = nullptr;     // pool row of each sorted particle
    float4 *pos_pool = nullptr;
    float4 *vel_pool = nullptr;
    int *flags = nullptr;             // device status word (wrap errors)
    // kModeKickLevels: kick count of each sorted particle, kick table
    const int32_t *levels = nullptr;
    KickTable kick{};
    // positions are in-cell offsets (precision variant): cell step w = ci_step,
    // and the remainder delta = L - nc w that a periodic wrap adds (ci_rem)
    bool cell_offset = false;
    float w = 0.0f;
    float delta = 0.0f;
    int variant = 0;            // pair-kernel variant (autotuned), 0..kForceVariants-1
    const int32_t *order = nullptr;   // non-null: the queue takes items[order[k]] (items_heavy_first)
};

constexpr int kForceVariants = 4;

cudaError_t sr_force_launch(const Geometry &g, const ForceConsts &fc, const ForceLaunch &fl, int num_sms,
                            cudaStream_t s);
hacc_status timed_force_launch(hacc_ctx *ctx, const Geometry &g, const ForceConsts &fc, const ForceLaunch &fl,
                               cudaStream_t s);

// FP64 sums: out[0..2] = sum m v, out[3] = sum m v^2 / 2, out[4] = sum phi.
cudaError_t diag_reduce(int64_t n, const float4 *pos, const float4 *vel, const float *phi, double *out,
                        cudaStream_t s);
// The same sums per box of a batch, over each box's range of the cell-sorted
// arrays (cells cell_base .. cell_base + nc^3 of cell_start), with a fixed
// partition of every range: out[5 orig + k] for each box (other entries are
// left as they are); partial: kDiagParts x 5 doubles per box of scratch.
constexpr int kDiagParts = 32;
cudaError_t diag_reduce_batch(int nbox, const BoxDev *boxes, const int32_t *cell_start, const float4 *pos,
                              const float4 *vel, const float *phi, double *partial, double *out, cudaStream_t s);
// FP64 sum of m x over (cell, offset) positions, x = (c + 1/2) w + off per axis: out[0..2] (added to).
cudaError_t diag_mass_moment_ci(int64_t n, const int32_t *cell, const float4 *off, int nc, double w, double *out,
                                cudaStream_t s);

// ---- PM (pm.cu) ------------------------------------------------------------
// Host copies of a full step overlapped with its PM stages (hacc_step_host):
// on the copy stream, positions are uploaded in kPmChunks chunks, each
// deposited as soon as it has landed, then the velocities in the same chunks,
// each kicked as soon as it has landed and the field is solved; at the
// closing kick the positions are downloaded while the field is solved, and
// the kicked velocities chunk by chunk as they are interpolated.  The deposit
// sums fixed-point integers, so the chunking changes no bit.
constexpr int kPmChunks = 16;
struct PmHostIO {
    cudaStream_t copy = nullptr;
    cudaEvent_t ev[kPmChunks] = {};
    const float4 *pos_up = nullptr;     // host positions to upload into pos
    const float4 *vel_up = nullptr;     // host velocities to upload into vel_kick, after the positions
    float4 *pos_down = nullptr;         // host: the positions, downloaded at the start of the stage
    float4 *vel_down = nullptr;         // host: the kicked velocities, downloaded chunk by chunk
};

// Long-range acceleration G * a_PM at pos; stored to acc (if non-null) and/or
// added as a kick vel += kick * a (if vel_kick is non-null).
// before_kick (nullable): an event the stream waits for between the field
// solve and the interpolation, which is the first use of vel_kick.  io
// (nullable): host copies overlapped with the stage (see PmHostIO).
hacc_status pm_accel(hacc_ctx *ctx, const hacc_box *box, const hacc_pm *pm, double G, int64_t n, const float4 *pos,
                     float4 *acc, float4 *vel_kick, float kick, cudaStream_t s, cudaEvent_t before_kick = nullptr,
                     const PmHostIO *io = nullptr);
void pm_destroy(hacc_ctx *ctx);

}  // namespace hacc
