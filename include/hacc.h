/*
 * hacc.h - C ABI of a GB300 (sm_103a) library for the short-range
 * particle-particle force of HACC's force-split N-body method
 * (Habib et al., arXiv 1410.2805).
 *
 * The method (Sec. 2.3-2.5, Sec. 3.1, Sec. 3.3 of the paper): particles in a
 * periodic cube of side L are binned into a chaining mesh of nc^3 cells of
 * width L/nc >= r_cut; each particle i then sums, over the particles j of the
 * 27 cells around its own (periodic minimum image),
 *
 *     a_i = G * sum_{j != i, s < r_cut^2} m_j r_ij f_SR(s),
 *     f_SR(s) = (s + eps)^(-3/2) - P5(s),   s = r_ij . r_ij,  r_ij = x_j - x_i
 *
 * (Eq. (force)), and the short-range map is sub-cycled with symmetric
 * stream-kick-stream steps (Sec. 2.5) inside a kick-sub-cycle-kick full step
 * around the long-range particle-mesh force (Eq. (tstep)).
 *
 * Units: grid units (the PM grid spacing is 1 when ng = L).  Positions and
 * velocities are FP32; arithmetic of the pair force is FP32 with FP32
 * accumulation; FP64 only in the diagnostics.
 *
 * Memory: every particle array is a DEVICE pointer owned by the caller
 * (unless an entry point's name ends in _host), 16-byte aligned, with one
 * 4-float row per particle:
 *     pos_m : (x, y, z, m)      positions in [-L, 2L) and masses
 *     vel   : (vx, vy, vz, w)   w is ignored and preserved as 0 on output
 *     acc   : (ax, ay, az, 0)
 * Row i of every output belongs to row i of the inputs (the library sorts
 * internally and un-permutes).  The library never frees caller memory.  The
 * context owns its scratch (a pool grown on demand and bounded by the HBM
 * budget given at creation) and reuses it across calls.
 *
 * Streams: each call enqueues its work on `stream` (NULL = legacy default
 * stream) and returns without synchronising, except the _host variants and
 * hacc_ctx_sync, which wait for their stream.  Calls on one context must not
 * run concurrently from several host threads.
 *
 * Errors: argument and domain errors are returned before anything is
 * enqueued.  Errors found on the device (a coordinate outside [-L, 2L) or
 * not finite) raise a flag that the next hacc_ctx_sync returns (and clears);
 * affected outputs are then undefined but every memory access stays in
 * bounds.  No kernel of the library waits on another kernel, a flag or a
 * peer, so no call can hang on the device.  hacc_last_error gives a message.
 */
#ifndef HACC_H
#define HACC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *hacc_stream_t;

typedef enum {
    HACC_OK = 0,
    HACC_EINVAL = 1,   /* null pointer, negative size, box side not an FP32 value, ... */
    HACC_EDOMAIN = 2,  /* nc < 3, cell width below r_cut, r_cut >= L/2, or a position
                          outside [-L, 2L) / not finite (reported by hacc_ctx_sync) */
    HACC_ENOMEM = 3,   /* scratch would exceed the context's HBM budget, or cudaMalloc failed */
    HACC_ECUDA = 4,    /* a CUDA runtime / cuFFT call failed */
    HACC_ETIMEOUT = 5  /* reserved for a bounded device-side wait that gave up; no call
                          returns it (the library has no device-side waits) */
} hacc_status;

/* Periodic box.  L: side in grid units; must be exactly representable in FP32
 * (the wrap and the minimum image are done in FP32).  nc: chaining-mesh cells
 * per side, 0 = floor(L / r_cut) (one fewer if the cell width would come
 * within a relative 1e-6 of r_cut); 3 <= nc <= 1024 and L/nc >= r_cut
 * (Sec. 2.4 "chaining mesh", Sec. 3.1 "26 neighbouring" cells).  ng: PM grid
 * points per side, used by hacc_step only (0 = round(L)). */
typedef struct {
    double L;
    int32_t nc;
    int32_t ng;
} hacc_box;

/* Force split of Sec. 2.3/3.1.  r_cut: matching scale (pairs with s >= r_cut^2
 * do not interact); eps: Plummer softening in units of length^2 (it is added
 * to s); poly: P5(s) = sum_k poly[k] s^k, ascending powers; G: prefactor.
 * Requires 0 < r_cut, eps >= 0. */
typedef struct {
    float r_cut;
    float eps;
    double poly[6];
    float G;
} hacc_split;

/* Long-range spectral PM parameters (Sec. 2.3): Gauss-sinc filter width sigma
 * and sinc power ns of Eq. (filter) (nominal 0.8 and 3). */
typedef struct {
    float sigma;
    int32_t ns;
} hacc_pm;

typedef struct hacc_ctx hacc_ctx;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * scratch the context may hold (0 = no bound beyond the device's memory).
 * *out receives the context or NULL on failure. */
hacc_status hacc_ctx_create(hacc_ctx **out, int device, size_t hbm_budget_bytes);

/* Free the context and its scratch (synchronises the device first).  NULL is a no-op. */
void hacc_ctx_destroy(hacc_ctx *ctx);

/* Message for the last error seen on this context ("" if none).  Owned by the context. */
const char *hacc_last_error(const hacc_ctx *ctx);

/* Wait for `stream`, then return and clear any flag raised on the device
 * (HACC_EDOMAIN) or a pending CUDA error. */
hacc_status hacc_ctx_sync(hacc_ctx *ctx, hacc_stream_t stream);

/* Bytes of scratch the context currently holds. */
size_t hacc_ctx_scratch_bytes(const hacc_ctx *ctx);

/* Default split parameters, computed on the host in FP64 from Eq. (fitform):
 * r_cut = root of r^2 F_grid(r) = 1 near three grid cells; P5 = least-squares
 * fit of F_grid(r)/r on (0, r_cut], residuals weighted by r^3, constrained to
 * P5(r_cut^2) = F_grid(r_cut)/r_cut; eps = 2.5e-4; G = 1. */
hacc_status hacc_split_default(hacc_split *out);

/* The chaining-mesh size hacc_box.nc = 0 resolves to, or -1 if the box is too
 * small (fewer than 3 cells of width >= r_cut). */
int32_t hacc_mesh_cells(double L, float r_cut);

/* Chaining-mesh build (Sec. 2.4 / Sec. 3.3; Hockney's chaining mesh):
 * wraps pos_m into [0, L) IN PLACE (x < 0 -> x + L, x >= L -> x - L, in FP32;
 * a result that rounds to L becomes 0), assigns each particle the cell
 * (ix, iy, iz) with ix the largest integer such that ix * L <= x * nc (exact),
 * linear id (iz*nc + iy)*nc + ix, and sorts stably by cell:
 *   cell_id    [n]       cell of each particle (input order)
 *   cell_start [nc^3+1]  first sorted slot of each cell; cell_start[nc^3] = n
 *   perm       [n]       perm[k] = input row of sorted slot k; within a cell,
 *                        ascending input row
 * All three are caller-owned device arrays. */
hacc_status hacc_bin(hacc_ctx *ctx, const hacc_box *box, float r_cut, int64_t n, float *pos_m,
                     int32_t *cell_id, int32_t *cell_start, int32_t *perm, hacc_stream_t stream);

/* Short-range force (Eq. (force)) on every particle from the particles of its
 * 27 neighbouring chaining-mesh cells, cut at r_cut, periodic minimum image.
 * pos_m is not modified.  acc[n] receives (ax, ay, az, 0).
 * pair_counts: NULL, or a device array of 2 uint64 that receives
 *   [0] candidate pairs of the 27-cell chaining mesh, sum_c n_c * sum_nbr n_j
 *       (self pairs included), exact;
 *   [1] ordered pairs (i, j), j != i, evaluated inside the cutoff.
 * Counting runs a slower kernel variant; forces are bitwise the same. */
hacc_status hacc_sr_force(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                          const float *pos_m, float *acc, uint64_t *pair_counts, hacc_stream_t stream);

/* n_sub short-range sub-cycles of step h = dt / n_sub (Sec. 2.5, SKS form):
 *   x += (h/2) v;  rebin;  v += h a_SR(x);  x += (h/2) v
 * Adjacent half streams are fused.  pos_m and vel are updated in place;
 * positions come back wrapped into [0, L).  n_sub >= 1. */
hacc_status hacc_subcycle(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                          float *pos_m, float *vel, double dt, int32_t n_sub, hacc_stream_t stream);

/* One full step of Eq. (tstep): M_lr(dt/2) (M_sr(dt/n_c))^n_c M_lr(dt/2), where
 * M_lr is a kick by the long-range spectral PM force (CIC deposit, Eq. (filter)
 * Gauss-sinc filter, Eq. (greenf) influence function, Eq. (sldiff) Super-Lanczos
 * gradient, CIC interpolation; Sec. 2.3) on an ng^3 grid, and M_sr the
 * sub-cycle above.  Both forces use split->G. */
hacc_status hacc_step(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, const hacc_pm *pm,
                      int64_t n, float *pos_m, float *vel, double dt, int32_t n_c, hacc_stream_t stream);

/* Multi-level short-range step (Sec. 3.1, Eq. (kicks)).  The step bins the
 * particles on a chaining mesh of nc_ml^3 cells, nc_ml = hacc_ml_mesh_cells(L,
 * r_cut, skin) (box->nc instead when that is nonzero), whose cells are at
 * least r_cut (1 + skin) wide.  The density of each particle's cell at the
 * start of the step, rho / rho0 = count nc_ml^3 / n, sets its kick count
 * l = floor(floor(rho/rho0) / d) + 1 (integers; d <= 0 gives every particle
 * lmax), clamped to [lmin, lmax] (1 <= lmin <= lmax <= 16; the paper's test
 * gives every particle at least two kicks).  A particle with l kicks is kicked by dt/l at
 * times (2k+1)/(2l) dt, k < l; all particles stream together between the union
 * of those times over the counts that occur, so each streams by dt in total.
 * The mesh is kept while the particles move (as the paper keeps its tree):
 * at each event the largest per-axis drift from the binned positions is
 * checked, and only when it passes half the cell's excess width over r_cut
 * are the particles rebinned (each cell then ordered by kick count).  At an
 * event only the particles kicked then get work items (as i; every particle
 * stays a j).  One host synchronisation per step reads which
 * kick counts occur; the events then run as one CUDA graph cached by the
 * context (the rebinnings are conditional nodes decided on the device), or,
 * with statistics timing or counting on, from the host with one
 * synchronisation per event (the same kernels in the same order).  skin must
 * be finite and >= 0.  level_out (nullable, device, n) receives the kick
 * counts. */
hacc_status hacc_subcycle_ml(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n, float *pos_m,
                             float *vel, double dt, int32_t d, int32_t lmin, int32_t lmax, float skin,
                             int32_t *level_out, hacc_stream_t stream);

/* Cells per side of the multi-level step's chaining mesh for box->nc = 0:
 * hacc_mesh_cells(L, r_cut (1 + skin)) when that gives at least 3 cells and
 * fewer than hacc_mesh_cells(L, r_cut), else hacc_mesh_cells(L, r_cut).
 * Returns -1 where hacc_mesh_cells(L, r_cut) does. */
int32_t hacc_ml_mesh_cells(double L, float r_cut, float skin);

/* Long-range PM acceleration alone (with G = 1): acc[n] receives (ax, ay, az, 0).
 * ng = 0 in the box means ng = round(L); ng must be even, 4 <= ng <= 2048.
 * The grid, its FFT plans and buffers are kept by the context between calls. */
hacc_status hacc_pm_force(hacc_ctx *ctx, const hacc_box *box, const hacc_pm *pm, int64_t n,
                          const float *pos_m, float *acc, hacc_stream_t stream);

/* FP64 diagnostics of one box: out (device, 5 doubles) receives
 * [0..2] sum m v, [3] kinetic energy sum m v^2/2, [4] short-range pair
 * potential energy sum_{i<j, s<r_cut^2} G m_i m_j phi(s), where
 * phi(s) = -(s+eps)^(-1/2) - sum_k poly[k] s^(k+1)/(2(k+1)) shifted so that
 * phi(r_cut^2) = 0 (so that -grad phi gives Eq. (force)). Per-pair terms are
 * FP32, per-particle sums FP32, the box sums FP64. */
hacc_status hacc_diagnostics(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                             const float *pos_m, const float *vel, double *out, hacc_stream_t stream);

/* Host-buffer variants: pos_m, vel (and acc) are HOST pointers (page-locked
 * memory gives the fastest copies).  Each call copies the inputs to scratch
 * on the device, runs the device entry point of the same name, copies the
 * results back and waits for the stream.  hacc_step_host runs its copies on a
 * second stream of the context, overlapped with the PM stages: the positions
 * go up in chunks that are deposited as they land, then the velocities; at
 * the end the positions come down while the closing field is solved and the
 * velocities chunk by chunk as they are kicked.  The results are the bits of
 * hacc_step's.  The host arrays must not be touched until the call returns. */
hacc_status hacc_sr_force_host(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                               const float *pos_m, float *acc, hacc_stream_t stream);
hacc_status hacc_subcycle_host(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                               float *pos_m, float *vel, double dt, int32_t n_sub, hacc_stream_t stream);
hacc_status hacc_step_host(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, const hacc_pm *pm,
                           int64_t n, float *pos_m, float *vel, double dt, int32_t n_c, hacc_stream_t stream);

/* ---- Precision variant: positions as (cell, in-cell offset) --------------
 * The paper's runs keep absolute positions in single precision; at box sides
 * of hundreds of cells FP32 rounds positions to ~3e-5 cells and every stream
 * adds that much again.  Here a position is stored as the int32 chaining-mesh
 * cell id of the box (nc from the box, as for hacc_bin) plus an FP32 offset
 * from the cell's centre, with the mass as the fourth float of off_m:
 * resolution ~1e-7 cells at any L.  The cells step by W = fl32(L / nc), the
 * FP32 value nearest the width: cell c (per axis) covers [c W, (c+1) W) and
 * the last cell [(nc-1) W, L), absorbing the remainder L - nc W (a few ulp of
 * W, of either sign); a coordinate is (c + 1/2) W + off, off in [-W/2, W/2]
 * (last cell: up to W/2 + L - nc W).  Because W is an FP32 value, moving a
 * neighbour's offset into i's cell frame by whole steps is exact for every
 * pair close enough to matter, so pair separations carry one rounding at most;
 * the wrap remainder is applied to i's offset, also exactly.  Pair arithmetic
 * and accumulation stay FP32; FP64 is used only inside the stream, on the
 * global position.  Requires W >= r_cut and W + (L - nc W) >= r_cut
 * (HACC_EDOMAIN otherwise).
 * pos64: n x 3 doubles (x, y, z); mass: n floats or NULL (all 1). */
hacc_status hacc_ci_from_f64(hacc_ctx *ctx, const hacc_box *box, float r_cut, int64_t n, const double *pos64,
                             const float *mass, int32_t *cell, float *off_m, hacc_stream_t stream);
hacc_status hacc_ci_to_f64(hacc_ctx *ctx, const hacc_box *box, float r_cut, int64_t n, const int32_t *cell,
                           const float *off_m, double *pos64, hacc_stream_t stream);
/* Eq. (force) as hacc_sr_force, from (cell, offset) positions; acc in input order. */
hacc_status hacc_sr_force_ci(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                             const int32_t *cell, const float *off_m, float *acc, hacc_stream_t stream);
/* SKS sub-cycles as hacc_subcycle on (cell, offset) positions, updated in place
 * (streams in FP64, kicks in FP32). */
/* FP64 diagnostics of a box stored as (cell, offset): out (device, 8 doubles)
 * receives [0..4] as hacc_diagnostics (sum m v, kinetic energy, short-range
 * pair potential energy; the pair terms from the offsets moved into one cell
 * frame, FP32) and [5..7] sum m x over the global positions (c + 1/2) W + off,
 * formed and summed in FP64 (the centre of mass times the total mass). */
hacc_status hacc_diagnostics_ci(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                                const int32_t *cell, const float *off_m, const float *vel, double *out,
                                hacc_stream_t stream);
hacc_status hacc_subcycle_ci(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n, int32_t *cell,
                             float *off_m, float *vel, double dt, int32_t n_sub, hacc_stream_t stream);

/* ---- Batches of independent boxes (serving / batching mode) --------------
 * The paper advances one domain per rank; serving many small boxes is this
 * library's extension.  Each box is an independent periodic cube whose rows
 * [offset, offset + n) live in shared pool arrays pos_pool / vel_pool (device,
 * caller-owned, same row layout as above).  All boxes of a call share one
 * binning pass and ONE persistent pair-kernel launch per sub-cycle, fed by a
 * single work queue of (box, cell) items; results are written back to the
 * boxes' rows, positions wrapped into [0, L).  Each box's result is bitwise
 * the same alone or in any mix.  One split for the whole batch.
 * Rows of different boxes must not overlap; limits: 2^31 particles and cells
 * per call. */
#define HACC_TICK_FIRST 1  /* this tick is the first sub-cycle of the box's run */
#define HACC_TICK_LAST 2   /* this tick is the last sub-cycle of the box's run */

typedef struct {
    double L;        /* box side (an FP32 value) */
    int32_t nc;      /* chaining-mesh cells per side, 0 = default */
    int32_t flags;   /* hacc_batch_tick only: HACC_TICK_FIRST | HACC_TICK_LAST */
    int64_t offset;  /* first row of the box in the pool arrays */
    int64_t n;       /* rows (0: box skipped) */
    double dt;       /* hacc_batch_subcycle: full step, split into n_sub sub-cycles;
                        hacc_batch_tick: the sub-cycle step h */
} hacc_batch_box;

/* n_sub SKS sub-cycles (as hacc_subcycle) of every box, dt / n_sub each.
 * use_graph != 0 captures the n_sub ticks as one CUDA graph, cached in the
 * context and replayed while the batch's geometry, rows, pool pointers and
 * split are unchanged (step sizes may change); the legacy default stream
 * (NULL) cannot be captured and runs the ticks directly. */
hacc_status hacc_batch_subcycle(hacc_ctx *ctx, const hacc_split *split, int32_t nbox,
                                const hacc_batch_box *boxes, float *pos_pool, float *vel_pool,
                                int32_t n_sub, int32_t use_graph, hacc_stream_t stream);

/* Autotuner of the batched launch (a tuning aid of the library; the paper has
 * no counterpart).  For every setting of work-item cap in {0 (cell-wide
 * items), 32, 64, 96, 128, 160} (see hacc_set_item_cap) x queue order (cell order,
 * largest first; see hacc_set_queue_order) x pair-kernel variant, times whole
 * batched ticks as hacc_batch_tick runs them (binning, gathers, the kick and
 * stream pass; each box one sub-cycle of step boxes[b].dt) on scratch copies
 * of the pools (reps ticks after one warm-up, CUDA events on `stream`);
 * setting k = (cap index * 2 + order) * HACC_FORCE_VARIANTS + variant.  The
 * fastest setting is kept for this batch geometry (the boxes' sides, cells and
 * sizes) and used by later hacc_batch_subcycle and hacc_batch_tick calls whose
 * non-empty boxes have that geometry (other batches use the context's
 * settings); a later tune replaces it.  times_ms (nullable, host,
 * HACC_BATCH_TUNE_SETTINGS doubles) receives each setting's mean tick time,
 * *chosen (nullable) the setting kept.  The pools are only read (the scratch
 * grows by 32 bytes per pool row).  Synchronises `stream`.  Every setting sums
 * the same pairs. */
#define HACC_BATCH_TUNE_SETTINGS 48
hacc_status hacc_batch_tune(hacc_ctx *ctx, const hacc_split *split, int32_t nbox, const hacc_batch_box *boxes,
                            const float *pos_pool, const float *vel_pool, int32_t reps, double *times_ms,
                            int32_t *chosen, hacc_stream_t stream);

/* FP64 diagnostics of every box of a batch (as hacc_diagnostics, per box):
 * out (device, 5 doubles per entry of `boxes`, including boxes with n = 0,
 * which get zeros) receives for box b at out[5 b]: sum m v (3), kinetic
 * energy, short-range pair potential energy of the box's own pairs.  One
 * batched binning pass and one pair-kernel launch over all boxes; each box's
 * sums are reduced over its own particles in a fixed order, so they are
 * bitwise the same alone or in any mix.  The pools are only read. */
hacc_status hacc_batch_diagnostics(hacc_ctx *ctx, const hacc_split *split, int32_t nbox,
                                   const hacc_batch_box *boxes, const float *pos_pool, const float *vel_pool,
                                   double *out, hacc_stream_t stream);

/* One sub-cycle of step boxes[b].dt for every box: stream h/2 first only if
 * HACC_TICK_FIRST (earlier ticks left positions streamed by h/2), kick h,
 * then stream h/2 if HACC_TICK_LAST, else h (fusing the next tick's opening
 * half stream).  A run of k ticks with FIRST on the first and LAST on the
 * last equals hacc_batch_subcycle with n_sub = k. */
hacc_status hacc_batch_tick(hacc_ctx *ctx, const hacc_split *split, int32_t nbox,
                            const hacc_batch_box *boxes, float *pos_pool, float *vel_pool,
                            hacc_stream_t stream);

/* ---- Serving: continuous batching of short-range runs -------------------
 * A server owns a device pool of `pool_bytes` (32 bytes per particle: one pos
 * and one vel row) and queues runs (a box of n particles, sub-cycle step h,
 * `steps` sub-cycles).  A queued run is admitted, in arrival order, while
 *   - its rows fit in the pool (first-fit, coalescing free list),
 *   - the particles advanced per tick stay within max_active_particles (if > 0),
 *   - and, when the context was created with an HBM budget, the pool plus the
 *     scratch that the batched tick of all resident runs takes from the
 *     context (hacc_batch_scratch_bytes; the larger of that and the arena the
 *     context already holds) plus the context's host-copy staging stay within
 *     the budget.
 * Each hacc_server_tick admits queued runs; advances every resident run by one
 * sub-cycle with hacc_batch_tick on `stream`; meanwhile admits further runs for
 * the next tick and copies their inputs to the device on a stream of the
 * server's own (so the upload overlaps the pass); copies runs whose last
 * sub-cycle ran back into their host arrays (in place) and releases their
 * rows; then waits for both streams.  The host arrays passed to
 * hacc_server_submit must stay valid until the run has been reported finished.
 * Server calls must not overlap other calls on its context. */
typedef struct hacc_server hacc_server;

typedef struct {
    int32_t admitted;   /* runs admitted this tick */
    int32_t finished;   /* runs retired this tick */
    int32_t active;     /* runs advanced this tick */
    int32_t queued;     /* runs still waiting */
    int64_t particles;  /* particles advanced this tick */
    int64_t free_rows;  /* pool rows free after the tick */
} hacc_server_tick_info;

hacc_status hacc_server_create(hacc_server **out, hacc_ctx *ctx, const hacc_split *split, size_t pool_bytes,
                               int64_t max_active_particles);
void hacc_server_destroy(hacc_server *sv);
/* Queue a run.  pos_host / vel_host: n rows each (host memory; page-locked
 * memory copies fastest), read at admission and overwritten with the result.
 * HACC_ENOMEM if the run alone exceeds the pool, the per-tick cap or the
 * budget. */
hacc_status hacc_server_submit(hacc_server *sv, int64_t id, double L, int64_t n, float *pos_host, float *vel_host,
                               double h, int32_t steps);
/* One tick (see above).  finished_ids (nullable, host, finished_cap entries)
 * receives the ids of the runs retired by this tick: at most finished_cap runs
 * are retired per tick; further finished runs stay resident (not advanced)
 * and are retired and reported by the next tick.  finished_ids NULL: every
 * finished run is retired.  info->finished counts the runs retired. */
hacc_status hacc_server_tick(hacc_server *sv, hacc_stream_t stream, hacc_server_tick_info *info,
                             int64_t *finished_ids, int32_t finished_cap);

/* Bytes of context scratch one batched tick (hacc_batch_tick) over these boxes
 * takes (the exact carving of its buffers; host arithmetic only, no device
 * call).  Boxes with n = 0 are skipped; 0 if none remain or a box is invalid. */
size_t hacc_batch_scratch_bytes(const hacc_split *split, int32_t nbox, const hacc_batch_box *boxes);

/* Size of the fixed device scratch behind hacc_sr_force_noalloc (16 MiB). */
#define HACC_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* Short-range force without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that may not call
 * cudaMalloc (their device memory is owned by another allocator or runtime,
 * or allocation is forbidden after their set-up), and so cannot create a
 * context.  It computes what hacc_sr_force computes (same kernels, no pair
 * counts), with all scratch taken from one fixed device array of
 * HACC_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits.  The caller owns pos_m
 * (n rows, not modified) and acc (n rows, receives (ax, ay, az, 0)).
 *   - Limit: about 49.3 bytes per particle plus 36 bytes per chaining-mesh cell
 *     must fit in the array (e.g. 262144 particles with up to 100000 cells);
 *     larger problems return HACC_ENOMEM before anything is enqueued.
 *   - Works on the current CUDA device; `stream` must belong to it
 *     (HACC_EINVAL otherwise, nothing enqueued).  Its first call on a device
 *     looks up the array's device address (once per device); make that first
 *     call before any stream capture.
 *   - All calls share the array and leave their data in it; calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on it and
 *     give wrong results, so serialise them.
 *   - Coordinates outside [-L, 2L) are not reported (no context holds the
 *     flag); the forces are then undefined but memory accesses stay in bounds.
 * Other errors as for hacc_sr_force (HACC_EINVAL, HACC_EDOMAIN, HACC_ECUDA). */
hacc_status hacc_sr_force_noalloc(const hacc_box *box, const hacc_split *split, int64_t n,
                                  const float *pos_m, float *acc, hacc_stream_t stream);

/* Number of pair-kernel variants: register budget (96 or 128 per thread) x
 * inner loop (indexed or pointer-stepped); all give bitwise the same forces. */
#define HACC_FORCE_VARIANTS 4

/* Autotuner (a tuning aid of the library; the paper has no counterpart):
 * for every setting of work-item cap in {0 (cell-wide items), 16, 24, 32, 48}
 * (see hacc_set_item_cap) x queue order (cell order, largest first; see
 * hacc_set_queue_order) x pair-kernel variant, times one sub-cycle's work on
 * pos_m as hacc_subcycle runs it: the chaining-mesh build (binning, gather
 * into cell order) and the pair-kernel launch that kicks and streams (with
 * zero velocities of its own; pos_m is not modified), reps times after a
 * warm-up sub-cycle from pos_m, each timed one binning what the previous one
 * left in cell order (as the sub-cycle loop does), CUDA events on `stream`; setting k = (cap index * 2 + order) *
 * HACC_FORCE_VARIANTS + variant.  Keeps the fastest setting for this
 * context's later calls (as hacc_set_item_cap, hacc_set_queue_order and
 * hacc_set_variant would).  times_ms (nullable, host, HACC_TUNE_SETTINGS
 * doubles) receives each setting's mean time, *chosen (nullable) the setting
 * kept.  Synchronises `stream`.  Every setting sums the same pairs (the
 * variants and orders in the same order; the caps in different orders, so
 * results differ by FP32 rounding). */
#define HACC_TUNE_SETTINGS 40
hacc_status hacc_tune(hacc_ctx *ctx, const hacc_box *box, const hacc_split *split, int64_t n,
                      const float *pos_m, int32_t reps, double *times_ms, int32_t *chosen,
                      hacc_stream_t stream);

/* Finer chaining mesh for the single-box force paths (hacc_sr_force,
 * hacc_subcycle, hacc_step, hacc_diagnostics, hacc_tune and their host forms):
 * cells_per_rcut = 1 (default) bins into cells at least r_cut wide and searches
 * the 27 cells around each particle's own (Sec. 3.3); 2 bins into cells at
 * least r_cut/2 wide (box->nc = 0: hacc_mesh_cells(L, r_cut/2); nc >= 5) and
 * searches the 125 cells within two cells, which covers the same sphere with a
 * smaller search volume (a variant of the library; the paper's own P3M search
 * is the 27-cell one).  The forces are those of the same pairs.  It also
 * takes boxes from 5 r_cut / 2 up (the 27-cell mesh needs 3 r_cut).  Batched,
 * served, multi-level, cell/offset and allocation-free paths always use 27
 * cells.  HACC_EINVAL for other values. */
hacc_status hacc_set_stencil(hacc_ctx *ctx, int32_t cells_per_rcut);

/* Work items of the pair kernel in the single-box force paths (hacc_sr_force,
 * hacc_subcycle, hacc_step, hacc_diagnostics, hacc_tune and their host forms),
 * the batched and served paths and the multi-level step (whose small events
 * split every cell into smaller items still); the cell/offset paths and
 * hacc_sr_force_noalloc use cap = 0.  A work item is a set of particles of
 * one chaining-mesh cell that one warp runs against the cell's neighbours; a
 * neighbour particle farther than r_cut from the item's bounding box is
 * skipped, so items that cover a small part of their cell evaluate fewer
 * pairs, but every item stages all of its neighbours.
 * cap in [16, 160]: within each cell of up to 512 particles the particles are
 * ordered by their 4x4x4 sub-cell (Morton order, ties by input row; larger
 * cells by input row alone), and a cell of m <= split_max particles becomes
 * ceil(m / cap) items of consecutive particles of near-equal size; a denser
 * cell becomes ceil(m / 160) items (split_max = 0: no such limit).
 * cap = 0: input row order within cells and items of up to 160 particles.
 * cap = -1 (the default): 48 for calls of up to 2^22 particles (short
 * launches, whose tail the longest items of dense cells set) and 0 above.
 * The forces are sums over the same pairs for every setting (the summation
 * order differs, so results differ by FP32 rounding).  HACC_EINVAL for a cap
 * outside {-1, 0} and [16, 160] or split_max < 0. */
hacc_status hacc_set_item_cap(hacc_ctx *ctx, int32_t cap, int32_t split_max);

/* Order in which the pair kernel's warps take the work items of a call of
 * 2^20 particles or more (single box or batch; smaller calls keep cell order):
 * heavy_first = 1 takes the largest items first, so that the items of dense
 * cells do not set the launch's tail; 0 (default) takes them in cell order
 * (neighbouring items on neighbouring warps, which share their neighbour
 * particles in the caches).  Results do not depend on it.  HACC_EINVAL for
 * other values. */
hacc_status hacc_set_queue_order(hacc_ctx *ctx, int32_t heavy_first);

/* Select the pair-kernel variant by hand (0 <= variant < HACC_FORCE_VARIANTS). */
hacc_status hacc_set_variant(hacc_ctx *ctx, int32_t variant);

/* Run statistics kept by a context (instrumentation, not part of the method). */
typedef struct {
    int64_t kernel_launches;  /* kernels this context launched */
    int64_t force_launches;   /* pair-force kernel launches */
    double force_ms;          /* summed CUDA-event durations of those launches (timing on) */
    uint64_t candidate_pairs; /* 27-cell candidate pairs of those launches (counting on) */
    uint64_t within_pairs;    /* ordered pairs (i, j != i) inside the cutoff (counting on) */
    uint64_t evaluated_pairs; /* ordered pairs the pair kernel evaluated: the candidates left after
                                 dropping j farther than r_cut from the item's bounds (counting on) */
    int64_t ml_rebins;        /* rebinnings inside multi-level steps after their first binning */
    double build_ms;          /* summed CUDA-event durations of the chaining-mesh builds (binning and
                                 the gather into cell order) of hacc_subcycle / hacc_step (timing on) */
    int64_t builds;           /* builds timed into build_ms */
} hacc_stats;

/* timing != 0: record a CUDA event pair on the call's stream around every
 * pair-force launch and every chaining-mesh build of the sub-cycle loop.  counting != 0: run the counting variant of the pair
 * kernel (bitwise the same forces) and accumulate pair counts.  Both off by
 * default. */
hacc_status hacc_stats_enable(hacc_ctx *ctx, int timing, int counting);

/* Wait for the device, fill *out, and zero the statistics if reset != 0. */
hacc_status hacc_stats_read(hacc_ctx *ctx, hacc_stats *out, int reset);

#ifdef __cplusplus
}
#endif

#endif /* HACC_H */
