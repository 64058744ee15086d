// Short-range pair force over the chaining mesh (Sec. 3.1, Eq. (force);
// Sec. 3.3: P3M with a chaining mesh on accelerators).
//
// For every particle i of a cell, the force from the particles of the 27
// cells around it (periodic):
//     a_i = G sum_j m_j r_ij f_SR(s),  f_SR(s) = (s+eps)^(-3/2) - P5(s),
// cut at s < r_cut^2 with a select instead of a branch (the paper folds the
// cutoff test into the force evaluation the same way, with fsel).
//
// GPU mapping.  Work item = up to 160 particles of one cell (one warp; K of
// them per lane, K = 1..5, in 1-8 lane groups, by cell occupancy).  Because
// cells are numbered x-fastest, the three cells (ix-1, ix, ix+1) of each of
// the 9 (dy, dz) rows are one contiguous run of the cell-sorted particle
// array (a second run when the row wraps in x).  The lanes first write the
// item's runs into a per-warp table; the runs are then staged as one stream,
// 32 candidates per round with coalesced 16-byte loads, into a per-warp
// shared-memory tile, keeping only the candidates within reach of the item's
// bounding box.  Every lane reads each staged j with one broadcast 16-byte
// shared load and evaluates it against its K particles, accumulating in FP32
// registers.  Work items are taken from an atomic counter so that clustered
// cells do not leave SMs idle.  With the finer mesh (stencil radius R = 2)
// the rows are 25 and the runs 5 cells long.
//
// Periodic images without rounding error: for a neighbour row that wraps on
// the low side (cell -1 -> nc-1), the staged j coordinates get -L (they lie in
// [2L/3, L), so x - L is exact); for a row that wraps on the high side
// (cell nc -> 0), the i coordinates get -L instead (same argument).  Either
// way r_ij = x_j' - x_i' carries only the rounding of one subtraction.
//
// Per evaluated pair (FP32): 3 FADD (r), 3 FFMA (t = s + eps), 1 MUFU rsqrt,
// 1 FMUL + 1 FFMA (t^-3/2 - P5), 5 FFMA (P5 in t), 1 FMUL (mass; dropped when
// all masses are equal), 1 compare, 3 predicated FFMA (accumulate inside the
// cutoff); P5 is re-expanded in t = s + eps on the host, and the cutoff test
// is t < fl(r_cut^2 + eps).
#include <cuda_runtime.h>
#include <stdint.h>

#include "hacc_internal.cuh"

namespace hacc {
namespace {

constexpr int kWarps = 4;
constexpr int kThreads = kWarps * 32;

struct KParams {
    const float4 *__restrict__ pos;
    const int4 *__restrict__ items;
    const int32_t *__restrict__ order;
    const int32_t *__restrict__ n_items;
    const int32_t *__restrict__ cell_start;
    int *work_counter;
    int nc;
    int R;            // neighbour cells per side of a cell's own (1: 27 cells, 2: 125 cells)
    float L;
    float T, eps, G;
    float q0, q1, q2, q3, q4, q5;
    float u0, u1, u2, u3, u4, u5, u6, phi0;
    int mode;
    float4 *out;
    const int32_t *__restrict__ perm;
    float4 *vel;
    float4 *pos_next;
    float h_kick, h_drift;
    float *phi_out;
    unsigned long long *within;
    unsigned long long *evaluated;
    const int *mass_flag;
    float w, delta;   // cell/offset form: cell step (an FP32 value) and the remainder L - nc w of a wrap
    const int32_t *levels;
    KickTable kick;
    const BoxDev *boxes;
    const int32_t *ids;
    float4 *pos_pool;
    float4 *vel_pool;
    int *flags;
};

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The pair-force constants, held in registers for the whole item.
struct PairConsts {
    float eps, T, q0, q1, q2, q3, q4, q5;
};

// Accumulate the interaction of one staged j (already image-shifted) with
// the K i-particles of this lane.  UM: all masses equal (the mass is applied
// once in the epilogue).
template <int K, bool COUNT, bool POT, bool EPS0, bool UM>
__device__ __forceinline__ void interact(const KParams &P, const PairConsts &C, float4 pj, int jidx, int iself, int lpg,
                                         const float (&xi)[K],
                                         const float (&yi)[K], const float (&zi)[K], float (&ax)[K],
                                         float (&ay)[K], float (&az)[K], unsigned &cnt) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float dx = pj.x - xi[k];
        float dy = pj.y - yi[k];
        float dz = pj.z - zi[k];
        float t = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, C.eps)));
        float r = rsqrt_approx(t);
        const bool in = t < C.T;
        if (POT) {
            // phi(s) = -(t)^(-1/2) - U(t) - phi0, U in t = s + eps
            float u = __fmaf_rn(P.u6, t, P.u5);
            u = __fmaf_rn(u, t, P.u4);
            u = __fmaf_rn(u, t, P.u3);
            u = __fmaf_rn(u, t, P.u2);
            u = __fmaf_rn(u, t, P.u1);
            u = __fmaf_rn(u, t, P.u0);
            float ph = -r - u - P.phi0;
            const bool self = jidx == iself + lpg * k;   // i's own row (sorted index)
            ax[k] += (in && !self) ? ph * pj.w : 0.0f;
        } else {
            float q = __fmaf_rn(C.q5, t, C.q4);
            q = __fmaf_rn(q, t, C.q3);
            q = __fmaf_rn(q, t, C.q2);
            q = __fmaf_rn(q, t, C.q1);
            q = __fmaf_rn(q, t, C.q0);
            float f = __fmaf_rn(r * r, r, -q);          // t^(-3/2) - P5
            if (!UM) f *= pj.w;
            // the cutoff as a predicate on the accumulating FMAs (the paper's
            // fsel select, without the select): pairs outside never touch the sums
            const bool use = EPS0 ? (t < C.T && t > 0.0f) : (t < C.T);
            if (use) {
                ax[k] = __fmaf_rn(f, dx, ax[k]);
                ay[k] = __fmaf_rn(f, dy, ay[k]);
                az[k] = __fmaf_rn(f, dz, az[k]);
            }
        }
        if (COUNT) cnt += (in && jidx != iself + lpg * k) ? 1u : 0u;   // j != i
    }
}

// Entries of a staged tile: up to 32 G entries, plus room for the up to 31
// that a compaction round carries past a full tile.
constexpr int kTileCap = 32 * 8 + 32;

// Tile steps per pass of the pair loop (the last tile is padded with far,
// massless entries to whole passes, so the loop has no remainder).
template <int K>
struct Unroll {
    static constexpr int F = K >= 5 ? 1 : (K >= 3 ? 2 : 4);
};

// Run the warp's i-particles against the staged entries [0, nj) of buf:
// group g takes entries g, g+G, g+2G, ... (consecutive float4 addresses
// across groups: no bank conflicts).  ids (nullable): sorted index of each
// entry, for the j != i tests of the counting and potential forms.
template <int K, bool COUNT, bool POT, bool EPS0, bool UM, int U>
__device__ __forceinline__ void run_tile(const KParams &P, const PairConsts &C, const float4 *buf, const int *ids,
                                         int nj, int iself, int lg, int grp, const float (&xs)[K],
                                         const float (&ys)[K], const float (&zs)[K], float (&ax)[K], float (&ay)[K],
                                         float (&az)[K], unsigned &cnt) {
    const int G = 1 << lg;
    const int lpg = 32 >> lg;
    // entries per group (interleaved); the pointer-stepped loop runs whole passes
    const int tg = U == 2 ? (nj + G * Unroll<K>::F - 1) / (G * Unroll<K>::F) * Unroll<K>::F : (nj + G - 1) >> lg;
    constexpr int kUnroll = U == 1 ? (K >= 3 ? 1 : 2) : (K >= 5 ? 1 : (K >= 3 ? 2 : 4));
    if (U == 2) {
        // pointer-stepped loop over the group's entries g, g+G, ..., F entries a
        // pass (the tile holds whole passes: no remainder)
        constexpr int F = Unroll<K>::F;
        const float4 *q = buf + grp;
        int e = grp;
#pragma unroll 1
        for (int t = 0; t < tg; t += F) {
#pragma unroll
            for (int u = 0; u < F; ++u) {
                const int jidx = (COUNT || POT) && e + u * G < nj ? ids[e + u * G] : -1;
                interact<K, COUNT, POT, EPS0, UM>(P, C, q[u * G], jidx, iself, lpg, xs, ys, zs, ax, ay, az, cnt);
            }
            q += F * G;
            e += F * G;
        }
    } else {
        const float4 *bp = buf + grp;
#pragma unroll kUnroll
        for (int t = 0; t < tg; ++t) {
            const int e = grp + (t << lg);
            const int jidx = (COUNT || POT) && e < nj ? ids[e] : -1;
            interact<K, COUNT, POT, EPS0, UM>(P, C, bp[t << lg], jidx, iself, lpg, xs, ys, zs, ax, ay, az, cnt);
        }
    }
}

// The neighbour cells of an item as x-runs of consecutive sorted particles:
// row (dz, dy) of the (2R+1)^2 rows gives run 2*row (cells cx-R..cx+R, or the
// part of them in [0, nc) when the row wraps in x) and run 2*row+1 (the
// wrapped part, else empty).  One table per warp in shared memory:
//   A = (exclusive end of the run in the item's concatenated stream,
//        offset j - t of its entries, shift bits, unused)
//   shift bits: 1/2/4 add -L to the staged j's x/y/z, 8/16/32 add -L to
//   the i side (runs of cells within R of a high face); with in-cell
//   offsets (CI) bits 0-3 and 4-7 hold dy + 2 and dz + 2 instead, bits 8-13
//   the same six wrap flags (there they move the i side by +delta for a low
//   wrap and -delta for a high one), and B = (b1, b2, d0): the x cell step of
//   entry j is d0 + (j >= b1) + (j >= b2).
constexpr int kMaxRuns = 64;   // 2 (2R+1)^2 <= 50 for R <= 2

struct RunTable {
    int4 *A;
    int4 *B;
    float4 *bnd;   // [0], [1]: the item's bounds (lx, ly, lz, -), (hx, hy, hz, -); [2], [3]: shifted, keep_r2 in [2].w
};


// Stream the runs [r0, r1) of the table (all with the same i shift tx, ty,
// tz) through the warp's shared tile.  The warp is split into G = 2^lg lane
// groups that share the i-particles and split the j.  Staging keeps only the
// j that can be within the cutoff of some i of the item: farther than r_cut
// (with a margin far above rounding) from the item's bounding box, a j is
// outside the cutoff of every i and would add exactly nothing, so dropping it
// leaves every pair sum unchanged; the kept j are compacted in stream order
// (ballot + prefix count) into full tiles, which carry over to the next call
// (fill, warp-uniform) until `last`.  With in-cell offsets (CI) the test runs
// in the frame of i's cell, where both the bounds and the staged j live.
// U selects the inner-loop form (the autotuner picks): 0 deep-unrolled and 1
// light-unrolled indexed loops, 2 pointer-stepped loop; every form visits the
// same entries in the same order.  (The lane-group count as a compile-time
// constant, four times the code, measured 2x slower from instruction-cache
// misses.)
template <int K, bool COUNT, bool POT, bool EPS0, bool UM, int U, bool CI>
__device__ __forceinline__ void process_runs(const KParams &P, const RunTable &rt, int r0, int r1, float L, float tx,
                                             float ty, float tz, int iself, int i_end, int lg, int grp,
                                             float (&xs)[K], float (&ys)[K], float (&zs)[K],
                                             float (&ax)[K], float (&ay)[K], float (&az)[K], unsigned &cnt,
                                             unsigned &jsum, float4 *buf, int *ids, int lane, int &fill, bool last) {
    const bool ishift = (tx != 0.0f) || (ty != 0.0f) || (tz != 0.0f);
    const int G = 1 << lg;
    // the i shift is applied in place and undone by reloading the coordinates
    // after the runs (no second copy of them in registers)
    if (ishift) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            xs[k] = __fadd_rn(xs[k], tx);
            ys[k] = __fadd_rn(ys[k], ty);
            zs[k] = __fadd_rn(zs[k], tz);
        }
    }
    const PairConsts C{P.eps, P.T, P.q0, P.q1, P.q2, P.q3, P.q4, P.q5};
    const float4 dummy = make_float4(1e18f, 1e18f, 1e18f, 0.0f);   // far away, zero mass
    const int tile = 32 << lg;
    // the item's bounds in this frame (monotone rounding keeps them bounds),
    // held in the warp's shared slots rather than in registers across the tiles
    if (lane == 0) {
        const float4 l = rt.bnd[0], h = rt.bnd[1];
        rt.bnd[2] = make_float4(__fadd_rn(l.x, tx), __fadd_rn(l.y, ty), __fadd_rn(l.z, tz), P.T * 1.001f + 1e-3f);
        rt.bnd[3] = make_float4(__fadd_rn(h.x, tx), __fadd_rn(h.y, ty), __fadd_rn(h.z, tz), 0.0f);
    }
    __syncwarp();
    const unsigned below = (1u << lane) - 1u;
    const int t_end = rt.A[r1 - 1].x;
    int t0 = r0 > 0 ? rt.A[r0 - 1].x : 0;
    int cur = r0;   // this lane's run
#pragma unroll 1
    while (true) {
        // stage 32 candidates at a time until a tile is full or the runs end
#pragma unroll 1
        while (fill < tile && t0 < t_end) {
            const int t = t0 + lane;
            bool keep = false;
            float4 v = dummy;
            int j = -1;
            if (t < t_end) {
                while (t >= rt.A[cur].x) ++cur;
                const int4 a = rt.A[cur];
                j = t + a.y;
                v = P.pos[j];
                if (CI) {
                    // in-cell offsets: move j into the frame of i's cell by whole
                    // cell steps of the FP32 width w (the x step depends on which of
                    // the run's cells j sits in).  For a j within reach of i's cell
                    // the sum lands in a binade no finer than the offset's, so it is
                    // exact: a close pair across a face gets its separation with one
                    // rounding at most, like a pair inside a cell.
                    const int4 b = rt.B[cur];
                    const float dlt = (float)(b.z + (j >= b.x) + (j >= b.y));
                    v.x = __fadd_rn(v.x, dlt * P.w);
                    v.y = __fadd_rn(v.y, (float)((a.z & 15) - 2) * P.w);
                    v.z = __fadd_rn(v.z, (float)(((a.z >> 4) & 15) - 2) * P.w);
                } else if (a.z & 7) {
                    if (a.z & 1) v.x = __fadd_rn(v.x, -L);
                    if (a.z & 2) v.y = __fadd_rn(v.y, -L);
                    if (a.z & 4) v.z = __fadd_rn(v.z, -L);
                }
                const float4 lo = rt.bnd[2], hi = rt.bnd[3];
                const float ex = fmaxf(fmaxf(lo.x - v.x, v.x - hi.x), 0.0f);
                const float ey = fmaxf(fmaxf(lo.y - v.y, v.y - hi.y), 0.0f);
                const float ez = fmaxf(fmaxf(lo.z - v.z, v.z - hi.z), 0.0f);
                keep = __fmaf_rn(ex, ex, __fmaf_rn(ey, ey, ez * ez)) < lo.w;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int at = fill + __popc(m & below);
                buf[at] = v;
                if (COUNT || POT) ids[at] = j;
            }
            fill += __popc(m);
            t0 += 32;
        }
        // a partial tile waits for the next call unless this is the last one
        if (fill < tile && !last) break;
        const int nj = min(fill, tile);
        if (nj == 0) break;
        // a short last tile is padded to whole passes of the pair loop (Unroll<K>::F
        // entries per lane group) with far, massless entries
        const int step = G * Unroll<K>::F;
        const int padded = (nj + step - 1) / step * step;
        if (nj < tile && lane < padded - nj) buf[nj + lane] = dummy;
        __syncwarp();
        run_tile<K, COUNT, POT, EPS0, UM, U>(P, C, buf, ids, nj, iself, lg, grp, xs, ys, zs, ax, ay, az, cnt);
        __syncwarp();
        if (COUNT) jsum += nj;
        // carry the entries past the tile to the front
        const int rest = fill - nj;
        float4 cv = dummy;
        int ci = 0;
        if (lane < rest) {
            cv = buf[nj + lane];
            if (COUNT || POT) ci = ids[nj + lane];
        }
        __syncwarp();
        if (lane < rest) {
            buf[lane] = cv;
            if (COUNT || POT) ids[lane] = ci;
        }
        fill = rest;
        if (t0 >= t_end && fill == 0) break;
    }
    __syncwarp();
    if (ishift) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = iself + (32 >> lg) * k;
            const float4 p = i < i_end ? P.pos[i] : make_float4(-1e30f, -1e30f, -1e30f, 0.0f);
            xs[k] = p.x;
            ys[k] = p.y;
            zs[k] = p.z;
        }
    }
}

// Write the run table of cell (cx, cy, cz) (of the box whose cells start at
// cbase) for stencil radius R, one run per lane; returns the number of runs.
template <bool CI>
__device__ __forceinline__ int build_runs(const KParams &P, const RunTable &rt, int cbase, int nc, int cx, int cy,
                                          int cz, int R, int lane) {
    const int span = 2 * R + 1;
    const int nrun = 2 * span * span;
    int run_end = 0;   // running total of the run lengths written so far
    for (int q0 = 0; q0 < nrun; q0 += 32) {
        const int q = q0 + lane;
        int ja = 0, jb = 0, bits = 0, b1 = 0, b2 = 0, d0 = 0;
        if (q < nrun) {
            const int rowi = q >> 1, r = q & 1;
            const int dz = rowi / span - R, dy = rowi % span - R;
            int rz = cz + dz, ry = cy + dy;
            int wb = 0;   // wrap flags: 1/2/4 low in x/y/z, 8/16/32 high
            if (rz < 0) { rz += nc; wb |= 4; }
            else if (rz >= nc) { rz -= nc; wb |= 32; }
            if (ry < 0) { ry += nc; wb |= 2; }
            else if (ry >= nc) { ry -= nc; wb |= 16; }
            const int32_t *row = P.cell_start + cbase + (rz * nc + ry) * nc;
            // cells lo..hi of this row: one run, or two when it wraps in x
            const int lo = cx - R, hi = cx + R;
            const bool wraps = lo < 0 || hi >= nc;
            if (lo < 0) {           // [0, hi], then [nc + lo, nc) with j shifted by -L
                ja = r ? row[nc + lo] : row[0];
                jb = r ? row[nc] : row[hi + 1];
                if (r) wb |= 1;
                b1 = r ? jb : row[1];
                d0 = r ? -1 : 0;
            } else if (hi >= nc) {  // [lo, nc), then [0, hi - nc] with i shifted by -L
                ja = r ? row[0] : row[lo];
                jb = r ? row[hi - nc + 1] : row[nc];
                if (r) wb |= 8;
                b1 = r ? jb : row[nc - 1];
                d0 = r ? 1 : -1;
            } else if (r == 0) {
                ja = row[lo];
                jb = row[hi + 1];
                b1 = row[cx];
                d0 = -1;
            }
            b2 = wraps ? jb : (r == 0 ? row[cx + 1] : 0);
            bits = CI ? ((dy + 2) | ((dz + 2) << 4) | (wb << 8)) : wb;
        }
        // exclusive ends of the runs in the concatenated stream
        int e = jb - ja;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, e, o);
            if (lane >= o) e += y;
        }
        e += run_end;
        if (q < nrun) {
            rt.A[q] = make_int4(e, ja - (e - (jb - ja)), bits, 0);
            if (CI) rt.B[q] = make_int4(b1, b2, d0, 0);
        }
        run_end = __shfl_sync(0xffffffffu, e, 31);
    }
    __syncwarp();
    return nrun;
}

// Apply the force on sorted particle i (position x, y, z, mass m) as the
// launch's mode says: store it, kick, or kick and stream.
__device__ __forceinline__ void write_result(const KParams &P, int i, float gx, float gy, float gz, float x, float y,
                                             float z, float m, float h_kick, float h_drift, float L) {
    if (P.mode == kModeForce) {
        int o = P.perm ? P.perm[i] : i;
        P.out[o] = make_float4(gx, gy, gz, 0.0f);
    } else if (P.mode == kModeKickLevels) {
        const float hk = P.kick.h[P.levels[i]];
        if (hk != 0.0f) {
            float4 v = P.vel[i];
            v.x = __fmaf_rn(hk, gx, v.x);
            v.y = __fmaf_rn(hk, gy, v.y);
            v.z = __fmaf_rn(hk, gz, v.z);
            if (P.ids) P.vel_pool[P.ids[i]] = v;   // back to input order
            else P.vel[i] = v;                      // in place, sorted order
        }
    } else if (P.mode == kModeKick) {
        const int row = P.ids[i];
        float4 v = P.vel[i];
        v.x = __fmaf_rn(h_kick, gx, v.x);
        v.y = __fmaf_rn(h_kick, gy, v.y);
        v.z = __fmaf_rn(h_kick, gz, v.z);
        P.vel_pool[row] = v;
    } else {
        float4 v = P.vel[i];
        v.x = __fmaf_rn(h_kick, gx, v.x);
        v.y = __fmaf_rn(h_kick, gy, v.y);
        v.z = __fmaf_rn(h_kick, gz, v.z);
        float4 p;
        p.x = __fmaf_rn(h_drift, v.x, x);
        p.y = __fmaf_rn(h_drift, v.y, y);
        p.z = __fmaf_rn(h_drift, v.z, z);
        p.w = m;
        if (P.mode == kModeBatch) {
            // back to the box's pool row, wrapped into [0, L)
            bool ok = wrap1(p.x, L);
            ok &= wrap1(p.y, L);
            ok &= wrap1(p.z, L);
            if (!ok) atomicOr(P.flags, kFlagDomain);
            const int row = P.ids[i];
            P.vel_pool[row] = v;
            P.pos_pool[row] = p;
        } else {
            P.vel[i] = v;
            P.pos_next[i] = p;
        }
    }
}

template <int K, bool COUNT, bool POT, bool EPS0, bool UM, int U, bool CI>
__device__ void process_item(const KParams &P, int4 item, float4 *buf, int *ids, const RunTable &rt, int lane,
                             float m_uniform) {
    // geometry: the single box of the call, or this item's box of a batch
    // (the kick and drift factors are read again in the epilogue)
    int nc = P.nc;
    float L = P.L;
    int cbase = 0;
    if (P.boxes) {
        const BoxDev &bx = P.boxes[item.w >> 8];
        nc = bx.nc;
        L = bx.L;
        cbase = bx.cell_base;
    }
    const int c = item.x - cbase, i0 = item.y, ni = item.z;
    const int lg = (item.w >> 4) & 15;    // 2^lg lane groups
    const int lpg = 32 >> lg;             // lanes per group
    const int grp = lane >> (5 - lg);
    const int slot = lane & (lpg - 1);
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);

    // every group holds the same K x lpg particles of the cell (their masses
    // are read again in the epilogue)
    float xi[K], yi[K], zi[K];
    float ax[K], ay[K], az[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int q = slot + lpg * k;
        float4 p = q < ni ? P.pos[i0 + q] : make_float4(-1e30f, -1e30f, -1e30f, 0.0f);
        xi[k] = p.x; yi[k] = p.y; zi[k] = p.z;
        ax[k] = 0.0f; ay[k] = 0.0f; az[k] = 0.0f;
    }
    unsigned cnt = 0, jsum = 0;           // pairs inside the cutoff; j evaluated (counting form)
    const int iself = i0 + slot;          // sorted index of this lane's k = 0 particle
    // bounding box of the item's particles (for the j culling of the runs),
    // kept in the warp's shared slots
    {
        float lx = 1e30f, ly = 1e30f, lz = 1e30f, hx = -1e30f, hy = -1e30f, hz = -1e30f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (slot + lpg * k < ni) {
                lx = fminf(lx, xi[k]);
                hx = fmaxf(hx, xi[k]);
                ly = fminf(ly, yi[k]);
                hy = fmaxf(hy, yi[k]);
                lz = fminf(lz, zi[k]);
                hz = fmaxf(hz, zi[k]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
            hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
            ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
            hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
            lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
            hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        }
        if (lane == 0) {
            rt.bnd[0] = make_float4(lx, ly, lz, 0.0f);
            rt.bnd[1] = make_float4(hx, hy, hz, 0.0f);
        }
        __syncwarp();
    }

    // neighbour cells cx-R..cx+R (R = 1: 27 cells; R = 2: 125 cells of a mesh twice as fine)
    const int R = P.boxes ? 1 : P.R;
    const int nrun = build_runs<CI>(P, rt, cbase, nc, cx, cy, cz, R, lane);
    // Tiles run on across all runs unless a run shifts the i side (cells
    // within R of the high faces; with in-cell offsets, cells next to any face
    // when the mesh has a wrap remainder): then every run ends its own tile.
    const bool carry = CI ? (P.delta == 0.0f || (cx >= R && cy >= R && cz >= R && cx + R < nc && cy + R < nc &&
                                                 cz + R < nc))
                          : (cx + R < nc && cy + R < nc && cz + R < nc);
    int fill = 0;
#pragma unroll 1
    for (int q = 0; q < nrun;) {
        // all runs at once, or one run with its own i shift
        const int q1 = carry ? nrun : q + 1;
        const int bits = carry ? 0 : rt.A[q].z;
        float tx, ty, tz;
        if (CI) {
            // a wrapped neighbour lies L - nc w beyond the whole cell steps:
            // moving i by it instead keeps the j side exact (the shifted i is
            // exact too for any i within reach of the face)
            const int wb = bits >> 8;
            tx = (wb & 1) ? P.delta : ((wb & 8) ? -P.delta : 0.0f);
            ty = (wb & 2) ? P.delta : ((wb & 16) ? -P.delta : 0.0f);
            tz = (wb & 4) ? P.delta : ((wb & 32) ? -P.delta : 0.0f);
        } else {
            tx = (bits & 8) ? -L : 0.0f;
            ty = (bits & 16) ? -L : 0.0f;
            tz = (bits & 32) ? -L : 0.0f;
        }
        if (rt.A[q1 - 1].x > (q > 0 ? rt.A[q - 1].x : 0))   // not empty
            process_runs<K, COUNT, POT, EPS0, UM, U, CI>(P, rt, q, q1, L, tx, ty, tz, iself, i0 + ni, lg, grp,
                                                         xi, yi, zi, ax, ay, az, cnt, jsum, buf, ids, lane, fill, true);
        q = q1;
    }

    // sum the groups' partial forces (the groups saw disjoint j)
    for (int o = 16; o >= lpg; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            ax[k] += __shfl_xor_sync(0xffffffffu, ax[k], o);
            ay[k] += __shfl_xor_sync(0xffffffffu, ay[k], o);
            az[k] += __shfl_xor_sync(0xffffffffu, az[k], o);
        }
    }

    // epilogue (group 0 writes)
    if (grp == 0) {
        float h_kick = P.h_kick, h_drift = P.h_drift;
        if (P.boxes) {
            const BoxDev &bx = P.boxes[item.w >> 8];
            h_kick = bx.h;
            h_drift = bx.post;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int q = slot + lpg * k;
            if (q >= ni) continue;
            int i = i0 + q;
            const float mi = P.pos[i].w;
            if (POT) {
                P.phi_out[i] = 0.5f * P.G * mi * ax[k];
                continue;
            }
            const float gm = UM ? P.G * m_uniform : P.G;
            write_result(P, i, gm * ax[k], gm * ay[k], gm * az[k], xi[k], yi[k], zi[k], mi, h_kick, h_drift, L);
        }
    }
    if (COUNT) {
        unsigned long long c64 = cnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c64 += __shfl_down_sync(0xffffffffu, c64, o);
        if (lane == 0) atomicAdd(P.within, c64);
        if (lane == 0 && P.evaluated) atomicAdd(P.evaluated, (unsigned long long)jsum * (unsigned long long)ni);
    }
}

template <bool COUNT, bool POT, bool EPS0, bool UM, int U, bool CI = false>
__device__ __forceinline__ void work_loop(const KParams &P, float4 *buf, int *ids, const RunTable &rt, int lane,
                                          float m_uniform) {
    const int n_items = *P.n_items;
    while (true) {
        int it = 0;
        if (lane == 0) it = atomicAdd(P.work_counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        int4 item = P.items[P.order ? P.order[it] : it];
        switch (item.w & 15) {
            case 1: process_item<1, COUNT, POT, EPS0, UM, U, CI>(P, item, buf, ids, rt, lane, m_uniform); break;
            case 2: process_item<2, COUNT, POT, EPS0, UM, U, CI>(P, item, buf, ids, rt, lane, m_uniform); break;
            case 3: process_item<3, COUNT, POT, EPS0, UM, U, CI>(P, item, buf, ids, rt, lane, m_uniform); break;
            case 4: process_item<4, COUNT, POT, EPS0, UM, U, CI>(P, item, buf, ids, rt, lane, m_uniform); break;
            default: process_item<5, COUNT, POT, EPS0, UM, U, CI>(P, item, buf, ids, rt, lane, m_uniform); break;
        }
    }
}

// MINB: blocks per SM the register allocation must allow (6 -> 80, 8 -> 64,
// 5 -> 96 registers per thread); U: unroll policy.  The autotuner picks.
template <bool COUNT, bool POT, bool EPS0, int MINB, int U>
__global__ void __launch_bounds__(kThreads, MINB) k_sr_force(KParams P) {
    __shared__ float4 tiles[kWarps][kTileCap];
    __shared__ int tile_ids[COUNT || POT ? kWarps : 1][kTileCap];
    __shared__ int4 runs[kWarps][kMaxRuns];
    __shared__ float4 bnd[kWarps][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *buf = tiles[w];
    int *ids = tile_ids[COUNT || POT ? w : 0];
    const RunTable rt{runs[w], nullptr, bnd[w]};
    // equal masses (flag left 0 by the binning pass): apply the mass once per i
    if (!POT && P.mass_flag && *P.mass_flag == 0 && *P.n_items > 0)
        work_loop<COUNT, POT, EPS0, true, U>(P, buf, ids, rt, lane, P.pos[0].w);
    else
        work_loop<COUNT, POT, EPS0, false, U>(P, buf, ids, rt, lane, 0.0f);
}

// Positions as (cell, in-cell offset): the precision variant.
template <bool EPS0>
__global__ void __launch_bounds__(kThreads, 5) k_sr_force_ci(KParams P) {
    __shared__ float4 tiles[kWarps][kTileCap];
    __shared__ int4 runs[kWarps][kMaxRuns];
    __shared__ int4 steps[kWarps][kMaxRuns];
    __shared__ float4 bnd[kWarps][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4 *buf = tiles[w];
    const RunTable rt{runs[w], steps[w], bnd[w]};
    if (P.mass_flag && *P.mass_flag == 0 && *P.n_items > 0)
        work_loop<false, false, EPS0, true, 0, true>(P, buf, nullptr, rt, lane, P.pos[0].w);
    else
        work_loop<false, false, EPS0, false, 0, true>(P, buf, nullptr, rt, lane, 0.0f);
}

// Pair potential (diagnostics) of the precision variant.
template <bool EPS0>
__global__ void __launch_bounds__(kThreads, 5) k_sr_pot_ci(KParams P) {
    __shared__ float4 tiles[kWarps][kTileCap];
    __shared__ int tile_ids[kWarps][kTileCap];
    __shared__ int4 runs[kWarps][kMaxRuns];
    __shared__ int4 steps[kWarps][kMaxRuns];
    __shared__ float4 bnd[kWarps][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const RunTable rt{runs[w], steps[w], bnd[w]};
    work_loop<false, true, EPS0, false, 0, true>(P, tiles[w], tile_ids[w], rt, lane, 0.0f);
}

template <bool COUNT, bool POT, bool EPS0, int MINB, int U>
cudaError_t launch_one(const KParams &P, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sr_force<COUNT, POT, EPS0, MINB, U>, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_sr_force<COUNT, POT, EPS0, MINB, U><<<num_sms * per_sm, kThreads, 0, s>>>(P);
    note_launch();
    return cudaGetLastError();
}

// Variants 0..kForceVariants-1: (MINB, U) = (5, 0), (4, 0), (5, 2), (4, 2);
// all give bitwise the same forces.
// (A blocked tile layout, each group's entries contiguous at a padded stride,
// measured 5% slower than these and changes the summation order.)
template <bool COUNT, bool POT, bool EPS0>
cudaError_t launch_variant(const KParams &P, int variant, int num_sms, cudaStream_t s) {
    switch (variant) {
        case 1: return launch_one<COUNT, POT, EPS0, 4, 0>(P, num_sms, s);
        case 2: return launch_one<COUNT, POT, EPS0, 5, 2>(P, num_sms, s);
        case 3: return launch_one<COUNT, POT, EPS0, 4, 2>(P, num_sms, s);
        default: return launch_one<COUNT, POT, EPS0, 5, 0>(P, num_sms, s);
    }
}

}  // namespace

cudaError_t sr_force_launch(const Geometry &g, const ForceConsts &fc, const ForceLaunch &fl, int num_sms,
                            cudaStream_t s) {
    const bool pot = fl.mode == kModePotential;
    cudaError_t e = cudaMemsetAsync(fl.work_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    KParams P;
    P.pos = fl.pos;
    P.items = fl.items;
    P.order = fl.order;
    P.n_items = fl.n_items;
    P.cell_start = fl.cell_start;
    P.work_counter = fl.work_counter;
    P.nc = g.nc;
    P.R = g.R;
    P.L = g.Lf;
    P.T = fc.T;
    P.eps = fc.eps;
    P.G = fc.G;
    P.q0 = fc.q[0]; P.q1 = fc.q[1]; P.q2 = fc.q[2]; P.q3 = fc.q[3]; P.q4 = fc.q[4]; P.q5 = fc.q[5];
    P.u0 = fc.u[0]; P.u1 = fc.u[1]; P.u2 = fc.u[2]; P.u3 = fc.u[3]; P.u4 = fc.u[4]; P.u5 = fc.u[5];
    P.u6 = fc.u[6];
    P.phi0 = fc.phi0;
    P.mode = fl.mode;
    P.out = fl.out;
    P.perm = fl.perm;
    P.vel = fl.vel;
    P.pos_next = fl.pos_next;
    P.h_kick = fl.h_kick;
    P.h_drift = fl.h_drift;
    P.phi_out = fl.phi_out;
    P.within = fl.within;
    P.evaluated = fl.evaluated;
    P.mass_flag = fl.mass_flag;
    P.boxes = fl.boxes;
    P.ids = fl.ids;
    P.pos_pool = fl.pos_pool;
    P.vel_pool = fl.vel_pool;
    P.flags = fl.flags;
    P.w = fl.w;
    P.levels = fl.levels;
    P.kick = fl.kick;
    P.delta = fl.delta;
    const bool eps0 = !(fc.eps > 0.0f);
    const bool count = fl.within != nullptr;
    const int v = fl.variant;
    if (fl.cell_offset && pot) {
        int per_sm = 0;
        cudaError_t e = eps0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sr_pot_ci<true>, kThreads, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sr_pot_ci<false>, kThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        if (eps0) k_sr_pot_ci<true><<<num_sms * per_sm, kThreads, 0, s>>>(P);
        else k_sr_pot_ci<false><<<num_sms * per_sm, kThreads, 0, s>>>(P);
        note_launch();
        return cudaGetLastError();
    }
    if (fl.cell_offset) {
        int per_sm = 0;
        cudaError_t e = eps0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sr_force_ci<true>, kThreads, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sr_force_ci<false>, kThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        if (eps0) k_sr_force_ci<true><<<num_sms * per_sm, kThreads, 0, s>>>(P);
        else k_sr_force_ci<false><<<num_sms * per_sm, kThreads, 0, s>>>(P);
        note_launch();
        return cudaGetLastError();
    }
    if (pot) return eps0 ? launch_one<false, true, true, 5, 0>(P, num_sms, s) : launch_one<false, true, false, 5, 0>(P, num_sms, s);
    if (count) return eps0 ? launch_variant<true, false, true>(P, v, num_sms, s) : launch_variant<true, false, false>(P, v, num_sms, s);
    return eps0 ? launch_variant<false, false, true>(P, v, num_sms, s) : launch_variant<false, false, false>(P, v, num_sms, s);
}

// ---- FP64 diagnostics ------------------------------------------------------
namespace {
__global__ void __launch_bounds__(256) k_diag(int64_t n, const float4 *__restrict__ pos,
                                               const float4 *__restrict__ vel, const float *__restrict__ phi,
                                               double *out) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float4 v = vel[i];
        double m = pos[i].w;
        s[0] += m * v.x;
        s[1] += m * v.y;
        s[2] += m * v.z;
        s[3] += 0.5 * m * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
        s[4] += phi ? (double)phi[i] : 0.0;
    }
    __shared__ double red[5][8];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double x = s[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double x = 0;
        for (int q = 0; q < (int)(blockDim.x / 32); ++q) x += red[threadIdx.x][q];
        atomicAdd(out + threadIdx.x, x);
    }
}
// Per box of a batch: block (box q, part k) sums part k of the box's sorted
// range (a fixed split into kDiagParts) in a fixed order; k_diag_combine adds
// the parts of each box in order.  Nothing depends on the other boxes.
__global__ void __launch_bounds__(256) k_diag_batch(const BoxDev *__restrict__ boxes,
                                                     const int32_t *__restrict__ cell_start,
                                                     const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                                                     const float *__restrict__ phi, double *__restrict__ partial) {
    const int q = blockIdx.x / kDiagParts, part = blockIdx.x % kDiagParts;
    const BoxDev bx = boxes[q];
    const int64_t a = cell_start[bx.cell_base];
    const int64_t len = (int64_t)cell_start[bx.cell_base + bx.nc * bx.nc * bx.nc] - a;
    const int64_t lo = a + len * part / kDiagParts, hi = a + len * (part + 1) / kDiagParts;
    double s[5] = {0, 0, 0, 0, 0};
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float4 v = vel[i];
        const double m = pos[i].w;
        s[0] += m * v.x;
        s[1] += m * v.y;
        s[2] += m * v.z;
        s[3] += 0.5 * m * ((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
        s[4] += (double)phi[i];
    }
    __shared__ double red[5][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double x = s[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double x = 0;
        for (int r = 0; r < (int)(blockDim.x / 32); ++r) x += red[threadIdx.x][r];
        partial[((int64_t)q * kDiagParts + part) * 5 + threadIdx.x] = x;
    }
}

__global__ void __launch_bounds__(256) k_diag_combine(int nbox, const BoxDev *__restrict__ boxes,
                                                       const double *__restrict__ partial, double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nbox * 5) return;
    const int q = (int)(t / 5), k = (int)(t % 5);
    double x = 0;
    for (int part = 0; part < kDiagParts; ++part) x += partial[((int64_t)q * kDiagParts + part) * 5 + k];
    out[(int64_t)boxes[q].orig * 5 + k] = x;
}

__global__ void __launch_bounds__(256) k_mass_moment_ci(int64_t n, const int32_t *__restrict__ cell,
                                                         const float4 *__restrict__ off, int nc, double w,
                                                         double *out) {
    double s[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cell[i];
        const float4 o = off[i];
        const double m = o.w;
        s[0] += m * fma((double)(c % nc) + 0.5, w, (double)o.x);
        s[1] += m * fma((double)((c / nc) % nc) + 0.5, w, (double)o.y);
        s[2] += m * fma((double)(c / (nc * nc)) + 0.5, w, (double)o.z);
    }
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = s[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][wp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double x = 0;
        for (int r = 0; r < (int)(blockDim.x / 32); ++r) x += red[threadIdx.x][r];
        atomicAdd(out + threadIdx.x, x);
    }
}
}  // namespace

cudaError_t diag_reduce_batch(int nbox, const BoxDev *boxes, const int32_t *cell_start, const float4 *pos,
                              const float4 *vel, const float *phi, double *partial, double *out, cudaStream_t s) {
    if (nbox <= 0) return cudaSuccess;
    k_diag_batch<<<(unsigned)nbox * kDiagParts, 256, 0, s>>>(boxes, cell_start, pos, vel, phi, partial);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_combine<<<(unsigned)((nbox * 5 + 255) / 256), 256, 0, s>>>(nbox, boxes, partial, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t diag_mass_moment_ci(int64_t n, const int32_t *cell, const float4 *off, int nc, double w, double *out,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_mass_moment_ci<<<blocks, 256, 0, s>>>(n, cell, off, nc, w, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t diag_reduce(int64_t n, const float4 *pos, const float4 *vel, const float *phi, double *out,
                        cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, 5 * sizeof(double), s);
    if (e != cudaSuccess || n <= 0) return e;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_diag<<<blocks, 256, 0, s>>>(n, pos, vel, phi, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace hacc
