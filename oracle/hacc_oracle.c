/*
 * FP64 CPU oracle for the short-range particle-particle force of the HACC
 * force split (Habib et al., "HACC: Simulating Sky Surveys on
 * State-of-the-Art Supercomputing Architectures", arXiv 1410.2805).
 *
 * TEST INFRASTRUCTURE ONLY.  The product path never links, loads or calls
 * this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * library under paper_1410_2805_gb300/.
 *
 * Plain and slow on purpose: every sum is FP64, loops follow the definitions,
 * OpenMP only splits the outer loop over particles (each particle's sum is
 * still taken in ascending j order by one thread).
 *
 * What each function follows:
 *   hacc_oracle_fsr          Sec. 3.1, Eq. (force): f_SR(s) = (s+eps)^(-3/2) - P5(s)
 *   hacc_oracle_phi          pair potential whose radial derivative gives f_SR
 *                            (phi'(s) = f_SR(s)/2), shifted to vanish at r_cut
 *   hacc_oracle_wrap_cell    periodic box + chaining-mesh cell of Sec. 2.4 / 3.3
 *                            (cell rule in exact arithmetic, see the comment there)
 *   hacc_oracle_bin          stable counting sort by cell (Hockney chaining mesh)
 *   hacc_oracle_force_brute  the plain definition: all pairs, minimum image
 *   hacc_oracle_force_mesh   same pair set through an FP64 cell list
 *   hacc_oracle_candidates   27-neighbour candidate-pair count of a binning
 *   hacc_oracle_subcycle     SKS short-range sub-cycle, Sec. 2.5 / Sec. 3.1
 *   hacc_oracle_diagnostics  momentum, kinetic and pair potential energy
 *
 * Conventions: positions in grid units in a periodic cube of side L; the
 * force on i is a_i = G sum_j m_j r_ij f_SR(|r_ij|^2), r_ij = x_j - x_i
 * (minimum image), over j != i with |r_ij|^2 < r_cut^2 (attractive).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math, no
 * contraction, so results agree between x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int hacc_oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void hacc_oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. (force): f_SR(s) = (s + eps)^(-3/2) - P5(s),  P5(s) = sum_k c_k s^k.  */
double hacc_oracle_fsr(double s, double eps, const double *c) {
    double t = s + eps;
    double newton = 1.0 / (t * sqrt(t));
    double p = 0.0, sk = 1.0;
    for (int k = 0; k < 6; ++k) { p += c[k] * sk; sk *= s; }
    return newton - p;
}

/* Pair potential phi(s) with d phi / d s = f_SR(s) / 2, so that the force on i
 * is -grad_i (G m_i m_j phi) / m_i = G m_j r_ij f_SR.  Integrating:
 *   phi(s) = -(s+eps)^(-1/2) - sum_k c_k s^(k+1) / (2(k+1)) + const,
 * with the constant chosen so that phi(r_cut^2) = 0. */
static double phi_raw(double s, double eps, const double *c) {
    double v = -1.0 / sqrt(s + eps);
    double sk = s;
    for (int k = 0; k < 6; ++k) { v -= c[k] * sk / (2.0 * (k + 1)); sk *= s; }
    return v;
}

double hacc_oracle_phi(double s, double eps, const double *c, double rcut) {
    return phi_raw(s, eps, c) - phi_raw(rcut * rcut, eps, c);
}

/* ------------------------------------------------------------------------ */
/* Wrap into the periodic box and find the chaining-mesh cell.
 *
 * Wrap rule (in the stored FP32 precision): a coordinate x in [-L, 2L) maps to
 * x + L if x < 0, x - L if x >= L, else x; a result that rounds up to L
 * becomes 0.  Anything outside [-L, 2L) or non-finite is an error.
 *
 * Cell rule (exact arithmetic on the FP32 value): the cell of x in [0, L) is
 * the largest integer k with k * L <= x * nc.  x * nc and k * L are exact in
 * FP64 here (24-bit mantissa times an integer below 2^11, and L is required to
 * be an FP32 value), so the comparisons below are exact.
 * Linear id = (iz * nc + iy) * nc + ix.
 *
 * pos4: n x 4 floats (x, y, z, m), wrapped in place.  Returns 0, or -1 if some
 * coordinate was out of range (cell of that particle is then -1). */
static int cell_1d(float x, double L, int nc) {
    double xn = (double)x * (double)nc;
    int k = (int)floor(xn / L);
    if (k < 0) k = 0;
    if (k > nc - 1) k = nc - 1;
    while (k > 0 && (double)k * L > xn) --k;
    while (k < nc - 1 && (double)(k + 1) * L <= xn) ++k;
    return k;
}

static int wrap_1d(float *x, float Lf) {
    float v = *x;
    if (!(v >= -Lf && v < 2.0f * Lf)) return -1;   /* also catches NaN */
    if (v < 0.0f) v = v + Lf;
    else if (v >= Lf) v = v - Lf;
    if (v >= Lf) v = 0.0f;
    *x = v;
    return 0;
}

int hacc_oracle_wrap_cell(int64_t n, float *pos4, double L, int nc, int32_t *cell) {
    float Lf = (float)L;
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        float *p = pos4 + 4 * i;
        int e = wrap_1d(p + 0, Lf) | wrap_1d(p + 1, Lf) | wrap_1d(p + 2, Lf);
        if (e) { cell[i] = -1; bad = 1; continue; }
        int ix = cell_1d(p[0], L, nc), iy = cell_1d(p[1], L, nc), iz = cell_1d(p[2], L, nc);
        cell[i] = (int32_t)(((int64_t)iz * nc + iy) * nc + ix);
    }
    return bad ? -1 : 0;
}

/* Stable counting sort by cell: count[c] = particles in c, start[c] = first
 * sorted slot of c (start has ncell+1 entries), perm[k] = original index of
 * the particle in sorted slot k; within a cell, ascending original index. */
void hacc_oracle_bin(int64_t n, const int32_t *cell, int64_t ncell,
                     int32_t *count, int32_t *start, int32_t *perm) {
    memset(count, 0, sizeof(int32_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) count[cell[i]]++;
    start[0] = 0;
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] = start[c] + count[c];
    int32_t *cursor = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    memcpy(cursor, start, sizeof(int32_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) perm[cursor[cell[i]]++] = (int32_t)i;
    free(cursor);
}

/* Candidate pairs of the 27-neighbour chaining mesh: sum over cells c of
 * n_c * (sum of n over the 27 cells around c, periodic).  Includes i == j. */
uint64_t hacc_oracle_candidates(const int32_t *count, int nc) {
    uint64_t total = 0;
    for (int iz = 0; iz < nc; ++iz)
        for (int iy = 0; iy < nc; ++iy)
            for (int ix = 0; ix < nc; ++ix) {
                uint64_t ni = (uint64_t)count[((int64_t)iz * nc + iy) * nc + ix];
                if (!ni) continue;
                uint64_t nb = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int jx = (ix + dx + nc) % nc, jy = (iy + dy + nc) % nc, jz = (iz + dz + nc) % nc;
                            nb += (uint64_t)count[((int64_t)jz * nc + jy) * nc + jx];
                        }
                total += ni * nb;
            }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Minimum image of a separation component in a periodic cube of side L. */
static double min_image(double d, double L) {
    return d - L * nearbyint(d / L);
}

/* The plain definition: a_i = G sum_{j != i, s < rcut^2} m_j r_ij f_SR(s).
 * x: n x 3 doubles, m: n doubles, acc: n x 3 doubles.
 * within (nullable): number of ordered pairs (i, j) inside the cutoff. */
void hacc_oracle_force_brute(int64_t n, const double *x, const double *m, double L,
                             double rcut, double eps, const double *c, double G,
                             double *acc, uint64_t *within) {
    double rc2 = rcut * rcut;
    uint64_t w = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : w)
    for (int64_t i = 0; i < n; ++i) {
        double ax = 0, ay = 0, az = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = min_image(x[3 * j + 0] - x[3 * i + 0], L);
            double dy = min_image(x[3 * j + 1] - x[3 * i + 1], L);
            double dz = min_image(x[3 * j + 2] - x[3 * i + 2], L);
            double s = dx * dx + dy * dy + dz * dz;
            if (!(s < rc2)) continue;
            double f = m[j] * hacc_oracle_fsr(s, eps, c);
            ax += f * dx; ay += f * dy; az += f * dz;
            ++w;
        }
        acc[3 * i + 0] = G * ax; acc[3 * i + 1] = G * ay; acc[3 * i + 2] = G * az;
    }
    if (within) *within = w;
}

/* The oracle's own cell list (independent of the GPU binning): nco cells per
 * side with width L/nco >= rcut (one cell fewer when the width would come
 * within 1e-9 of rcut, so FP64 rounding at cell faces cannot split a pair
 * that lies inside the cutoff), positions wrapped into [0, L) in FP64. */
typedef struct {
    int nco;
    int32_t *start;   /* nco^3 + 1 */
    int32_t *idx;     /* n, particles by cell, ascending index inside a cell */
} oracle_mesh;

static int mesh_nc(double L, double rcut) {
    int nco = (int)floor(L / rcut);
    if (nco >= 1 && L / nco < rcut * (1.0 + 1e-9)) --nco;
    return nco;
}

static double wrap64(double v, double L) {
    double w = v - L * floor(v / L);
    if (w >= L) w -= L;
    if (w < 0) w = 0;
    return w;
}

static int mesh_cell_1d(double v, double L, int nco) {
    int k = (int)floor(wrap64(v, L) * nco / L);
    if (k < 0) k = 0;
    if (k >= nco) k = nco - 1;
    return k;
}

static void mesh_build(oracle_mesh *M, int64_t n, const double *x, double L, double rcut) {
    int nco = mesh_nc(L, rcut);
    M->nco = nco;
    int64_t ncell = (int64_t)nco * nco * nco;
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    M->start = (int32_t *)calloc((size_t)ncell + 1, sizeof(int32_t));
    M->idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        int ix = mesh_cell_1d(x[3 * i + 0], L, nco);
        int iy = mesh_cell_1d(x[3 * i + 1], L, nco);
        int iz = mesh_cell_1d(x[3 * i + 2], L, nco);
        cell[i] = (int32_t)(((int64_t)iz * nco + iy) * nco + ix);
        M->start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) M->start[c + 1] += M->start[c];
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    memcpy(cur, M->start, sizeof(int32_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) M->idx[cur[cell[i]]++] = (int32_t)i;
    free(cur);
    free(cell);
}

static void mesh_free(oracle_mesh *M) { free(M->start); free(M->idx); }

/* Force on one particle i through the cell list (same pair set as brute force;
 * the 27 neighbour cells are distinct because nco >= 3). */
static void mesh_force_one(const oracle_mesh *M, int64_t i, const double *x, const double *m,
                           double L, double rc2, double eps, const double *c, double G,
                           double *a, uint64_t *w) {
    int nco = M->nco;
    int ix = mesh_cell_1d(x[3 * i + 0], L, nco);
    int iy = mesh_cell_1d(x[3 * i + 1], L, nco);
    int iz = mesh_cell_1d(x[3 * i + 2], L, nco);
    double ax = 0, ay = 0, az = 0;
    uint64_t cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx_ = -1; dx_ <= 1; ++dx_) {
                int jx = (ix + dx_ + nco) % nco, jy = (iy + dy + nco) % nco, jz = (iz + dz + nco) % nco;
                int64_t cj = ((int64_t)jz * nco + jy) * nco + jx;
                for (int32_t q = M->start[cj]; q < M->start[cj + 1]; ++q) {
                    int64_t j = M->idx[q];
                    if (j == i) continue;
                    double ddx = min_image(x[3 * j + 0] - x[3 * i + 0], L);
                    double ddy = min_image(x[3 * j + 1] - x[3 * i + 1], L);
                    double ddz = min_image(x[3 * j + 2] - x[3 * i + 2], L);
                    double s = ddx * ddx + ddy * ddy + ddz * ddz;
                    if (!(s < rc2)) continue;
                    double f = m[j] * hacc_oracle_fsr(s, eps, c);
                    ax += f * ddx; ay += f * ddy; az += f * ddz;
                    ++cnt;
                }
            }
    a[0] = G * ax; a[1] = G * ay; a[2] = G * az;
    *w = cnt;
}

/* Forces through the cell list, for all particles (sel == NULL, nsel == n) or
 * for the nsel particles listed in sel.  acc: nsel x 3.  Falls back to brute
 * force over all j when the box holds fewer than 3 cells per side. */
void hacc_oracle_force_mesh(int64_t n, const double *x, const double *m, double L,
                            double rcut, double eps, const double *c, double G,
                            int64_t nsel, const int64_t *sel, double *acc, uint64_t *within) {
    double rc2 = rcut * rcut;
    uint64_t w = 0;
    if (mesh_nc(L, rcut) < 3) {
        double *full = (double *)malloc(sizeof(double) * 3 * (size_t)(n ? n : 1));
        hacc_oracle_force_brute(n, x, m, L, rcut, eps, c, G, full, NULL);
        for (int64_t k = 0; k < nsel; ++k) {
            int64_t i = sel ? sel[k] : k;
            acc[3 * k + 0] = full[3 * i + 0]; acc[3 * k + 1] = full[3 * i + 1]; acc[3 * k + 2] = full[3 * i + 2];
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double dx = min_image(x[3 * j + 0] - x[3 * i + 0], L);
                double dy = min_image(x[3 * j + 1] - x[3 * i + 1], L);
                double dz = min_image(x[3 * j + 2] - x[3 * i + 2], L);
                if (dx * dx + dy * dy + dz * dz < rc2) ++w;
            }
        }
        free(full);
        if (within) *within = w;
        return;
    }
    oracle_mesh M;
    mesh_build(&M, n, x, L, rcut);
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : w)
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t i = sel ? sel[k] : k;
        uint64_t cnt;
        mesh_force_one(&M, i, x, m, L, rc2, eps, c, G, acc + 3 * k, &cnt);
        w += cnt;
    }
    mesh_free(&M);
    if (within) *within = w;
}

/* ------------------------------------------------------------------------ */
/* Short-range sub-cycle of Sec. 2.5: n_sub symmetric stream-kick-stream maps
 * of step h = dt / n_sub each:  x += (h/2) v;  v += h a(x);  x += (h/2) v,
 * wrapping positions into [0, L) after every stream.  Static (non-expanding)
 * time, FP64 throughout.  x, v: n x 3 doubles, updated in place. */
void hacc_oracle_subcycle(int64_t n, double *x, double *v, const double *m, double L,
                          double rcut, double eps, const double *c, double G,
                          double dt, int nsub) {
    double h = dt / nsub;
    double *a = (double *)malloc(sizeof(double) * 3 * (size_t)(n ? n : 1));
    for (int k = 0; k < nsub; ++k) {
        for (int64_t i = 0; i < 3 * n; ++i) x[i] = wrap64(x[i] + 0.5 * h * v[i], L);
        hacc_oracle_force_mesh(n, x, m, L, rcut, eps, c, G, n, NULL, a, NULL);
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += h * a[i];
        for (int64_t i = 0; i < 3 * n; ++i) x[i] = wrap64(x[i] + 0.5 * h * v[i], L);
    }
    free(a);
}

/* Diagnostics: out[0..2] = sum m v, out[3] = kinetic energy sum m v^2 / 2,
 * out[4] = pair potential energy sum_{i<j, s<rcut^2} G m_i m_j phi(s). */
void hacc_oracle_diagnostics(int64_t n, const double *x, const double *v, const double *m,
                             double L, double rcut, double eps, const double *c, double G,
                             double *out) {
    double px = 0, py = 0, pz = 0, ke = 0;
    for (int64_t i = 0; i < n; ++i) {
        px += m[i] * v[3 * i + 0]; py += m[i] * v[3 * i + 1]; pz += m[i] * v[3 * i + 2];
        ke += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    }
    double rc2 = rcut * rcut, pe = 0;
    if (mesh_nc(L, rcut) < 3) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j) {
                double dx = min_image(x[3 * j] - x[3 * i], L);
                double dy = min_image(x[3 * j + 1] - x[3 * i + 1], L);
                double dz = min_image(x[3 * j + 2] - x[3 * i + 2], L);
                double s = dx * dx + dy * dy + dz * dz;
                if (s < rc2) pe += G * m[i] * m[j] * hacc_oracle_phi(s, eps, c, rcut);
            }
    } else {
        oracle_mesh M;
        mesh_build(&M, n, x, L, rcut);
        int nco = M.nco;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : pe)
        for (int64_t i = 0; i < n; ++i) {
            int ix = mesh_cell_1d(x[3 * i + 0], L, nco);
            int iy = mesh_cell_1d(x[3 * i + 1], L, nco);
            int iz = mesh_cell_1d(x[3 * i + 2], L, nco);
            double local = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx_ = -1; dx_ <= 1; ++dx_) {
                        int jx = (ix + dx_ + nco) % nco, jy = (iy + dy + nco) % nco, jz = (iz + dz + nco) % nco;
                        int64_t cj = ((int64_t)jz * nco + jy) * nco + jx;
                        for (int32_t q = M.start[cj]; q < M.start[cj + 1]; ++q) {
                            int64_t j = M.idx[q];
                            if (j <= i) continue;
                            double ddx = min_image(x[3 * j] - x[3 * i], L);
                            double ddy = min_image(x[3 * j + 1] - x[3 * i + 1], L);
                            double ddz = min_image(x[3 * j + 2] - x[3 * i + 2], L);
                            double s = ddx * ddx + ddy * ddy + ddz * ddz;
                            if (s < rc2) local += G * m[i] * m[j] * hacc_oracle_phi(s, eps, c, rcut);
                        }
                    }
            pe += local;
        }
        mesh_free(&M);
    }
    out[0] = px; out[1] = py; out[2] = pz; out[3] = ke; out[4] = pe;
}

/* ------------------------------------------------------------------------ */
/* Multi-level short-range step (Sec. 3.1, Eq. (kicks)).
 *
 * Levels: with the chaining mesh of hacc_oracle_wrap_cell on the FP32 start
 * positions, a cell holding count particles has density rho / rho0 =
 * count nc^3 / n; its particles get l = floor(floor(rho/rho0) / d) + 1 kicks
 * (integer arithmetic), capped at lmax and raised to at least lmin (the paper
 * runs its test with every particle taking at least two sub-cycles and up to two
 * more levels in the densest regions).  d <= 0 gives every particle lmax.
 * pos32: n x 4 floats (wrapped copy is made internally); level: n ints out. */
void hacc_oracle_ml_levels(int64_t n, const float *pos32, double L, int nc, int d, int lmin, int lmax,
                           int32_t *level) {
    int64_t ncell = (int64_t)nc * nc * nc;
    float *p = (float *)malloc(sizeof(float) * 4 * (size_t)(n ? n : 1));
    memcpy(p, pos32, sizeof(float) * 4 * (size_t)n);
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    hacc_oracle_wrap_cell(n, p, L, nc, cell);
    int64_t *count = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) count[cell[i]]++;
    for (int64_t i = 0; i < n; ++i) {
        int64_t l = lmax;
        if (d > 0) {
            int64_t ratio = count[cell[i]] * ncell / n;   /* floor(rho / rho0) */
            l = ratio / d + 1;
            if (l > lmax) l = lmax;
        }
        if (l < lmin) l = lmin;
        level[i] = (int32_t)l;
    }
    free(count);
    free(cell);
    free(p);
}

/* One multi-level step of length dt with fixed per-particle kick counts
 * level[i] in [1, lmax]: a particle with l kicks is kicked by dt/l at the
 * times (2k+1)/(2l) dt, k = 0..l-1 (the midpoints of its own SKS steps); all
 * particles stream together between consecutive event times (the union of
 * those times over the levels present), so each is streamed by the same
 * total dt.  FP64. */
void hacc_oracle_subcycle_ml(int64_t n, double *x, double *v, const double *m, double L, double rcut, double eps,
                             const double *c, double G, double dt, int lmax, const int32_t *level) {
    /* event times, as reduced fractions num/den of dt, of the levels present */
    int cap = lmax * (lmax + 1) / 2, ne = 0;
    int64_t *num = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t *den = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    char *present = (char *)calloc((size_t)lmax + 1, 1);
    for (int64_t i = 0; i < n; ++i)
        if (level[i] >= 1 && level[i] <= lmax) present[level[i]] = 1;
    for (int l = 1; l <= lmax; ++l)
        for (int k = 0; k < l && present[l]; ++k) {
            int64_t a = 2 * k + 1, b = 2 * l, g = a, h = b;
            while (h) { int64_t t = g % h; g = h; h = t; }
            a /= g; b /= g;
            int dup = 0;
            for (int e = 0; e < ne; ++e) if (num[e] == a && den[e] == b) dup = 1;
            if (!dup) { num[ne] = a; den[ne] = b; ++ne; }
        }
    for (int i = 1; i < ne; ++i)          /* insertion sort by value (exact cross products) */
        for (int j = i; j > 0 && num[j] * den[j - 1] < num[j - 1] * den[j]; --j) {
            int64_t t = num[j]; num[j] = num[j - 1]; num[j - 1] = t;
            t = den[j]; den[j] = den[j - 1]; den[j - 1] = t;
        }
    int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    double *a = (double *)malloc(sizeof(double) * 3 * (size_t)(n ? n : 1));
    double t_prev = 0.0;
    for (int e = 0; e < ne; ++e) {
        double te = dt * (double)num[e] / (double)den[e];
        for (int64_t i = 0; i < 3 * n; ++i) x[i] = wrap64(x[i] + (te - t_prev) * v[i], L);
        t_prev = te;
        int64_t ns = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t l = level[i];
            /* kicked now iff 2 l num / den is an odd integer */
            if ((2 * l * num[e]) % den[e] == 0 && ((2 * l * num[e]) / den[e]) % 2 == 1) sel[ns++] = i;
        }
        if (ns == 0) continue;
        hacc_oracle_force_mesh(n, x, m, L, rcut, eps, c, G, ns, sel, a, NULL);
        for (int64_t q = 0; q < ns; ++q) {
            int64_t i = sel[q];
            double h = dt / level[i];
            v[3 * i] += h * a[3 * q]; v[3 * i + 1] += h * a[3 * q + 1]; v[3 * i + 2] += h * a[3 * q + 2];
        }
    }
    for (int64_t i = 0; i < 3 * n; ++i) x[i] = wrap64(x[i] + (dt - t_prev) * v[i], L);
    free(a); free(sel); free(num); free(den); free(present);
}
