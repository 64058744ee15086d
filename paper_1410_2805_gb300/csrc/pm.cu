// Long-range spectral particle-mesh force (Sec. 2.3): a plain GPU stage
// around cuFFT, not the optimisation target of the library.
//
//   k_deposit   CIC deposit of the masses on the ng^3 grid (64-bit fixed-point
//               integer atomics: order-independent, so reproducible)
//   cuFFT R2C   density -> rho(k)
//   k_kspace    phi(k) = 4 pi G G6(k) S(k) rho(k) / ng^3 (Eq. (greenf),
//               Eq. (filter)) and a_c(k) = -i D_c(k) phi(k), the fourth-order
//               Super-Lanczos derivative of Eq. (sldiff), for c = x, y, z
//   cuFFT C2R   x3, one per component
//   k_interp    CIC interpolation of (a_x, a_y, a_z) at the particles, then
//               either a store or a kick v += kick * a
//
// Accuracy: the bracket of Eq. (greenf) is a sum of O(1) cosines that cancels
// to O((k D)^2) at low k, so its per-axis parts are tabulated in FP64 by
// k_tables (t(k) = cos(ph) - 5/64 cos(2ph) + 1/1024 cos(4ph) - 945/1024, which
// is <= 0 and needs no further cancellation in FP32), as are the Super-Lanczos
// factors and the squared wavenumbers.
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "hacc_internal.cuh"

namespace hacc {
namespace {

constexpr int kBlock = 256;

struct PmState {
    int ng = 0;
    cufftHandle r2c = 0, c2r = 0;
    bool have_plans = false;
    float *rho = nullptr;        // ng^3
    unsigned long long *mass = nullptr;  // ng^3 fixed-point mass per grid point
    cufftComplex *rk = nullptr;  // ng*ng*(ng/2+1)
    cufftComplex *ak = nullptr;  // 3 x ng*ng*(ng/2+1)
    float4 *field = nullptr;     // ng^3 (a_x, a_y, a_z, 0): one 16-byte load per CIC corner
    float *tab = nullptr;        // per-axis tables: t[ng], sl[ng], K2[ng]
    size_t bytes = 0;
};

__device__ __forceinline__ void cic_setup(float x, float inv_d, int ng, int &i0, int &i1, float &f) {
    float u = x * inv_d;
    float fl = floorf(u);
    f = u - fl;
    int i = (int)fl % ng;
    if (i < 0) i += ng;
    i0 = i;
    i1 = i + 1 == ng ? 0 : i + 1;
}

// Masses are accumulated as 64-bit fixed-point integers (units of 2^-32 of
// mass): integer addition is associative, so the grid does not depend on the
// order in which the atomics land and every step is reproducible bit for bit.
constexpr double kFix = 4294967296.0;  // 2^32

__global__ void __launch_bounds__(kBlock) k_deposit(int64_t n, const float4 *__restrict__ pos, float inv_d, int ng,
                                                     unsigned long long *__restrict__ acc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = pos[i];
    int a0, a1, b0, b1, c0, c1;
    float fa, fb, fc;
    cic_setup(p.x, inv_d, ng, a0, a1, fa);
    cic_setup(p.y, inv_d, ng, b0, b1, fb);
    cic_setup(p.z, inv_d, ng, c0, c1, fc);
    const int64_t ng2 = (int64_t)ng * ng;
    const int ia[2] = {a0, a1}, ib[2] = {b0, b1}, ic[2] = {c0, c1};
    const float wa[2] = {1.f - fa, fa}, wb[2] = {1.f - fb, fb}, wc[2] = {1.f - fc, fc};
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y)
#pragma unroll
            for (int z = 0; z < 2; ++z) {
                // FP32 product, scaled by 2^32 exactly; float values >= 2^24 are integers
                long long q = __float2ll_rn(p.w * (wa[x] * wb[y] * wc[z]) * 4294967296.0f);
                atomicAdd(acc + ia[x] * ng2 + (int64_t)ib[y] * ng + ic[z], (unsigned long long)q);
            }
}

__global__ void __launch_bounds__(kBlock) k_fix_to_density(int64_t ng3, const unsigned long long *__restrict__ acc,
                                                            double scale, float *__restrict__ rho) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng3) return;
    rho[g] = (float)((double)(long long)acc[g] * scale);
}

// Per-axis tables in FP64 (rounded to FP32 once): mode number k of index q is
// q for q <= ng/2, q - ng above.
__global__ void k_tables(int ng, double L, float *tab) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ng) return;
    const double pi = 3.14159265358979323846;
    double k = q <= ng / 2 ? (double)q : (double)(q - ng);
    double ph = 2.0 * pi * k / ng;                 // K D with K = 2 pi k / L, D = L / ng
    double t = cos(ph) - (5.0 / 64.0) * cos(2.0 * ph) + (1.0 / 1024.0) * cos(4.0 * ph) - 945.0 / 1024.0;
    double D = L / ng;
    double K = 2.0 * pi * k / L;
    tab[q] = (float)t;
    tab[ng + q] = (float)(((4.0 / 3.0) * sin(K * D) - (1.0 / 6.0) * sin(2.0 * K * D)) / D);
    tab[2 * ng + q] = (float)(K * K);
}

__global__ void __launch_bounds__(kBlock) k_kspace(int ng, float D, float sigma, int ns, float pref,
                                                    const float *__restrict__ tab,
                                                    const cufftComplex *__restrict__ rk,
                                                    cufftComplex *__restrict__ ak) {
    const int nh = ng / 2 + 1;
    const int64_t nmodes = (int64_t)ng * ng * nh;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nmodes) return;
    int qz = (int)(idx % nh);
    int qy = (int)((idx / nh) % ng);
    int qx = (int)(idx / ((int64_t)nh * ng));
    const float *t = tab, *sl = tab + ng, *K2 = tab + 2 * ng;
    float br = t[qx] + t[qy] + t[qz];
    cufftComplex r = rk[idx];
    float phr = 0.f, phi = 0.f;
    if (br < 0.f) {
        float g6 = (45.0f / 128.0f) * D * D / br;
        float k2 = K2[qx] + K2[qy] + K2[qz];
        float kd = sqrtf(k2) * D;
        float sinc = kd > 0.f ? (2.0f / kd) * sinf(0.5f * kd) : 1.0f;
        float s = expf(-k2 * sigma * sigma * D * D * 0.25f);
        for (int i = 0; i < ns; ++i) s *= sinc;
        float f = pref * g6 * s;
        phr = f * r.x;
        phi = f * r.y;
    }
    // a_c = -i D_c phi  ->  (re, im) = (D_c phi_im, -D_c phi_re)
    const float dc[3] = {sl[qx], sl[qy], sl[qz]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cufftComplex o;
        o.x = dc[c] * phi;
        o.y = -dc[c] * phr;
        ak[c * nmodes + idx] = o;
    }
}

// The three force components from real ng^3 arrays into the interleaved grid.
__global__ void __launch_bounds__(kBlock) k_pack_components(int64_t ng3, const float *__restrict__ fx,
                                                             const float *__restrict__ fy,
                                                             const float *__restrict__ fz,
                                                             float4 *__restrict__ field) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng3) return;
    field[g] = make_float4(fx[g], fy[g], fz[g], 0.0f);
}

__global__ void __launch_bounds__(kBlock) k_interp(int64_t n, const float4 *__restrict__ pos, float inv_d, int ng,
                                                    const float4 *__restrict__ field, float4 *acc, float4 *vel,
                                                    float kick) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = pos[i];
    int a0, a1, b0, b1, c0, c1;
    float fa, fb, fc;
    cic_setup(p.x, inv_d, ng, a0, a1, fa);
    cic_setup(p.y, inv_d, ng, b0, b1, fb);
    cic_setup(p.z, inv_d, ng, c0, c1, fc);
    const int64_t ng2 = (int64_t)ng * ng;
    const int ia[2] = {a0, a1}, ib[2] = {b0, b1}, ic[2] = {c0, c1};
    const float wa[2] = {1.f - fa, fa}, wb[2] = {1.f - fb, fb}, wc[2] = {1.f - fc, fc};
    float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y)
#pragma unroll
            for (int z = 0; z < 2; ++z) {
                int64_t g = ia[x] * ng2 + (int64_t)ib[y] * ng + ic[z];
                float w = wa[x] * wb[y] * wc[z];
                const float4 fg = field[g];
                s[0] = __fmaf_rn(w, fg.x, s[0]);
                s[1] = __fmaf_rn(w, fg.y, s[1]);
                s[2] = __fmaf_rn(w, fg.z, s[2]);
            }
    if (acc) acc[i] = make_float4(s[0], s[1], s[2], 0.f);
    if (vel) {
        float4 v = vel[i];
        v.x = __fmaf_rn(kick, s[0], v.x);
        v.y = __fmaf_rn(kick, s[1], v.y);
        v.z = __fmaf_rn(kick, s[2], v.z);
        vel[i] = v;
    }
}

void free_state(PmState *st) {
    if (!st) return;
    if (st->have_plans) {
        cufftDestroy(st->r2c);
        cufftDestroy(st->c2r);
    }
    cudaFree(st->rho);
    cudaFree(st->mass);
    cudaFree(st->rk);
    cudaFree(st->ak);
    cudaFree(st->field);
    cudaFree(st->tab);
    *st = PmState();
}

hacc_status get_state(hacc_ctx *ctx, int ng, double L, cudaStream_t s, PmState **out) {
    PmState *st = static_cast<PmState *>(ctx->pm_state);
    if (!st) {
        st = new PmState();
        ctx->pm_state = st;
    }
    if (st->ng != ng) {
        cudaStreamSynchronize(s);
        free_state(st);
        const size_t ng3 = (size_t)ng * ng * ng, nm = (size_t)ng * ng * (ng / 2 + 1);
        size_t bytes = ng3 * 4 + ng3 * 8 + nm * 8 * 4 + ng3 * 16 + 3 * ng * 4;
        if (ctx->budget && ctx->scratch.cap + bytes > ctx->budget)
            return set_error(ctx, HACC_ENOMEM, "PM grid exceeds the context budget");
        if (cudaMalloc(&st->rho, ng3 * 4) != cudaSuccess || cudaMalloc(&st->mass, ng3 * 8) != cudaSuccess ||
            cudaMalloc(&st->rk, nm * 8) != cudaSuccess ||
            cudaMalloc(&st->ak, 3 * nm * 8) != cudaSuccess || cudaMalloc(&st->field, ng3 * 16) != cudaSuccess ||
            cudaMalloc(&st->tab, 3 * ng * 4) != cudaSuccess) {
            cudaGetLastError();
            free_state(st);
            return set_error(ctx, HACC_ENOMEM, "cudaMalloc of the PM grid failed");
        }
        if (cufftPlan3d(&st->r2c, ng, ng, ng, CUFFT_R2C) != CUFFT_SUCCESS) {
            free_state(st);
            return set_error(ctx, HACC_ECUDA, "cufftPlan3d R2C failed");
        }
        if (cufftPlan3d(&st->c2r, ng, ng, ng, CUFFT_C2R) != CUFFT_SUCCESS) {
            cufftDestroy(st->r2c);
            free_state(st);
            return set_error(ctx, HACC_ECUDA, "cufftPlan3d C2R failed");
        }
        st->have_plans = true;
        st->ng = ng;
        st->bytes = bytes;
    }
    *out = st;
    return HACC_OK;
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace

hacc_status pm_accel(hacc_ctx *ctx, const hacc_box *box, const hacc_pm *pm, double G, int64_t n, const float4 *pos,
                     float4 *acc, float4 *vel_kick, float kick, cudaStream_t s, cudaEvent_t before_kick,
                     const PmHostIO *io) {
    if (!box || !pm) return set_error(ctx, HACC_EINVAL, "box or pm is NULL");
    const double L = box->L;
    if (!(L > 0) || !std::isfinite(L)) return set_error(ctx, HACC_EINVAL, "box side L must be finite and > 0");
    int ng = box->ng ? box->ng : (int)std::lround(L);
    if (ng < 4 || ng > 2048 || (ng & 1)) return set_error(ctx, HACC_EINVAL, "PM grid ng must be even, in [4, 2048]");
    if (pm->ns < 0 || pm->ns > 16 || !(pm->sigma >= 0)) return set_error(ctx, HACC_EINVAL, "bad PM filter parameters");
    if (n == 0) return HACC_OK;
    PmState *st = nullptr;
    hacc_status r = get_state(ctx, ng, L, s, &st);
    if (r != HACC_OK) return r;
    const size_t ng3 = (size_t)ng * ng * ng;
    const int64_t nm = (int64_t)ng * ng * (ng / 2 + 1);
    const double D = L / ng;
    const float inv_d = (float)(ng / L);
    cudaError_t e;
    // chunk c of the particles: [lo, hi)
    const int nch = io ? kPmChunks : 1;
    const int64_t per = (n + nch - 1) / nch;
    auto bounds = [&](int c, int64_t *lo, int64_t *hi) {
        *lo = std::min<int64_t>(n, c * per);
        *hi = std::min<int64_t>(n, (c + 1) * per);
    };
    if (io && io->pos_down) {
        // the positions are final: download them while the field is solved
        if ((e = cudaEventRecord(io->ev[0], s)) != cudaSuccess) return check_cuda(ctx, e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(io->copy, io->ev[0], 0)) != cudaSuccess)
            return check_cuda(ctx, e, "cudaStreamWaitEvent");
        if ((e = cudaMemcpyAsync(io->pos_down, pos, (size_t)n * 16, cudaMemcpyDeviceToHost, io->copy)) != cudaSuccess)
            return check_cuda(ctx, e, "D2H copy");
    }
    if ((e = cudaMemsetAsync(st->mass, 0, ng3 * 8, s)) != cudaSuccess) return check_cuda(ctx, e, "PM memset");
    for (int c = 0; c < nch; ++c) {
        int64_t lo, hi;
        bounds(c, &lo, &hi);
        if (hi <= lo) continue;
        if (io && io->pos_up) {
            if ((e = cudaMemcpyAsync(const_cast<float4 *>(pos) + lo, io->pos_up + lo, (size_t)(hi - lo) * 16,
                                     cudaMemcpyHostToDevice, io->copy)) != cudaSuccess)
                return check_cuda(ctx, e, "H2D copy");
            if ((e = cudaEventRecord(io->ev[c], io->copy)) != cudaSuccess) return check_cuda(ctx, e, "cudaEventRecord");
            if ((e = cudaStreamWaitEvent(s, io->ev[c], 0)) != cudaSuccess) return check_cuda(ctx, e, "cudaStreamWaitEvent");
        }
        k_deposit<<<blocks_for(hi - lo), kBlock, 0, s>>>(hi - lo, pos + lo, inv_d, ng, st->mass);
        note_launch();
    }
    if (io && io->vel_up) {
        // the velocities follow in the same chunks; each chunk's kick waits for
        // its own (the events are reused: the deposits' waits were enqueued
        // against the position records already)
        for (int c = 0; c < nch; ++c) {
            int64_t lo, hi;
            bounds(c, &lo, &hi);
            if (hi <= lo) continue;
            if ((e = cudaMemcpyAsync(vel_kick + lo, io->vel_up + lo, (size_t)(hi - lo) * 16, cudaMemcpyHostToDevice,
                                     io->copy)) != cudaSuccess)
                return check_cuda(ctx, e, "H2D copy");
            if ((e = cudaEventRecord(io->ev[c], io->copy)) != cudaSuccess) return check_cuda(ctx, e, "cudaEventRecord");
        }
    }
    k_fix_to_density<<<blocks_for((int64_t)ng3), kBlock, 0, s>>>((int64_t)ng3, st->mass, 1.0 / (kFix * D * D * D),
                                                                   st->rho);
    note_launch();
    k_tables<<<(ng + 127) / 128, 128, 0, s>>>(ng, L, st->tab);
    note_launch();
    if (cufftSetStream(st->r2c, s) != CUFFT_SUCCESS || cufftSetStream(st->c2r, s) != CUFFT_SUCCESS)
        return set_error(ctx, HACC_ECUDA, "cufftSetStream failed");
    if (cufftExecR2C(st->r2c, st->rho, st->rk) != CUFFT_SUCCESS) return set_error(ctx, HACC_ECUDA, "cufftExecR2C failed");
    const float pref = (float)(4.0 * 3.14159265358979323846 * G / (double)ng3);
    k_kspace<<<blocks_for(nm), kBlock, 0, s>>>(ng, (float)D, pm->sigma, pm->ns, pref, st->tab, st->rk, st->ak);
    note_launch();
    // the components back to real space into arrays free at this point (the
    // density, and the fixed-point mass grid as two real arrays), then
    // interleaved into the field grid in one pass
    float *comp[3] = {st->rho, reinterpret_cast<float *>(st->mass), reinterpret_cast<float *>(st->mass) + ng3};
    for (int c = 0; c < 3; ++c)
        if (cufftExecC2R(st->c2r, st->ak + c * nm, comp[c]) != CUFFT_SUCCESS)
            return set_error(ctx, HACC_ECUDA, "cufftExecC2R failed");
    k_pack_components<<<blocks_for((int64_t)ng3), kBlock, 0, s>>>((int64_t)ng3, comp[0], comp[1], comp[2], st->field);
    note_launch();
    if (before_kick && (e = cudaStreamWaitEvent(s, before_kick, 0)) != cudaSuccess)
        return check_cuda(ctx, e, "cudaStreamWaitEvent");
    for (int c = 0; c < nch; ++c) {
        int64_t lo, hi;
        bounds(c, &lo, &hi);
        if (hi <= lo) continue;
        if (io && io->vel_up && (e = cudaStreamWaitEvent(s, io->ev[c], 0)) != cudaSuccess)
            return check_cuda(ctx, e, "cudaStreamWaitEvent");
        k_interp<<<blocks_for(hi - lo), kBlock, 0, s>>>(hi - lo, pos + lo, inv_d, ng, st->field, acc ? acc + lo : nullptr,
                                                        vel_kick ? vel_kick + lo : nullptr, kick);
        note_launch();
        if (io && io->vel_down) {
            if ((e = cudaEventRecord(io->ev[c], s)) != cudaSuccess) return check_cuda(ctx, e, "cudaEventRecord");
            if ((e = cudaStreamWaitEvent(io->copy, io->ev[c], 0)) != cudaSuccess)
                return check_cuda(ctx, e, "cudaStreamWaitEvent");
            if ((e = cudaMemcpyAsync(io->vel_down + lo, vel_kick + lo, (size_t)(hi - lo) * 16, cudaMemcpyDeviceToHost,
                                     io->copy)) != cudaSuccess)
                return check_cuda(ctx, e, "D2H copy");
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return check_cuda(ctx, e, "PM kernels");
    return HACC_OK;
}

void pm_destroy(hacc_ctx *ctx) {
    PmState *st = static_cast<PmState *>(ctx->pm_state);
    if (st) {
        free_state(st);
        delete st;
        ctx->pm_state = nullptr;
    }
}

}  // namespace hacc
