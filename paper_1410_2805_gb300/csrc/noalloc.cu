// hacc_sr_force_noalloc: the short-range force of hacc_sr_force for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs under a memory
// manager that owns every device allocation (a pool or arena another runtime
// has already carved up), or code embedded where allocation is forbidden
// once set-up has finished.  This entry point needs no context and allocates
// nothing: all of its scratch (binning keys, counts, cell starts, the sorted
// copy of the positions, work items, counters) lives in one fixed array of
// device memory compiled into the library.  The caller still owns and passes
// the input positions and the output accelerations.
//
// Costs and rules of the fixed array:
//   * every GPU that loads the library holds kNoAllocScratchBytes of device
//     memory for the array until the process exits;
//   * all calls share the one array, and each call leaves its contents
//     behind; so two calls whose work overlaps on the GPU (different streams,
//     or several host threads) race on it and give wrong results: serialise
//     them;
//   * the first call on a device looks up the array's device address (set-up,
//     once per device); make that first call before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "hacc_internal.cuh"

namespace hacc {
namespace {

constexpr size_t kNoAllocScratchBytes = HACC_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The fixed scratch.  In host code this name is only a stand-in for the
// symbol, not a device address: host code must use the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceSetup {
    bool done = false;
    char *base = nullptr;
    int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: the device address of the array.
cudaError_t setup_device(int dev, DeviceSetup **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        s.base = static_cast<char *>(ptr);
        s.done = true;
    }
    *out = &s;
    return cudaSuccess;
}

// Layout of the fixed scratch for one call (same carving as the context path).
size_t carve_noalloc(char *base, int64_t n, int64_t ncell, float4 **P, float4 **Ps, int **counter, int **flags,
                     BinBuffers *b) {
    Carver c(base);
    *P = c.take<float4>(n);
    *Ps = c.take<float4>(n);
    *counter = c.take<int>(1);
    *flags = c.take<int>(4);
    carve_bin(c, n, ncell, b, false);
    return c.off;
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" hacc_status hacc_sr_force_noalloc(const hacc_box *box, const hacc_split *split, int64_t n,
                                             const float *pos_m, float *acc, hacc_stream_t stream) {
    tl_launches = nullptr;  // no context: launches are not counted anywhere
    if (!split || !box) return HACC_EINVAL;
    if (n < 0 || n >= ((int64_t)1 << 31)) return HACC_EINVAL;
    if (n > 0 && (!pos_m || !acc)) return HACC_EINVAL;
    if (n > 0 && (((uintptr_t)pos_m | (uintptr_t)acc) & 15u)) return HACC_EINVAL;
    Geometry g;
    hacc_status st = make_geometry(nullptr, box, split->r_cut, &g);
    if (st != HACC_OK) return st;
    ForceConsts fc;
    st = make_force_consts(nullptr, split, g, &fc);
    if (st != HACC_OK) return st;
    float4 *P, *Ps;
    int *counter, *flags;
    BinBuffers b;
    // sizes beyond the fixed array are refused before anything is enqueued
    if (carve_noalloc(nullptr, n, g.ncell, &P, &Ps, &counter, &flags, &b) > kNoAllocScratchBytes)
        return HACC_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HACC_ECUDA;
    // the array's address belongs to the current device: a stream of another
    // device would run the kernels there with this device's address
    int stream_dev = -1;
    if (cudaStreamGetDevice(reinterpret_cast<cudaStream_t>(stream), &stream_dev) != cudaSuccess) {
        cudaGetLastError();
        return HACC_EINVAL;
    }
    if (stream_dev != dev) return HACC_EINVAL;
    DeviceSetup *ds = nullptr;
    if (setup_device(dev, &ds) != cudaSuccess) return HACC_ECUDA;
    carve_noalloc(ds->base, n, g.ncell, &P, &Ps, &counter, &flags, &b);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the flags word keeps the previous call's value: start it at zero
    if (cudaMemsetAsync(flags, 0, 4 * sizeof(int), s) != cudaSuccess) return HACC_ECUDA;
    const float4 *src = reinterpret_cast<const float4 *>(pos_m);
    if (bin_build(g, n, src, nullptr, 0.0f, P, b, flags, true, s) != cudaSuccess) return HACC_ECUDA;
    if (n == 0) return HACC_OK;
    if (gather_sorted(n, b.perm, P, Ps, nullptr, nullptr, nullptr, nullptr, s) != cudaSuccess) return HACC_ECUDA;
    ForceLaunch fl;
    fl.pos = Ps;
    fl.items = b.items;
    fl.n_items = b.n_items;
    fl.cell_start = b.cell_start;
    fl.work_counter = counter;
    fl.mode = kModeForce;
    fl.out = reinterpret_cast<float4 *>(acc);
    fl.perm = b.perm;
    fl.vel = nullptr;
    fl.pos_next = nullptr;
    fl.h_kick = 0.f;
    fl.h_drift = 0.f;
    fl.phi_out = nullptr;
    fl.within = nullptr;
    fl.mass_flag = b.mass_flag;
    if (sr_force_launch(g, fc, fl, ds->num_sms, s) != cudaSuccess) return HACC_ECUDA;
    return HACC_OK;
}
