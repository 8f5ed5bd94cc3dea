// kn_noalloc.cu -- kn_integrate_noalloc: the batched integrator for callers
// that cannot allocate GPU memory at integration time.
//
// Who needs it: host simulation codes that own all device memory through
// their own pool or arena (allocated once at start-up and accounted for
// there), and codes whose per-step path must not call cudaMalloc/cudaFree,
// because those calls can synchronise the whole device and stall the hydro
// work the code overlaps with the network integration.  kn_integrate_batch
// keeps per-network zone state and work-queue buffers that it (re)allocates;
// this entry point instead reads and writes only the caller's device buffers
// and keeps its one piece of scratch -- the work-queue counter and the queue
// order -- in a fixed, file-scope device array.
//
// The scratch array is shared by every call in the process on a device and
// holds the previous call's contents; each call clears the counters it needs.
// Two calls whose work overlaps on the GPU (different streams, or threads)
// race on it: serialise them on one stream.
#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/kn.h"
#include "kn_internal.h"

#include <cstdio>

namespace kn {
kn_status noalloc_prepare(kn_network* n, const kn_opts* o, int32_t n_zones, const kn_zone_conditions* zc,
                          double* Y_out, double* t_out, double* dt_next, int64_t* steps, int64_t* rejects,
                          int32_t* status, const int* order, int* queue_head, LaunchParams& lp, int& grid,
                          int& block, double& nbar, double& rbar);
kn_status noalloc_fail(kn_status s, const char* msg);
}  // namespace kn

using namespace kn;

namespace {

constexpr int kBuckets = 64;

// Scratch layout (ints): [0, KN_NOALLOC_MAX_ZONES) queue order;
// then kBuckets bucket counts, kBuckets bucket offsets, the queue head, and
// the ordering key's min and max (order-preserving integer encoding).
constexpr int kOffCount = KN_NOALLOC_MAX_ZONES;
constexpr int kOffOffset = kOffCount + kBuckets;
constexpr int kOffHead = kOffOffset + kBuckets;
constexpr int kOffMinMax = kOffHead + 1;
constexpr int kScratchInts = kOffMinMax + 2;

static __device__ __align__(256) int g_scratch[kScratchInts];

// Address of g_scratch on each device, looked up on the first call with that
// device current and again whenever the device's current context differs from
// the one the address was taken in (after cudaDeviceReset the old address is
// stale).  Guarded so that threads racing on a device's first call agree.
struct ScratchAddr {
    CUcontext ctx = nullptr;
    int* addr = nullptr;
};
static ScratchAddr g_scratch_addr[64];
static std::mutex g_scratch_mu;

// The calling thread's current context, through the driver entry point the
// runtime hands out (the library does not link the driver library itself).
static CUcontext current_context() {
    typedef CUresult (*GetCurrent)(CUcontext*);
    static GetCurrent fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (GetCurrent)p;
        looked = true;
    }
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

__device__ __forceinline__ unsigned int key_bits(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // monotone in f
}

__device__ __forceinline__ float zone_key(const double* T0, const double* rho0, int z, double nbar, double rbar) {
    const double t = T0[z], r = rho0[z];
    const double k = (t > 0.0 && r > 0.0) ? nbar * log(t) + rbar * log(r) : 0.0;
    return isfinite(k) ? (float)k : 0.f;
}

// clears the counters this call needs (the queue order is fully rewritten)
__global__ void noalloc_clear() {
    const int i = threadIdx.x;
    if (i < 2 * kBuckets) g_scratch[kOffCount + i] = 0;
    if (i == 0) {
        g_scratch[kOffHead] = 0;
        g_scratch[kOffMinMax] = (int)0xffffffffu;  // min (as unsigned) starts high
        g_scratch[kOffMinMax + 1] = 0;             // max starts low
    }
}

__global__ void noalloc_minmax(const double* T0, const double* rho0, int n, double nbar, double rbar) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < n) {
        const unsigned int b = key_bits(zone_key(T0, rho0, z, nbar, rbar));
        atomicMin((unsigned int*)&g_scratch[kOffMinMax], b);
        atomicMax((unsigned int*)&g_scratch[kOffMinMax + 1], b);
    }
}

__device__ __forceinline__ float bits_key(unsigned int b) {
    const unsigned int u = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
    return __uint_as_float(u);
}

// bucket of zone z, bucket 0 = largest key (longest predicted zones first)
__device__ __forceinline__ int zone_bucket(const double* T0, const double* rho0, int z, double nbar, double rbar) {
    const float lo = bits_key((unsigned int)g_scratch[kOffMinMax]);
    const float hi = bits_key((unsigned int)g_scratch[kOffMinMax + 1]);
    const float k = zone_key(T0, rho0, z, nbar, rbar);
    int b = hi > lo ? (int)((hi - k) / (hi - lo) * (kBuckets - 1) + 0.5f) : 0;
    return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

__global__ void noalloc_count(const double* T0, const double* rho0, int n, double nbar, double rbar) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < n) atomicAdd(&g_scratch[kOffCount + zone_bucket(T0, rho0, z, nbar, rbar)], 1);
}

__global__ void noalloc_scan() {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < kBuckets; ++b) {
            g_scratch[kOffOffset + b] = acc;
            acc += g_scratch[kOffCount + b];
        }
    }
}

__global__ void noalloc_scatter(const double* T0, const double* rho0, int n, double nbar, double rbar) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < n) {
        const int pos = atomicAdd(&g_scratch[kOffOffset + zone_bucket(T0, rho0, z, nbar, rbar)], 1);
        g_scratch[pos] = z;
    }
}

// Once per device (and context), with that device current: the device address
// of g_scratch.  In host code the name g_scratch is only a host-side stand-in.
static kn_status scratch_address(int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(KN_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: device id out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    CUcontext ctx = current_context();
    ScratchAddr& a = g_scratch_addr[dev];
    if (!a.addr || !ctx || ctx != a.ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);  // makes the device's context current if it was not
        if (e != cudaSuccess || !p) return noalloc_fail(KN_ERR_CUDA, "cudaGetSymbolAddress(g_scratch) failed");
        ctx = current_context();
        a.addr = (int*)p;
        a.ctx = ctx;
    }
    *out = a.addr;
    return KN_OK;
}

// A pointer the integrator may dereference: device (or managed) memory of the
// current device.  Host memory, and memory of another device, are refused on
// the host before any launch.
static bool on_current_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // the failed query's error is not sticky: clear it
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" kn_status kn_integrate_noalloc(kn_network* net, int32_t n_zones, const kn_zone_conditions* zc,
                                          const kn_opts* opts, double* Y, double* t, double* dt_next,
                                          int64_t* steps, int64_t* rejects, int32_t* status, void* stream_) {
    if (!net || !zc || !opts) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: NULL argument");
    if (n_zones < 1) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: n_zones must be >= 1");
    if (n_zones > KN_NOALLOC_MAX_ZONES)
        return noalloc_fail(KN_ERR_INVALID_ARG,
                            "kn_integrate_noalloc: n_zones exceeds KN_NOALLOC_MAX_ZONES (65536); split the batch");
    if (!zc->Y0 || !zc->T0 || !zc->rho0 || !zc->tau || !zc->t_start || !zc->t_end || !zc->dt_trial || !Y || !t ||
        !dt_next || !steps || !rejects || !status)
        return noalloc_fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: every input and output must be a device pointer");
    cudaStream_t st = (cudaStream_t)stream_;
    int* scratch = nullptr;
    kn_status s = scratch_address(&scratch);
    if (s != KN_OK) return s;
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return noalloc_fail(KN_ERR_CUDA, cudaGetErrorString(e));
        const void* ptrs[13] = {zc->Y0, zc->T0, zc->rho0, zc->tau, zc->t_start, zc->t_end, zc->dt_trial,
                                Y, t, dt_next, steps, rejects, status};
        static const char* names[13] = {"Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial",
                                        "Y", "t", "dt_next", "steps", "rejects", "status"};
        for (int k = 0; k < 13; ++k)
            if (!on_current_device(ptrs[k], dev)) {
                char msg[160];
                snprintf(msg, sizeof msg,
                         "kn_integrate_noalloc: %s is not device memory of the current device", names[k]);
                return noalloc_fail(KN_ERR_INVALID_ARG, msg);
            }
    }
    LaunchParams lp;
    int grid = 0, block = 0, n_species = 0;
    double nbar = 0, rbar = 0;
    s = noalloc_prepare(net, opts, n_zones, zc, Y, t, dt_next, steps, rejects, status, scratch,
                        scratch + kOffHead, lp, grid, block, nbar, rbar);
    if (s != KN_OK) return s;
    n_species = lp.plans[0].N;
    // Y may be Y0 itself (integrated in place); any other overlap is refused
    const size_t ybytes = sizeof(double) * (size_t)n_zones * n_species;
    const char* yb = (const char*)Y;
    const char* y0b = (const char*)zc->Y0;
    cudaError_t e = cudaSuccess;
    if (yb != y0b) {
        if (yb < y0b + ybytes && y0b < yb + ybytes)
            return noalloc_fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: Y overlaps Y0 without being Y0");
        e = cudaMemcpyAsync(Y, zc->Y0, ybytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return noalloc_fail(KN_ERR_CUDA, cudaGetErrorString(e));
    }
    const int nb = (n_zones + 255) / 256;
    noalloc_clear<<<1, 2 * kBuckets, 0, st>>>();
    noalloc_minmax<<<nb, 256, 0, st>>>(zc->T0, zc->rho0, n_zones, nbar, rbar);
    noalloc_count<<<nb, 256, 0, st>>>(zc->T0, zc->rho0, n_zones, nbar, rbar);
    noalloc_scan<<<1, 32, 0, st>>>();
    noalloc_scatter<<<nb, 256, 0, st>>>(zc->T0, zc->rho0, n_zones, nbar, rbar);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(KN_ERR_CUDA, cudaGetErrorString(e));
    e = launch_integrator(lp, opts->precision, grid, block, st);
    if (e != cudaSuccess) return noalloc_fail(KN_ERR_CUDA, cudaGetErrorString(e));
    return KN_OK;
}
