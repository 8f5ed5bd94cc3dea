// kn_host.h -- host-side pieces shared by the runtime's translation units:
// error reporting, the device-buffer helper, a network's host and device
// state, and the table builder's entry points.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/kn.h"
#include "kn_internal.h"

namespace kn {
// Record a formatted message for kn_last_error and return s.
kn_status fail(kn_status s, const char* fmt, ...);
const char* last_error();

inline int pad16(int x) { return (x + 15) & ~15; }

// a device buffer that grows on demand
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t b) {
        if (b <= bytes && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, b ? b : 16);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    template <class T> T* as() const { return (T*)p; }
};

struct Tables {
    std::unique_ptr<DevBuf> blob;
    TableLayout tl{};
    int L = 0, n_slices = 0, warp_len = 0;  // piece cap, slices, longest warp's terms per lane
};
}  // namespace kn

#define KN_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return kn::fail(e_ == cudaErrorMemoryAllocation ? KN_ERR_NOMEM : KN_ERR_CUDA,  \
                            "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

struct kn_network {
    int N = 0, R = 0, S_r = 0, S_p = 0;
    std::vector<double> A, lnk0, tn;
    std::vector<int> reac, prod, nr, slot0;  // in the caller's reaction order
    std::vector<int> perm;                   // sorted position -> caller's reaction index
    int R1 = 0, R12 = 0;                     // 1-body reactions [0,R1), 2-body [R1,R12)
    double cmax = 0;
    kn::DevBuf rate0;                            // double2[R] (ln k0, n), sorted order
    double nbar = 0, rbar = 0;
    std::map<std::pair<int, int>, kn::Tables> tables;  // (precision, Q) -> device blob
    // zone state
    int Z = 0, capZ = 0;
    kn::DevBuf Y, T0, rho0, tau, ts, te, dtt, tout, dtn, steps, rej, props, status, energy;
    kn::DevBuf bind;            // [N] binding energies, when set
    bool has_bind = false;
    kn::DevBuf key_in, key_out, idx_in, order, cub_tmp, qhead;
    bool has_const = true;  // conservative until zones are known
    bool zones_set = false;
    int trial_Z = 0;        // > 0 during autotune trials: integrate only the first trial_Z zones of the queue
    int tuned_P[3][3] = {};  // [precision][plain, learned, QSS]: autotuned CTA size
    int tuned_G[3][3] = {};  // ... and zone group size
};

namespace kn {
// kn_tables.cu: validation and the sorted reaction order (no device work), and
// one network's tables for (precision, threads per zone group), built and
// checked on the host; `blob` is what goes to the device.
kn_status network_host_setup(const kn_network_desc* d, std::unique_ptr<kn_network>& n, std::vector<double>& r0);
kn_status build_tables_host(const kn_network* n, int prec, int Q, std::vector<unsigned char>& blob, Tables& T);
}  // namespace kn
