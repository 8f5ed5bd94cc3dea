// kn_api.cu -- host runtime behind include/kn.h: networks and their device
// state, zone upload, launch geometry and the autotuner, work-queue ordering,
// CUDA-graph capture/replay, result read-back, operator split and energy.
// The tables themselves are built in kn_tables.cu.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "kn_host.h"

using namespace kn;

namespace kn {
void mlp_device_view(const void* h, const float** P, const void** Wb, const float** norm);  // kn_mlp.cu
}

namespace kn {
static thread_local std::string g_err;

kn_status fail(kn_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

const char* last_error() { return g_err.c_str(); }
}  // namespace kn

namespace {

static kn_status build_tables(kn_network* n, int prec, int Q, Tables& T) {
    std::vector<unsigned char> blob;
    kn_status s = build_tables_host(n, prec, Q, blob, T);
    if (s != KN_OK) return s;
    T.blob.reset(new DevBuf());
    KN_CUDA(T.blob->ensure(blob.size()));
    KN_CUDA(cudaMemcpy(T.blob->p, blob.data(), blob.size(), cudaMemcpyHostToDevice));
    return KN_OK;
}

static kn_status get_tables(kn_network* n, int prec, int Q, Tables** out) {
    auto key = std::make_pair(prec, Q);
    auto it = n->tables.find(key);
    if (it == n->tables.end()) {
        Tables T;
        kn_status s = build_tables(n, prec, Q, T);
        if (s != KN_OK) return s;
        it = n->tables.emplace(key, std::move(T)).first;
    }
    *out = &it->second;
    return KN_OK;
}

// The FP32-flux forms keep a per-group cache of the current rates (4 R bytes)
// only for networks of up to 2048 reactions: beyond that the cache would cost
// a zone group per SM, which is worth more than the saved rate evaluations.
static bool rate_cache_on(const kn_network* n, int prec) { return prec != kPrecFP64 && 4 * n->R <= 8192; }

// Optional parts of a group's region: kLayoutFeat the learned proposal's and
// the records' scratch, kLayoutQss the (F+, k) pairs of the QSS predicted state.
enum { kLayoutFeat = 1, kLayoutQss = 2 };

static GroupLayout group_layout(const kn_network* n, int prec, int G, int extras) {
    const int real = prec == kPrecFP64 ? 8 : 4;
    GroupLayout g{};
    int off = 0;
    g.off_V = off;
    off = pad16(off + real * (n->R + n->S_r + 1));
    g.off_K = off;
    off = pad16(off + real * n->R);
    g.off_Kc = off;
    if (rate_cache_on(n, prec)) off = pad16(off + 4 * n->R);
    g.off_Y = off;
    off = pad16(off + (prec == kPrecMixed ? 4 : 8) * 2 * (n->N + 1));
    g.off_Y32 = off;
    if (prec != kPrecFP64) off = pad16(off + 4 * 2 * (n->N + 1));
    g.off_Fk = off;
    off = pad16(off + real * 2 * n->N);
    g.off_carry = off;  // directly after Fk: the tables' spare slot fk_span
    off = pad16(off + real);
    g.off_Fk2 = off;    // the same span and spare slot again
    if (extras & kLayoutQss) off = pad16(pad16(off + real * 2 * n->N) + real);
    g.off_red = off;
    off = pad16(off + (G / 32) * (8 * 3 + 4 + 4));
    g.off_feat = off;
    if (extras & kLayoutFeat) off = pad16(off + 4 * 384 + 4 * (3 * 64 + 4));
    g.off_state = off;
    off = pad16(off + (int)sizeof(GroupState));
    g.bytes = off;
    return g;
}

// ---------------------------------------------------------------------------
// launch configuration
// ---------------------------------------------------------------------------
struct DeviceInfo {
    int dev = -1, sms = 0, smem_optin = 0;
};
static DeviceInfo g_dev;
static int g_smem_limit_set = 0;

static kn_status device_info(DeviceInfo& d) {
    int dev;
    KN_CUDA(cudaGetDevice(&dev));
    if (g_dev.dev != dev) {
        g_dev.dev = dev;
        KN_CUDA(cudaDeviceGetAttribute(&g_dev.sms, cudaDevAttrMultiProcessorCount, dev));
        KN_CUDA(cudaDeviceGetAttribute(&g_dev.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        g_smem_limit_set = 0;
    }
    if (!g_smem_limit_set) {
        KN_CUDA(integrator_set_smem_limit(g_dev.smem_optin - 1024));
        g_smem_limit_set = 1;
    }
    d = g_dev;
    return KN_OK;
}

struct Tiling {
    int G = 0, M = 0, smem_tables = 1, bytes = 0;
};

// Smallest zone group for a network: one warp for small networks; otherwise
// enough threads (a multiple of 32, at least a warp group) that the FP64
// update touches every species in a single pass.
static int base_group(const kn_network* n) {
    if (n->R + n->S_r + n->S_p <= 512) return 32;
    return std::max(128, (n->N + 31) / 32 * 32);
}

// For CTA size P, the tiling of one network: the smallest group size
// G >= base_group that divides P with at most kMaxGroups groups, preferring
// tables staged in shared memory; bytes = dynamic shared memory per CTA.
static kn_status plan_tiling(kn_network* n, int prec, int P, int budget, int G_fixed, int extras, Tiling& out,
                             bool& ok) {
    ok = false;
    Tiling best;
    bool have = false;
    for (int G = G_fixed ? G_fixed : base_group(n); G <= P; G += 32) {
        if (P % G) continue;
        const int M = P / G;
        if (M > kMaxGroups) continue;
        Tables* tb;
        kn_status s = get_tables(n, prec, G, &tb);
        if (s != KN_OK) return s;
        const GroupLayout gl = group_layout(n, prec, G, extras);
        if (tb->tl.bytes + M * gl.bytes <= budget) {
            out = Tiling{G, M, 1, tb->tl.bytes + M * gl.bytes};
            ok = true;
            return KN_OK;
        }
        if (!have && M * gl.bytes <= budget) {
            best = Tiling{G, M, 0, M * gl.bytes};
            have = true;
        }
        if (G_fixed) break;
    }
    if (have) {
        out = best;
        ok = true;
    }
    return KN_OK;
}

struct GraphEntry {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
};
static std::map<std::string, GraphEntry> g_graphs;

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void kn_default_opts(kn_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = KN_PREC_MIXED;
    o->max_reject = 60;
    o->kappa = 1.0;
    o->eps_r = 0.05;
    o->eps_c = 1e-6;
    o->y_min = 1e-10;
    o->grow_max = 1.5;
    o->safety = 0.9;
    o->shrink = 0.5;
    o->dt_min_frac = 1e-30;
    o->max_steps = 10000000;
    o->use_graph = 0;
    o->lockstep = 0;
    o->mlp_margin = 0.5;
}

const char* kn_last_error(void) { return kn::last_error(); }

kn_status kn_create_network(const kn_network_desc* d, kn_network** out) {
    if (!d || !out) return fail(KN_ERR_INVALID_ARG, "kn_create_network: NULL argument");
    *out = nullptr;
    std::unique_ptr<kn_network> n;
    std::vector<double> r0;
    kn_status s = network_host_setup(d, n, r0);
    if (s != KN_OK) return s;
    KN_CUDA(n->rate0.ensure(8 * r0.size()));
    KN_CUDA(cudaMemcpy(n->rate0.p, r0.data(), 8 * r0.size(), cudaMemcpyHostToDevice));
    KN_CUDA(n->qhead.ensure(64));
    *out = n.release();
    return KN_OK;
}

kn_status kn_check_gather_tables(const kn_network_desc* d, int32_t precision, int32_t threads_per_zone,
                                 int32_t stats[4]) {
    if (!d || !stats) return fail(KN_ERR_INVALID_ARG, "kn_check_gather_tables: NULL argument");
    if (precision != KN_PREC_FP64 && precision != KN_PREC_MIXED && precision != KN_PREC_MIXED_FP64)
        return fail(KN_ERR_INVALID_ARG, "kn_check_gather_tables: bad precision");
    if (threads_per_zone < 32 || threads_per_zone > 1024 || threads_per_zone % 32)
        return fail(KN_ERR_INVALID_ARG, "kn_check_gather_tables: threads_per_zone must be a multiple of 32 in [32, 1024]");
    std::unique_ptr<kn_network> n;
    std::vector<double> r0;
    kn_status s = network_host_setup(d, n, r0);
    if (s != KN_OK) return s;
    std::vector<unsigned char> blob;
    Tables T;
    s = build_tables_host(n.get(), precision, threads_per_zone, blob, T);
    if (s != KN_OK) return s;
    stats[0] = T.L;
    stats[1] = T.n_slices;
    stats[2] = T.warp_len;
    stats[3] = (int)blob.size();
    return KN_OK;
}

kn_status kn_destroy_network(kn_network* net) {
    if (!net) return KN_OK;
    cudaDeviceSynchronize();
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        // graphs may reference this network's buffers: drop them all (cheap to recapture)
        if (it->second.x) cudaGraphExecDestroy(it->second.x);
        if (it->second.g) cudaGraphDestroy(it->second.g);
        it = g_graphs.erase(it);
    }
    delete net;
    return KN_OK;
}

kn_status kn_network_info(const kn_network* net, int32_t* ns, int32_t* nr, int32_t* srs, int32_t* sps) {
    if (!net) return fail(KN_ERR_INVALID_ARG, "kn_network_info: NULL network");
    if (ns) *ns = net->N;
    if (nr) *nr = net->R;
    if (srs) *srs = net->S_r;
    if (sps) *sps = net->S_p;
    return KN_OK;
}

kn_status kn_set_zone_conditions(kn_network* n, int32_t Z, const kn_zone_conditions* zc, int32_t mem,
                                 void* stream_) {
    if (!n || !zc) return fail(KN_ERR_INVALID_ARG, "kn_set_zone_conditions: NULL argument");
    if (Z < 1) return fail(KN_ERR_INVALID_ARG, "n_zones must be >= 1");
    if (mem != KN_MEM_HOST && mem != KN_MEM_DEVICE) return fail(KN_ERR_INVALID_ARG, "bad kn_mem");
    if (!zc->Y0 || !zc->T0 || !zc->rho0 || !zc->tau || !zc->t_start || !zc->t_end || !zc->dt_trial)
        return fail(KN_ERR_INVALID_ARG, "kn_zone_conditions has a NULL array");
    cudaStream_t st = (cudaStream_t)stream_;
    const int N = n->N;
    bool has_const = true;
    if (mem == KN_MEM_HOST) {
        has_const = false;
        for (int z = 0; z < Z; ++z) {
            for (int i = 0; i < N; ++i) {
                const double y = zc->Y0[(size_t)z * N + i];
                if (!(std::isfinite(y) && y >= 0))
                    return fail(KN_ERR_INVALID_ARG, "zone %d: Y0[%d] must be finite and >= 0", z, i);
            }
            const double T0 = zc->T0[z], r0 = zc->rho0[z], tau = zc->tau[z], ts = zc->t_start[z],
                         te = zc->t_end[z], dt = zc->dt_trial[z];
            if (!(std::isfinite(T0) && T0 > 0 && std::isfinite(r0) && r0 > 0))
                return fail(KN_ERR_INVALID_ARG, "zone %d: T0 and rho0 must be finite and > 0", z);
            if (!(std::isfinite(tau) && std::isfinite(ts) && std::isfinite(te) && ts >= 0 && te > ts))
                return fail(KN_ERR_INVALID_ARG, "zone %d: need finite tau and 0 <= t_start < t_end", z);
            if (!(std::isfinite(dt) && (ts > 0 || dt > 0)))
                return fail(KN_ERR_INVALID_ARG, "zone %d: need t_start > 0 or dt_trial > 0", z);
            if (!(tau > 0)) has_const = true;
        }
    }
    if (Z > n->capZ) {
        const size_t zd = 8 * (size_t)Z;
        KN_CUDA(n->Y.ensure(zd * N));
        KN_CUDA(n->T0.ensure(zd));
        KN_CUDA(n->rho0.ensure(zd));
        KN_CUDA(n->tau.ensure(zd));
        KN_CUDA(n->ts.ensure(zd));
        KN_CUDA(n->te.ensure(zd));
        KN_CUDA(n->dtt.ensure(zd));
        KN_CUDA(n->tout.ensure(zd));
        KN_CUDA(n->dtn.ensure(zd));
        KN_CUDA(n->steps.ensure(zd));
        KN_CUDA(n->rej.ensure(zd));
        KN_CUDA(n->props.ensure(zd));
        KN_CUDA(n->energy.ensure(zd));
        KN_CUDA(n->status.ensure(4 * (size_t)Z));
        KN_CUDA(n->key_in.ensure(4 * (size_t)Z));
        KN_CUDA(n->key_out.ensure(4 * (size_t)Z));
        KN_CUDA(n->idx_in.ensure(4 * (size_t)Z));
        KN_CUDA(n->order.ensure(4 * (size_t)Z));
        size_t tmp = 0;
        KN_CUDA(cub::DeviceRadixSort::SortPairsDescending(nullptr, tmp, (const float*)nullptr, (float*)nullptr,
                                                          (const int*)nullptr, (int*)nullptr, Z));
        KN_CUDA(n->cub_tmp.ensure(tmp));
        n->capZ = Z;
    }
    const cudaMemcpyKind kind = mem == KN_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t zd = 8 * (size_t)Z;
    KN_CUDA(cudaMemcpyAsync(n->Y.p, zc->Y0, zd * N, kind, st));
    KN_CUDA(cudaMemcpyAsync(n->T0.p, zc->T0, zd, kind, st));
    KN_CUDA(cudaMemcpyAsync(n->rho0.p, zc->rho0, zd, kind, st));
    KN_CUDA(cudaMemcpyAsync(n->tau.p, zc->tau, zd, kind, st));
    KN_CUDA(cudaMemcpyAsync(n->ts.p, zc->t_start, zd, kind, st));
    KN_CUDA(cudaMemcpyAsync(n->te.p, zc->t_end, zd, kind, st));
    KN_CUDA(cudaMemcpyAsync(n->dtt.p, zc->dt_trial, zd, kind, st));
    KN_CUDA(launch_fill_int(n->status.as<int>(), Z, KN_ZONE_PENDING, st));
    KN_CUDA(cudaMemsetAsync(n->energy.p, 0, 8 * (size_t)Z, st));
    // work-queue order: predicted longest zones first
    KN_CUDA(launch_zone_cost_simple(n->T0.as<double>(), n->rho0.as<double>(), Z, n->nbar, n->rbar,
                                    n->key_in.as<float>(), n->idx_in.as<int>(), st));
    size_t tmp = n->cub_tmp.bytes;
    KN_CUDA(cub::DeviceRadixSort::SortPairsDescending(n->cub_tmp.p, tmp, n->key_in.as<float>(),
                                                      n->key_out.as<float>(), n->idx_in.as<int>(),
                                                      n->order.as<int>(), Z, 0, 32, st));
    n->Z = Z;
    n->has_const = has_const;
    n->zones_set = true;
    return KN_OK;
}

}  // extern "C"

namespace {

// The FP32-flux forms reuse a zone's cached rates K_j 2^(-c_j u_ref) while
// |u - u_ref| <= tol: then every rate differs from K_j 2^(-c_j u) by less
// than c_max ln 2 tol = 2^-26 relative, a quarter of an FP32 ulp.
static float rate_cache_tol(double cmax) {
    return cmax > 0.0 ? (float)(1.4901161193847656e-08 / (cmax * 0.6931471805599453)) : 3.0e38f;
}

// Which autotuned tiling a call uses: the plain form's, the learned form's or
// the QSS form's (they differ in shared memory per group and in work per step).
static int tuned_slot(const kn_opts* o, bool learn) { return learn ? 1 : (o->method == KN_METHOD_QSS ? 2 : 0); }

static kn_status validate_opts(const kn_opts* o) {
    if (!o) return fail(KN_ERR_INVALID_ARG, "NULL opts");
    if (o->precision != KN_PREC_FP64 && o->precision != KN_PREC_MIXED && o->precision != KN_PREC_MIXED_FP64)
        return fail(KN_ERR_INVALID_ARG, "opts.precision must be KN_PREC_FP64, KN_PREC_MIXED or KN_PREC_MIXED_FP64");
    if (!(o->kappa > 0 && o->eps_r > 0 && o->eps_c > 0 && o->y_min >= 0 && o->grow_max >= 1 &&
          o->safety > 0 && o->shrink > 0 && o->shrink < 1 && o->dt_min_frac >= 0 && o->max_steps >= 0 &&
          o->max_reject >= 0))
        return fail(KN_ERR_INVALID_ARG, "opts: a controller parameter is out of range");
    if (o->threads_per_zone && (o->threads_per_zone % 32 || o->threads_per_zone > 1024))
        return fail(KN_ERR_INVALID_ARG, "opts.threads_per_zone must be a multiple of 32, <= 1024");
    if (o->threads_per_cta && (o->threads_per_cta % 32 || o->threads_per_cta > 1024))
        return fail(KN_ERR_INVALID_ARG, "opts.threads_per_cta must be a multiple of 32, <= 1024");
    if (o->lockstep) return fail(KN_ERR_INVALID_ARG, "opts.lockstep is reserved and must be 0");
    if (o->record_features && (!o->record_labels || !o->record_count || o->record_capacity < 0))
        return fail(KN_ERR_INVALID_ARG, "opts.record_features needs record_labels, record_count, capacity >= 0");
    if (o->record_features && o->mlp)
        return fail(KN_ERR_INVALID_ARG, "opts.record_features and opts.mlp are not combined");
    if (o->trace_features || o->trace_out || o->trace_dt || o->trace_count) {
        if (!o->mlp) return fail(KN_ERR_INVALID_ARG, "opts.trace_* needs opts.mlp");
        if (!o->trace_features || !o->trace_out || !o->trace_dt || !o->trace_count || o->trace_capacity < 0)
            return fail(KN_ERR_INVALID_ARG, "opts.trace_* must be set together, with trace_capacity >= 0");
    }
    if (o->follow_label && !o->record_features)
        return fail(KN_ERR_INVALID_ARG, "opts.follow_label needs opts.record_features");
    if (o->method != KN_METHOD_ASYMPTOTIC && o->method != KN_METHOD_QSS)
        return fail(KN_ERR_INVALID_ARG, "opts.method must be KN_METHOD_ASYMPTOTIC or KN_METHOD_QSS");
    if (o->method == KN_METHOD_QSS &&
        (o->precision == KN_PREC_MIXED_FP64 || o->mlp || o->record_features))
        return fail(KN_ERR_INVALID_ARG,
                    "opts.method KN_METHOD_QSS runs in KN_PREC_FP64 or KN_PREC_MIXED, without mlp or records");
    if ((o->replay_dt != nullptr) != (o->replay_off != nullptr) ||
        (o->replay_dt != nullptr) != (o->replay_len != nullptr))
        return fail(KN_ERR_INVALID_ARG, "opts.replay_dt/off/len must be set together");
    return KN_OK;
}

// FP32 guard band of the mixed form's accept test.  y, y', their max m and the
// difference d of the FP32 copies carry relative errors of at most 2^-24 each,
// so |d32 - d| <= 2^-23 m + 2^-24 |d|; near the threshold |d| ~ eps_r m this is
// a relative error of 2^-23 / eps_r + 2^-24, plus the roundings of eps_r and
// eps_r m.  Outside 8x that band the FP32 compare decides as the FP64 one does.
static void set_guard_band(OptsDev& D, const kn_opts* o) {
    const double u = 5.9604644775390625e-08;  // 2^-24
    // the test compares the ratio |d| / m, itself within 2 ulp (__fdividef)
    const double band = 8.0 * (2.0 * u / o->eps_r + 4.0 * u) + 8.0 * u;
    D.eps_r32 = (float)o->eps_r;
    D.kappa32 = (float)o->kappa;
    D.eps_c32 = (float)o->eps_c;
    D.ga32 = (float)(o->safety * o->eps_r);
    D.gb32 = (float)(o->safety * o->eps_c);
    D.grow32 = (float)o->grow_max;
    D.shrink32 = (float)o->shrink;
    D.band_lo32 = (float)(1.0 - band);
    D.band_hi32 = (float)(1.0 + band);
    D.thr_lo32 = (float)(o->eps_r * (1.0 - band));
    D.thr_hi32 = (float)(o->eps_r * (1.0 + band));
    D.ymin_lo32 = (float)(o->y_min * (1.0 - 8.0 * u));
    D.ymin_hi32 = (float)(o->y_min * (1.0 + 8.0 * u));
}

// Fill lp for the listed networks; returns grid/block.
static kn_status prepare_launch(kn_network* const* nets, int n_nets, const kn_opts* o, LaunchParams& lp,
                                int& grid, int& block, bool probe) {
    DeviceInfo di;
    kn_status s = device_info(di);
    if (s != KN_OK) return s;
    const int prec = o->precision;
    const bool learn = o->mlp != nullptr && !probe;
    const bool record = o->record_features != nullptr && !probe;
    const int extras = (learn || record ? kLayoutFeat : 0) | (o->method == KN_METHOD_QSS ? kLayoutQss : 0);
    // the staged network takes the front of the CTA's shared memory
    const int budget = di.smem_optin - 1024 - 64 - (learn ? kMlpSmemBytes : 0);
    memset(&lp, 0, sizeof lp);
    lp.n_plans = n_nets;
    // one CTA size P for the launch; per network the group size G | P
    Tiling tl[kMaxPlans];
    int P_best = 0;
    for (int p = 0; p < n_nets; ++p)
        if (!nets[p]->zones_set) return fail(KN_ERR_STATE, "network %d has no zones (kn_set_zone_conditions)", p);
    {
        int P_lo = 32, P_hi = 1024;
        if (o->threads_per_cta) P_lo = P_hi = o->threads_per_cta;
        else if (o->threads_per_zone) P_lo = P_hi = o->threads_per_zone;
        // an autotuned tiling (kn_autotune) when the caller gives none
        if (!o->threads_per_cta && !o->threads_per_zone) {
            const int tP = nets[0]->tuned_P[prec][tuned_slot(o, learn)];
            bool all = tP > 0;
            Tiling cand[kMaxPlans];
            for (int p = 0; p < n_nets && all; ++p) {
                const int tG = nets[p]->tuned_G[prec][tuned_slot(o, learn)];
                bool ok = false;
                all = nets[p]->tuned_P[prec][tuned_slot(o, learn)] == tP && tG > 0;
                if (all && (s = plan_tiling(nets[p], prec, tP, budget, tG, extras, cand[p], ok)) != KN_OK) return s;
                all = all && ok;
            }
            if (all) {
                P_best = tP;
                for (int p = 0; p < n_nets; ++p) tl[p] = cand[p];
            }
        }
        if (!P_best && n_nets == 1 && !o->threads_per_cta) {
            // one network, no explicit CTA size, tables staged in shared memory.
            // FP64 form, and single-warp groups (small networks): the most
            // groups per CTA, then the smallest group -- the FP64 pipe, or the
            // groups' short serial sections, are best shared by many groups.
            // Mixed form with larger groups: up to kTargetGroups groups, then
            // the largest group (fewer gather slices per warp); measured on the
            // 150-species network, mixed 5 x 192 beats 6 x 160, 5 x 160 and
            // 3 x 320 threads, while FP64 3 x 128 beats 3 x 320.
            kn_network* n = nets[0];
            Tiling best;
            const int g0 = o->threads_per_zone ? o->threads_per_zone : base_group(n);
            const int g1 = o->threads_per_zone ? o->threads_per_zone : 512;
            const bool small = g0 == 32 || prec != kPrecMixed;
            constexpr int kTargetGroups = 5;
            for (int G = g0; G <= g1; G += 32) {
                Tables* tb;
                if ((s = get_tables(n, prec, G, &tb)) != KN_OK) return s;
                const GroupLayout gl = group_layout(n, prec, G, extras);
                int M = std::min(kMaxGroups, 1024 / G);
                if (!small) M = std::min(M, kTargetGroups);
                while (M > 0 && tb->tl.bytes + M * gl.bytes > budget) --M;
                const bool better = small ? M > best.M : (M > best.M || (M == best.M && M > 0));
                if (better) best = Tiling{G, M, 1, tb->tl.bytes + M * gl.bytes};
            }
            if (best.M > 0) {
                P_best = best.G * best.M;
                tl[0] = best;
            }
        }
        // without an explicit tiling: the largest CTA that stages every network's tables
        for (int pass = 0; pass < 2 && !P_best; ++pass) {  // (skipped when a tiling is already chosen)
            for (int P = P_hi; P >= P_lo && !P_best; P -= 32) {
                bool all = true, all_smem = true;
                Tiling cand[kMaxPlans];
                for (int p = 0; p < n_nets && all; ++p) {
                    bool ok;
                    if ((s = plan_tiling(nets[p], prec, P, budget, o->threads_per_zone, extras, cand[p], ok)) != KN_OK)
                        return s;
                    all = ok;
                    all_smem = all_smem && ok && cand[p].smem_tables;
                }
                if (all && (all_smem || pass == 1 || P_lo == P_hi)) {
                    P_best = P;
                    for (int p = 0; p < n_nets; ++p) tl[p] = cand[p];
                }
            }
        }
        if (!P_best) return fail(KN_ERR_INVALID_ARG, "no tiling fits in %d B of shared memory per CTA", budget);
    }
    int max_smem = 0;
    double work[kMaxPlans];
    double total_work = 0;
    int zone_base = 0;
    for (int p = 0; p < n_nets; ++p) {
        kn_network* n = nets[p];
        const Tiling t = tl[p];
        Tables* tb;
        if ((s = get_tables(n, prec, t.G, &tb)) != KN_OK) return s;
        const GroupLayout gl = group_layout(n, prec, t.G, extras);
        PlanDev& P = lp.plans[p];
        P.blob = (const unsigned char*)tb->blob->p;
        P.tl = tb->tl;
        P.rate0 = n->rate0.as<const double2>();
        P.R1 = n->R1;
        P.R12 = n->R12;
        P.cmax = n->cmax;
        P.u_tol = rate_cache_tol(n->cmax);
        P.rate_cache = rate_cache_on(n, prec) ? 1 : 0;
        P.N = n->N;
        P.R = n->R;
        P.S_r = n->S_r;
        P.zero_idx = n->R + n->S_r;
        P.smem_tables = t.smem_tables;
        P.G = t.G;
        P.M = t.M;
        P.gl = gl;
        P.Y = n->Y.as<double>();
        P.T0 = n->T0.as<double>();
        P.rho0 = n->rho0.as<double>();
        P.tau = n->tau.as<double>();
        P.t_start = n->ts.as<double>();
        P.t_end = n->te.as<double>();
        P.dt_trial = n->dtt.as<double>();
        P.t_out = n->tout.as<double>();
        P.dt_next = n->dtn.as<double>();
        P.steps = n->steps.as<long long>();
        P.rejects = n->rej.as<long long>();
        P.props = n->props.as<long long>();
        P.bind = n->has_bind ? n->bind.as<const double>() : nullptr;
        P.energy = n->energy.as<double>();
        P.status = n->status.as<int>();
        P.n_zones = n->trial_Z > 0 ? std::min(n->Z, n->trial_Z) : n->Z;
        P.zone_base = zone_base;
        P.order = n->order.as<int>();
        P.queue_head = n->qhead.as<int>();
        zone_base += n->Z;
        max_smem = std::max(max_smem, t.bytes);
        work[p] = (double)n->Z * (n->R + n->S_r + n->S_p) / (double)t.M;
        total_work += work[p];
    }
    const int max_block = P_best;
    // one block size for the launch: every plan must fill it exactly
    block = max_block;
    for (int p = 0; p < n_nets; ++p)
        if (lp.plans[p].G * lp.plans[p].M != block)
            return fail(KN_ERR_INVALID_ARG, "networks in one launch need equal threads per CTA (got %d and %d)",
                        lp.plans[p].G * lp.plans[p].M, block);
    lp.smem_bytes = max_smem + (learn ? kMlpSmemBytes : 0);
    int bps = 0;
    {
        cudaError_t e = integrator_occupancy(prec, block, lp.smem_bytes, &bps);
        if (e != cudaSuccess) return fail(KN_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
    }
    if (bps < 1)
        return fail(KN_ERR_INVALID_ARG, "tiling does not fit on an SM (block %d, smem %d)", block, lp.smem_bytes);
    grid = di.sms * bps;
    int zones_total = 0;
    for (int p = 0; p < n_nets; ++p) zones_total += lp.plans[p].n_zones;
    if (probe) grid = std::min(grid, std::max(1, zones_total));
    // home CTAs proportional to each plan's work
    int b = 0;
    for (int p = 0; p < n_nets; ++p) {
        int cnt = (p == n_nets - 1) ? grid - b : (int)std::lround(grid * work[p] / total_work);
        cnt = std::max(0, std::min(cnt, grid - b));
        lp.plans[p].cta_begin = b;
        lp.plans[p].cta_end = b + cnt;
        b += cnt;
    }
    OptsDev& D = lp.o;
    D.kappa = o->kappa;
    D.eps_r = o->eps_r;
    D.eps_c = o->eps_c;
    D.y_min = o->y_min;
    D.grow_max = o->grow_max;
    D.safety = o->safety;
    D.shrink = o->shrink;
    D.dt_min_frac = o->dt_min_frac;
    D.max_steps = o->max_steps;
    D.max_reject = o->max_reject;
    D.lockstep = o->lockstep;
    D.method = o->method;
    set_guard_band(D, o);
    D.zone_ns = probe ? nullptr : (long long*)o->zone_ns;
    D.replay_dt = o->replay_dt;
    D.replay_off = (const long long*)o->replay_off;
    D.replay_len = (const long long*)o->replay_len;
    if (learn) {
        D.learn = 1;
        D.mlp_margin = (float)o->mlp_margin;
        const void* W;
        mlp_device_view(o->mlp, &D.mlpP, &W, &D.mlpNorm);
        D.mlpW = W;
        if (o->trace_features) {
            D.trace_feat = o->trace_features;
            D.trace_out = o->trace_out;
            D.trace_dt = o->trace_dt;
            D.trace_cap = o->trace_capacity;
            D.trace_count = (unsigned long long*)o->trace_count;
        }
    }
    if (record) {
        D.record = 1;
        D.rec_feat = o->record_features;
        D.rec_label = o->record_labels;
        D.rec_cap = o->record_capacity;
        D.rec_count = (unsigned long long*)o->record_count;
        D.follow_label = o->follow_label ? 1 : 0;
    }
    return KN_OK;
}

static kn_status enqueue(kn_network* const* nets, int n_nets, const LaunchParams& lp, int prec, int grid,
                         int block, cudaStream_t st) {
    for (int p = 0; p < n_nets; ++p) KN_CUDA(cudaMemsetAsync(nets[p]->qhead.p, 0, sizeof(int), st));
    KN_CUDA(launch_integrator(lp, prec, grid, block, st));
    return KN_OK;
}

}  // namespace

extern "C" {

kn_status kn_integrate_batch(kn_network* const* nets, int32_t n_nets, const kn_opts* o, void* stream_) {
    if (!nets || n_nets < 1 || n_nets > kMaxPlans)
        return fail(KN_ERR_INVALID_ARG, "need 1..%d networks", kMaxPlans);
    for (int p = 0; p < n_nets; ++p) {
        if (!nets[p]) return fail(KN_ERR_INVALID_ARG, "network %d is NULL", p);
        for (int q = 0; q < p; ++q)
            if (nets[q] == nets[p]) return fail(KN_ERR_INVALID_ARG, "networks must be distinct");
    }
    kn_status s = validate_opts(o);
    if (s != KN_OK) return s;
    cudaStream_t st = (cudaStream_t)stream_;
    LaunchParams lp;
    int grid, block;
    if ((s = prepare_launch(nets, n_nets, o, lp, grid, block, false)) != KN_OK) return s;
    if (!o->use_graph) return enqueue(nets, n_nets, lp, o->precision, grid, block, st);
    // CUDA graph keyed by the full launch description
    std::string key((const char*)&lp, sizeof lp);
    key.append((const char*)&grid, sizeof grid);
    key.append((const char*)&block, sizeof block);
    key.append((const char*)&o->precision, sizeof o->precision);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        if (g_graphs.size() >= 32) {
            for (auto& kv : g_graphs) {
                if (kv.second.x) cudaGraphExecDestroy(kv.second.x);
                if (kv.second.g) cudaGraphDestroy(kv.second.g);
            }
            g_graphs.clear();
        }
        cudaStream_t cs;
        KN_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        GraphEntry ge;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            kn_status es = enqueue(nets, n_nets, lp, o->precision, grid, block, cs);
            e = cudaStreamEndCapture(cs, &ge.g);
            if (es != KN_OK) {
                cudaStreamDestroy(cs);
                return es;
            }
        }
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return fail(KN_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        KN_CUDA(cudaGraphInstantiate(&ge.x, ge.g, 0));
        it = g_graphs.emplace(key, ge).first;
    }
    KN_CUDA(cudaGraphLaunch(it->second.x, st));
    return KN_OK;
}

kn_status kn_probe_step(kn_network* net, const kn_opts* o, double* Fp, double* k, double* Y1, double* cons,
                        double* rel, void* stream_) {
    if (!net) return fail(KN_ERR_INVALID_ARG, "kn_probe_step: NULL network");
    kn_status s = validate_opts(o);
    if (s != KN_OK) return s;
    if (!net->zones_set) return fail(KN_ERR_STATE, "kn_probe_step: no zones set");
    cudaStream_t st = (cudaStream_t)stream_;
    const size_t zn = 8 * (size_t)net->Z * net->N, zd = 8 * (size_t)net->Z;
    // outputs the caller did not ask for go to scratch
    DevBuf scratch;
    KN_CUDA(scratch.ensure(3 * zn + 2 * zd));
    double* sp = scratch.as<double>();
    kn_opts oo = *o;
    oo.replay_dt = nullptr;
    oo.replay_off = nullptr;
    oo.replay_len = nullptr;
    LaunchParams lp;
    int grid, block;
    kn_network* nets[1] = {net};
    if ((s = prepare_launch(nets, 1, &oo, lp, grid, block, true)) != KN_OK) return s;
    lp.o.probe = 1;
    lp.o.probe_Fp = Fp ? Fp : sp;
    lp.o.probe_k = k ? k : sp + zn / 8;
    lp.o.probe_Y1 = Y1 ? Y1 : sp + 2 * zn / 8;
    lp.o.probe_cons = cons ? cons : sp + 3 * zn / 8;
    lp.o.probe_rel = rel ? rel : sp + 3 * zn / 8 + zd / 8;
    if ((s = enqueue(nets, 1, lp, o->precision, grid, block, st)) != KN_OK) return s;
    KN_CUDA(cudaStreamSynchronize(st));  // scratch is freed on return
    return KN_OK;
}

kn_status kn_get_abundances(const kn_network* n, double* Y, double* t, double* dt_next, int64_t* steps,
                            int64_t* rejects, int32_t* status, int32_t mem, void* stream_) {
    if (!n) return fail(KN_ERR_INVALID_ARG, "kn_get_abundances: NULL network");
    if (mem != KN_MEM_HOST && mem != KN_MEM_DEVICE) return fail(KN_ERR_INVALID_ARG, "bad kn_mem");
    if (!n->zones_set) return fail(KN_ERR_STATE, "kn_get_abundances: no zones set");
    cudaStream_t st = (cudaStream_t)stream_;
    const cudaMemcpyKind kind = mem == KN_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t zd = 8 * (size_t)n->Z;
    if (Y) KN_CUDA(cudaMemcpyAsync(Y, n->Y.p, zd * n->N, kind, st));
    if (t) KN_CUDA(cudaMemcpyAsync(t, n->tout.p, zd, kind, st));
    if (dt_next) KN_CUDA(cudaMemcpyAsync(dt_next, n->dtn.p, zd, kind, st));
    if (steps) KN_CUDA(cudaMemcpyAsync(steps, n->steps.p, zd, kind, st));
    if (rejects) KN_CUDA(cudaMemcpyAsync(rejects, n->rej.p, zd, kind, st));
    if (status) KN_CUDA(cudaMemcpyAsync(status, n->status.p, 4 * (size_t)n->Z, kind, st));
    KN_CUDA(cudaStreamSynchronize(st));
    return KN_OK;
}

kn_status kn_get_batch_stats(kn_network* const* nets, int32_t n_nets, void* stream_, kn_batch_stats* stats) {
    if (!nets || n_nets < 1 || !stats) return fail(KN_ERR_INVALID_ARG, "kn_get_batch_stats: bad arguments");
    memset(stats, 0, sizeof *stats);
    for (int p = 0; p < n_nets; ++p) {
        const kn_network* n = nets[p];
        if (!n || !n->zones_set) return fail(KN_ERR_STATE, "network %d has no zones", p);
        std::vector<int64_t> st(n->Z), rj(n->Z), pr(n->Z);
        std::vector<int32_t> ss(n->Z);
        kn_status s = kn_get_abundances(n, nullptr, nullptr, nullptr, st.data(), rj.data(), ss.data(),
                                        KN_MEM_HOST, stream_);
        if (s != KN_OK) return s;
        KN_CUDA(cudaMemcpy(pr.data(), n->props.p, 8 * (size_t)n->Z, cudaMemcpyDeviceToHost));
        for (int z = 0; z < n->Z; ++z) {
            stats->zones += 1;
            stats->zones_ok += ss[z] == KN_ZONE_OK;
            stats->steps += st[z];
            stats->rejects += rj[z];
            stats->proposals_used += pr[z];
        }
    }
    return KN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Support for kn_integrate_noalloc (kn_noalloc.cu): fill the launch of one
// network from tables that already exist, pointing the zone state at the
// caller's device buffers and the work queue at caller-given scratch.  It
// builds no tables and allocates nothing; a missing table is an error.
// ---------------------------------------------------------------------------
namespace kn {
kn_status noalloc_prepare(kn_network* n, const kn_opts* o, int32_t n_zones, const kn_zone_conditions* zc,
                          double* Y_out, double* t_out, double* dt_next, int64_t* steps, int64_t* rejects,
                          int32_t* status, const int* order, int* queue_head, LaunchParams& lp, int& grid,
                          int& block, double& nbar, double& rbar) {
    kn_status s = validate_opts(o);
    if (s != KN_OK) return s;
    if (o->use_graph) return fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: use_graph must be 0");
    if (o->replay_dt) return fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: replay is not supported");
    if (o->mlp || o->record_features)
        return fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: learned proposal and records not supported");
    const int G = o->threads_per_zone, P = o->threads_per_cta ? o->threads_per_cta : o->threads_per_zone;
    if (G <= 0) return fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: set opts.threads_per_zone (and threads_per_cta)");
    if (P % G || P / G > kMaxGroups) return fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: bad tiling %d/%d", P, G);
    DeviceInfo di;
    if ((s = device_info(di)) != KN_OK) return s;
    auto it = n->tables.find(std::make_pair((int)o->precision, G));
    if (it == n->tables.end())
        return fail(KN_ERR_STATE,
                    "kn_integrate_noalloc: the tables for this precision and threads_per_zone are not built; "
                    "call kn_integrate_batch or kn_probe_step once with the same opts during set-up");
    const Tables& tb = it->second;
    const int budget = di.smem_optin - 1024 - 64;
    const int M = P / G;
    const GroupLayout gl = group_layout(n, o->precision, G, o->method == KN_METHOD_QSS ? kLayoutQss : 0);
    int smem_tables = tb.tl.bytes + M * gl.bytes <= budget;
    const int bytes = (smem_tables ? tb.tl.bytes : 0) + M * gl.bytes;
    if (bytes > budget) return fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: tiling needs %d B of shared memory", bytes);
    memset(&lp, 0, sizeof lp);
    lp.n_plans = 1;
    lp.smem_bytes = bytes;
    PlanDev& Pd = lp.plans[0];
    Pd.blob = (const unsigned char*)tb.blob->p;
    Pd.tl = tb.tl;
    Pd.rate0 = n->rate0.as<const double2>();
    Pd.R1 = n->R1;
    Pd.R12 = n->R12;
    Pd.cmax = n->cmax;
    Pd.u_tol = rate_cache_tol(n->cmax);
    Pd.rate_cache = rate_cache_on(n, o->precision) ? 1 : 0;
    Pd.N = n->N;
    Pd.R = n->R;
    Pd.S_r = n->S_r;
    Pd.zero_idx = n->R + n->S_r;
    Pd.smem_tables = smem_tables;
    Pd.G = G;
    Pd.M = M;
    Pd.gl = gl;
    Pd.Y = Y_out;
    Pd.T0 = zc->T0;
    Pd.rho0 = zc->rho0;
    Pd.tau = zc->tau;
    Pd.t_start = zc->t_start;
    Pd.t_end = zc->t_end;
    Pd.dt_trial = zc->dt_trial;
    Pd.t_out = t_out;
    Pd.dt_next = dt_next;
    Pd.steps = (long long*)steps;
    Pd.rejects = (long long*)rejects;
    Pd.status = status;
    Pd.n_zones = n_zones;
    Pd.zone_base = 0;
    Pd.order = order;
    Pd.queue_head = queue_head;
    int bps = 0;
    cudaError_t e = integrator_occupancy(o->precision, P, bytes, &bps);
    if (e != cudaSuccess) return fail(KN_ERR_CUDA, "occupancy: %s", cudaGetErrorString(e));
    if (bps < 1) return fail(KN_ERR_INVALID_ARG, "kn_integrate_noalloc: tiling does not fit on an SM");
    grid = di.sms * bps;
    block = P;
    Pd.cta_begin = 0;
    Pd.cta_end = grid;
    OptsDev& D = lp.o;
    D.kappa = o->kappa;
    D.eps_r = o->eps_r;
    D.eps_c = o->eps_c;
    D.y_min = o->y_min;
    D.grow_max = o->grow_max;
    D.safety = o->safety;
    D.shrink = o->shrink;
    D.dt_min_frac = o->dt_min_frac;
    D.max_steps = o->max_steps;
    D.max_reject = o->max_reject;
    D.method = o->method;
    set_guard_band(D, o);
    nbar = n->nbar;
    rbar = n->rbar;
    return KN_OK;
}

kn_status noalloc_fail(kn_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace kn


namespace kn {
cudaError_t launch_fp64_peak(double* out, int blocks, int threads, int iters, cudaStream_t st);
}

namespace {
// Candidate (P, G) tilings for the listed networks.
static kn_status tiling_candidates(kn_network* const* nets, int n_nets, int prec, int extras, int budget,
                                   std::vector<std::pair<int, int>>& out) {
    kn_status s;
    if (n_nets == 1) {
        kn_network* n = nets[0];
        for (int G = base_group(n); G <= 512; G += 32) {
            Tables* tb;
            if ((s = get_tables(n, prec, G, &tb)) != KN_OK) return s;
            const GroupLayout gl = group_layout(n, prec, G, extras);
            int M = std::min(kMaxGroups, 1024 / G);
            while (M > 0 && tb->tl.bytes + M * gl.bytes > budget) --M;
            if (M == 0) {  // tables in global memory
                M = std::min(kMaxGroups, 1024 / G);
                while (M > 0 && M * gl.bytes > budget) --M;
            }
            for (int m = M; m >= std::max(1, M - 1); --m) out.push_back({G * m, G});
        }
    } else {
        for (int P = 1024; P >= 128; P -= 64) out.push_back({P, 0});
    }
    return KN_OK;
}
}  // namespace

extern "C" {

kn_status kn_measure_fp64_peak(double* tflops, void* stream_) {
    if (!tflops) return fail(KN_ERR_INVALID_ARG, "kn_measure_fp64_peak: NULL argument");
    DeviceInfo di;
    kn_status s = device_info(di);
    if (s != KN_OK) return s;
    cudaStream_t st = (cudaStream_t)stream_;
    const int blocks = di.sms * 4, threads = 512, iters = 4096;
    DevBuf out;
    KN_CUDA(out.ensure(sizeof(double) * (size_t)blocks * threads));
    cudaEvent_t e0, e1;
    KN_CUDA(cudaEventCreate(&e0));
    KN_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        KN_CUDA(cudaEventRecord(e0, st));
        KN_CUDA(launch_fp64_peak(out.as<double>(), blocks, threads, iters, st));
        KN_CUDA(cudaEventRecord(e1, st));
        KN_CUDA(cudaEventSynchronize(e1));
        float ms;
        KN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)blocks * threads * 8.0 * iters;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return KN_OK;
}

kn_status kn_autotune(kn_network* const* nets, int32_t n_nets, const kn_opts* o, int64_t max_steps, void* stream_,
                      kn_tiling* best) {
    if (!nets || n_nets < 1 || n_nets > kMaxPlans || !o || !best || max_steps < 0)
        return fail(KN_ERR_INVALID_ARG, "kn_autotune: bad arguments");
    const bool full = max_steps == 0;  // whole-batch trials
    kn_status s = validate_opts(o);
    if (s != KN_OK) return s;
    if (o->replay_dt || o->record_features) return fail(KN_ERR_INVALID_ARG, "kn_autotune: replay/records must be off");
    for (int p = 0; p < n_nets; ++p)
        if (!nets[p] || !nets[p]->zones_set) return fail(KN_ERR_STATE, "kn_autotune: network %d has no zones", p);
    DeviceInfo di;
    if ((s = device_info(di)) != KN_OK) return s;
    cudaStream_t st = (cudaStream_t)stream_;
    const int prec = o->precision;
    const bool learn = o->mlp != nullptr;
    const int budget = di.smem_optin - 1024 - 64 - (learn ? kMlpSmemBytes : 0);
    std::vector<std::pair<int, int>> cands;
    const int extras = (learn ? kLayoutFeat : 0) | (o->method == KN_METHOD_QSS ? kLayoutQss : 0);
    if ((s = tiling_candidates(nets, n_nets, prec, extras, budget, cands)) != KN_OK) return s;
    // save the zone abundances (the trials integrate in place)
    std::vector<std::unique_ptr<DevBuf>> saved(n_nets);
    for (int p = 0; p < n_nets; ++p) {
        saved[p].reset(new DevBuf());
        const size_t bytes = 8 * (size_t)nets[p]->Z * nets[p]->N;
        KN_CUDA(saved[p]->ensure(bytes));
        KN_CUDA(cudaMemcpyAsync(saved[p]->p, nets[p]->Y.p, bytes, cudaMemcpyDeviceToDevice, st));
    }
    cudaEvent_t e0, e1;
    KN_CUDA(cudaEventCreate(&e0));
    KN_CUDA(cudaEventCreate(&e1));
    // A trial runs the longest predicted zones (the head of the queue, about
    // twelve per SM) for up to max_steps steps each, which resembles the
    // steady state that dominates a real batch better than every zone's first
    // steps do (those over-weight the once-per-zone set-up).  Zones outside
    // the trial keep zeroed counters, so the batch statistics count the trial.
    const int trial_Z = full ? 0 : 12 * di.sms;
    auto clear_counters = [&]() -> kn_status {
        for (int p = 0; p < n_nets; ++p) {
            KN_CUDA(cudaMemsetAsync(nets[p]->steps.p, 0, 8 * (size_t)nets[p]->Z, st));
            KN_CUDA(cudaMemsetAsync(nets[p]->rej.p, 0, 8 * (size_t)nets[p]->Z, st));
        }
        return KN_OK;
    };
    for (int p = 0; p < n_nets; ++p) nets[p]->trial_Z = trial_Z;
    kn_tiling win{0, 0, 0.0, 0, 0};
    for (const auto& c : cands) {
        kn_opts t = *o;
        t.threads_per_cta = c.first;
        t.threads_per_zone = c.second;
        t.use_graph = 0;
        // Untimed first run of one step: builds and uploads the candidate's
        // tables (host work that would otherwise sit between the events) and
        // sets the kernel's shared-memory limit.  Then the better of two
        // timed trials of up to max_steps steps, each from the saved state.
        t.max_steps = 1;
        for (int p = 0; p < n_nets; ++p)
            KN_CUDA(cudaMemcpyAsync(nets[p]->Y.p, saved[p]->p, 8 * (size_t)nets[p]->Z * nets[p]->N,
                                    cudaMemcpyDeviceToDevice, st));
        if (kn_integrate_batch(nets, n_nets, &t, st) != KN_OK) continue;  // does not fit: skipped
        t.max_steps = full ? o->max_steps : std::min<int64_t>(o->max_steps, max_steps);
        double rate = 0.0;
        for (int rep = 0; rep < (full ? 1 : 2) && s == KN_OK; ++rep) {
            for (int p = 0; p < n_nets; ++p)
                KN_CUDA(cudaMemcpyAsync(nets[p]->Y.p, saved[p]->p, 8 * (size_t)nets[p]->Z * nets[p]->N,
                                        cudaMemcpyDeviceToDevice, st));
            if ((s = clear_counters()) != KN_OK) break;
            KN_CUDA(cudaEventRecord(e0, st));
            s = kn_integrate_batch(nets, n_nets, &t, st);
            if (s != KN_OK) break;
            KN_CUDA(cudaEventRecord(e1, st));
            KN_CUDA(cudaEventSynchronize(e1));
            float ms;
            KN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            kn_batch_stats bs;
            if ((s = kn_get_batch_stats(nets, n_nets, st, &bs)) != KN_OK) return s;
            rate = std::max(rate, (double)bs.steps / (ms * 1e-3));
        }
        if (s != KN_OK) {
            s = KN_OK;
            continue;
        }
        win.candidates += 1;
        if (rate > win.zone_steps_per_s) {
            win.zone_steps_per_s = rate;
            win.threads_per_cta = c.first;
            // resolve the group size the launch used for each network
            win.threads_per_zone = c.second;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int p = 0; p < n_nets; ++p) nets[p]->trial_Z = 0;
    if ((s = clear_counters()) != KN_OK) return s;
    for (int p = 0; p < n_nets; ++p) {
        KN_CUDA(cudaMemcpyAsync(nets[p]->Y.p, saved[p]->p, 8 * (size_t)nets[p]->Z * nets[p]->N,
                                cudaMemcpyDeviceToDevice, st));
        KN_CUDA(launch_fill_int(nets[p]->status.as<int>(), nets[p]->Z, KN_ZONE_PENDING, st));
    }
    KN_CUDA(cudaStreamSynchronize(st));
    if (win.threads_per_cta == 0) return fail(KN_ERR_INVALID_ARG, "kn_autotune: no candidate tiling ran");
    // remember the winner: per network, the group size that CTA size gives it
    for (int p = 0; p < n_nets; ++p) {
        int G = win.threads_per_zone;
        if (G == 0) {
            Tiling tlp;
            bool ok = false;
            if ((s = plan_tiling(nets[p], prec, win.threads_per_cta, budget, 0, extras, tlp, ok)) != KN_OK) return s;
            if (!ok) return fail(KN_ERR_STATE, "kn_autotune: winning tiling no longer fits");
            G = tlp.G;
        }
        nets[p]->tuned_P[prec][tuned_slot(o, learn)] = win.threads_per_cta;
        nets[p]->tuned_G[prec][tuned_slot(o, learn)] = G;
    }
    *best = win;
    return KN_OK;
}

}  // extern "C"


namespace kn {
cudaError_t launch_advance(int n, const double* T9, const double* rho, const double* te, const double* t_out,
                           const double* dt_next, double* T0, double* rho0, double* tau, double* ts, double* tend,
                           double* dtt, int* status, cudaStream_t st);
}

extern "C" {

kn_status kn_advance_zones(kn_network* n, int32_t Z, const double* T9, const double* rho, const double* t_end,
                           int32_t mem, void* stream_) {
    if (!n || !T9 || !rho || !t_end) return fail(KN_ERR_INVALID_ARG, "kn_advance_zones: NULL argument");
    if (!n->zones_set) return fail(KN_ERR_STATE, "kn_advance_zones: no zones set");
    if (Z != n->Z) return fail(KN_ERR_INVALID_ARG, "kn_advance_zones: n_zones %d != zones set %d", Z, n->Z);
    if (mem != KN_MEM_HOST && mem != KN_MEM_DEVICE) return fail(KN_ERR_INVALID_ARG, "bad kn_mem");
    cudaStream_t st = (cudaStream_t)stream_;
    const double *dT = T9, *dR = rho, *dE = t_end;
    DevBuf tmp;
    if (mem == KN_MEM_HOST) {
        for (int z = 0; z < Z; ++z)
            if (!(std::isfinite(T9[z]) && T9[z] > 0 && std::isfinite(rho[z]) && rho[z] > 0 && std::isfinite(t_end[z])))
                return fail(KN_ERR_INVALID_ARG, "kn_advance_zones: zone %d needs finite T9, rho > 0 and t_end", z);
        KN_CUDA(tmp.ensure(3 * 8 * (size_t)Z));
        double* p = tmp.as<double>();
        KN_CUDA(cudaMemcpyAsync(p, T9, 8 * (size_t)Z, cudaMemcpyHostToDevice, st));
        KN_CUDA(cudaMemcpyAsync(p + Z, rho, 8 * (size_t)Z, cudaMemcpyHostToDevice, st));
        KN_CUDA(cudaMemcpyAsync(p + 2 * Z, t_end, 8 * (size_t)Z, cudaMemcpyHostToDevice, st));
        dT = p;
        dR = p + Z;
        dE = p + 2 * Z;
    }
    KN_CUDA(launch_advance(Z, dT, dR, dE, n->tout.as<double>(), n->dtn.as<double>(), n->T0.as<double>(),
                           n->rho0.as<double>(), n->tau.as<double>(), n->ts.as<double>(), n->te.as<double>(),
                           n->dtt.as<double>(), n->status.as<int>(), st));
    KN_CUDA(cudaMemsetAsync(n->energy.p, 0, 8 * (size_t)Z, st));
    n->has_const = true;
    if (mem == KN_MEM_HOST) KN_CUDA(cudaStreamSynchronize(st));  // tmp is freed on return
    return KN_OK;
}

kn_status kn_set_binding_energies(kn_network* n, const double* B) {
    if (!n || !B) return fail(KN_ERR_INVALID_ARG, "kn_set_binding_energies: NULL argument");
    for (int i = 0; i < n->N; ++i)
        if (!std::isfinite(B[i])) return fail(KN_ERR_INVALID_ARG, "kn_set_binding_energies: B[%d] not finite", i);
    KN_CUDA(n->bind.ensure(8 * (size_t)n->N));
    KN_CUDA(cudaMemcpy(n->bind.p, B, 8 * (size_t)n->N, cudaMemcpyHostToDevice));
    n->has_bind = true;
    return KN_OK;
}

kn_status kn_get_energy(const kn_network* n, double* E, int32_t mem, void* stream_) {
    if (!n || !E) return fail(KN_ERR_INVALID_ARG, "kn_get_energy: NULL argument");
    if (!n->zones_set) return fail(KN_ERR_STATE, "kn_get_energy: no zones set");
    cudaStream_t st = (cudaStream_t)stream_;
    KN_CUDA(cudaMemcpyAsync(E, n->energy.p, 8 * (size_t)n->Z,
                            mem == KN_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    KN_CUDA(cudaStreamSynchronize(st));
    return KN_OK;
}

}  // extern "C"
