// kn_internal.h -- library-internal layouts shared by the host runtime and the
// integrator kernel.  Nothing here is part of the C ABI (include/kn.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kn {

// Sliced gather list (the SELL-C-sigma layout of Kreutzer et al., SIAM J.
// Sci. Comput. 36 (2014), with slices of C = 32 rows, one per warp lane).
// The 2N row sums -- F+_i (rows 0..N-1: a flux f_j per product slot naming
// i) and k_i (rows N..2N-1: a reactant-slot partial per slot naming i) --
// are cut into pieces of at most L terms; a row's pieces occupy consecutive
// lanes of one slice.  Slice s has length len_s and holds lane l's term k at
// sidx[base_s + 32 k + l] (the value's byte offset in V when every offset
// fits 16 bits, else its index; shorter pieces are padded with the
// constant-zero entry).  Warp w of a zone group sums slices wsl[w] ..
// wsl[w + 1] - 1; in a slice flagged as holding a split row, a segmented
// warp reduction adds each row's pieces into its first lane.  Each row's sum
// is stored at byte offset sdst[32 s + l] from the zone's Fk array (padding
// lanes store to the spare slot fk_span).

// Fk holds 2N values of `real_bytes` each, padded to 16 bytes; the spare slot
// that padding lanes of the gather store to follows directly, at slot fk_span.
constexpr int fk_span(int N, int real_bytes) { return ((real_bytes * 2 * N + 15) & ~15) / real_bytes; }

constexpr int kMaxSpecies = 1023;
constexpr int kMaxPlans = 4;      // networks per launch
constexpr int kMaxGroups = 15;    // named barriers 1..15
constexpr int kPrecFP64 = 0;
constexpr int kPrecMixed = 1;
constexpr int kPrecMixed64 = 2;  // FP32 rates, fluxes and Kahan gathers; FP64 update, conservation sum and test
constexpr int kMlpFeatures = 64;   // learned-proposal network: 64 -> 128 -> 128 -> 1
constexpr int kMlpHidden = 128;
constexpr int kMlpParams = kMlpFeatures * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpHidden + 1;
// shared memory of the staged network: BF16 W1, W2 + FP32 b1, b2, w3, b3 (+3 pad), mu, 1/sigma
constexpr int kMlpSmemBytes = (kMlpFeatures * kMlpHidden + kMlpHidden * kMlpHidden) * 2 +
                              (3 * kMlpHidden + 4 + 2 * kMlpFeatures) * 4;

// One network's tables, as one contiguous device blob per (precision, zone
// group size); the kernel stages the blob into shared memory when it fits.
// Reactions are stored sorted by reactant count (1-body, 2-body, 3-body) so
// that the flux loop is warp-uniform and multiplies by no sentinel.
struct TableLayout {
    int32_t bytes;        // total (multiple of 16)
    int32_t off_A;        // mass numbers (integers, exact): float[N] in the mixed form, double[N] in the
                          //   forms with an FP64 update
    int32_t off_rspec;    // uint32[R]: reactant species a | b << 10 | c << 20 (N = none)
    int32_t off_cexp;     // real[R]: c_j = n_j + 3 (r_j - 1), so that along the profile
                          //   k_j(t) = k_j(T0, rho0) exp(-c_j t / tau)
    int32_t off_wsl;      // uint16[W + 1]: slice range of each warp (W = G / 32)
    int32_t off_shdr;     // uint2[n_slices]: (base into sidx, length | split-row flag << 31)
    int32_t off_sdst;     // uint16[32 n_slices]: destination byte offsets from Fk
    int32_t off_sidx;     // uint16[sum_s 32 len_s]: terms, lane-interleaved: byte offsets into V
                          //   when sidx_bytes, else V indices
    int32_t sidx_bytes;   // 1: sidx holds byte offsets
};

// Per-group shared-memory layout (byte offsets inside one group's region).
struct GroupLayout {
    int32_t bytes;
    int32_t off_V;      // real[R + S_r + 1]: fluxes f_j, partial planes 0, 1, 2 (reactions with
                        //   more than 0, 1, 2 reactants), constant 0
    int32_t off_K;      // real[R]: the zone's rates at (T0, rho0)
    int32_t off_Kc;     // float[R] (FP32-flux forms with the rate cache): the rates at u_ref
    int32_t off_Y;      // FP64 and mixed-FP64: double[2][N + 1], entry N the constant 1; mixed:
                        //   float[2][N + 1], the low parts of the float-float abundances (0 at N)
    int32_t off_Y32;    // float[2][N + 1] (FP32-flux forms): the FP32 copy the flux pass reads (the
                        //   high parts in the mixed form), entry N the constant 1
    int32_t off_Fk;     // real[N][2]: (F+_i, k_i) pairs
    int32_t off_carry;  // real[1]: the spare slot padding lanes of the gather store to
    int32_t off_Fk2;    // real[N][2] + spare slot (QSS): (F+_i, k_i) of the predicted state, at the
                        //   same distance from its spare slot as Fk (absent otherwise)
    int32_t off_red;    // per-warp reduction scratch, W = G/32 warps: double[W] x 3, float[W], int[W]
    int32_t off_feat;   // learned proposal / records: float[64 feats, 64 inputs, 128 h1, 128 h2],
                        //   int[3][64] histograms + 4 counters (absent when unused)
    int32_t off_state;  // GroupState
};

struct GroupState {
    double t, dt, t_end, h;
    double lnT0, lnR0, inv_tau, s;  // s = t / tau at the current step start
    double T0, rho0, tau;
    double cons, rel;
    long long steps, rejects;
    int zone, status, nrej, rhs_valid;
    int cur, done, valid, clipped;
    int constant, poly, poly_p, refresh_p;  // poly: 0 none (constant), 2/5 Taylor degree, 9 full exp;
                                            //   poly_p: the same at t + h (QSS predicted state);
                                            //   refresh_p: the QSS predicted pass recomputes Kc
    float u;                         // s / ln 2 for the mixed rate factor
    float pad2[3];
    // learned proposal / records
    double h_prev;     // the last accepted step
    double dt_plain;   // the plain controller's proposal for the current state
    long long props;   // accepted steps whose dt came from the learned proposal
    int fresh;         // current state was reached by an accepted step: features due
    int mlp_try;       // the current attempt uses the learned proposal
    int found;         // label search: a grid step passed
    float u_spec;      // FP32-flux forms: (t + h)/(tau ln 2) of the candidate state
    float u_scale;     // FP32-flux forms: 1/(tau ln 2)
    float u_ref;       // FP32-flux forms: the u at which the cached rates Kc were computed
    int refresh_spec;  // the speculative flux pass recomputes Kc
    double h_best;     // label search: the last grid step that passed (0: none)
    long long t_fetch_ns;  // global timer when the zone was taken from the queue
    // mixed form: the step sizes in FP32 (the update runs in FP32 and takes h as FP32)
    float h32;      // the current attempt's step
    float dt32;     // the controller's next step
    float dtp32;    // the plain controller's proposal for the current state
    float u_p;      // QSS, FP32-flux forms: (t + h)/(tau ln 2) of the predicted state
    double s_p;     // QSS: (t + h) / tau, the profile time of the predicted state
};

struct PlanDev {
    // tables
    const unsigned char* blob;  // device
    TableLayout tl;
    const double2* rate0;        // [R] (ln k0_j, n_j), sorted order, global: zone-load rates
    int32_t N, R, S_r;
    int32_t R1, R12;             // reactions [0,R1) 1-body, [R1,R12) 2-body, [R12,R) 3-body
    double cmax;                 // max_j c_j
    float u_tol;                 // FP32-flux forms: cached rates are reused while |u - u_ref| <= u_tol,
                                 //   i.e. while no rate would move by a quarter ulp: 2^-26 / (cmax ln 2)
    int32_t rate_cache;          // 1: the groups keep the cache Kc (FP32-flux forms, small enough R)
    int32_t zero_idx;            // V index of the constant zero (= R + S_r)
    int32_t smem_tables;         // 1: stage blob into shared memory
    int32_t G, M;                // threads per zone group, groups per CTA
    GroupLayout gl;
    // zone state (device, library-owned)
    double* Y;                   // [Z][N] in: Y0, out: Y at t
    const double* T0;
    const double* rho0;
    const double* tau;
    const double* t_start;
    const double* t_end;
    const double* dt_trial;
    double* t_out;
    double* dt_next;
    long long* steps;
    long long* rejects;
    long long* props;            // [Z] accepted steps proposed by the network
    const double* bind;          // [N] binding energies (NULL: no energy output)
    double* energy;              // [Z] sum_i B_i (Y_end - Y_start)
    int* status;
    int32_t n_zones;
    int32_t zone_base;           // first global zone index of this plan (replay arrays)
    const int* order;            // work-queue order of zones (longest first)
    int* queue_head;             // work-queue counter (reset to 0 before each launch)
    int32_t cta_begin, cta_end;  // CTAs whose home is this plan
};

struct OptsDev {
    double kappa, eps_r, eps_c, y_min, grow_max, safety, shrink, dt_min_frac;
    long long max_steps;
    int max_reject;
    int lockstep;
    // replay
    const double* replay_dt;
    const long long* replay_off;
    const long long* replay_len;
    // probe (one step, no test): outputs [zones][N] / [zones]
    double* probe_Fp;
    double* probe_k;
    double* probe_Y1;
    double* probe_cons;
    double* probe_rel;
    int probe;
    // records for training the learned proposal: features [cap][64] and labels
    float* rec_feat;
    float* rec_label;
    long long rec_cap;
    unsigned long long* rec_count;
    // learned proposal: device parameters of the network (FP32 layout of kn.h),
    // BF16 W1 [64][128] then W2 [128][128], normalisation mu [64], 1/sigma [64]
    const float* mlpP;
    const void* mlpW;
    const float* mlpNorm;
    float mlp_margin;  // the proposal uses e^(out - margin)
    // FP32 guard band of the mixed form's accept test (see update_reduce)
    float eps_r32, ymin_lo32, ymin_hi32, band_lo32, band_hi32, kappa32;
    float eps_c32, ga32, gb32, grow32;  // mixed form: eps_c and the growth factor's terms in FP32
    float shrink32;                     // mixed form: the reject factor in FP32
    float thr_lo32, thr_hi32;           // mixed form: eps_r times the guard band's ends
    // trace of the learned proposal: features [cap][64], output [cap], dt record [cap][6]
    float* trace_feat;
    float* trace_out;
    double* trace_dt;
    long long trace_cap;
    unsigned long long* trace_count;
    int follow_label;  // records: the attempt takes the label's step (perfect proposal)
    int method;        // 0: Eq. (3) with the kappa switch; 1: alpha-QSS (FP64 and mixed forms)
    long long* zone_ns;  // [zones][2]: global timer at queue fetch and at write-back (NULL: off)
    int learn;   // 1: propose with the network
    int record;  // 1: write (features, label) at every accepted state
    int mlp_smem_off;  // byte offset of the staged network in the CTA's shared memory
};

struct LaunchParams {
    int32_t n_plans;
    int32_t smem_bytes;
    PlanDev plans[kMaxPlans];
    OptsDev o;
};

// Host-side launch of the integrator kernel (kn_integrate.cu).
cudaError_t launch_integrator(const LaunchParams& lp, int precision, int grid, int block,
                              cudaStream_t stream);
// Occupancy query for a given precision, block size and shared memory.
cudaError_t integrator_occupancy(int precision, int block, int smem, int* blocks_per_sm);
// Enable the large dynamic shared memory carve-out for both kernel variants.
cudaError_t integrator_set_smem_limit(int bytes);
// Work-queue ordering key per zone (mean log-rate at the initial conditions)
// and the identity permutation, for a descending sort.
cudaError_t launch_zone_cost_simple(const double* T0, const double* rho0, int n, double nbar,
                                    double rbar, float* key, int* idx, cudaStream_t stream);
cudaError_t launch_fill_int(int* p, int n, int v, cudaStream_t stream);

}  // namespace kn
