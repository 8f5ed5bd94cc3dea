/*
 * kn.h -- C ABI of libkn: batched explicit asymptotic integration of many
 * independent stiff reaction networks ("zones") on one NVIDIA GB300 (sm_103a).
 *
 * Method (Brock, Belt, Billings & Guidry, "Explicit Integration with GPU
 * Acceleration for Large Kinetic Networks"):
 *   Eq. (1)  dY_i/dt = F+_i - F-_i = F+_i - k_i Y_i
 *   Eq. (3)  Y_i' = (Y_i + dt F+_i) / (1 + k_i dt)      if k_i dt >= kappa  (Sec. 3)
 *            Y_i' = Y_i + dt (F+_i - k_i Y_i)           otherwise (forward Euler)
 *   Sec. 4   adaptive network timestep dt inside one hydro interval
 *   Sec. 6   per zone the host sends abundances, T, rho, the interval and a
 *            trial dt, and gets back abundances and a final dt.
 *
 * Conventions for every entry point:
 *   - Return codes only (kn_status); no exception or abort crosses the ABI.
 *     On any code other than KN_OK, kn_last_error() describes the failure.
 *   - Inputs are copied; the caller keeps ownership of everything it passes.
 *   - Pointers marked "host or device" are read according to the kn_mem
 *     argument of the call.  Device pointers must be addressable from the
 *     current CUDA device (e.g. torch tensors' data_ptr()).
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *     Calls that enqueue GPU work are asynchronous on that stream unless the
 *     entry point says it synchronises.
 *   - Not thread-safe per object: one network object must not be used from
 *     two host threads at once.  Different objects are independent.
 */
#ifndef KN_H
#define KN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KN_OK = 0,
    KN_ERR_INVALID_ARG = 1, /* bad pointer, size, value or layout */
    KN_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
    KN_ERR_NOMEM = 3,       /* device or host allocation failed */
    KN_ERR_STATE = 4,       /* call out of order (e.g. integrate before zones are set) */
    KN_ERR_INTERNAL = 5     /* a self-check of the library failed before any device work
                               (a bug; the message names the check) */
} kn_status;

/* Per-zone outcome, written by kn_integrate_batch. */
typedef enum {
    KN_ZONE_OK = 0,           /* reached t_end */
    KN_ZONE_STEP_LIMIT = 1,   /* max_steps accepted steps before t_end */
    KN_ZONE_DT_UNDERFLOW = 2, /* dt fell below dt_min_frac * t */
    KN_ZONE_NONFINITE = 3,    /* max_reject consecutive rejects, the last one non-finite */
    KN_ZONE_MAX_REJECT = 4,   /* max_reject consecutive rejects */
    KN_ZONE_INVALID = 5,      /* zone inputs failed validation on the device */
    KN_ZONE_PENDING = 6       /* set but not yet integrated */
} kn_zone_status;

typedef enum { KN_MEM_HOST = 0, KN_MEM_DEVICE = 1 } kn_mem;

typedef enum {
    KN_PREC_FP64 = 0, /* every step of the path in FP64 */
    KN_PREC_MIXED = 1, /* FP32 rates, fluxes and gathers (every row sum of positive
                          terms within (L + 5) 2^-24 relative, L <= the longest row;
                          for networks of up to 2048 reactions the FP32 rates are
                          cached and refreshed before any moves by 2^-26 relative);
                          abundances kept as FP32 high/low pairs (~48 bits); the
                          kappa-switched update in FP32; the conservation sum as a
                          float-float sum of exact products; the relative-error
                          test in FP32 outside a guard band, FP64 inside it */
    KN_PREC_MIXED_FP64 = 2 /* FP32 rates and fluxes, Kahan-compensated FP32 gathers;
                              the kappa-switched update, the conservation sum and the
                              error test in FP64 (FP64 abundances) */
} kn_precision;

typedef enum {
    KN_METHOD_ASYMPTOTIC = 0, /* the kappa-switched update of Sec. 3, Eq. (3) */
    KN_METHOD_QSS = 1         /* the alpha-QSS predictor-corrector (kn_opts.method) */
} kn_method;

/*
 * Network description (Sec. 2 and Sec. 6: the rate-library parameters that are
 * copied to the GPU once and stay resident).  Reaction j has 1..3 reactant
 * slots and 1..3 product slots; a species id repeated in a list is a repeated
 * reactant/product (i + i -> k).  Its rate is
 *     k_j(T9, rho) = exp(ln_k0[j]) * T9^t9_exp[j] * rho^(r_j - 1),
 * r_j = number of reactant slots, and its flux is f_j = k_j * prod(Y of reactant slots).
 * Limits: 1 <= n_species <= 1023, 1 <= n_reactions <= 16383, and
 * n_reactions + (reactant slots) < 65535.
 */
typedef struct {
    int32_t n_species;
    int32_t n_reactions;
    const double *A;       /* [n_species] mass number of each species, > 0 */
    const int32_t *reac;   /* [n_reactions][3] reactant species ids, -1 padded (ids first) */
    const int32_t *prod;   /* [n_reactions][3] product species ids, -1 padded */
    const double *ln_k0;   /* [n_reactions] natural log of k0_j */
    const double *t9_exp;  /* [n_reactions] temperature exponent n_j */
} kn_network_desc;

/*
 * Per-zone initial conditions (Sec. 6, item 1: abundances, temperature,
 * density, hydro interval and trial timestep).  All arrays host or device
 * (kn_mem argument), row-major:
 *   Y0 [n_zones][n_species]  molar abundances (mass fraction X_i = A_i Y_i)
 *   T0, rho0  [n_zones]      T9 and density at t = 0
 *   tau       [n_zones]      profile time scale: T9(t) = T0 exp(-t/tau),
 *                            rho(t) = rho0 exp(-3t/tau); tau <= 0 holds T9 and
 *                            rho constant (the operator-split setting, Sec. 4)
 *   t_start, t_end [n_zones] the interval to integrate
 *   dt_trial  [n_zones]      first trial dt; <= 0 means t_start
 */
typedef struct {
    const double *Y0;
    const double *T0;
    const double *rho0;
    const double *tau;
    const double *t_start;
    const double *t_end;
    const double *dt_trial;
} kn_zone_conditions;

/*
 * Integration options.  kn_default_opts() fills the defaults listed here.
 * The accept test and the timestep update are the library's reading of
 * Sec. 4 (the paper states no criterion):
 *   accept iff |sum_i A_i (Y'_i - Y_i)| <= eps_c and
 *              max_{i: max(Y_i,Y'_i) > y_min} |Y'_i - Y_i| / max(Y_i,Y'_i) <= eps_r
 *   accept: t += dt; dt *= min(grow_max, safety*eps_r/rel, safety*eps_c/cons)
 *   reject: dt *= shrink, retry from the same state
 */
typedef struct {
    int32_t precision;     /* kn_precision, default KN_PREC_MIXED */
    int32_t max_reject;    /* consecutive rejects before KN_ZONE_MAX_REJECT, default 60 */
    double kappa;          /* asymptotic switch (Sec. 3), default 1 */
    double eps_r;          /* default 0.05 */
    double eps_c;          /* default 1e-6 */
    double y_min;          /* default 1e-10 */
    double grow_max;       /* default 1.5 */
    double safety;         /* default 0.9 */
    double shrink;         /* default 0.5 */
    double dt_min_frac;    /* default 1e-30 */
    int64_t max_steps;     /* accepted steps per zone, default 10^7 */
    /* Tiling (0 = the kn_autotune winner if there is one, else the built-in
       default): threads per CTA and threads per zone group.  A CTA holds
       threads_per_cta/threads_per_zone zone slots; threads_per_zone ==
       threads_per_cta is CTA-per-zone.  The built-in default for one network
       stages the tables in shared memory and takes, in KN_PREC_MIXED with
       groups of more than one warp, up to 5 groups per CTA and then the largest
       group; otherwise the most groups per CTA and then the smallest group. */
    int32_t threads_per_cta;
    int32_t threads_per_zone;
    int32_t use_graph;     /* 1: capture the launch sequence in a CUDA graph and replay it */
    int32_t lockstep;      /* reserved, must be 0 */
    /* Replay (validation): zone z takes exactly replay_len[z] accepted steps
       with dt = replay_dt[replay_off[z] + s], no accept test.  Device pointers;
       zones are numbered across the nets of the call in order. NULL = off. */
    const double *replay_dt;
    const int64_t *replay_off;
    const int64_t *replay_len;
    /* Learned dt proposal (kn_mlp handle from kn_mlp_create), NULL = off.
       At every state reached by an accepted step the network proposes
       dt_mlp = clip(dt_prev e^(out - mlp_margin), dt_plain, 16 dt_plain);
       the accept test judges it, and a rejected proposal is retried with
       dt_plain. */
    const void *mlp;
    /* Training records for the proposal network: at every state reached by an
       accepted step, the 64 features and the label ln(dt_best / dt_prev)
       (dt_best the last step of the grid dt_prev 2^(q/4), q = -8 .. 16, before
       the first one that fails the accept test from that state; -2 ln 2 if
       the smallest fails) are appended to these device arrays.
       *record_count (device, zeroed by the caller) counts every record; those
       beyond record_capacity are counted but not written.  NULL = off; not
       combined with mlp. */
    float *record_features;   /* [record_capacity][64] */
    float *record_labels;     /* [record_capacity] */
    int64_t record_capacity;
    int64_t *record_count;
    double mlp_margin;        /* ln-units safety margin of the learned proposal, default 0.5 */
    /* Trace of the learned proposal (validation; needs mlp): every time the
       network proposes a step, one record is appended:
         trace_features [cap][64]  the features it was given (FP32)
         trace_out [cap]           its output (FP32)
         trace_dt [cap][6]         dt_prev; dt_plain; the unclipped proposal
                                   dt_prev e^min(out - mlp_margin, 20); the step
                                   the attempt then takes; 1 if that step is the
                                   proposal, else 0; t_end - t
       *trace_count (device, zeroed by the caller) counts every record; those
       beyond trace_capacity are counted but not written.  NULL = off. */
    float *trace_features;
    float *trace_out;
    double *trace_dt;
    int64_t trace_capacity;
    int64_t *trace_count;
    /* Perfect-proposal run (measurement; needs record_features): at every state
       reached by an accepted step, the attempt takes the step of the record's
       label -- the last grid step before the first that fails the accept test
       from that state -- clipped to [dt_plain, 16 dt_plain] like a learned
       proposal with margin 0, and falls back to dt_plain if that step is not
       above it.  Its step count bounds what any learned proposal of this form
       can save.  0 = off. */
    int32_t follow_label;
    /* kn_method, default KN_METHOD_ASYMPTOTIC.  KN_METHOD_QSS replaces the
       update of Eq. (3) by the explicit quasi-steady-state update that Sec. 11
       proposes to try; the paper defers its formula to its QSS reference, and
       the library takes the alpha-QSS predictor-corrector of Mott, Oran &
       van Leer (J. Comput. Phys. 164 (2000) 407), with the production F+ and
       the depletion rate k of Eq. (1):
         alpha(x) = (180 r^3 + 60 r^2 + 11 r + 1) / (360 r^3 + 60 r^2 + 12 r + 1),
                    r = 1/x
         predictor  Yp = Y + dt (F+ - k Y) / (1 + alpha(k dt) k dt)
                    (F+, k of Y at t)
         corrector  kbar = (k + kp)/2, a = alpha(kbar dt),
                    Y' = Y + dt (a F+p + (1 - a) F+ - kbar Y) / (1 + a kbar dt)
                    (F+p, kp of Yp at t + dt)
       and the same accept test and step control.  Each update
       y + h (f - k y) / (1 + alpha k h) is evaluated in an algebraically equal
       form without its cancellation at k h >> 1, which is non-negative for
       non-negative inputs.  Each attempt evaluates the right-hand side twice.
       With KN_PREC_FP64 every step is FP64; with KN_PREC_MIXED the predictor
       and the predicted state's fluxes and gathers are FP32 and the corrector
       updates the float-float pairs as Eq. (3) does (the change added up to
       k dt = 1, y' itself above).  Not with KN_PREC_MIXED_FP64, mlp,
       record_features or follow_label (KN_ERR_INVALID_ARG). */
    int32_t method;
    /* Per-zone timing (measurement): zone_ns [total zones][2] (device int64)
       receives the GPU global timer, in ns, when a zone group takes the zone
       from the work queue and when it has written the zone back.  Zones are
       numbered across the nets of the call in order.  NULL = off. */
    int64_t *zone_ns;
} kn_opts;

/* Aggregate counters of the last kn_integrate_batch on these networks. */
typedef struct {
    int64_t zones;          /* zones integrated */
    int64_t zones_ok;       /* of which reached t_end (KN_ZONE_OK) */
    int64_t steps;          /* accepted steps, summed over zones */
    int64_t rejects;        /* rejected attempts, summed over zones */
    int64_t proposals_used; /* accepted steps whose dt came from the learned proposal */
} kn_batch_stats;

typedef struct kn_network kn_network; /* opaque, library-owned host + device copies */

/* Fill *opts with the defaults documented on kn_opts.  Never fails. */
void kn_default_opts(kn_opts *opts);

/*
 * Validate the description, build the species<->reaction maps (the CSR
 * gathers behind the F+ and F- sums of Sec. 10 item (2)) and upload the
 * rate parameters to the current device, where they stay resident until
 * kn_destroy_network (Sec. 6: "copied to the GPU and resident ... for the
 * duration of the calculation").  *out receives the new object.
 * Errors: KN_ERR_INVALID_ARG (NULL pointers, sizes beyond the limits, a
 * species id out of range, a reaction with no reactant or product, a
 * non-finite parameter, A <= 0), KN_ERR_NOMEM, KN_ERR_CUDA.
 */
kn_status kn_create_network(const kn_network_desc *desc, kn_network **out);

/* Free all host and device memory of the network (after synchronising the
   device).  NULL is accepted and ignored. */
kn_status kn_destroy_network(kn_network *net);

/* Sizes of a network: n_species, n_reactions, reactant slots, product slots
   (any pointer may be NULL). */
kn_status kn_network_info(const kn_network *net, int32_t *n_species, int32_t *n_reactions,
                          int32_t *n_reactant_slots, int32_t *n_product_slots);

/*
 * Host-only check of the gather tables the integrator would use for this
 * description at `precision` with zone groups of `threads_per_zone` threads
 * (a multiple of 32 in [32, 1024]); no device is touched.  The F+ and k sums
 * of Eq. 1 (Sec. 10 item (2)) are laid out as warp slices of row pieces; the
 * builder verifies every index and destination and, running the gather on
 * the host with V[v] = v + 1, that every row's sum comes out exactly once.
 * stats (4 int32, caller-owned) receives: the piece length cap L, the number
 * of slices, the longest warp's terms per lane, and the table bytes.
 * Errors: KN_ERR_INVALID_ARG (as kn_create_network, or a bad precision or
 * group size), KN_ERR_INTERNAL (a table check failed; the message names it).
 */
kn_status kn_check_gather_tables(const kn_network_desc *desc, int32_t precision, int32_t threads_per_zone,
                                 int32_t stats[4]);

/*
 * Load n_zones zones into the network's device state (Sec. 6, step 1: the
 * host-to-device copy of abundances, T, rho, interval and trial dt), replacing
 * any previous zones.  Enqueued on `stream`.  Host inputs are validated on the
 * host (finite, Y0 >= 0, T0 > 0, rho0 > 0, t_end > t_start >= 0, and
 * t_start > 0 or dt_trial > 0) and an invalid zone fails the call with
 * KN_ERR_INVALID_ARG; device inputs are validated by the integrator, which
 * marks an invalid zone KN_ZONE_INVALID.  Device state is (re)allocated only
 * when n_zones grows.
 * Errors: KN_ERR_INVALID_ARG, KN_ERR_NOMEM, KN_ERR_CUDA.
 */
kn_status kn_set_zone_conditions(kn_network *net, int32_t n_zones, const kn_zone_conditions *zc,
                                 int32_t mem, void *stream);

/*
 * Integrate every zone of every listed network from t_start to t_end
 * (Sec. 3 update, Sec. 4 adaptive steps, Sec. 9 many networks at once),
 * entirely on the GPU in one persistent-kernel launch fed by a work queue.
 * Zones of networks of different sizes share the launch.  Asynchronous on
 * `stream`: results are in the networks' device state when the stream
 * reaches this point; read them with kn_get_abundances.  Results overwrite
 * the zone abundances in place, so a second call continues from them once
 * new conditions are set.  nets must be distinct.
 * Errors: KN_ERR_INVALID_ARG (bad opts or tiling), KN_ERR_STATE (a network
 * without zones), KN_ERR_CUDA.
 */
kn_status kn_integrate_batch(kn_network *const *nets, int32_t n_nets, const kn_opts *opts,
                             void *stream);

/*
 * Copy results out (Sec. 6, step 3: abundances and the final dt, plus
 * per-zone counters).  Synchronises `stream` first.  Any output pointer may
 * be NULL.  Layouts: Y [n_zones][n_species]; t, dt_next [n_zones] double;
 * steps, rejects [n_zones] int64; status [n_zones] int32 (kn_zone_status).
 * dt_next is the controller's proposal after the last accepted step, the
 * trial dt for the next hydro interval.
 * Errors: KN_ERR_INVALID_ARG, KN_ERR_STATE, KN_ERR_CUDA.
 */
kn_status kn_get_abundances(const kn_network *net, double *Y, double *t, double *dt_next,
                            int64_t *steps, int64_t *rejects, int32_t *status, int32_t mem,
                            void *stream);

/* Sum the per-zone counters of the listed networks into *stats.
   Synchronises `stream`.  Errors: KN_ERR_INVALID_ARG, KN_ERR_CUDA. */
kn_status kn_get_batch_stats(kn_network *const *nets, int32_t n_nets, void *stream,
                             kn_batch_stats *stats);

/*
 * Diagnostic single step (Eq. 1 and Eq. 3 from one state): for every zone of
 * `net`, evaluate the rates at (T9, rho)(t_start), the fluxes and the F+/k
 * gathers at Y0, and apply one kappa-switched update with dt = dt_trial,
 * without the accept test, through the same device code as the integrator.
 * Outputs (device pointers, any may be NULL): Fp, k [n_zones][n_species]
 * double, Y1 [n_zones][n_species] double, cons [n_zones] (|sum A dY|),
 * rel [n_zones] (max relative change, as in the accept test).  The zone
 * state is left as set.  Asynchronous on `stream`.
 * Errors: KN_ERR_INVALID_ARG, KN_ERR_STATE, KN_ERR_CUDA.
 */
kn_status kn_probe_step(kn_network *net, const kn_opts *opts, double *Fp, double *k, double *Y1,
                        double *cons, double *rel, void *stream);

/* ---------------------------------------------------------------------------
 * Learned timestep proposal (the paper has no learned component; this is the
 * library's addition on top of the Sec. 4 controller, which stays the judge
 * of every step).  A small network maps 64 per-zone features to
 * ln(dt_next / dt_prev): 64 -> 128 (ReLU) -> 128 (ReLU) -> 1, BF16 weights
 * and activations, FP32 accumulation, FP32 master weights trained by Adam.
 * Parameters are one FP32 array of KN_MLP_PARAMS values, in this order:
 *   W1 [64][128] (input-major), b1 [128], W2 [128][128], b2 [128], w3 [128], b3 [1].
 * Features are normalised as (f - mu) / sigma before the first layer.
 * ------------------------------------------------------------------------- */
#define KN_MLP_FEATURES 64
#define KN_MLP_HIDDEN 128
#define KN_MLP_PARAMS 24961

typedef struct kn_mlp kn_mlp; /* opaque: device parameters, Adam state, activations */

/* Create a network with all parameters zero, mu = 0, sigma = 1 (on the
   current device).  Errors: KN_ERR_INVALID_ARG, KN_ERR_CUDA. */
kn_status kn_mlp_create(kn_mlp **out);

/* Free the network (after synchronising the device); NULL is ignored. */
kn_status kn_mlp_destroy(kn_mlp *mlp);

/* Set the FP32 parameters (host array of KN_MLP_PARAMS) and the feature
   normalisation mu, sigma (host arrays of KN_MLP_FEATURES, sigma > 0); resets
   the Adam state.  Synchronous.  Errors: KN_ERR_INVALID_ARG, KN_ERR_CUDA. */
kn_status kn_mlp_set_params(kn_mlp *mlp, const float *params, const float *mu, const float *sigma);

/* Copy the FP32 parameters and the last gradients to host arrays of
   KN_MLP_PARAMS (either may be NULL).  Synchronises the device. */
kn_status kn_mlp_get_params(const kn_mlp *mlp, float *params, float *grads);

/* Inference on a batch: features [B][64] and out [B] are device FP32 arrays
   (features 16-byte aligned).  Asynchronous on `stream`.
   Errors: KN_ERR_INVALID_ARG, KN_ERR_CUDA. */
kn_status kn_mlp_forward(kn_mlp *mlp, const float *features, int32_t B, float *out, void *stream);

/* Forward and backward pass of the mean squared error against labels [B]
   (device FP32; features as for kn_mlp_forward); the gradients stay in the
   handle for kn_mlp_adam, and the loss is written to *loss (device FP32
   scalar) when loss is not NULL.  Tiles of 64 rows are processed by one CTA
   each and their partial gradients added in a fixed order, so a call is
   deterministic.  Asynchronous on `stream`. */
kn_status kn_mlp_backward(kn_mlp *mlp, const float *features, const float *labels, int32_t B, float *loss,
                          void *stream);

/* One Adam step on the FP32 master weights with the handle's gradients
   (bias-corrected, Kingma & Ba), then refresh the BF16 copies.  Asynchronous. */
kn_status kn_mlp_adam(kn_mlp *mlp, float lr, float beta1, float beta2, float eps, void *stream);

/* ---------------------------------------------------------------------------
 * Autotuner and measurement helpers (library additions; the paper has none).
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t threads_per_cta;   /* CTA size P */
    int32_t threads_per_zone;  /* zone group size G (G == P: CTA-per-zone) */
    double zone_steps_per_s;   /* measured on the trial batch */
    int32_t candidates;        /* tilings timed */
    int32_t pad;
} kn_tiling;

/*
 * Time candidate tilings on the networks' current zones and keep the fastest
 * as the default for later kn_integrate_batch calls with the same precision
 * and learned/plain form (a tiling in opts still overrides it).  Candidates:
 * zone groups from one warp (small networks) or the smallest warp multiple
 * covering the species, up to CTA-per-zone, each with the most groups per CTA
 * that fit in shared memory and with fewer.  Each candidate runs once for one
 * step (building its tables), then is timed.  max_steps > 0: two trials, each
 * integrating the longest predicted zones (the head of the work queue, twelve
 * per SM) for at most max_steps accepted steps -- the steady state of a long
 * batch -- and the better one counts.  max_steps == 0: one trial that
 * integrates the whole batch, which also weighs the tail, where the longest
 * zone's per-step latency rather than throughput can set the batch time.  The
 * zone state is saved before and restored after the trials.  *best receives
 * the winner.  Synchronises
 * `stream`.  Errors: KN_ERR_INVALID_ARG, KN_ERR_STATE (no zones), KN_ERR_NOMEM,
 * KN_ERR_CUDA.
 */
kn_status kn_autotune(kn_network *const *nets, int32_t n_nets, const kn_opts *opts, int64_t max_steps,
                      void *stream, kn_tiling *best);

/* Measured FP64 FMA throughput of the current device (independent DFMA
   chains on every SM, timed with CUDA events), in TFLOP/s (2 flops per FMA).
   The roofline denominator for the FP64-bound integrator.  Synchronises
   `stream`. */
kn_status kn_measure_fp64_peak(double *tflops, void *stream);

/* Largest batch kn_integrate_noalloc accepts (its fixed scratch holds one
   queue slot per zone: 256 KB of device memory, kept until process exit). */
#define KN_NOALLOC_MAX_ZONES 65536

/*
 * kn_integrate_noalloc -- the batched integrator for callers that cannot
 * allocate GPU memory when they integrate.  The paper has no counterpart:
 * this is a library convenience.  Typical callers are host simulation codes
 * that hand out all device memory from their own pre-allocated pool, or whose
 * per-step path must avoid cudaMalloc/cudaFree (those can synchronise the
 * device and stall work the code overlaps with the network integration).
 *
 * Same integration as kn_integrate_batch for one network, but every zone
 * array is the caller's (device memory of the current device, row-major as
 * in kn_zone_conditions / kn_get_abundances; each pointer is checked on the
 * host and anything else -- host memory, another device's memory -- is
 * refused before any launch): zc holds the inputs; Y [n_zones][n_species]
 * receives the abundances at t (Y0 is copied there first; Y may be Y0 itself,
 * which integrates in place, but must not otherwise overlap it), t,
 * dt_next [n_zones] double, steps, rejects [n_zones] int64, status
 * [n_zones] int32.  The network's resident tables must already exist for
 * opts->precision and opts->threads_per_zone (built by any earlier
 * kn_integrate_batch or kn_probe_step call with those opts, e.g. at set-up);
 * opts->threads_per_zone must be set (threads_per_cta 0 means one zone group
 * per CTA); use_graph, replay and mlp must be off.
 *
 * Its only scratch (work-queue counter and order) is a fixed device array in
 * the library, 256 KB per device: no call allocates device memory.  The
 * first call on each device (and again after the device's context changes,
 * e.g. after cudaDeviceReset) looks up that array's address; make that first
 * call before any stream capture.  Every call shares the array and clears
 * what it needs, so calls whose GPU work overlaps (different streams or
 * threads) race: serialise them.  Asynchronous on `stream`.
 * Errors: KN_ERR_INVALID_ARG (NULL or non-device pointer, Y partly
 * overlapping Y0, n_zones < 1 or above KN_NOALLOC_MAX_ZONES, bad opts or
 * tiling), KN_ERR_STATE (tables not built), KN_ERR_CUDA.
 */
kn_status kn_integrate_noalloc(kn_network *net, int32_t n_zones, const kn_zone_conditions *zc,
                               const kn_opts *opts, double *Y, double *t, double *dt_next,
                               int64_t *steps, int64_t *rejects, int32_t *status, void *stream);

/*
 * Operator splitting (Sec. 4, Sec. 6): continue every zone of `net` into the
 * next hydro interval.  The abundances stay where the last integration left
 * them; each zone starts at its last time t, runs to t_end[z] at constant
 * T9[z], rho[z] (the hydro values held fixed over the interval), and takes
 * the last dt_next as its trial step.  Arrays [n_zones] host or device (mem),
 * n_zones must equal the zones set.  Asynchronous on `stream`.
 * Errors: KN_ERR_INVALID_ARG, KN_ERR_STATE (no zones), KN_ERR_CUDA.
 */
kn_status kn_advance_zones(kn_network *net, int32_t n_zones, const double *T9, const double *rho,
                           const double *t_end, int32_t mem, void *stream);

/*
 * Integrated energy release (Sec. 6 item 3).  With per-species binding
 * energies B_i (any unit per nucleus; host array [n_species]) set, every
 * integration also records per zone E = sum_i B_i (Y_i(t) - Y_i(t_start)),
 * which for an A-conserving network equals the time integral of
 * sum_j Q_j f_j with Q_j the reaction's binding-energy gain.  Synchronous.
 */
kn_status kn_set_binding_energies(kn_network *net, const double *B);

/* Copy the per-zone energy release of the last integration (see above) to
   E [n_zones] (host or device per mem); synchronises `stream`.  Zones without
   binding energies set report 0. */
kn_status kn_get_energy(const kn_network *net, double *E, int32_t mem, void *stream);

/* Human-readable description of the most recent failure on this host thread
   (empty string if none).  The pointer stays valid until the next call on
   the same thread. */
const char *kn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KN_H */
