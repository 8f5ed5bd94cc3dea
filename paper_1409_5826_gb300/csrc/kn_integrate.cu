// kn_integrate.cu -- persistent batched integrator for the explicit asymptotic
// method (Brock, Belt, Billings & Guidry: Eq. 1, Eq. 3 and the kappa switch of
// Sec. 3, adaptive network steps of Sec. 4, many networks on one GPU, Sec. 9).
//
// Execution model (sm_103a):
//   * one persistent launch; each CTA is split into M zone groups of G
//     threads (G = CTA size: CTA-per-zone; G = 128: warp-group-per-zone);
//   * every group pulls zones from its network's work queue (one atomic per
//     zone, longest predicted zones first) and keeps the zone resident in
//     shared memory for its whole integration;
//   * a network's tables (reactant lists, rate parameters, the sliced gather
//     list) are staged once per CTA into shared memory and shared by all
//     groups;
//   * per step: rates + fluxes + reactant-slot partials (one pass over
//     reactions), sliced gathers of F+ and k (each lane sums one row piece
//     per slice with no per-term branch; a long row's pieces are combined
//     by a segmented warp reduction), then the kappa-switched update with
//     deterministic group reductions for the accept test.
//   * no spin-waits: every loop is bounded by the zone's step and reject limits.
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "kn_internal.h"

namespace kn {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
struct GroupSync {
    int id, n, whole;
    __device__ __forceinline__ void sync() const {
        if (whole) {
            __syncthreads();
        } else if (n == 32) {
            __syncwarp();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
        }
    }
};

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exp(-x) for 0 <= x <= 2^-10 by its Taylor series (degree 5: the next term,
// x^6/720, is below 2^-69 relative), or degree 2 for x <= 1e-6 (x^3/6 below
// 2^-62).  Written from the series; callers fall back to exp() beyond.
__device__ __forceinline__ double exp_neg_small(double x, int degree) {
    if (degree == 2) return fma(x, fma(x, 0.5, -1.0), 1.0);
    double p = fma(x, -1.0 / 120.0, 1.0 / 24.0);
    p = fma(x, p, -1.0 / 6.0);
    p = fma(x, p, 0.5);
    p = fma(x, p, -1.0);
    return fma(x, p, 1.0);
}

// Kahan-compensated FP32 sum (the gathers of the mixed form with the FP64 update).
struct AccKahan {
    float s, c;  // sum and (negated) lost low part: value = s - c
    __device__ __forceinline__ void reset() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float v) {
        float y = __fsub_rn(v, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

template <int PREC> struct PrecTraits;
template <> struct PrecTraits<kPrecFP64> {
    using real = double;
};
template <> struct PrecTraits<kPrecMixed> {
    using real = float;
};
template <> struct PrecTraits<kPrecMixed64> {
    using real = float;
};

// ---------------------------------------------------------------------------
// leader-only: set up the next attempt (clipped dt, profile factor at t)
// ---------------------------------------------------------------------------
template <int PREC>
__device__ __forceinline__ void leader_prepare(GroupState& S, const PlanDev& P, const OptsDev& O) {
    if (S.done) return;
    const int zg = P.zone_base + S.zone;
    if (O.replay_dt) {
        if (S.steps >= O.replay_len[zg]) {
            S.done = 1;
            return;
        }
        const double h = O.replay_dt[O.replay_off[zg] + S.steps];
        S.clipped = h >= S.t_end - S.t;
        S.h = h;
    } else {
        if (!(S.t < S.t_end)) {
            S.done = 1;
            return;
        }
        if (S.steps >= O.max_steps) {
            S.status = 1;  // STEP_LIMIT
            S.done = 1;
            return;
        }
        const double rem = S.t_end - S.t;
        S.clipped = S.dt >= rem;
        S.h = S.clipped ? rem : S.dt;
    }
    if (!S.rhs_valid && !S.constant) {
        // k_j(t) = K_j exp(-c_j s), s = t / tau: T9 = T0 e^{-s}, rho = rho0 e^{-3s}
        const double s = S.t * S.inv_tau;
        S.s = s;
        if (PREC != kPrecFP64) {
            S.u = __fmul_rn(__double2float_rn(S.t), S.u_scale);
        } else {
            const double xm = P.cmax * s;
            S.poly = xm <= 1e-6 ? 2 : (xm <= 0.0009765625 ? 5 : 9);
        }
    }
}

// ---------------------------------------------------------------------------
// one zone group: fetch zones until the queue is empty
// ---------------------------------------------------------------------------
struct GroupPtrs {
    const void* A;  // real[N]
    const uint32_t* rspec;  // reactants a | b << 10 | c << 20 (N = none)
    const void* cexp;
    const uint16_t* wsl;
    const uint2* shdr;
    const uint16_t* sdst;
    const uint16_t* sidx;
    unsigned char* gbase;
    void* V;
    void* K;
    float* Kc;  // FP32-flux forms: the rates at u_ref
    double* Y64;  // FP64 form: the abundances
    float* Ylo;   // mixed form: low parts of the float-float abundances (high parts: Y32)
    float* Y32;
    void* Fk;
    void* Fk2;  // QSS: (F+, k) pairs of the predicted state
    double* red_c;
    double* red_n;
    double* red_d;
    float* red_r;
    int* red_f;
    float* feat;  // [64] features, [64] normalised inputs, [128] h1, [128] h2
    int* hist;    // [3][64] + [4] counters
};

// ---------------------------------------------------------------------------
// The explicit quasi-steady-state update (Sec. 11 proposes it as the
// alternative to Eq. 3; its formula is the alpha-QSS predictor-corrector of
// Mott, Oran & van Leer, J. Comput. Phys. 164 (2000) 407).  FP64 and mixed forms.
// ---------------------------------------------------------------------------

// alpha(x), x = k dt >= 0, is the rational approximation
// N/D = (180 r^3 + 60 r^2 + 11 r + 1) / (360 r^3 + 60 r^2 + 12 r + 1), r = 1/x,
// of 1/(1 - e^-x) - 1/x, the alpha that makes the step exact for constant F+
// and k; times x^3, N = x^3 + 11 x^2 + 60 x + 180, D = x^3 + 12 x^2 + 60 x + 360
// and D - N = x^2 + 180.
//
// The scheme's update of one species is y + h (f - k y) / (1 + alpha(k h) k h),
// with f the production term (F+ in the predictor, the corrector's blend
// a F+p + (1 - a) F+).  As printed it is a difference of nearly equal terms
// once k h >> 1 (the result is about 12 y / (k h)^2 + f / k), which rounding
// would leave with a relative error of about eps (k h)^2 / 12; the same
// function is evaluated as (c0 y + c1 h f) / c2 from 1 + alpha x = (D + x N)/D
// and 1 - (1 - alpha) x = (D - x (D - N))/D:
//   c0 = 12 x^2 - 120 x + 360 (> 0 for every x), c1 = D,
//   c2 = D + x N = x^4 + 12 x^3 + 72 x^2 + 240 x + 360,
// so y, f >= 0 give a result >= 0.  In the corrector c1 h f = h (N F+p +
// (D - N) F+): the blend's denominator cancels and each update costs one
// division.  Up to x = 2^100 these polynomials in x cannot overflow; above,
// the same functions are taken in powers of r = 1/x (divided through by x^4).
constexpr double kQssXMax = 1.2676506002282294e30;  // 2^100

__device__ __forceinline__ void qss_coeffs_x(double x, double& c0, double& c2) {
    c0 = fma(fma(12.0, x, -120.0), x, 360.0);
    c2 = fma(fma(fma(x + 12.0, x, 72.0), x, 240.0), x, 360.0);
}

// The predictor's update, production f.
__device__ __forceinline__ double qss_update1(double y, double f, double k, double h) {
    const double x = k * h;
    if (x <= kQssXMax) {
        double c0, c2;
        qss_coeffs_x(x, c0, c2);
        const double c1 = fma(fma(x + 12.0, x, 60.0), x, 360.0);
        return fma(c0, y, c1 * (h * f)) / c2;
    }
    const double r = 1.0 / x;
    const double c0 = fma(fma(360.0, r, -120.0), r, 12.0) * (r * r);
    const double c1 = fma(fma(fma(360.0, r, 60.0), r, 12.0), r, 1.0) * r;
    const double c2 = fma(fma(fma(fma(360.0, r, 240.0), r, 72.0), r, 12.0), r, 1.0);
    return fma(c0, y, c1 * (h * f)) / c2;
}

// The corrector's update: kbar, the predicted state's F+p and the current
// state's F+ (f0).
__device__ __forceinline__ double qss_correct1(double y, double fp, double f0, double kbar, double h) {
    const double x = kbar * h;
    if (x <= kQssXMax) {
        double c0, c2;
        qss_coeffs_x(x, c0, c2);
        const double n = fma(fma(x + 11.0, x, 60.0), x, 180.0);
        const double dn = fma(x, x, 180.0);
        return fma(c0, y, h * fma(n, fp, dn * f0)) / c2;
    }
    // weights a = N/D and 1 - a = (D - N)/D in powers of r, then the update
    const double r = 1.0 / x;
    const double n = fma(fma(fma(180.0, r, 60.0), r, 11.0), r, 1.0);
    const double d = fma(fma(fma(360.0, r, 60.0), r, 12.0), r, 1.0);
    const double dn = r * fma(180.0 * r, r, 1.0);
    return qss_update1(y, fma(n, fp, dn * f0) / d, kbar, h);
}

// Predictor: Yp = Y + h (F+ - k Y) / (1 + alpha(k h) k h) from buffer cur into
// nxt, with (F+, k) of the current state.  No barrier inside.
__device__ __forceinline__ void qss_predict(const PlanDev& P, const GroupPtrs& g, int lane, int cur, double h) {
    const int N = P.N, G = P.G, NP1 = N + 1;
    const double* Fk = (const double*)g.Fk;
    const double* Yc = g.Y64 + cur * NP1;
    double* Yp = g.Y64 + (cur ^ 1) * NP1;
    for (int i = lane; i < N; i += G) Yp[i] = qss_update1(Yc[i], Fk[2 * i], Fk[2 * i + 1], h);
}

// FP32 versions for the mixed form.  In powers of r = 1/x above x = 1 the
// c1 h f term is written (c1 / r) (f / k), since h r = 1/k: nothing then
// overflows or underflows before the result does (x up to FLT_MAX).  The
// denominators d and c2 lie in [1, 685], so the approximate division
// __fdividef (2 ulp) is exact enough; f / k and 1/x use the correctly rounded
// division and reciprocal.
__device__ __forceinline__ void qss_weights32(float x, float& a, float& b) {
    float n, d, dn;
    if (x <= 1.f) {
        n = fmaf(fmaf(x + 11.f, x, 60.f), x, 180.f);
        d = fmaf(fmaf(x + 12.f, x, 60.f), x, 360.f);
        dn = fmaf(x, x, 180.f);
    } else {
        const float r = __frcp_rn(x);
        n = fmaf(fmaf(fmaf(180.f, r, 60.f), r, 11.f), r, 1.f);
        d = fmaf(fmaf(fmaf(360.f, r, 60.f), r, 12.f), r, 1.f);
        dn = r * fmaf(180.f * r, r, 1.f);
    }
    a = __fdividef(n, d);
    b = __fdividef(dn, d);
}

__device__ __forceinline__ float qss_update1_32(float y, float f, float k, float h) {
    const float x = __fmul_rn(k, h);
    if (x <= 1.f) {
        const float c0 = fmaf(fmaf(12.f, x, -120.f), x, 360.f);
        const float c1 = fmaf(fmaf(x + 12.f, x, 60.f), x, 360.f);
        const float c2 = fmaf(fmaf(fmaf(x + 12.f, x, 72.f), x, 240.f), x, 360.f);
        return __fdividef(fmaf(c0, y, c1 * __fmul_rn(h, f)), c2);
    }
    const float r = __frcp_rn(x);
    const float c0 = fmaf(fmaf(360.f, r, -120.f), r, 12.f) * __fmul_rn(r, r);
    const float c1r = fmaf(fmaf(fmaf(360.f, r, 60.f), r, 12.f), r, 1.f);  // c1 / r
    const float c2 = fmaf(fmaf(fmaf(fmaf(360.f, r, 240.f), r, 72.f), r, 12.f), r, 1.f);
    return __fdividef(fmaf(c0, y, c1r * __fdiv_rn(f, k)), c2);
}

// Mixed form predictor: the FP32 copy of Yp (all the predicted state's flux
// pass reads) into buffer nxt, from the high parts of the current pairs.
__device__ __forceinline__ void qss_predict_mixed(const PlanDev& P, const GroupPtrs& g, int lane, int cur,
                                                  float h32) {
    const int N = P.N, G = P.G, NP1 = N + 1;
    const float2* Fk = (const float2*)g.Fk;
    const float* Yh = g.Y32 + cur * NP1;
    float* Yp = g.Y32 + (cur ^ 1) * NP1;
    for (int i = lane; i < N; i += G) {
        const float2 fk = Fk[i];
        Yp[i] = qss_update1_32(Yh[i], fk.x, fk.y, h32);
    }
}

// Warps of a group that hold species (species i goes to lane i mod G): a warp
// whose first lane is at or past N has none, skips the update and its
// reductions, and is left out of the combine.
__device__ __forceinline__ int species_warps(const PlanDev& P) { return (min(P.G, P.N) + 31) >> 5; }

// (d) the update with step h from buffer cur into nxt, and each warp's share
// of the error measures (no barrier inside).  FP64 form: every step in FP64,
// in the order of the definitions.  QSS = false: the kappa-switched update
// (Sec. 3, Eq. 3).  QSS = true: the alpha-QSS corrector from the current
// state's (F+, k) and the predicted state's (F+p, kp) in Fk2:
//   kbar = (k + kp)/2, a = alpha(kbar h),
//   Y' = Y + h (a F+p + (1 - a) F+ - kbar Y) / (1 + a kbar h).
template <bool QSS>
__device__ __forceinline__ void update_reduce_fp64(const PlanDev& P, const OptsDev& O, const GroupPtrs& g, int lane,
                                                   int cur, double h, int z) {
    if ((lane & ~31) >= P.N) return;  // a warp without species
    const int N = P.N, G = P.G, NP1 = N + 1;
    const double* Fk = (const double*)g.Fk;
    const double* Fk2 = (const double*)g.Fk2;
    const double* A = (const double*)g.A;
    const double* Yc = g.Y64 + cur * NP1;
    double* Yn64 = g.Y64 + (cur ^ 1) * NP1;
    const double kappa = O.kappa, ymin = O.y_min;
    double csum = 0.0, bn = 0.0, bd = 1.0;
    for (int i = lane; i < N; i += G) {
        const double y = Yc[i], fp = Fk[2 * i], kk = Fk[2 * i + 1];
        double yn;
        if (QSS) {
            yn = qss_correct1(y, Fk2[2 * i], fp, 0.5 * (kk + Fk2[2 * i + 1]), h);
        } else {
            const double kdt = kk * h;
            yn = (kdt >= kappa) ? (y + h * fp) / (1.0 + kdt) : y + h * (fp - kk * y);
        }
        Yn64[i] = yn;
        const double d = yn - y;
        csum = fma(A[i], d, csum);
        if ((y > yn ? y : yn) > ymin) {
            const double m = y > yn ? y : yn;
            const double ad = fabs(d);
            if (ad * bd > bn * m) {
                bn = ad;
                bd = m;
            }
        }
        if (O.probe) {
            O.probe_Fp[(size_t)z * N + i] = fp;
            O.probe_k[(size_t)z * N + i] = kk;
            O.probe_Y1[(size_t)z * N + i] = yn;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        csum += __shfl_xor_sync(0xffffffffu, csum, off);
        const double on = __shfl_xor_sync(0xffffffffu, bn, off);
        const double od = __shfl_xor_sync(0xffffffffu, bd, off);
        if (on * bd > bn * od) {
            bn = on;
            bd = od;
        }
    }
    if ((lane & 31) == 0) {
        const int w = lane >> 5;
        g.red_c[w] = csum;
        g.red_n[w] = bn;
        g.red_d[w] = bd;
    }
}

// Knuth's TwoSum (TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact rounding
// error e = (a + b) - s, for any a, b (no ordering condition).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// Mixed form.  The abundances are float-float pairs y = yh + yl (|yl| at most
// half an ulp of yh, so yh is the FP32 copy the flux pass reads; about 48
// significant bits), and the update runs in FP32, the precision F+ and k
// arrive in: on the asymptotic branch y' itself (relative accuracy,
// positivity), on the explicit branch the change dt (F+ - k y), added to the
// pair exactly up to one rounding of the low part.  The conservation sum
// sum A (y' - y) is a float-float sum of exact products, so it resolves the
// stored change far below eps_c; no FP64 instruction runs per species.
// QSS: the alpha-QSS corrector in place of Eq. 3 (F+p, kp of the predicted
// state in Fk2).  Up to k h = 1 its change h (f~ - kbar y)/(1 + a k h) is added
// to the pair as on Eq. 3's explicit branch; above, y' itself is computed in
// the form without cancellation, as on Eq. 3's asymptotic branch.
template <bool QSS>
__device__ __forceinline__ void update_reduce_mixed(const PlanDev& P, const OptsDev& O, const GroupPtrs& g, int lane,
                                                    int cur, float h32, int z) {
    if ((lane & ~31) >= P.N) return;  // a warp without species
    const int N = P.N, G = P.G, NP1 = N + 1;
    const float2* Fk = (const float2*)g.Fk;    // (F+_i, k_i)
    const float2* Fk2 = (const float2*)g.Fk2;  // the same for the QSS predicted state
    const float* A = (const float*)g.A;
    const float* Yh = g.Y32 + cur * NP1;
    const float* Yl = g.Ylo + cur * NP1;
    float* Nh = g.Y32 + (cur ^ 1) * NP1;
    float* Nl = g.Ylo + (cur ^ 1) * NP1;
    float cs_h = 0.f, cs_l = 0.f, rmax = 0.f;
    int ok = 1;
    // species i; FIRST: the lane's first species starts the sums
    auto body = [&](int i, auto first) {
        const float2 fk = Fk[i];
        const float yh = Yh[i], yl = Yl[i], fp = fk.x, kk = fk.y;
        const float kdt = __fmul_rn(kk, h32);
        float nh, nl, dh, dl;
        if (QSS) {
            const float2 fkp = Fk2[i];
            const float kbar = 0.5f * (kk + fkp.y);
            const float x = __fmul_rn(kbar, h32);
            float a, b;
            qss_weights32(x, a, b);
            const float ft = fmaf(a, fkp.x, b * fp);
            if (x <= 1.f) {
                dh = __fdividef(__fmul_rn(h32, fmaf(-kbar, yh, ft)), fmaf(a, x, 1.f));
                dl = 0.f;
                float s, e;
                two_sum(yh, dh, s, e);
                two_sum(s, __fadd_rn(e, yl), nh, nl);
            } else {
                nh = qss_update1_32(yh, ft, kbar, h32);
                nl = 0.f;
                two_sum(nh, -yh, dh, dl);
                dl = __fsub_rn(dl, yl);
            }
        } else if (kdt >= O.kappa32) {
            // 1 + k dt >= 2; __fdividef is within 2 ulp below 2^126 and gives
            // 0 above it (an abundance below 2^-126 of y + dt F+)
            nh = __fdividef(fmaf(h32, fp, yh), __fadd_rn(1.f, kdt));
            nl = 0.f;
            two_sum(nh, -yh, dh, dl);
            dl = __fsub_rn(dl, yl);
        } else {
            dh = __fmul_rn(h32, fmaf(-kk, yh, fp));
            dl = 0.f;
            float s, e;
            two_sum(yh, dh, s, e);
            two_sum(s, __fadd_rn(e, yl), nh, nl);
        }
        Nh[i] = nh;
        Nl[i] = nl;
        // A (dh + dl): the product a dh split exactly by an FMA
        const float a = A[i];
        const float p = __fmul_rn(a, dh);
        const float pe = fmaf(a, dh, -p);
        if (decltype(first)::value) {
            cs_h = p;
            cs_l = fmaf(a, dl, pe);
        } else {
            float s, e;
            two_sum(cs_h, p, s, e);
            cs_h = s;
            cs_l = __fadd_rn(cs_l, __fadd_rn(e, fmaf(a, dl, pe)));
        }
        // The accept test's decisions are those of the compares m > y_min
        // and |d| <= eps_r m on the pairs; they are taken on the high parts
        // when those lie clearly on one side (outside a guard band that
        // bounds their rounding and the ratio's division), and on the pairs
        // in FP64 inside the band.
        const float m32 = fmaxf(yh, nh);
        int tested;
        if (m32 > O.ymin_hi32) tested = 1;
        else if (m32 < O.ymin_lo32) tested = 0;
        else tested = fmax((double)yh + (double)yl, (double)nh + (double)nl) > O.y_min;
        if (tested) {
            const float r = __fdividef(fabsf(__fsub_rn(nh, yh)), m32);
            int pass_i;
            if (r < O.thr_lo32) {
                pass_i = 1;
            } else if (r > O.thr_hi32) {
                pass_i = 0;
            } else {
                const double y = (double)yh + (double)yl, yn = (double)nh + (double)nl;
                pass_i = fabs(yn - y) <= O.eps_r * (y > yn ? y : yn);
            }
            ok &= pass_i;
            rmax = fmaxf(rmax, r);  // the dt proposal, FP32
        }
        if (O.probe) {
            O.probe_Fp[(size_t)z * N + i] = (double)fp;
            O.probe_k[(size_t)z * N + i] = (double)kk;
            O.probe_Y1[(size_t)z * N + i] = (double)nh + (double)nl;
        }
    };
    if (lane < N) body(lane, std::true_type{});
    for (int i = lane + G; i < N; i += G) body(i, std::false_type{});
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, cs_h, off);
        const float ol = __shfl_xor_sync(0xffffffffu, cs_l, off);
        float s, e;
        two_sum(cs_h, oh, s, e);
        cs_h = s;
        cs_l = __fadd_rn(__fadd_rn(cs_l, ol), e);
    }
    // rmax >= 0, so its bit pattern orders as an unsigned integer
    const unsigned int rbits = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));
    ok = __all_sync(0xffffffffu, ok);
    if ((lane & 31) == 0) {
        const int w = lane >> 5;
        ((float2*)g.red_c)[w] = make_float2(cs_h, cs_l);
        g.red_r[w] = __uint_as_float(rbits);
        g.red_f[w] = ok;
    }
}

// Mixed form with the FP64 update: F+ and k arrive from the Kahan-compensated
// FP32 gathers and are widened; the kappa-switched update runs in FP64 on FP64
// abundances (an FP32 copy of y' is kept for the FP32 flux pass), and the
// conservation sum sum A (y' - y) is an FP64 sum.  The relative test's
// decisions are those of the FP64 compares max(y, y') > y_min and
// |y' - y| <= eps_r max(y, y'): taken on the FP32 copies when these lie
// outside a guard band that bounds the copies' rounding and the ratio's
// division (as in the mixed form), and in FP64 inside it.  Per warp the
// reductions carry the FP64 sum, an all-pass flag and the FP32 maximum ratio
// (the step proposal), so no FP64 compare or product runs in them.
__device__ __forceinline__ void update_reduce_mixed64(const PlanDev& P, const OptsDev& O, const GroupPtrs& g,
                                                      int lane, int cur, double h, int z) {
    if ((lane & ~31) >= P.N) return;  // a warp without species
    const int N = P.N, G = P.G, NP1 = N + 1;
    const float2* Fk = (const float2*)g.Fk;  // (F+_i, k_i)
    const double* A = (const double*)g.A;
    const double* Yc = g.Y64 + cur * NP1;
    const float* Yc32 = g.Y32 + cur * NP1;
    double* Yn64 = g.Y64 + (cur ^ 1) * NP1;
    float* Yn32 = g.Y32 + (cur ^ 1) * NP1;
    const double kappa = O.kappa;
    double csum = 0.0;
    float rmax = 0.f;
    int ok = 1;
    for (int i = lane; i < N; i += G) {
        const float2 fk = Fk[i];
        const double y = Yc[i], fp = (double)fk.x, kk = (double)fk.y;
        const double kdt = kk * h;
        const double yn = (kdt >= kappa) ? (y + h * fp) / (1.0 + kdt) : y + h * (fp - kk * y);
        const float yn32 = (float)yn;
        Yn64[i] = yn;
        Yn32[i] = yn32;
        const double d = yn - y;
        csum = fma(A[i], d, csum);
        // y32 = fl32(y) and yn32 = fl32(y'): each within 2^-24 relative, so the
        // band of set_guard_band covers their difference and the ratio
        const float y32 = Yc32[i];
        const float m32 = fmaxf(y32, yn32);
        int tested;
        if (m32 > O.ymin_hi32) tested = 1;
        else if (m32 < O.ymin_lo32) tested = 0;
        else tested = (y > yn ? y : yn) > O.y_min;
        if (tested) {
            const float r = __fdividef(fabsf(__fsub_rn(yn32, y32)), m32);
            int pass_i;
            if (r < O.thr_lo32) pass_i = 1;
            else if (r > O.thr_hi32) pass_i = 0;
            else pass_i = fabs(d) <= O.eps_r * (y > yn ? y : yn);
            ok &= pass_i;
            rmax = fmaxf(rmax, r);
        }
        if (O.probe) {
            O.probe_Fp[(size_t)z * N + i] = fp;
            O.probe_k[(size_t)z * N + i] = kk;
            O.probe_Y1[(size_t)z * N + i] = yn;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) csum += __shfl_xor_sync(0xffffffffu, csum, off);
    const unsigned int rbits = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));
    ok = __all_sync(0xffffffffu, ok);
    if ((lane & 31) == 0) {
        const int w = lane >> 5;
        g.red_c[w] = csum;
        g.red_r[w] = __uint_as_float(rbits);
        g.red_f[w] = ok;
    }
}

// h: the step (FP64 forms); h32: the same step in FP32 (the mixed form's update);
// QSS: the alpha-QSS corrector instead of Eq. 3 (FP64 form)
template <int PREC, bool QSS = false>
__device__ __forceinline__ void update_reduce(const PlanDev& P, const OptsDev& O, const GroupPtrs& g, int lane,
                                              int cur, double h, float h32, int z) {
    if (PREC == kPrecMixed)
        update_reduce_mixed<QSS>(P, O, g, lane, cur, h32, z);
    else if (PREC == kPrecMixed64)
        update_reduce_mixed64(P, O, g, lane, cur, h, z);
    else
        update_reduce_fp64<QSS>(P, O, g, lane, cur, h, z);
}

// lane 0, after the barrier that follows update_reduce: combine the warps.
// A non-finite abundance makes the conservation sum non-finite, so the
// finiteness test reads that sum.
struct TestOutcome {
    double cons, bn, bd;
    float rmax, cons32;
    int fin, pass;
};
template <int PREC>
__device__ __forceinline__ TestOutcome combine(const PlanDev& P, const OptsDev& O, const GroupPtrs& g) {
    const int nw = species_warps(P);
    TestOutcome v{0.0, 0.0, 1.0, 0.f, 0.f, 1, 0};
    if (PREC == kPrecMixed) {
        float ch = 0.f, cl = 0.f;
        int ok = 1;
        for (int w = 0; w < nw; ++w) {
            const float2 c = ((const float2*)g.red_c)[w];
            float s, e;
            two_sum(ch, c.x, s, e);
            ch = s;
            cl = __fadd_rn(__fadd_rn(cl, c.y), e);
            v.rmax = fmaxf(v.rmax, g.red_r[w]);
            ok &= g.red_f[w];
        }
        const float cs = __fadd_rn(ch, cl);
        v.fin = isfinite(cs) ? 1 : 0;
        v.cons32 = fabsf(cs);
        v.pass = v.fin && ok && v.cons32 <= O.eps_c32;
    } else if (PREC == kPrecMixed64) {
        double cs = 0.0;
        int ok = 1;
        for (int w = 0; w < nw; ++w) {
            cs += g.red_c[w];
            v.rmax = fmaxf(v.rmax, g.red_r[w]);
            ok &= g.red_f[w];
        }
        v.fin = isfinite(cs) ? 1 : 0;
        v.cons = fabs(cs);
        v.cons32 = (float)v.cons;
        v.pass = v.fin && ok && v.cons <= O.eps_c;
    } else {
        double cs = 0.0;
        for (int w = 0; w < nw; ++w) {
            cs += g.red_c[w];
            const double on = g.red_n[w], od = g.red_d[w];
            if (on * v.bd > v.bn * od) {
                v.bn = on;
                v.bd = od;
            }
        }
        v.fin = isfinite(cs) ? 1 : 0;
        v.cons = fabs(cs);
        v.pass = v.fin && v.cons <= O.eps_c && v.bn <= O.eps_r * v.bd;
    }
    return v;
}

// lane 0, mixed form, plain integration (no probe, no replay): accept or
// reject the attempt just tested and set up the next one.  The step sizes are
// FP32 (the mixed update takes h in FP32 anyway) and the time axis FP64.  The
// FP64 work that does not depend on the outcome -- the time an accept would
// reach, the remaining interval after an accept or a reject, the profile
// factor there -- is issued before the warp combine so that its latency
// overlaps it; after the combine the chain to the next step is FP32 only.
// Clipping to t_end compares in FP32; a step that an FP32 compare leaves a
// hair past t_end ends the zone at t_end all the same.
template <bool FEAT>
__device__ __forceinline__ void decide_mixed(GroupState& S, const PlanDev& P, const OptsDev& O, const GroupPtrs& g,
                                             int nxt, bool spec) {
    const float h32 = S.h32;
    const double t = S.t, te = S.t_end;
    const int was_clipped = S.clipped;
    const double t_acc = was_clipped ? te : t + (double)h32;
    const float rem_acc = (float)(te - t_acc);
    const float rem_cur = (float)(te - t);
    const float u_acc = S.constant ? 0.f : __fmul_rn(__double2float_rn(t_acc), S.u_scale);
    if (spec && S.refresh_spec) S.u_ref = S.u_spec;  // the speculative pass refreshed Kc
    const TestOutcome v = combine<kPrecMixed>(P, O, g);
    if (v.pass) {
        const float ga = __fdiv_rn(O.ga32, fmaxf(v.rmax, 1e-30f));
        const float gb = __fdiv_rn(O.gb32, fmaxf(v.cons32, 1e-30f));
        const float dt = __fmul_rn(h32, fminf(O.grow32, fminf(ga, gb)));
        S.dt32 = dt;
        S.dtp32 = dt;
        S.cur = nxt;
        S.steps += 1;
        S.nrej = 0;
        S.rhs_valid = 0;
        if (FEAT) {
            if (S.mlp_try) S.props += 1;
            S.mlp_try = 0;
            S.h_prev = (double)h32;
            S.dt_plain = (double)dt;
            S.fresh = 1;
        }
        if (was_clipped || !(t_acc < te)) {
            S.t = te;
            S.done = 1;
        } else {
            S.t = t_acc;
            S.u = u_acc;
            if (S.steps >= O.max_steps) {
                S.status = 1;  // STEP_LIMIT
                S.done = 1;
            } else {
                const int c = dt >= rem_acc;
                S.clipped = c;
                S.h32 = c ? rem_acc : dt;
            }
        }
    } else {
        S.rejects += 1;
        S.rhs_valid = 1;
        float dt;
        if (FEAT && S.mlp_try) {
            // a rejected learned proposal: retry with the plain controller's dt
            S.mlp_try = 0;
            dt = S.dtp32;
        } else {
            S.nrej += 1;
            dt = __fmul_rn(h32, O.shrink32);
            if (S.nrej > O.max_reject) {
                S.status = v.fin ? 4 : 3;  // MAX_REJECT : NONFINITE
                S.done = 1;
            } else if ((double)dt < O.dt_min_frac * t) {
                S.status = 2;  // DT_UNDERFLOW
                S.done = 1;
            }
        }
        S.dt32 = dt;
        const int c = dt >= rem_cur;
        S.clipped = c;
        S.h32 = c ? rem_cur : dt;
    }
}

// FP32 exponent histogram bin (4 octaves per bin, values below 2^-100 in bin 0)
__device__ __forceinline__ int exp_bin(float x) {
    const unsigned int b = __float_as_uint(x);
    const int ef = (int)((b >> 23) & 0xffu);
    if (ef == 0) return 0;  // zero or subnormal
    const int bin = (ef - 127 + 100) >> 2;
    return bin < 0 ? 0 : (bin > 63 ? 63 : bin);
}

__constant__ float kQuantileP[20] = {0.025f, 0.075f, 0.125f, 0.175f, 0.225f, 0.275f, 0.325f,
                                     0.375f, 0.425f, 0.475f, 0.525f, 0.575f, 0.625f, 0.675f,
                                     0.725f, 0.775f, 0.825f, 0.875f, 0.925f, 0.975f};

// The 64 features of the current state (group-wide; barriers inside):
// ln T9, ln rho, ln dt_prev, the fraction of species with k dt_prev >= kappa,
// and 20 quantiles each of Y, F+ and F- = k Y from FP32 exponent histograms.
template <int PREC>
__device__ void compute_features(const PlanDev& P, const OptsDev& O, const GroupPtrs& g, GroupState& S, int lane,
                                 int cur, const GroupSync& gs) {
    using real = typename PrecTraits<PREC>::real;
    const int N = P.N, G = P.G, NP1 = N + 1;
    const real* Fk = (const real*)g.Fk;
    for (int i = lane; i < 3 * 64 + 4; i += G) g.hist[i] = 0;
    gs.sync();
    const double hp = S.h_prev, kappa = O.kappa;
    for (int i0 = 0; i0 < N; i0 += G) {
        const int i = i0 + lane;
        int asy = 0;
        if (i < N) {
            const float y32 = PREC != kPrecFP64 ? g.Y32[cur * NP1 + i] : (float)g.Y64[cur * NP1 + i];
            const float fp = (float)Fk[2 * i], kk = (float)Fk[2 * i + 1];
            atomicAdd(&g.hist[exp_bin(y32)], 1);
            atomicAdd(&g.hist[64 + exp_bin(fp)], 1);
            atomicAdd(&g.hist[128 + exp_bin(__fmul_rn(kk, y32))], 1);
            asy = (double)Fk[2 * i + 1] * hp >= kappa;
        }
        const unsigned int bal = __ballot_sync(0xffffffffu, asy);
        if ((lane & 31) == 0 && bal) atomicAdd(&g.hist[192], __popc(bal));
    }
    gs.sync();
    for (int j = lane; j < 61; j += G) {
        if (j < 60) {
            const int q = j / 20, m = j - q * 20;
            const int* h = g.hist + 64 * q;
            const float target = __fmul_rn(kQuantileP[m], (float)N);
            int cum = 0;
            float val = 64.f;
            for (int b = 0; b < 64; ++b) {
                const int c = h[b];
                if (c > 0 && (float)(cum + c) > target) {
                    val = __fadd_rn((float)b, __fdiv_rn(__fsub_rn(target, (float)cum), (float)c));
                    break;
                }
                cum += c;
            }
            g.feat[4 + j] = __fmul_rn(__fsub_rn(__fmul_rn(val, 4.f), 100.f), 0.30102999566398120f);
        } else {
            g.feat[0] = (float)(S.lnT0 - S.s);
            g.feat[1] = (float)(S.lnR0 - 3.0 * S.s);
            g.feat[2] = logf((float)hp);
            g.feat[3] = __fdiv_rn((float)g.hist[192], (float)N);
        }
    }
    gs.sync();
}

// lane 0: append (features, label) to the record buffer
__device__ __forceinline__ void write_record(const OptsDev& O, const GroupPtrs& g, float label) {
    const unsigned long long slot = atomicAdd(O.rec_count, 1ull);
    if ((long long)slot < O.rec_cap) {
        float* f = O.rec_feat + slot * 64;
        for (int k = 0; k < 64; ++k) f[k] = g.feat[k];
        O.rec_label[slot] = label;
    }
}

// The network on the group's threads (CUDA cores; one row): BF16 weights
// staged in shared memory, FP32 accumulation, BF16 activations; returns the
// network output on lane 0.
__device__ float mlp_forward_group(const OptsDev& O, const GroupPtrs& g, const unsigned char* mlp_smem, int lane,
                                   int G, const GroupSync& gs) {
    const __nv_bfloat16* W1 = (const __nv_bfloat16*)mlp_smem;              // [64][128]
    const __nv_bfloat16* W2 = W1 + 64 * 128;                                // [128][128]
    const float* Pb = (const float*)(W2 + 128 * 128);                       // b1 [128], b2 [128], w3 [128], b3
    const float* nrm = Pb + 3 * 128 + 4;                                    // mu [64], 1/sigma [64]
    float* x = g.feat + 64;
    float* h1 = g.feat + 128;
    float* h2 = g.feat + 256;
    for (int k = lane; k < 64; k += G) x[k] = __bfloat162float(__float2bfloat16((g.feat[k] - nrm[k]) * nrm[64 + k]));
    gs.sync();
    for (int n = lane; n < 128; n += G) {
        float acc = Pb[n];
        for (int k = 0; k < 64; ++k) acc = fmaf(x[k], __bfloat162float(W1[k * 128 + n]), acc);
        h1[n] = __bfloat162float(__float2bfloat16(acc > 0.f ? acc : 0.f));
    }
    gs.sync();
    for (int n = lane; n < 128; n += G) {
        float acc = Pb[128 + n];
        for (int k = 0; k < 128; ++k) acc = fmaf(h1[k], __bfloat162float(W2[k * 128 + n]), acc);
        h2[n] = __bfloat162float(__float2bfloat16(acc > 0.f ? acc : 0.f));
    }
    gs.sync();
    float s = 0.f;
    if (lane < 32) {
        for (int n = lane; n < 128; n += 32) s = fmaf(h2[n], Pb[256 + n], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    }
    return s + Pb[384];
}

// FP32-flux forms, one reactant-count class of the sorted reactions:
// reactions j, j + stride, ... below j_end; returns the first index at or
// past j_end, where the next class continues.  The rates come from the
// group's cache Kc; REFRESH recomputes them, K_j 2^(-c_j u), and stores them
// to Kc when the plan keeps the cache (`store`).
// The flux goes to V[j] and partial q (the product of k_j and the other
// reactants' abundances) to plane q at Pq[j], so a warp's stores are
// contiguous.
template <bool REFRESH, int NB>
__device__ __forceinline__ int flux_class(int j, int j_end, int stride, const uint32_t* __restrict__ rspec,
                                          const float* __restrict__ cexp, const float* __restrict__ Kz,
                                          float* __restrict__ Kc, const float* __restrict__ Y,
                                          float* __restrict__ V, float* __restrict__ P0, float* __restrict__ P1,
                                          float* __restrict__ P2, float u, bool store) {
#pragma unroll 1
    for (; j < j_end; j += stride) {
        const uint32_t rs = rspec[j];
        float k;
        if (REFRESH) {
            k = __fmul_rn(Kz[j], ex2_approx(-__fmul_rn(cexp[j], u)));
            if (store) Kc[j] = k;
        } else {
            k = Kc[j];
        }
        const float ya = Y[rs & 1023u];
        if (NB == 1) {
            V[j] = __fmul_rn(k, ya);
            P0[j] = k;
        } else if (NB == 2) {
            const float yb = Y[(rs >> 10) & 1023u];
            V[j] = __fmul_rn(__fmul_rn(k, ya), yb);
            P0[j] = __fmul_rn(k, yb);
            P1[j] = __fmul_rn(k, ya);
        } else {
            const float yb = Y[(rs >> 10) & 1023u], yc = Y[rs >> 20];
            const float ka = __fmul_rn(k, ya);
            V[j] = __fmul_rn(__fmul_rn(ka, yb), yc);
            P0[j] = __fmul_rn(__fmul_rn(k, yb), yc);
            P1[j] = __fmul_rn(ka, yc);
            P2[j] = __fmul_rn(ka, yb);
        }
    }
    return j;
}

// (a) rates k_j(t), fluxes f_j and reactant-slot partials (Eq. 1) of the state
// in buffer `buf`, over reactions j0, j0 + stride, ...; reactions are sorted
// 1-, 2-, 3-body, so no multiply by an absent reactant.  s = t / tau (FP64
// form: poly selects the series for exp(-c_j s)); u = s / ln 2 (mixed form).
template <int PREC>
// refresh (FP32-flux forms): recompute the cached rates at u before use; each
// thread refreshes exactly the reactions it then reads, so no barrier is needed.
__device__ __forceinline__ void flux_pass(const PlanDev& P, const GroupPtrs& g, int j0, int stride, int buf,
                                          int constant, double s, float u, int poly, bool refresh) {
    using real = typename PrecTraits<PREC>::real;
    const int N = P.N, R = P.R, R1 = P.R1, R12 = P.R12, NP1 = N + 1;
    const uint32_t* __restrict__ rspec = g.rspec;
    const real* __restrict__ cexp = (const real*)g.cexp;
    const real* __restrict__ Kz = (const real*)g.K;
    real* __restrict__ Vw = (real*)g.V;
    const int pb1 = 2 * R - R1, pb2 = 3 * R - R1 - R12;  // bases of partial planes 1 and 2
    if (PREC == kPrecFP64) {
        const double* __restrict__ Yr = g.Y64 + buf * NP1;
#pragma unroll 2
        for (int j = j0; j < R; j += stride) {
            const uint32_t rs = rspec[j];
            double k = (double)Kz[j];
            if (poly == 2 || poly == 5)
                k *= exp_neg_small((double)cexp[j] * s, poly);
            else if (poly == 9)
                k *= exp(-(double)cexp[j] * s);
            const double ya = Yr[rs & 1023u];
            if (j < R1) {
                Vw[j] = (real)(k * ya);
                Vw[R + j] = (real)k;
            } else if (j < R12) {
                const double yb = Yr[(rs >> 10) & 1023u];
                Vw[j] = (real)(k * ya * yb);
                Vw[R + j] = (real)(k * yb);
                Vw[pb1 + j] = (real)(k * ya);
            } else {
                const double yb = Yr[(rs >> 10) & 1023u], yc = Yr[rs >> 20];
                const double ka = k * ya;
                Vw[j] = (real)(ka * yb * yc);
                Vw[R + j] = (real)(k * yb * yc);
                Vw[pb1 + j] = (real)(ka * yc);
                Vw[pb2 + j] = (real)(ka * yb);
            }
        }
    } else {
        const float* __restrict__ Yc32 = g.Y32 + buf * NP1;
        const float* __restrict__ cf = (const float*)g.cexp;
        const float* __restrict__ Kf = (const float*)g.K;
        float* __restrict__ Vf = (float*)g.V;
        float* __restrict__ Kc = g.Kc;
        float* P0 = Vf + R;
        float* P1 = Vf + pb1;
        float* P2 = Vf + pb2;
        if (refresh) {
            int j = flux_class<true, 1>(j0, R1, stride, rspec, cf, Kf, Kc, Yc32, Vf, P0, P1, P2, u, P.rate_cache != 0);
            j = flux_class<true, 2>(j, R12, stride, rspec, cf, Kf, Kc, Yc32, Vf, P0, P1, P2, u, P.rate_cache != 0);
            flux_class<true, 3>(j, R, stride, rspec, cf, Kf, Kc, Yc32, Vf, P0, P1, P2, u, P.rate_cache != 0);
        } else {
            int j = flux_class<false, 1>(j0, R1, stride, rspec, cf, Kf, Kc, Yc32, Vf, P0, P1, P2, u, P.rate_cache != 0);
            j = flux_class<false, 2>(j, R12, stride, rspec, cf, Kf, Kc, Yc32, Vf, P0, P1, P2, u, P.rate_cache != 0);
            flux_class<false, 3>(j, R, stride, rspec, cf, Kf, Kc, Yc32, Vf, P0, P1, P2, u, P.rate_cache != 0);
        }
    }
}

// (b) sliced gathers of the row sums F+_i and k_i into the (F+, k) pairs at
// Fb: warp w sums its slices, one row piece per lane; the pieces of a split
// row (consecutive lanes, same destination) are added by a segmented
// reduction into the first one.  FP64 form: FP64 sums.  Mixed form: plain
// FP32 sums -- every term of a row is positive, so a row of k pieces of at
// most L terms is within (L - 1 + ceil(log2 k)) 2^-24 of its value, relative.
// Mixed form with the FP64 update: Kahan-compensated FP32 sums, and the
// pieces' (sum, compensation) pairs added with TwoSum.  Padding lanes store
// to the spare slot after the pairs.  No barrier inside.
template <int PREC>
__device__ __forceinline__ void gather_pass(const PlanDev& P, const GroupPtrs& g, int lane, unsigned char* Fb_) {
    using real = typename PrecTraits<PREC>::real;
    const real* V = (const real*)g.V;
    const int w = lane >> 5, l = lane & 31;
    const int s1 = g.wsl[w + 1];
    const bool boff = P.tl.sidx_bytes != 0;
    unsigned char* __restrict__ Fb = Fb_;
    const real* __restrict__ Vr = V;
    for (int sl = g.wsl[w]; sl < s1; ++sl) {
        const uint2 hd = g.shdr[sl];
        const uint16_t* __restrict__ ix = g.sidx + hd.x + l;
        const int len = (int)(hd.y & 0x7fffffffu);
        const unsigned int d = g.sdst[32 * sl + l];
        if (PREC == kPrecMixed64) {
            AccKahan ak;
            ak.reset();
            if (boff) {
                const unsigned char* __restrict__ Vb = (const unsigned char*)Vr;
#pragma unroll 4
                for (int k = 0; k < len; ++k) ak.add((float)*(const real*)(Vb + ix[32 * k]));
            } else {
#pragma unroll 4
                for (int k = 0; k < len; ++k) ak.add((float)Vr[ix[32 * k]]);
            }
            float hi = ak.s, lo = -ak.c;
            bool first = true;
            if (hd.y >> 31) {  // warp-uniform
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float oh = __shfl_down_sync(0xffffffffu, hi, off);
                    const float ol = __shfl_down_sync(0xffffffffu, lo, off);
                    const unsigned int od = __shfl_down_sync(0xffffffffu, d, off);
                    if (l + off < 32 && od == d) {
                        float s2, e2;
                        two_sum(hi, oh, s2, e2);
                        hi = s2;
                        lo = __fadd_rn(__fadd_rn(lo, ol), e2);
                    }
                }
                const unsigned int ud = __shfl_up_sync(0xffffffffu, d, 1);
                first = l == 0 || ud != d;
            }
            if (first) *(real*)(Fb + d) = (real)__fadd_rn(hi, lo);
            continue;
        }
        real acc = (real)0;
        if (boff) {  // byte offsets into V (uniform per table)
            const unsigned char* __restrict__ Vb = (const unsigned char*)Vr;
#pragma unroll 4
            for (int k = 0; k < len; ++k) acc = acc + *(const real*)(Vb + ix[32 * k]);
        } else {
#pragma unroll 4
            for (int k = 0; k < len; ++k) acc = acc + Vr[ix[32 * k]];
        }
        bool first = true;
        if (hd.y >> 31) {  // warp-uniform
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const real o = __shfl_down_sync(0xffffffffu, acc, off);
                const unsigned int od = __shfl_down_sync(0xffffffffu, d, off);
                if (l + off < 32 && od == d) acc = acc + o;
            }
            const unsigned int ud = __shfl_up_sync(0xffffffffu, d, 1);
            first = l == 0 || ud != d;
        }
        if (first) *(real*)(Fb + d) = acc;
    }
}

// TB_SHARED: the caller passes tb derived from the CTA's shared-memory array
// (staged tables), so that the compiler addresses the tables as shared memory
// rather than through generic pointers; the code is the same otherwise.
template <int PREC, bool FEAT, bool QSS, bool TB_SHARED>
__device__ void run_group(const PlanDev& P, const OptsDev& O, const unsigned char* tb, const unsigned char* mlp_smem,
                          unsigned char* gbase, const int lane, const GroupSync gs) {
    using real = typename PrecTraits<PREC>::real;
    const int N = P.N, R = P.R, G = P.G, NP1 = N + 1;
    const int R1 = P.R1, R12 = P.R12;
    const bool feats_on = FEAT && (O.learn || O.record);

    GroupPtrs g;
    g.A = tb + P.tl.off_A;
    g.rspec = (const uint32_t*)(tb + P.tl.off_rspec);
    g.cexp = tb + P.tl.off_cexp;
    g.wsl = (const uint16_t*)(tb + P.tl.off_wsl);
    g.shdr = (const uint2*)(tb + P.tl.off_shdr);
    g.sdst = (const uint16_t*)(tb + P.tl.off_sdst);
    g.sidx = (const uint16_t*)(tb + P.tl.off_sidx);
    g.gbase = gbase;
    g.V = gbase + P.gl.off_V;
    g.K = gbase + P.gl.off_K;
    g.Kc = (float*)(gbase + P.gl.off_Kc);
    g.Y64 = (double*)(gbase + P.gl.off_Y);
    g.Ylo = (float*)(gbase + P.gl.off_Y);
    g.Y32 = (float*)(gbase + P.gl.off_Y32);
    g.Fk = gbase + P.gl.off_Fk;
    g.Fk2 = gbase + P.gl.off_Fk2;
    {
        const int nw = G >> 5;
        g.red_c = (double*)(gbase + P.gl.off_red);
        g.red_n = g.red_c + nw;
        g.red_d = g.red_n + nw;
        g.red_r = (float*)(g.red_d + nw);
        g.red_f = (int*)(g.red_r + nw);
    }
    g.feat = (float*)(gbase + P.gl.off_feat);
    g.hist = (int*)(g.feat + 384);

    real* V = (real*)g.V;
    real* K = (real*)g.K;
    double* Y64 = g.Y64;
    float* Ylo = g.Ylo;
    float* Y32 = g.Y32;
    real* Fk = (real*)g.Fk;
    GroupState& S = *(GroupState*)(gbase + P.gl.off_state);

    if (lane == 0) V[P.zero_idx] = (real)0;

    for (;;) {
        if (lane == 0) {
            const int q = atomicAdd(P.queue_head, 1);
            S.zone = q < P.n_zones ? P.order[q] : -1;
            S.valid = 1;
            if (O.zone_ns) S.t_fetch_ns = global_ns();
        }
        gs.sync();
        const int z = S.zone;
        if (z < 0) break;

        // ---- load the zone (Sec. 6 step 1 inputs, already on the device) ----
        {
            const double* Yg = P.Y + (size_t)z * N;
            int bad = 0;
            for (int i = lane; i < N; i += G) {
                const double y = Yg[i];
                if (PREC == kPrecMixed) {
                    const float hi = __double2float_rn(y);
                    Y32[i] = hi;
                    Ylo[i] = __double2float_rn(y - (double)hi);
                } else {
                    Y64[i] = y;
                    if (PREC == kPrecMixed64) Y32[i] = (float)y;
                }
                bad |= !(isfinite(y) && y >= 0.0);
            }
            if (lane == 0) {
                if (PREC == kPrecMixed) {
                    Y32[N] = 1.0f;
                    Y32[NP1 + N] = 1.0f;
                    Ylo[N] = 0.0f;
                    Ylo[NP1 + N] = 0.0f;
                } else {
                    Y64[N] = 1.0;
                    Y64[NP1 + N] = 1.0;
                    if (PREC == kPrecMixed64) {
                        Y32[N] = 1.0f;
                        Y32[NP1 + N] = 1.0f;
                    }
                }
                const double T0 = P.T0[z], rho0 = P.rho0[z], tau = P.tau[z];
                const double ts = P.t_start[z], te = P.t_end[z], dtt = P.dt_trial[z];
                S.T0 = T0;
                S.rho0 = rho0;
                S.tau = tau;
                S.t = ts;
                S.t_end = te;
                S.dt = dtt > 0.0 ? dtt : ts;
                S.constant = !(tau > 0.0);
                S.inv_tau = S.constant ? 0.0 : 1.0 / tau;
                S.u_scale = S.constant ? 0.f : __double2float_rn(S.inv_tau * 1.4426950408889634);
                S.s = 0.0;
                S.poly = 0;
                S.s_p = 0.0;
                S.poly_p = 0;
                S.u_p = 0.f;
                S.refresh_p = 0;
                S.u = 0.f;
                S.u_ref = -1e30f;  // the first flux pass computes the cached rates
                S.steps = 0;
                S.rejects = 0;
                S.props = 0;
                S.nrej = 0;
                S.status = 0;
                S.rhs_valid = 0;
                S.cur = 0;
                S.done = 0;
                S.fresh = 0;
                S.mlp_try = 0;
                S.h_prev = 0.0;
                S.dt_plain = 0.0;
                const bool ok = isfinite(T0) && T0 > 0.0 && isfinite(rho0) && rho0 > 0.0 &&
                                isfinite(tau) && isfinite(ts) && isfinite(te) && ts >= 0.0 &&
                                te > ts && isfinite(dtt) && (ts > 0.0 || dtt > 0.0);
                if (ok) {
                    S.lnT0 = log(T0);
                    S.lnR0 = log(rho0);
                } else {
                    S.valid = 0;
                }
            }
            if (bad) S.valid = 0;  // benign race: every writer stores 0
        }
        gs.sync();
        if (!S.valid) {
            if (lane == 0) {
                S.status = 5;  // INVALID
                S.done = 1;
            }
        } else {
            // the zone's rates at (T0, rho0), once per zone (Sec. 10 item (2))
            const double lnT0 = S.lnT0, lnR0 = S.lnR0;
            for (int j = lane; j < R; j += G) {
                const double2 p = P.rate0[j];
                const double r1 = (double)((j >= R1) + (j >= R12));
                K[j] = (real)exp(fma(p.y, lnT0, p.x) + r1 * lnR0);
            }
        }
        if (lane == 0) {
            leader_prepare<PREC>(S, P, O);
            if (PREC == kPrecMixed) {
                S.h32 = (float)S.h;
                S.dt32 = (float)S.dt;
                S.dtp32 = S.dt32;
            }
        }
        gs.sync();

        // ---- step loop (Sec. 4: adaptive network timesteps) ----
        // have_a: phase (a) of the current state was already computed, by the
        // speculative pass that overlapped the previous decision
        bool have_a = false;
        const bool spec = G >= 64 && PREC != kPrecFP64;
        while (!S.done) {
            const int cur = S.cur, nxt = cur ^ 1;

            if (!S.rhs_valid) {
                if (!have_a) {
                    // (a) rates, fluxes and reactant-slot partials at this state
                    // FP32-flux forms: refresh the cached rates when u has moved
                    // by more than u_tol since they were computed (a rate change
                    // below a quarter ulp), or at the zone's first pass
                    const bool refresh = PREC != kPrecFP64 && (!P.rate_cache || !(fabsf(S.u - S.u_ref) <= P.u_tol));
                    flux_pass<PREC>(P, g, lane, G, cur, S.constant, S.s, S.u, S.poly, refresh);
                    gs.sync();
                    if (lane == 0 && refresh) S.u_ref = S.u;
                }
                // (b) sliced gathers into the (F+, k) pairs
                gather_pass<PREC>(P, g, lane, (unsigned char*)Fk);
                gs.sync();
            }

            // features of a state reached by an accepted step: training records
            // (label by grid search) or the learned proposal
            if (FEAT && feats_on && S.fresh) {
                compute_features<PREC>(P, O, g, S, lane, cur, gs);
                if (O.record) {
                    // walk the grid dt_prev 2^(q/4), q = -8 .. 16, up from the
                    // smallest step; the label is the last step before the first
                    // failure (or the step that reaches t_end)
                    float label = -1.3862943611198906f;
                    if (lane == 0) S.h_best = 0.0;
                    for (int q = -8; q <= 16; ++q) {
                        double hq = S.h_prev * exp2(0.25 * q);
                        const double rem = S.t_end - S.t;
                        const bool last = hq >= rem;
                        if (last) hq = rem;
                        update_reduce<PREC>(P, O, g, lane, cur, hq, (float)hq, z);
                        gs.sync();
                        if (lane == 0) {
                            const TestOutcome v = combine<PREC>(P, O, g);
                            if (v.pass) {
                                label = (float)log(hq / S.h_prev);
                                S.h_best = hq;
                            }
                            S.found = !v.pass || last;  // stop
                        }
                        gs.sync();
                        if (S.found) break;
                    }
                    if (lane == 0) {
                        write_record(O, g, label);
                        if (O.follow_label) {
                            // the perfect proposal: the label's step, clipped like a learned one
                            const double lo = S.dt_plain, hi = 16.0 * S.dt_plain;
                            double hb = S.h_best;
                            if (hb > lo) {
                                hb = hb > hi ? hi : hb;
                                const double rem = S.t_end - S.t;
                                S.clipped = hb >= rem;
                                S.h = S.clipped ? rem : hb;
                                if (PREC == kPrecMixed) S.h32 = (float)S.h;
                                S.mlp_try = S.h > lo;
                            }
                        }
                    }
                }
                if (O.learn) {
                    const float out = mlp_forward_group(O, g, mlp_smem, lane, G, gs);
                    if (lane == 0) {
                        // dt_mlp = clip(dt_prev e^out, dt_plain, 16 dt_plain), then clipped to t_end
                        double hm = S.h_prev * (double)expf(fminf(out - O.mlp_margin, 20.f));
                        const double lo = S.dt_plain, hi = 16.0 * S.dt_plain;
                        // a proposal at or below the plain step is the plain attempt itself
                        const double raw = hm;
                        if (hm > lo) {
                            hm = hm > hi ? hi : hm;
                            const double rem = S.t_end - S.t;
                            S.clipped = hm >= rem;
                            S.h = S.clipped ? rem : hm;
                            if (PREC == kPrecMixed) S.h32 = (float)S.h;
                            S.mlp_try = S.h > lo;  // clipping to t_end can leave only the plain step
                        }
                        if (O.trace_out) {
                            const unsigned long long slot = atomicAdd(O.trace_count, 1ull);
                            if ((long long)slot < O.trace_cap) {
                                float* f = O.trace_feat + slot * 64;
                                for (int k = 0; k < 64; ++k) f[k] = g.feat[k];
                                O.trace_out[slot] = out;
                                double* d = O.trace_dt + slot * 6;
                                d[0] = S.h_prev;
                                d[1] = S.dt_plain;
                                d[2] = raw;
                                d[3] = PREC == kPrecMixed ? (double)S.h32 : S.h;  // the step the update takes
                                d[4] = S.mlp_try ? 1.0 : 0.0;
                                d[5] = S.t_end - S.t;
                            }
                        }
                    }
                }
                if (lane == 0) S.fresh = 0;
                gs.sync();
            }

            // QSS: the predictor into nxt, then (a) and (b) of the predicted
            // state at t + h into Fk2; the corrector in (d) then overwrites
            // nxt.  (F+, k) of the current state stay in Fk, so a rejected
            // attempt repeats only this part.  FP32-flux form: the predictor
            // writes the FP32 copy the flux pass reads, and the predicted
            // pass refreshes the cached rates at (t + h) when they are stale
            // (each thread the reactions it reads, as in the main pass).
            if (QSS) {
                if (PREC == kPrecFP64)
                    qss_predict(P, g, lane, cur, S.h);
                else
                    qss_predict_mixed(P, g, lane, cur, S.h32);
                if (lane == 0 && !S.constant) {
                    if (PREC == kPrecFP64) {
                        const double sp = (S.t + S.h) * S.inv_tau;
                        const double xm = P.cmax * sp;
                        S.s_p = sp;
                        S.poly_p = xm <= 1e-6 ? 2 : (xm <= 0.0009765625 ? 5 : 9);
                    } else {
                        S.u_p = __fmul_rn(__double2float_rn(S.t + (double)S.h32), S.u_scale);
                    }
                }
                if (lane == 0 && PREC != kPrecFP64)
                    S.refresh_p = !P.rate_cache || !(fabsf(S.u_p - S.u_ref) <= P.u_tol);
                gs.sync();
                flux_pass<PREC>(P, g, lane, G, nxt, S.constant, S.s_p, S.u_p, S.poly_p,
                                PREC != kPrecFP64 && S.refresh_p != 0);
                gs.sync();
                if (lane == 0 && PREC != kPrecFP64 && S.refresh_p) S.u_ref = S.u_p;
                gather_pass<PREC>(P, g, lane, (unsigned char*)g.Fk2);
                gs.sync();
            }

            // (d) update and error measures, then (e) the decision (lane 0)
            // while warps 1.. compute (a) for the candidate state at t + h,
            // as the next step needs it if this one is accepted
            const double h_now = PREC == kPrecMixed ? (double)S.h32 : S.h;
            if (spec && lane == 32) {
                // the candidate state's profile factor (t + h) / (tau ln 2), once per group
                S.u_spec = S.constant ? 0.f : __fmul_rn(__double2float_rn(S.t + h_now), S.u_scale);
                S.refresh_spec = !P.rate_cache || !(fabsf(S.u_spec - S.u_ref) <= P.u_tol);
            }
            update_reduce<PREC, QSS>(P, O, g, lane, cur, h_now, PREC == kPrecMixed ? S.h32 : (float)h_now, z);
            gs.sync();
            if (spec && lane >= 32)
                flux_pass<PREC>(P, g, lane - 32, G - 32, nxt, S.constant, 0.0, S.u_spec, 0, S.refresh_spec != 0);
            have_a = spec;
            if (PREC == kPrecMixed && lane == 0 && !O.probe && !O.replay_dt) {
                decide_mixed<FEAT>(S, P, O, g, nxt, spec);
            } else if (lane == 0) {
                if (spec && S.refresh_spec) S.u_ref = S.u_spec;  // the speculative pass refreshed Kc
                const TestOutcome v = combine<PREC>(P, O, g);
                const double h = S.h;  // FP64 (replay steps are FP64 even in the mixed form)
                if (O.probe) {
                    O.probe_cons[z] = PREC == kPrecMixed ? (double)v.cons32 : v.cons;
                    O.probe_rel[z] = PREC == kPrecFP64 ? v.bn / v.bd : (double)v.rmax;
                    S.done = 1;
                } else if (O.replay_dt || v.pass) {
                    S.t = S.clipped ? S.t_end : S.t + h;
                    S.cur = nxt;
                    S.steps += 1;
                    S.nrej = 0;
                    S.rhs_valid = 0;
                    if (S.mlp_try) S.props += 1;
                    S.mlp_try = 0;
                    S.h_prev = h;
                    S.fresh = 1;
                    if (O.replay_dt) {
                        S.dt = h;
                    } else if (PREC == kPrecFP64) {
                        // FP64 form: the proposal in FP64 as well
                        const double rel = v.bn / v.bd;
                        double gfac = O.grow_max;
                        const double ga = O.safety * O.eps_r / (rel > 1e-300 ? rel : 1e-300);
                        const double gb = O.safety * O.eps_c / (v.cons > 1e-300 ? v.cons : 1e-300);
                        if (ga < gfac) gfac = ga;
                        if (gb < gfac) gfac = gb;
                        S.dt = h * gfac;
                    } else {
                        // FP32-flux forms: the growth factor in FP32
                        const float ga = __fdiv_rn(O.ga32, fmaxf(v.rmax, 1e-30f));
                        const float gb = __fdiv_rn(O.gb32, fmaxf(v.cons32, 1e-30f));
                        const float gfac = fminf(O.grow32, fminf(ga, gb));
                        S.dt = h * (double)gfac;
                    }
                    S.dt_plain = S.dt;
                } else if (S.mlp_try) {
                    // a rejected learned proposal: retry with the plain controller's dt
                    S.rejects += 1;
                    S.rhs_valid = 1;
                    S.mlp_try = 0;
                    S.dt = S.dt_plain;
                } else {
                    S.rejects += 1;
                    S.nrej += 1;
                    S.rhs_valid = 1;
                    S.dt = h * O.shrink;
                    if (S.nrej > O.max_reject) {
                        S.status = v.fin ? 4 : 3;  // MAX_REJECT : NONFINITE
                        S.done = 1;
                    } else if (S.dt < O.dt_min_frac * S.t) {
                        S.status = 2;  // DT_UNDERFLOW
                        S.done = 1;
                    }
                }
                leader_prepare<PREC>(S, P, O);
                if (PREC == kPrecMixed) {
                    S.h32 = (float)S.h;
                    S.dt32 = (float)S.dt;
                }
            }
            gs.sync();
        }

        // ---- write back (Sec. 6 step 3 outputs: abundances, energy, final dt) ----
        if (!O.probe) {
            double* Yg = P.Y + (size_t)z * N;
            double e = 0.0;
            if (S.status != 5) {
                for (int i = lane; i < N; i += G) {
                    const double y0 = Yg[i];  // still Y(t_start)
                    double y;
                    if (PREC == kPrecMixed) {
                        // a pair that never changed returns the FP64 input bit for bit
                        const float hi = Y32[S.cur * NP1 + i], lo = Ylo[S.cur * NP1 + i];
                        const float hi0 = __double2float_rn(y0);
                        const float lo0 = __double2float_rn(y0 - (double)hi0);
                        y = (hi == hi0 && lo == lo0) ? y0 : (double)hi + (double)lo;
                    } else {
                        y = Y64[S.cur * NP1 + i];
                    }
                    if (P.bind) e = fma(P.bind[i], y - y0, e);
                    Yg[i] = y;
                }
            }
            if (P.bind) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
                if ((lane & 31) == 0) g.red_c[lane >> 5] = e;
                gs.sync();
                if (lane == 0) {
                    double es = 0.0;
                    for (int w = 0; w < (G >> 5); ++w) es += g.red_c[w];
                    P.energy[z] = es;
                }
            }
            if (lane == 0) {
                P.t_out[z] = S.t;
                P.dt_next[z] = PREC == kPrecMixed ? (double)S.dt32 : S.dt;
                P.steps[z] = S.steps;
                P.rejects[z] = S.rejects;
                if (P.props) P.props[z] = S.props;
                P.status[z] = S.status;
                if (O.zone_ns) {
                    long long* tz = O.zone_ns + 2 * (size_t)(P.zone_base + z);
                    tz[0] = S.t_fetch_ns;
                    tz[1] = global_ns();
                }
            }
        }
        gs.sync();
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <int PREC, bool FEAT, bool QSS>
__global__ void __launch_bounds__(1024, 1) integrate_kernel(const __grid_constant__ LaunchParams lp) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_go;
    const int np = lp.n_plans;
    // the learned proposal's network, staged once per CTA: BF16 W1, W2, then
    // FP32 b1, b2, w3, b3 (+3 pad) and mu, 1/sigma
    const int moff = FEAT && lp.o.learn ? kMlpSmemBytes : 0;
    if (FEAT && lp.o.learn) {
        const int4* src = (const int4*)lp.o.mlpW;
        int4* dst = (int4*)smem;
        const int nw = (kMlpFeatures * kMlpHidden + kMlpHidden * kMlpHidden) * 2 / 16;
        for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
        float* Pb = (float*)(smem + nw * 16);
        const float* P = lp.o.mlpP;
        const int ob1 = kMlpFeatures * kMlpHidden, ob2 = ob1 + kMlpHidden + kMlpHidden * kMlpHidden,
                  ow3 = ob2 + kMlpHidden, ob3 = ow3 + kMlpHidden;
        for (int i = threadIdx.x; i < kMlpHidden; i += blockDim.x) {
            Pb[i] = P[ob1 + i];
            Pb[kMlpHidden + i] = P[ob2 + i];
            Pb[2 * kMlpHidden + i] = P[ow3 + i];
        }
        if (threadIdx.x == 0) Pb[3 * kMlpHidden] = P[ob3];
        for (int i = threadIdx.x; i < 2 * kMlpFeatures; i += blockDim.x) Pb[3 * kMlpHidden + 4 + i] = lp.o.mlpNorm[i];
    }
    int home = 0;
    for (int p = 0; p < np; ++p)
        if ((int)blockIdx.x >= lp.plans[p].cta_begin && (int)blockIdx.x < lp.plans[p].cta_end) home = p;
    for (int a = 0; a < np; ++a) {
        const PlanDev& P = lp.plans[(home + a) % np];
        if (threadIdx.x == 0) s_go = *((volatile int*)P.queue_head) < P.n_zones;
        __syncthreads();
        const int go = s_go;
        __syncthreads();
        if (!go) continue;
        const unsigned char* tb = P.blob;
        int toff = moff;
        if (P.smem_tables) {
            const int4* src = (const int4*)P.blob;
            int4* dst = (int4*)(smem + moff);
            for (int i = threadIdx.x; i < P.tl.bytes / 16; i += blockDim.x) dst[i] = src[i];
            tb = smem + moff;
            toff += P.tl.bytes;
        }
        __syncthreads();
        const int g = threadIdx.x / P.G, lane = threadIdx.x - g * P.G;
        if (g < P.M) {
            GroupSync gs{1 + g, P.G, P.M == 1 && P.G == (int)blockDim.x};
            unsigned char* gbase = smem + toff + g * P.gl.bytes;
            // the FP32-flux forms with staged tables (the common case) get their
            // own copy of the group loop with the tables known to be shared
            // memory (measured: mixed +2.9 %, mixed with the FP64 update +0.7 %;
            // the FP64 form, FP64-pipe bound, within noise)
            if (PREC != kPrecFP64 && P.smem_tables)
                run_group<PREC, FEAT, QSS, true>(P, lp.o, smem + moff, smem, gbase, lane, gs);
            else
                run_group<PREC, FEAT, QSS, false>(P, lp.o, tb, smem, gbase, lane, gs);
        }
        __syncthreads();
    }
}

cudaError_t launch_integrator(const LaunchParams& lp, int precision, int grid, int block,
                              cudaStream_t stream) {
    const bool feat = lp.o.learn || lp.o.record;
    if (precision == kPrecFP64 && lp.o.method) {
        integrate_kernel<kPrecFP64, false, true><<<grid, block, lp.smem_bytes, stream>>>(lp);
    } else if (precision == kPrecMixed && lp.o.method) {
        integrate_kernel<kPrecMixed, false, true><<<grid, block, lp.smem_bytes, stream>>>(lp);
    } else if (precision == kPrecFP64) {
        if (feat)
            integrate_kernel<kPrecFP64, true, false><<<grid, block, lp.smem_bytes, stream>>>(lp);
        else
            integrate_kernel<kPrecFP64, false, false><<<grid, block, lp.smem_bytes, stream>>>(lp);
    } else if (precision == kPrecMixed64) {
        if (feat)
            integrate_kernel<kPrecMixed64, true, false><<<grid, block, lp.smem_bytes, stream>>>(lp);
        else
            integrate_kernel<kPrecMixed64, false, false><<<grid, block, lp.smem_bytes, stream>>>(lp);
    } else {
        if (feat)
            integrate_kernel<kPrecMixed, true, false><<<grid, block, lp.smem_bytes, stream>>>(lp);
        else
            integrate_kernel<kPrecMixed, false, false><<<grid, block, lp.smem_bytes, stream>>>(lp);
    }
    return cudaGetLastError();
}

cudaError_t integrator_set_smem_limit(int bytes) {
    const void* fns[] = {(const void*)integrate_kernel<kPrecFP64, false, false>,
                         (const void*)integrate_kernel<kPrecFP64, true, false>,
                         (const void*)integrate_kernel<kPrecMixed, false, false>,
                         (const void*)integrate_kernel<kPrecMixed, true, false>,
                         (const void*)integrate_kernel<kPrecMixed64, false, false>,
                         (const void*)integrate_kernel<kPrecMixed64, true, false>,
                         (const void*)integrate_kernel<kPrecFP64, false, true>,
                         (const void*)integrate_kernel<kPrecMixed, false, true>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t integrator_occupancy(int precision, int block, int smem, int* blocks_per_sm) {
    // the FEAT variants use the same shared memory model; occupancy is governed
    // by shared memory and block size
    if (precision == kPrecFP64)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, integrate_kernel<kPrecFP64, false, false>,
                                                             block, smem);
    if (precision == kPrecMixed64)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, integrate_kernel<kPrecMixed64, false, false>,
                                                             block, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, integrate_kernel<kPrecMixed, false, false>, block,
                                                         smem);
}

// ---------------------------------------------------------------------------
// work-queue ordering key: mean log-rate at the zone's initial conditions,
// nbar ln T0 + rbar ln rho0 (the constant mean ln k0 drops out of a ranking)
// ---------------------------------------------------------------------------
__global__ void zone_cost_kernel(const double* T0, const double* rho0, int n, double nbar,
                                 double rbar, float* key, int* idx) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < n) {
        const double t = T0[z], r = rho0[z];
        double k = (t > 0.0 && r > 0.0) ? nbar * log(t) + rbar * log(r) : 0.0;
        key[z] = isfinite(k) ? (float)k : 0.f;
        idx[z] = z;
    }
}

cudaError_t launch_zone_cost_simple(const double* T0, const double* rho0, int n, double nbar,
                                    double rbar, float* key, int* idx, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    zone_cost_kernel<<<(n + 255) / 256, 256, 0, stream>>>(T0, rho0, n, nbar, rbar, key, idx);
    return cudaGetLastError();
}

__global__ void fill_int_kernel(int* p, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

cudaError_t launch_fill_int(int* p, int n, int v, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    fill_int_kernel<<<(n + 255) / 256, 256, 0, stream>>>(p, n, v);
    return cudaGetLastError();
}

}  // namespace kn

namespace kn {
// FP64 FMA throughput probe: 8 independent DFMA chains per thread
__global__ void fp64_peak_kernel(double* out, double a, double b, int iters) {
    double x0 = a + threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
           x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, b, a);
        x1 = fma(x1, b, a);
        x2 = fma(x2, b, a);
        x3 = fma(x3, b, a);
        x4 = fma(x4, b, a);
        x5 = fma(x5, b, a);
        x6 = fma(x6, b, a);
        x7 = fma(x7, b, a);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

cudaError_t launch_fp64_peak(double* out, int blocks, int threads, int iters, cudaStream_t st) {
    fp64_peak_kernel<<<blocks, threads, 0, st>>>(out, 0.5, 0.999, iters);
    return cudaGetLastError();
}
}  // namespace kn

namespace kn {
// operator-split continuation: the next hydro interval starts where the last ended
__global__ void advance_kernel(int n, const double* T9, const double* rho, const double* te, const double* t_out,
                               const double* dt_next, double* T0, double* rho0, double* tau, double* ts, double* tend,
                               double* dtt, int* status) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z < n) {
        T0[z] = T9[z];
        rho0[z] = rho[z];
        tau[z] = 0.0;
        ts[z] = t_out[z];
        tend[z] = te[z];
        dtt[z] = dt_next[z];
        status[z] = 6;  // PENDING
    }
}

cudaError_t launch_advance(int n, const double* T9, const double* rho, const double* te, const double* t_out,
                           const double* dt_next, double* T0, double* rho0, double* tau, double* ts, double* tend,
                           double* dtt, int* status, cudaStream_t st) {
    advance_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, T9, rho, te, t_out, dt_next, T0, rho0, tau, ts, tend, dtt,
                                                    status);
    return cudaGetLastError();
}
}  // namespace kn
