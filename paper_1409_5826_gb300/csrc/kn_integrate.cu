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
//   * a network's tables (reactant lists, rate parameters, the flat gather
//     list) are staged once per CTA into shared memory and shared by all
//     groups;
//   * per step: rates + fluxes + reactant-slot partials (one pass over
//     reactions), balanced chunked gathers of F+ and k (every thread sums the
//     same number of terms; rows cut by a chunk boundary are fixed up from
//     per-chunk carries), then the kappa-switched FP64 update with
//     deterministic group reductions for the accept test.
//   * no spin-waits: every loop is bounded by the zone's step and reject limits.
#include <cstdint>

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

// Gather accumulators: plain FP64, or FP32 with Kahan compensation.
struct AccD {
    double s;
    __device__ __forceinline__ void reset() { s = 0.0; }
    __device__ __forceinline__ void add(double v) { s += v; }
};
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
    using Acc = AccD;
};
template <> struct PrecTraits<kPrecMixed> {
    using real = float;
    using Acc = AccKahan;
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
        if (PREC == kPrecMixed) {
            S.u = (float)(s * 1.4426950408889634);
        } else {
            const double xm = P.cmax * s;
            S.poly = xm <= 1e-6 ? 2 : (xm <= 0.0009765625 ? 5 : 9);
        }
    }
}

// ---------------------------------------------------------------------------
// one zone group: fetch zones until the queue is empty
// ---------------------------------------------------------------------------
template <int PREC>
__device__ void run_group(const PlanDev& P, const OptsDev& O, const unsigned char* tb,
                          unsigned char* gbase, const int lane, const GroupSync gs) {
    using real = typename PrecTraits<PREC>::real;
    using Acc = typename PrecTraits<PREC>::Acc;
    const int N = P.N, R = P.R, G = P.G, Q = P.Q, C = P.C, NP1 = N + 1;
    const int R1 = P.R1, R12 = P.R12;

    const double* __restrict__ A = (const double*)(tb + P.tl.off_A);
    const ushort4* __restrict__ rspec = (const ushort4*)(tb + P.tl.off_rspec);
    const real* __restrict__ cexp = (const real*)(tb + P.tl.off_cexp);
    const uint32_t* __restrict__ terms = (const uint32_t*)(tb + P.tl.off_terms);
    const ushort4* __restrict__ fix = (const ushort4*)(tb + P.tl.off_fix);

    real* V = (real*)(gbase + P.gl.off_V);
    real* K = (real*)(gbase + P.gl.off_K);
    double* Y64 = (double*)(gbase + P.gl.off_Y64);
    float* Y32 = (float*)(gbase + P.gl.off_Y32);
    real* Fk = (real*)(gbase + P.gl.off_Fk);
    double* red_c = (double*)(gbase + P.gl.off_red);  // [32] per-warp cons sums
    double* red_n = red_c + 32;                        // [32] per-warp ratio numerators (FP64 form)
    double* red_d = red_n + 32;                        // [32] per-warp ratio denominators
    float* red_r = (float*)(red_d + 32);               // [32] per-warp max ratio (mixed form)
    int* red_f = (int*)(red_r + 32);                   // [32] per-warp finite | accept flags
    GroupState& S = *(GroupState*)(gbase + P.gl.off_state);

    if (lane == 0) V[P.zero_idx] = (real)0;

    for (;;) {
        if (lane == 0) {
            const int q = atomicAdd(P.queue_head, 1);
            S.zone = q < P.n_zones ? P.order[q] : -1;
            S.valid = 1;
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
                Y64[i] = y;
                if (PREC == kPrecMixed) Y32[i] = (float)y;
                bad |= !(isfinite(y) && y >= 0.0);
            }
            if (lane == 0) {
                Y64[N] = 1.0;
                Y64[NP1 + N] = 1.0;
                if (PREC == kPrecMixed) {
                    Y32[N] = 1.0f;
                    Y32[NP1 + N] = 1.0f;
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
                S.poly = 0;
                S.u = 0.f;
                S.steps = 0;
                S.rejects = 0;
                S.nrej = 0;
                S.status = 0;
                S.rhs_valid = 0;
                S.cur = 0;
                S.done = 0;
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
        if (lane == 0) leader_prepare<PREC>(S, P, O);
        gs.sync();

        // ---- step loop (Sec. 4: adaptive network timesteps) ----
        while (!S.done) {
            const int cur = S.cur, nxt = cur ^ 1;
            const double* Yc = Y64 + cur * NP1;
            double* Yn64 = Y64 + nxt * NP1;

            if (!S.rhs_valid) {
                // (a) rates k_j(t), fluxes f_j and reactant-slot partials (Eq. 1),
                //     reactions sorted 1-, 2-, 3-body: no multiply by a missing reactant
                if (PREC == kPrecFP64) {
                    const int poly = S.poly;
                    const double s = S.s;
                    const double* __restrict__ Yr = Yc;
                    const real* __restrict__ Kz = K;
                    real* __restrict__ Vw = V;
#pragma unroll 2
                    for (int j = lane; j < R; j += G) {
                        const ushort4 rs = rspec[j];
                        double k = (double)Kz[j];
                        if (poly == 2 || poly == 5)
                            k *= exp_neg_small((double)cexp[j] * s, poly);
                        else if (poly == 9)
                            k *= exp(-(double)cexp[j] * s);
                        const double ya = Yr[rs.x];
                        if (j < R1) {
                            Vw[j] = (real)(k * ya);
                            Vw[rs.w] = (real)k;
                        } else if (j < R12) {
                            const double yb = Yr[rs.y];
                            Vw[j] = (real)(k * ya * yb);
                            Vw[rs.w] = (real)(k * yb);
                            Vw[rs.w + 1] = (real)(k * ya);
                        } else {
                            const double yb = Yr[rs.y], yc = Yr[rs.z];
                            const double ka = k * ya;
                            Vw[j] = (real)(ka * yb * yc);
                            Vw[rs.w] = (real)(k * yb * yc);
                            Vw[rs.w + 1] = (real)(ka * yc);
                            Vw[rs.w + 2] = (real)(ka * yb);
                        }
                    }
                } else {
                    const float* __restrict__ Yc32 = Y32 + cur * NP1;
                    const real* __restrict__ Kz = K;
                    real* __restrict__ Vw = V;
                    const float u = S.u;
                    const bool varying = !S.constant;
#pragma unroll 2
                    for (int j = lane; j < R; j += G) {
                        const ushort4 rs = rspec[j];
                        float k = (float)Kz[j];
                        if (varying) k = __fmul_rn(k, ex2_approx(-__fmul_rn((float)cexp[j], u)));
                        const float ya = Yc32[rs.x];
                        if (j < R1) {
                            Vw[j] = (real)__fmul_rn(k, ya);
                            Vw[rs.w] = (real)k;
                        } else if (j < R12) {
                            const float yb = Yc32[rs.y];
                            Vw[j] = (real)__fmul_rn(__fmul_rn(k, ya), yb);
                            Vw[rs.w] = (real)__fmul_rn(k, yb);
                            Vw[rs.w + 1] = (real)__fmul_rn(k, ya);
                        } else {
                            const float yb = Yc32[rs.y], yc = Yc32[rs.z];
                            const float ka = __fmul_rn(k, ya);
                            Vw[j] = (real)__fmul_rn(__fmul_rn(ka, yb), yc);
                            Vw[rs.w] = (real)__fmul_rn(__fmul_rn(k, yb), yc);
                            Vw[rs.w + 1] = (real)__fmul_rn(ka, yc);
                            Vw[rs.w + 2] = (real)__fmul_rn(ka, yb);
                        }
                    }
                }
                gs.sync();
                // (b) balanced gathers: chunk `lane` of the flat term list; the
                //     next two terms are loaded ahead of the current one's store
                if (lane < Q) {
                    const uint32_t* __restrict__ tp = terms + lane;
                    const real* __restrict__ Vr = V;
                    real* __restrict__ Fw = Fk;
                    const uint32_t zterm = (uint32_t)P.zero_idx;
                    uint32_t w0 = tp[0];
                    uint32_t w1 = C > 1 ? tp[Q] : zterm;
                    real v0 = Vr[w0 & 0xffffu];
                    real v1 = Vr[w1 & 0xffffu];
                    if (PREC == kPrecFP64) {
                        double* __restrict__ carry = (double*)(gbase + P.gl.off_carry);
                        double acc = 0.0;
                        for (int k = 0; k < C; ++k) {
                            const uint32_t w2 = k + 2 < C ? tp[(k + 2) * Q] : zterm;
                            const real v2 = Vr[w2 & 0xffffu];
                            acc += (double)v0;
                            if (w0 & kTermEnd) {
                                if (w0 & kTermHead)
                                    carry[lane] = acc;
                                else
                                    Fw[(w0 >> kTermRowShift) & kTermRowMask] = (real)acc;
                                acc = 0.0;
                            }
                            w0 = w1;
                            v0 = v1;
                            w1 = w2;
                            v1 = v2;
                        }
                        carry[Q + lane] = acc;
                    } else {
                        // FP32 Kahan sums; no FP64 instruction in this loop
                        float2* __restrict__ carry = (float2*)(gbase + P.gl.off_carry);
                        AccKahan ak;
                        ak.reset();
                        for (int k = 0; k < C; ++k) {
                            const uint32_t w2 = k + 2 < C ? tp[(k + 2) * Q] : zterm;
                            const real v2 = Vr[w2 & 0xffffu];
                            ak.add((float)v0);
                            if (w0 & kTermEnd) {
                                if (w0 & kTermHead)
                                    carry[lane] = make_float2(ak.s, ak.c);
                                else
                                    Fw[(w0 >> kTermRowShift) & kTermRowMask] = (real)__fsub_rn(ak.s, ak.c);
                                ak.reset();
                            }
                            w0 = w1;
                            v0 = v1;
                            w1 = w2;
                            v1 = v2;
                        }
                        carry[Q + lane] = make_float2(ak.s, ak.c);
                    }
                }
                gs.sync();
                // (c) rows that cross chunk boundaries: tails of c0..c1-1, head of c1
                for (int f = lane; f < P.n_fix; f += G) {
                    const ushort4 fx = fix[f];
                    if (PREC == kPrecFP64) {
                        const double* carry = (const double*)(gbase + P.gl.off_carry);
                        double s = 0.0;
                        for (int c = fx.y; c < fx.z; ++c) s += carry[Q + c];
                        s += carry[fx.z];
                        Fk[fx.x] = (real)s;
                    } else {
                        const float2* carry = (const float2*)(gbase + P.gl.off_carry);
                        AccKahan ak;
                        ak.reset();
                        for (int c = fx.y; c < fx.z; ++c) {
                            ak.add(carry[Q + c].x);
                            ak.add(-carry[Q + c].y);
                        }
                        ak.add(carry[fx.z].x);
                        ak.add(-carry[fx.z].y);
                        Fk[fx.x] = (real)__fsub_rn(ak.s, ak.c);
                    }
                }
                gs.sync();
            }

            // (d) kappa-switched update (Sec. 3, Eq. 3) and error measures, FP64;
            //     each warp reduces its own lanes
            {
                const double h = S.h, kappa = O.kappa, ymin = O.y_min, eps_r = O.eps_r;
                double csum = 0.0, bn = 0.0, bd = 1.0;
                float rmax = 0.f;
                int fin = 1, ok = 1;
                float* Yn32 = Y32 + nxt * NP1;
                const float* Yc32 = Y32 + cur * NP1;
                for (int i = lane; i < N; i += G) {
                    const double y = Yc[i], fp = (double)Fk[i], kk = (double)Fk[N + i];
                    const double kdt = kk * h;
                    const double yn = (kdt >= kappa) ? (y + h * fp) / (1.0 + kdt) : y + h * (fp - kk * y);
                    Yn64[i] = yn;
                    const double d = yn - y;
                    csum = fma(A[i], d, csum);
                    const double m = y > yn ? y : yn;
                    if (PREC == kPrecMixed) {
                        const float yn32 = (float)yn;
                        Yn32[i] = yn32;
                        if (m > ymin) {
                            ok &= fabs(d) <= eps_r * m ? 1 : 0;  // the accept test, FP64
                            const float y32 = Yc32[i];           // the dt proposal, FP32
                            rmax = fmaxf(rmax, __fdividef(fabsf(yn32 - y32), fmaxf(y32, yn32)));
                        }
                    } else if (m > ymin) {
                        const double ad = fabs(d);
                        if (ad * bd > bn * m) {
                            bn = ad;
                            bd = m;
                        }
                    }
                    fin &= isfinite(yn) ? 1 : 0;
                    if (O.probe) {
                        O.probe_Fp[(size_t)z * N + i] = fp;
                        O.probe_k[(size_t)z * N + i] = kk;
                        O.probe_Y1[(size_t)z * N + i] = yn;
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    csum += __shfl_xor_sync(0xffffffffu, csum, off);
                    if (PREC == kPrecMixed) {
                        rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
                    } else {
                        const double on = __shfl_xor_sync(0xffffffffu, bn, off);
                        const double od = __shfl_xor_sync(0xffffffffu, bd, off);
                        if (on * bd > bn * od) {
                            bn = on;
                            bd = od;
                        }
                    }
                }
                fin = __all_sync(0xffffffffu, fin);
                ok = __all_sync(0xffffffffu, ok);
                if ((lane & 31) == 0) {
                    const int w = lane >> 5;
                    red_c[w] = csum;
                    red_n[w] = bn;
                    red_d[w] = bd;
                    red_r[w] = rmax;
                    red_f[w] = fin | (ok << 1);
                }
            }
            gs.sync();

            // (e) accept / reject and the next dt (lane 0 combines the warps)
            if (lane == 0) {
                const int nw = G >> 5;
                double cs = 0.0, bn = 0.0, bd = 1.0;
                float rmax = 0.f;
                int fin = 1, ok = 1;
                for (int w = 0; w < nw; ++w) {
                    cs += red_c[w];
                    if (PREC == kPrecMixed) {
                        rmax = fmaxf(rmax, red_r[w]);
                    } else {
                        const double on = red_n[w], od = red_d[w];
                        if (on * bd > bn * od) {
                            bn = on;
                            bd = od;
                        }
                    }
                    fin &= red_f[w] & 1;
                    ok &= (red_f[w] >> 1) & 1;
                }
                const double cons = fabs(cs);
                const double h = S.h;
                const bool pass = PREC == kPrecMixed ? (fin && ok && cons <= O.eps_c)
                                                     : (fin && cons <= O.eps_c && bn <= O.eps_r * bd);
                if (O.probe) {
                    O.probe_cons[z] = cons;
                    O.probe_rel[z] = PREC == kPrecMixed ? (double)rmax : bn / bd;
                    S.done = 1;
                } else if (O.replay_dt || pass) {
                    S.t = S.clipped ? S.t_end : S.t + h;
                    S.cur = nxt;
                    S.steps += 1;
                    S.nrej = 0;
                    S.rhs_valid = 0;
                    if (O.replay_dt) {
                        S.dt = h;
                    } else if (PREC == kPrecFP64) {
                        // FP64 form: the proposal in FP64 as well
                        const double rel = bn / bd;
                        double gfac = O.grow_max;
                        const double ga = O.safety * O.eps_r / (rel > 1e-300 ? rel : 1e-300);
                        const double gb = O.safety * O.eps_c / (cons > 1e-300 ? cons : 1e-300);
                        if (ga < gfac) gfac = ga;
                        if (gb < gfac) gfac = gb;
                        S.dt = h * gfac;
                    } else {
                        // mixed form: the accept test above is FP64; the growth
                        // factor is proposed in FP32
                        float gfac = (float)O.grow_max;
                        const float ga = __fdiv_rn((float)(O.safety * O.eps_r), fmaxf(rmax, 1e-30f));
                        const float gb = __fdiv_rn((float)(O.safety * O.eps_c), fmaxf((float)cons, 1e-30f));
                        gfac = fminf(gfac, fminf(ga, gb));
                        S.dt = h * (double)gfac;
                    }
                } else {
                    S.rejects += 1;
                    S.nrej += 1;
                    S.rhs_valid = 1;
                    S.dt = h * O.shrink;
                    if (S.nrej > O.max_reject) {
                        S.status = fin ? 4 : 3;  // MAX_REJECT : NONFINITE
                        S.done = 1;
                    } else if (S.dt < O.dt_min_frac * S.t) {
                        S.status = 2;  // DT_UNDERFLOW
                        S.done = 1;
                    }
                }
                leader_prepare<PREC>(S, P, O);
            }
            gs.sync();
        }

        // ---- write back (Sec. 6 step 3 outputs) ----
        if (!O.probe) {
            const double* Yc = Y64 + S.cur * NP1;
            double* Yg = P.Y + (size_t)z * N;
            if (S.status != 5)
                for (int i = lane; i < N; i += G) Yg[i] = Yc[i];
            if (lane == 0) {
                P.t_out[z] = S.t;
                P.dt_next[z] = S.dt;
                P.steps[z] = S.steps;
                P.rejects[z] = S.rejects;
                P.status[z] = S.status;
            }
        }
        gs.sync();
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(1024, 1) integrate_kernel(const __grid_constant__ LaunchParams lp) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_go;
    const int np = lp.n_plans;
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
        int toff = 0;
        if (P.smem_tables) {
            const int4* src = (const int4*)P.blob;
            int4* dst = (int4*)smem;
            for (int i = threadIdx.x; i < P.tl.bytes / 16; i += blockDim.x) dst[i] = src[i];
            tb = smem;
            toff = P.tl.bytes;
        }
        __syncthreads();
        const int g = threadIdx.x / P.G, lane = threadIdx.x - g * P.G;
        if (g < P.M) {
            GroupSync gs{1 + g, P.G, P.M == 1 && P.G == (int)blockDim.x};
            run_group<PREC>(P, lp.o, tb, smem + toff + g * P.gl.bytes, lane, gs);
        }
        __syncthreads();
    }
}

cudaError_t launch_integrator(const LaunchParams& lp, int precision, int grid, int block,
                              cudaStream_t stream) {
    if (precision == kPrecFP64)
        integrate_kernel<kPrecFP64><<<grid, block, lp.smem_bytes, stream>>>(lp);
    else
        integrate_kernel<kPrecMixed><<<grid, block, lp.smem_bytes, stream>>>(lp);
    return cudaGetLastError();
}

cudaError_t integrator_set_smem_limit(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(integrate_kernel<kPrecFP64>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(integrate_kernel<kPrecMixed>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t integrator_occupancy(int precision, int block, int smem, int* blocks_per_sm) {
    if (precision == kPrecFP64)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, integrate_kernel<kPrecFP64>,
                                                             block, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, integrate_kernel<kPrecMixed>,
                                                         block, smem);
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
