/*
 * kn_oracle.c -- plain, slow, FP64 CPU oracle for explicit asymptotic
 * integration of reaction networks (Brock, Belt, Billings & Guidry,
 * "Explicit Integration with GPU Acceleration for Large Kinetic Networks").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * table with the library: it reads the network as plain arrays and recomputes
 * everything with loops over reactions in index order.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fopenmp -shared -fPIC
 * (no FMA contraction, no fast-math: every sum is a left-to-right loop).
 *
 * What each function follows:
 *   or_conditions   T9(t) = T0 exp(-t/tau), rho(t) = rho0 exp(-3t/tau); tau <= 0
 *                   holds both constant, as in the operator-split setting of
 *                   Sec. 4 and footnote 2 of Sec. 10.
 *   or_rates        k_j = k0_j T9^n_j rho^(r_j-1): the rate-library step of Sec. 6
 *                   and Sec. 10 item (2), with the synthetic parameterisation.
 *   or_rhs          Eq. (1): dY_i/dt = F+_i - F-_i = F+_i - k_i Y_i, with the flux
 *                   of reaction j f_j = k_j prod(reactant Y), F+_i the sum of the
 *                   fluxes producing i, and k_i the effective depletion rate
 *                   (each reactant slot s of j naming i adds k_j times the
 *                   product of the OTHER reactant abundances), so F-_i = k_i Y_i
 *                   even when Y_i = 0.
 *   or_update       Sec. 3: k_i dt >= kappa -> the asymptotic formula, Eq. (3),
 *                   Y' = (Y + dt F+)/(1 + k dt); otherwise forward Euler
 *                   Y' = Y + dt (F+ - k Y).  Ties go asymptotic (the text says >=).
 *   or_test         adaptive network timestep (Sec. 4).  The paper gives no
 *                   criterion; the reading implemented is: accept iff
 *                   |sum_i A_i (Y'_i - Y_i)| <= eps_c and
 *                   max over species with max(Y, Y') > y_min of
 *                   |Y' - Y| / max(Y, Y') <= eps_r.
 *   or_integrate    the step loop: accept -> t += dt, grow dt by
 *                   min(grow_max, safety eps_r/rel, safety eps_c/cons);
 *                   reject -> dt *= shrink and retry from the same state.
 *   or_qss_*        the explicit QSS update that Sec. 11 proposes as the
 *                   alternative to Eq. (3); its formula is not in the paper,
 *                   and the reading implemented is the alpha-QSS
 *                   predictor-corrector of Mott, Oran & van Leer (2000), under
 *                   the same accept test and step control (opts.method).
 *   or_be_*         backward Euler with Newton iterations and dense LU with
 *                   partial pivoting: the implicit comparison method of Sec. 7
 *                   (the paper's Xnet is sparse; dense is the brute-force form).
 *
 * Parity pins (checked by the CPU test-suite, not by this file): hand-computed
 * single steps in exact rational arithmetic, hand-worked cases of or_test and
 * or_growth and a hand-worked run of the step loop (each case built so that a
 * plausible slip changes its outcome), the A<->B closed form, FE and
 * asymptotic linear maps against matrix powers, conservation of sum A_i Y_i,
 * equilibrium ratios of reversible pairs, positivity, rate scaling laws,
 * backward Euler with Richardson extrapolation on tiny networks, and for the
 * QSS update: alpha's Taylor series at x = 0 and limit at infinity, the
 * single-step error of one linear decay against e^-x (O(x^7)), second-order
 * convergence on a nonlinear network, and the trapezoidal rule for a
 * species with no depletion.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXR 3

typedef struct {
    int32_t N, R;
    const double *A;       /* [N] */
    const int32_t *reac;   /* [R][3], -1 padded */
    const int32_t *prod;   /* [R][3], -1 padded */
    const double *ln_k0;   /* [R] */
    const double *t9_exp;  /* [R] */
} or_net;

typedef struct {
    double kappa;       /* asymptotic switch, 1 in the paper */
    double eps_r;       /* max relative change per accepted step */
    double eps_c;       /* max |sum A dY| per accepted step */
    double y_min;       /* abundances at or below this are not tested */
    double grow_max;    /* max growth factor of dt after an accept */
    double safety;      /* safety factor on the ratio proposal */
    double shrink;      /* dt factor after a reject */
    int32_t max_reject; /* consecutive rejects before giving up */
    int32_t method;     /* OR_ASYMPTOTIC: Eq. (3) with the kappa switch; OR_QSS: alpha-QSS */
    int64_t max_steps;  /* accepted steps before giving up */
    double dt_min_frac; /* dt < dt_min_frac * t is an underflow */
} or_opts;

enum { OR_OK = 0, OR_STEP_LIMIT = 1, OR_DT_UNDERFLOW = 2, OR_NONFINITE = 3, OR_MAX_REJECT = 4 };
enum { OR_ASYMPTOTIC = 0, OR_QSS = 1 };

void or_default_opts(or_opts *o)
{
    o->kappa = 1.0;
    o->eps_r = 0.05;
    o->eps_c = 1e-6;
    o->y_min = 1e-10;
    o->grow_max = 1.5;
    o->safety = 0.9;
    o->shrink = 0.5;
    o->max_reject = 60;
    o->method = OR_ASYMPTOTIC;
    o->max_steps = 10000000;
    o->dt_min_frac = 1e-30;
}

static int n_reactants(const or_net *n, int j)
{
    int c = 0;
    for (int q = 0; q < OR_MAXR; ++q)
        if (n->reac[j * OR_MAXR + q] >= 0) ++c;
    return c;
}

void or_conditions(double T0, double rho0, double tau, double t, double *T9, double *rho)
{
    if (tau > 0.0) {
        *T9 = T0 * exp(-t / tau);
        *rho = rho0 * exp(-3.0 * t / tau);
    } else {
        *T9 = T0;
        *rho = rho0;
    }
}

void or_rates(const or_net *n, double T9, double rho, double *k)
{
    for (int j = 0; j < n->R; ++j) {
        int r = n_reactants(n, j);
        k[j] = exp(n->ln_k0[j]) * pow(T9, n->t9_exp[j]) * pow(rho, (double)(r - 1));
    }
}

/* Fluxes f_j, production F+_i and effective depletion rate k_i (Eq. 1). */
void or_rhs(const or_net *n, const double *k, const double *Y, double *Fp, double *kk, double *f)
{
    for (int i = 0; i < n->N; ++i) {
        Fp[i] = 0.0;
        kk[i] = 0.0;
    }
    for (int j = 0; j < n->R; ++j) {
        const int32_t *rs = n->reac + j * OR_MAXR;
        double fj = k[j];
        for (int q = 0; q < OR_MAXR; ++q)
            if (rs[q] >= 0) fj = fj * Y[rs[q]];
        if (f) f[j] = fj;
        for (int q = 0; q < OR_MAXR; ++q) {
            int p = n->prod[j * OR_MAXR + q];
            if (p >= 0) Fp[p] = Fp[p] + fj;
        }
        for (int s = 0; s < OR_MAXR; ++s) {
            if (rs[s] < 0) continue;
            double ps = k[j];
            for (int q = 0; q < OR_MAXR; ++q)
                if (q != s && rs[q] >= 0) ps = ps * Y[rs[q]];
            kk[rs[s]] = kk[rs[s]] + ps;
        }
    }
}

/* Sec. 3: kappa-switched update of every species.  asy[i] = 1 where the
 * asymptotic formula was used (may be NULL). */
void or_update(int N, const double *Y, const double *Fp, const double *kk, double dt,
               double kappa, double *Yn, int8_t *asy)
{
    for (int i = 0; i < N; ++i) {
        double kdt = kk[i] * dt;
        if (kdt >= kappa) {
            Yn[i] = (Y[i] + dt * Fp[i]) / (1.0 + kdt);
            if (asy) asy[i] = 1;
        } else {
            Yn[i] = Y[i] + dt * (Fp[i] - kk[i] * Y[i]);
            if (asy) asy[i] = 0;
        }
    }
}

/* Error measures of a trial update: cons = |sum_i A_i (Y'_i - Y_i)|,
 * rel = max relative change over tested species.  Returns 1 if accepted. */
int or_test(int N, const double *A, const double *Y, const double *Yn, const or_opts *o,
            double *cons_out, double *rel_out, int *finite_out)
{
    double cons = 0.0, rel = 0.0;
    int finite = 1;
    for (int i = 0; i < N; ++i) {
        double d = Yn[i] - Y[i];
        if (!isfinite(Yn[i])) finite = 0;
        cons = cons + A[i] * d;
        double m = Y[i] > Yn[i] ? Y[i] : Yn[i];
        if (m > o->y_min) {
            double r = fabs(d) / m;
            if (r > rel) rel = r;
        }
    }
    cons = fabs(cons);
    if (cons_out) *cons_out = cons;
    if (rel_out) *rel_out = rel;
    if (finite_out) *finite_out = finite;
    return finite && cons <= o->eps_c && rel <= o->eps_r;
}

/* Factor applied to an accepted dt to propose the next one. */
double or_growth(double rel, double cons, const or_opts *o)
{
    double g = o->grow_max;
    double a = o->safety * o->eps_r / (rel > 1e-300 ? rel : 1e-300);
    double b = o->safety * o->eps_c / (cons > 1e-300 ? cons : 1e-300);
    if (a < g) g = a;
    if (b < g) g = b;
    return g;
}

/* ---------------------------------------------------------------------------
 * The explicit quasi-steady-state (QSS) update, the alternative to Eq. (3)
 * that Sec. 11 proposes to try on the GPU.  The paper defers its formula to
 * its QSS reference; the reading implemented is the alpha-QSS
 * predictor-corrector of Mott, Oran & van Leer (J. Comput. Phys. 164 (2000)
 * 407), the QSS scheme that reference applies, written in this file's
 * notation: production F+_i and depletion rate k_i (F-_i = k_i Y_i).
 *
 * For dY/dt = F+ - k Y with F+ and k constant, the exact step is
 *   Y(dt) = Y + dt (F+ - k Y) / (1 + alpha k dt),
 *   alpha(x) = 1/(1 - e^-x) - 1/x,   x = k dt,
 * and the scheme replaces alpha by its rational approximation in r = 1/x
 *   alpha = (180 r^3 + 60 r^2 + 11 r + 1) / (360 r^3 + 60 r^2 + 12 r + 1),
 * which tends to 1/2 as x -> 0 (the trapezoidal rule) and to 1 as x -> inf.
 * ------------------------------------------------------------------------- */

/* alpha as a function of x = k dt >= 0.  The same rational function is
 * evaluated in powers of x for x <= 1 (multiplying through by x^3, so x = 0
 * gives 1/2) and in powers of r = 1/x above, so neither form overflows. */
double or_qss_alpha(double x)
{
    if (x <= 1.0)
        return (180.0 + 60.0 * x + 11.0 * x * x + x * x * x) /
               (360.0 + 60.0 * x + 12.0 * x * x + x * x * x);
    double r = 1.0 / x;
    return (180.0 * r * r * r + 60.0 * r * r + 11.0 * r + 1.0) /
           (360.0 * r * r * r + 60.0 * r * r + 12.0 * r + 1.0);
}

/* 1 - alpha(x), from the same rational function: (D - N)/D with
 * D - N = 180 + x^2 (powers of x) or 180 r^3 + r (powers of r), so that it
 * keeps its relative accuracy as alpha -> 1. */
static double qss_one_minus_alpha(double x)
{
    if (x <= 1.0)
        return (180.0 + x * x) / (360.0 + 60.0 * x + 12.0 * x * x + x * x * x);
    double r = 1.0 / x;
    return (180.0 * r * r * r + r) / (360.0 * r * r * r + 60.0 * r * r + 12.0 * r + 1.0);
}

/* The scheme's update of one species, Y + dt (F - k Y) / (1 + alpha(x) x),
 * x = k dt, with F the production term (F+ in the predictor, F~ in the
 * corrector).  Written that way it is a difference of nearly equal terms
 * once x >> 1 (Y and dt k Y / (1 + alpha x) are both about Y, the result
 * about 12 Y / x^2 + F / k), and rounding leaves it a relative error of about
 * eps x^2 / 12.  With alpha = N/D, 1 + alpha x = (D + x N)/D and
 * 1 - (1 - alpha) x = (D - x (D - N))/D, so the same function is
 *   (c0 Y + c1 dt F) / c2,
 *   x <= 1:  c0 = D - x (D - N) = 360 - 120 x + 12 x^2,
 *            c1 = D             = 360 + 60 x + 12 x^2 + x^3,
 *            c2 = D + x N       = 360 + 240 x + 72 x^2 + 12 x^3 + x^4;
 *   x > 1 (numerator and denominator divided by x^4, r = 1/x):
 *            c0 = 360 r^4 - 120 r^3 + 12 r^2,
 *            c1 = 360 r^4 + 60 r^3 + 12 r^2 + r,
 *            c2 = 360 r^4 + 240 r^3 + 72 r^2 + 12 r + 1,
 * a sum of non-negative terms: c0 = 12 (30 - 10 x + x^2) (or r^2 times it in
 * r) has no real root, so Y, F >= 0 give a result >= 0. */
static double qss_update1(double Y, double F, double k, double dt)
{
    double x = k * dt, c0, c1, c2;
    if (x <= 1.0) {
        c0 = 360.0 - 120.0 * x + 12.0 * x * x;
        c1 = 360.0 + 60.0 * x + 12.0 * x * x + x * x * x;
        c2 = 360.0 + 240.0 * x + 72.0 * x * x + 12.0 * x * x * x + x * x * x * x;
    } else {
        double r = 1.0 / x, r2 = r * r, r3 = r2 * r, r4 = r3 * r;
        c0 = 360.0 * r4 - 120.0 * r3 + 12.0 * r2;
        c1 = 360.0 * r4 + 60.0 * r3 + 12.0 * r2 + r;
        c2 = 360.0 * r4 + 240.0 * r3 + 72.0 * r2 + 12.0 * r + 1.0;
    }
    return (c0 * Y + c1 * (dt * F)) / c2;
}

/* Predictor: Yp_i = Y_i + dt (F+_i - k_i Y_i) / (1 + alpha(k_i dt) k_i dt),
 * with F+ and k of the state Y at the start of the step. */
void or_qss_predict(int N, const double *Y, const double *Fp, const double *kk, double dt,
                    double *Yp)
{
    for (int i = 0; i < N; ++i)
        Yp[i] = qss_update1(Y[i], Fp[i], kk[i], dt);
}

/* Corrector, from the start state (F+0, k0 of Y) and the predicted state
 * (F+p, kp of Yp at t + dt):
 *   kbar = (k0 + kp)/2,  abar = alpha(kbar dt),
 *   F~   = abar F+p + (1 - abar) F+0,
 *   Yc_i = Y_i + dt (F~_i - kbar_i Y_i) / (1 + abar kbar_i dt). */
void or_qss_correct(int N, const double *Y, const double *Fp0, const double *k0,
                    const double *Fpp, const double *kp, double dt, double *Yc)
{
    for (int i = 0; i < N; ++i) {
        double kbar = 0.5 * (k0[i] + kp[i]);
        double x = kbar * dt;
        double ft = or_qss_alpha(x) * Fpp[i] + qss_one_minus_alpha(x) * Fp0[i];
        Yc[i] = qss_update1(Y[i], ft, kbar, dt);
    }
}

typedef struct {
    double T0, rho0, tau, t_start, t_end, dt_trial;
} or_zone;

/* One QSS trial step of length h from (Y, t), with F+0 and k0 already
 * evaluated at (Y, t): the rates at t + h (recomputed only when the
 * conditions vary), the right-hand side at the predicted state, then the
 * corrector into Yn.  Work arrays: kr [R], Yp, Fpp, kp [N]. */
static void qss_attempt(const or_net *n, const or_zone *z, double t, double h, const double *Y,
                        const double *Fp0, const double *k0, const double *k_rates,
                        double *kr, double *Yp, double *Fpp, double *kp, double *Yn)
{
    const int N = n->N;
    or_qss_predict(N, Y, Fp0, k0, h, Yp);
    const double *kq = k_rates;
    if (z->tau > 0.0) {
        double T9, rho;
        or_conditions(z->T0, z->rho0, z->tau, t + h, &T9, &rho);
        or_rates(n, T9, rho, kr);
        kq = kr;
    }
    or_rhs(n, kq, Yp, Fpp, kp, NULL);
    or_qss_correct(N, Y, Fp0, k0, Fpp, kp, h, Yn);
}

typedef struct {
    double t;          /* time reached */
    double dt_next;    /* proposed next dt (unclipped), the trial for the next interval */
    int64_t steps;     /* accepted steps */
    int64_t rejects;   /* rejected attempts */
    int32_t status;
    int32_t pad;
} or_result;

/*
 * Integrate one zone from t_start to t_end.  Y [N] holds Y0 on entry and the
 * end state on exit.  If rec_dt is non-NULL, the dt of every accepted step is
 * written there (up to rec_cap entries); the count is steps.
 */
void or_integrate(const or_net *n, const or_opts *o, const or_zone *z, double *Y,
                  or_result *res, double *rec_dt, int64_t rec_cap)
{
    const int N = n->N, R = n->R;
    double *k = (double *)malloc(sizeof(double) * (size_t)R);
    double *Fp = (double *)malloc(sizeof(double) * (size_t)N);
    double *kk = (double *)malloc(sizeof(double) * (size_t)N);
    double *Yn = (double *)malloc(sizeof(double) * (size_t)N);
    const int qss = o->method == OR_QSS;
    double *kr = NULL, *Yp = NULL, *Fpp = NULL, *kp = NULL;
    if (qss) {
        kr = (double *)malloc(sizeof(double) * (size_t)R);
        Yp = (double *)malloc(sizeof(double) * (size_t)N);
        Fpp = (double *)malloc(sizeof(double) * (size_t)N);
        kp = (double *)malloc(sizeof(double) * (size_t)N);
    }
    double t = z->t_start, dt = z->dt_trial > 0.0 ? z->dt_trial : z->t_start;
    int64_t steps = 0, rejects = 0;
    int nrej = 0, status = OR_OK, rhs_valid = 0, last_finite = 1;
    double T9, rho;
    int constant = !(z->tau > 0.0);
    if (constant) {
        or_conditions(z->T0, z->rho0, z->tau, t, &T9, &rho);
        or_rates(n, T9, rho, k);
    }
    while (t < z->t_end) {
        if (steps >= o->max_steps) { status = OR_STEP_LIMIT; break; }
        if (!rhs_valid) {
            if (!constant) {
                or_conditions(z->T0, z->rho0, z->tau, t, &T9, &rho);
                or_rates(n, T9, rho, k);
            }
            or_rhs(n, k, Y, Fp, kk, NULL);
            rhs_valid = 1;
        }
        double rem = z->t_end - t;
        int clipped = dt >= rem;
        double h = clipped ? rem : dt;
        if (qss)
            qss_attempt(n, z, t, h, Y, Fp, kk, k, kr, Yp, Fpp, kp, Yn);
        else
            or_update(N, Y, Fp, kk, h, o->kappa, Yn, NULL);
        double cons, rel;
        int finite;
        if (or_test(N, n->A, Y, Yn, o, &cons, &rel, &finite)) {
            if (rec_dt && steps < rec_cap) rec_dt[steps] = h;
            t = clipped ? z->t_end : t + h;
            memcpy(Y, Yn, sizeof(double) * (size_t)N);
            ++steps;
            nrej = 0;
            rhs_valid = 0;
            dt = h * or_growth(rel, cons, o);
        } else {
            ++rejects;
            ++nrej;
            last_finite = finite;
            dt = h * o->shrink;
            if (nrej > o->max_reject) { status = last_finite ? OR_MAX_REJECT : OR_NONFINITE; break; }
            if (dt < o->dt_min_frac * t) { status = OR_DT_UNDERFLOW; break; }
        }
    }
    res->t = t;
    res->dt_next = dt;
    res->steps = steps;
    res->rejects = rejects;
    res->status = status;
    res->pad = 0;
    free(k); free(Fp); free(kk); free(Yn);
    free(kr); free(Yp); free(Fpp); free(kp);
}

/* Replay: apply accepted steps with the given dt sequence, no tests. */
void or_replay(const or_net *n, const or_opts *o, const or_zone *z, double *Y,
               const double *dts, int64_t n_steps, double *t_out)
{
    const int N = n->N, R = n->R;
    double *k = (double *)malloc(sizeof(double) * (size_t)R);
    double *Fp = (double *)malloc(sizeof(double) * (size_t)N);
    double *kk = (double *)malloc(sizeof(double) * (size_t)N);
    double *Yn = (double *)malloc(sizeof(double) * (size_t)N);
    const int qss = o->method == OR_QSS;
    double *kr = NULL, *Yp = NULL, *Fpp = NULL, *kp = NULL;
    if (qss) {
        kr = (double *)malloc(sizeof(double) * (size_t)R);
        Yp = (double *)malloc(sizeof(double) * (size_t)N);
        Fpp = (double *)malloc(sizeof(double) * (size_t)N);
        kp = (double *)malloc(sizeof(double) * (size_t)N);
    }
    double t = z->t_start, T9, rho;
    for (int64_t s = 0; s < n_steps; ++s) {
        or_conditions(z->T0, z->rho0, z->tau, t, &T9, &rho);
        or_rates(n, T9, rho, k);
        or_rhs(n, k, Y, Fp, kk, NULL);
        double h = dts[s];
        if (qss)
            qss_attempt(n, z, t, h, Y, Fp, kk, k, kr, Yp, Fpp, kp, Yn);
        else
            or_update(N, Y, Fp, kk, h, o->kappa, Yn, NULL);
        memcpy(Y, Yn, sizeof(double) * (size_t)N);
        t = (h >= z->t_end - t) ? z->t_end : t + h;
    }
    *t_out = t;
    free(k); free(Fp); free(kk); free(Yn);
    free(kr); free(Yp); free(Fpp); free(kp);
}

/* Many zones, one thread each (OpenMP over zones when built with -fopenmp). */
void or_integrate_batch(const or_net *n, const or_opts *o, int32_t n_zones, const or_zone *zones,
                        double *Y, or_result *res, int32_t n_threads)
{
    (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int32_t z = 0; z < n_zones; ++z)
        or_integrate(n, o, &zones[z], Y + (size_t)z * (size_t)n->N, &res[z], NULL, 0);
}

/* ---------------------------------------------------------------------------
 * Backward Euler: Y' = Y + dt F(Y'), solved by Newton with the dense Jacobian
 * J = I - dt dF/dY and an LU factorisation with partial pivoting.
 * dF_i/dY_m = sum_j (nu_prod(i,j) - nu_reac(i,j)) df_j/dY_m, with
 * df_j/dY_m = sum over reactant slots of j naming m of the slot partial.
 * ------------------------------------------------------------------------- */

static void be_residual_jac(const or_net *n, const double *k, const double *Y0, const double *Y,
                            double dt, double *G, double *J, double *fbuf)
{
    const int N = n->N;
    for (int i = 0; i < N; ++i) G[i] = Y[i] - Y0[i];
    for (int i = 0; i < N * N; ++i) J[i] = 0.0;
    for (int i = 0; i < N; ++i) J[i * N + i] = 1.0;
    for (int j = 0; j < n->R; ++j) {
        const int32_t *rs = n->reac + j * OR_MAXR;
        const int32_t *ps = n->prod + j * OR_MAXR;
        double fj = k[j];
        for (int q = 0; q < OR_MAXR; ++q)
            if (rs[q] >= 0) fj = fj * Y[rs[q]];
        fbuf[j] = fj;
        for (int q = 0; q < OR_MAXR; ++q) {
            if (ps[q] >= 0) G[ps[q]] = G[ps[q]] - dt * fj;
            if (rs[q] >= 0) G[rs[q]] = G[rs[q]] + dt * fj;
        }
        for (int s = 0; s < OR_MAXR; ++s) {
            if (rs[s] < 0) continue;
            int m = rs[s];
            double part = k[j];
            for (int q = 0; q < OR_MAXR; ++q)
                if (q != s && rs[q] >= 0) part = part * Y[rs[q]];
            /* d f_j / d Y_m contribution of this slot: goes to every species j touches */
            for (int q = 0; q < OR_MAXR; ++q) {
                if (ps[q] >= 0) J[ps[q] * N + m] = J[ps[q] * N + m] - dt * part;
                if (rs[q] >= 0) J[rs[q] * N + m] = J[rs[q] * N + m] + dt * part;
            }
        }
    }
}

/* In-place LU with partial pivoting; solves J x = b, b overwritten by x.
 * Returns 0 on success, -1 on a zero pivot. */
int or_lu_solve(int N, double *J, double *b)
{
    for (int c = 0; c < N; ++c) {
        int piv = c;
        double best = fabs(J[c * N + c]);
        for (int r = c + 1; r < N; ++r)
            if (fabs(J[r * N + c]) > best) { best = fabs(J[r * N + c]); piv = r; }
        if (best == 0.0) return -1;
        if (piv != c) {
            for (int q = 0; q < N; ++q) {
                double tmp = J[c * N + q]; J[c * N + q] = J[piv * N + q]; J[piv * N + q] = tmp;
            }
            double tb = b[c]; b[c] = b[piv]; b[piv] = tb;
        }
        for (int r = c + 1; r < N; ++r) {
            double l = J[r * N + c] / J[c * N + c];
            J[r * N + c] = l;
            for (int q = c + 1; q < N; ++q) J[r * N + q] = J[r * N + q] - l * J[c * N + q];
            b[r] = b[r] - l * b[c];
        }
    }
    for (int r = N - 1; r >= 0; --r) {
        double s = b[r];
        for (int q = r + 1; q < N; ++q) s = s - J[r * N + q] * b[q];
        b[r] = s / J[r * N + r];
    }
    return 0;
}

/* One backward-Euler step from Y0 with rates k.  Newton from Y = Y0 until
 * max |dY| / max(|Y|, y_floor) <= tol or max_iter.  Returns iterations used,
 * or -1 if it did not converge (Y then holds the last iterate). */
int or_be_step(const or_net *n, const double *k, const double *Y0, double dt, double *Y,
               double tol, double y_floor, int max_iter)
{
    const int N = n->N;
    double *G = (double *)malloc(sizeof(double) * (size_t)N);
    double *J = (double *)malloc(sizeof(double) * (size_t)N * (size_t)N);
    double *fb = (double *)malloc(sizeof(double) * (size_t)n->R);
    memcpy(Y, Y0, sizeof(double) * (size_t)N);
    int it, ok = -1;
    for (it = 1; it <= max_iter; ++it) {
        be_residual_jac(n, k, Y0, Y, dt, G, J, fb);
        for (int i = 0; i < N; ++i) G[i] = -G[i];
        if (or_lu_solve(N, J, G) != 0) break;
        double err = 0.0;
        for (int i = 0; i < N; ++i) {
            Y[i] = Y[i] + G[i];
            double sc = fabs(Y[i]) > y_floor ? fabs(Y[i]) : y_floor;
            double e = fabs(G[i]) / sc;
            if (e > err) err = e;
        }
        if (!(err == err)) break;
        if (err <= tol) { ok = it; break; }
    }
    free(G); free(J); free(fb);
    return ok;
}

/* Fixed-step backward Euler over [t_start, t_end] with n_steps equal steps
 * (constant or profiled conditions evaluated at each step's end time). */
int or_be_fixed(const or_net *n, const or_zone *z, double *Y, int64_t n_steps, double tol,
                double y_floor, int max_iter)
{
    const int N = n->N;
    double *k = (double *)malloc(sizeof(double) * (size_t)n->R);
    double *Yn = (double *)malloc(sizeof(double) * (size_t)N);
    double h = (z->t_end - z->t_start) / (double)n_steps, T9, rho;
    int worst = 0;
    for (int64_t s = 0; s < n_steps; ++s) {
        double t1 = z->t_start + (double)(s + 1) * h;
        or_conditions(z->T0, z->rho0, z->tau, t1, &T9, &rho);
        or_rates(n, T9, rho, k);
        int it = or_be_step(n, k, Y, h, Yn, tol, y_floor, max_iter);
        if (it < 0) { worst = -1; break; }
        if (it > worst) worst = it;
        memcpy(Y, Yn, sizeof(double) * (size_t)N);
    }
    free(k); free(Yn);
    return worst;
}

/* Adaptive backward Euler (the CPU implicit baseline): same accept test on
 * relative change (all species above y_min) as the explicit controller, and a
 * Newton failure (more than max_iter iterations) counts as a reject.
 * Implicit Euler conserves sum A Y up to the Newton tolerance, so eps_c is
 * not tested. */
void or_be_integrate(const or_net *n, const or_opts *o, const or_zone *z, double *Y,
                     or_result *res, int max_iter)
{
    const int N = n->N;
    double *k = (double *)malloc(sizeof(double) * (size_t)n->R);
    double *Yn = (double *)malloc(sizeof(double) * (size_t)N);
    double t = z->t_start, dt = z->dt_trial > 0.0 ? z->dt_trial : z->t_start, T9, rho;
    int64_t steps = 0, rejects = 0;
    int nrej = 0, status = OR_OK;
    while (t < z->t_end) {
        if (steps >= o->max_steps) { status = OR_STEP_LIMIT; break; }
        double rem = z->t_end - t;
        int clipped = dt >= rem;
        double h = clipped ? rem : dt;
        or_conditions(z->T0, z->rho0, z->tau, t + h, &T9, &rho);
        or_rates(n, T9, rho, k);
        int it = or_be_step(n, k, Y, h, Yn, 1e-10, o->y_min, max_iter);
        double rel = 0.0;
        int finite = 1;
        for (int i = 0; i < N; ++i) {
            if (!isfinite(Yn[i])) finite = 0;
            double m = Y[i] > Yn[i] ? Y[i] : Yn[i];
            if (m > o->y_min) {
                double r = fabs(Yn[i] - Y[i]) / m;
                if (r > rel) rel = r;
            }
        }
        if (it > 0 && finite && rel <= o->eps_r) {
            t = clipped ? z->t_end : t + h;
            memcpy(Y, Yn, sizeof(double) * (size_t)N);
            ++steps;
            nrej = 0;
            double g = o->safety * o->eps_r / (rel > 1e-300 ? rel : 1e-300);
            dt = h * (g < o->grow_max ? g : o->grow_max);
        } else {
            ++rejects;
            ++nrej;
            dt = h * o->shrink;
            if (nrej > o->max_reject) { status = OR_MAX_REJECT; break; }
            if (dt < o->dt_min_frac * t) { status = OR_DT_UNDERFLOW; break; }
        }
    }
    res->t = t;
    res->dt_next = dt;
    res->steps = steps;
    res->rejects = rejects;
    res->status = status;
    res->pad = 0;
    free(k); free(Yn);
}

void or_be_integrate_batch(const or_net *n, const or_opts *o, int32_t n_zones, const or_zone *zones,
                           double *Y, or_result *res, int32_t max_iter, int32_t n_threads)
{
    (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int32_t z = 0; z < n_zones; ++z)
        or_be_integrate(n, o, &zones[z], Y + (size_t)z * (size_t)n->N, &res[z], max_iter);
}
