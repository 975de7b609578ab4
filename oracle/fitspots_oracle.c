/*
 * FP64 oracle for implicit-amplitude Levenberg-Marquardt fitting of 2-D Gaussian
 * spots (Leutenegger & Weber, "Least-squares fitting of Gaussian spots on graphics
 * processing units", arXiv 2106.02045).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously-correct CPU
 * statement of what the GPU path computes. Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it. It shares no code, header, table or
 * constant with the CUDA library; the two agree only through the paper.
 *
 * Everything is double precision and per spot, in the paper's order:
 *   profile f_i(p) and its derivatives ............ Eq. 10, Eq. 11 (elliptic: by analogy)
 *   sums F, G, F(bold), G(bold) ................... Eq. 5
 *   implicit amplitudes alpha^, beta^ ............. Eq. 6
 *   squared error chi^2 ........................... Eq. 2
 *   derivative sums and gamma_j ................... Eq. 7
 *   amplitude derivatives d alpha^/dp, d beta^/dp . Eq. 8
 *   per-pixel Jacobian J_ij = dh_i/dp_j ........... second factor of Eq. 9
 *   damped normal equations ....................... Eq. 12, Eq. 14 (J^T J, J^T (g - h))
 *   damping schedule, stop criteria ............... Sec. "Levenberg-Marquardt algorithm",
 *                                                   the Fit2DGaussian listing (Sec.
 *                                                   "Implementation") and the criteria of
 *                                                   Sec. "Results and Discussion".
 * The Jacobian is formed explicitly pixel by pixel (Eq. 9 form); no sum expansion.
 *
 * Readings where the paper is silent or garbled (the CUDA path follows the same ones):
 *   R1  Eq. 12 sign: J = dh/dp, right-hand side J^T (g - h), p' = p + delta.
 *   R2  Eq. 13 "Jacobian" is the per-pixel J_ij = dh_i/dp_j; J^T J is P x P.
 *   R3  inside the lambda-escalation loop the re-evaluated error is the trial error.
 *   R4  the listing's "NotConverged" after that loop is split: a step below minStep
 *       without decrease -> NO_DECREASE (converged class); otherwise NOT_CONVERGED.
 *   R6  minStep is relative: |delta_j| < min_step * |best_j| (benchmark criterion iii).
 *   R7  maxError ("A/3") is an absolute, caller-supplied chi^2 threshold.
 *   R8  limit(): x in [-0.5, W-0.5], y in [-0.5, H-0.5], each sigma in [0.25, max(W,H)].
 *   R9  normalised chi^2 = chi^2 / (N - P - 2).
 *   R10 stop tests after an accepted step in the order MAX_ERROR, MIN_DELTA, MIN_STEP;
 *       a trial error equal to the best error is accepted (and then meets MIN_DELTA).
 *   R11 lambda = 10^k with integer k, k = -2 at the start of each fit; "lambda < 10^4"
 *       is k < 4 (exactly the paper's schedule, free of rounding in the comparison).
 *   R12 the elliptic (axis-aligned) model, parameters (x, y, sigma_x, sigma_y).
 *   R13 a ROI has at most 1024 pixels (the paper's bound on the pixels of one fit) and
 *       both sides at least 3, so the longer side is at most 341; the explicit and weighted
 *       comparison fits keep both sides at most 32.
 * Pixel i of a W x H spot sits at x_i = i mod W, y_i = floor(i / W) (row-major).
 *
 * parity unpinned: limit() bounds (R8) and the maxError default (R7) are conventions; the
 * CUDA path follows the same readings, nothing in the paper fixes them. The normalised chi^2
 * (R9) is pinned statistically: chi^2 / (N - P - 2) is the unbiased residual variance, mean
 * 1 for unit white noise (tests/test_oracle_pins.py). The damping schedule (R11) is not pinned by a printed value either: changes
 * to it leave the fits and the paper's statistics unchanged (only the GPU-vs-oracle
 * iteration histograms compare it). The NO_DECREASE exit (R4), the escalation loop's exit
 * and the order of the stop tests are pinned by the stop-condition shares the paper
 * reports, through the second build below.
 *
 * A second build of this file, with -DOR_PAPER_ARITHMETIC, serves one pin only: the stop
 * conditions the paper reports for its own implementation (Results, "Number of
 * Levenberg-Marquardt iterations"). Two things change there and nothing else:
 *   chi^2 is formed as that implementation forms it (Sec. "Implementation": every value a
 *       32-bit float, one thread per pixel, per-fit sums over the threads): each residual
 *       in FP32 from the FP32-rounded alpha^, beta^, f_i and g_i, the squares summed in
 *       FP32 by a pairwise tree over a power-of-two number of threads (a reading: the
 *       reduction order is not given);
 *   the minStep test takes x and y relative to the ROI centre, |delta_j| <
 *       min_step |p_j - c_j| with c = ((W-1)/2, (H-1)/2) (a reading of criterion iii).
 * The default build keeps FP64 and the pixel-index origin of R6.
 *
 * A third build, with -DOR_FP32_PROFILE, also serves one measurement only: how far the fit
 * moves when the profile f_i and its derivatives df_i/dp_j (Eq. 10, 11) are rounded to the
 * nearest FP32 value, with everything after them (amplitudes, chi^2, normal equations,
 * solve) in FP64. It measures how well any implementation that evaluates the model in
 * 32-bit floats (as the paper's does, Sec. "Implementation") can agree with the FP64 fit.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_PIXELS 1024
#define OR_MAX_SIDE 32 /* sides of the explicit and weighted comparison fits */

/* spot models */
#define OR_MODEL_ISO 0
#define OR_MODEL_ELLIPTIC 1
/* image element types (the oracle also takes fp64 images for exact-recovery tests) */
#define OR_U16 0
#define OR_F32 1
#define OR_F64 2
/* per-spot outcome */
#define OR_MAX_ITER 0
#define OR_MIN_DELTA 1
#define OR_MIN_STEP 2
#define OR_MAX_ERROR 3
#define OR_NO_DECREASE 4
#define OR_NOT_CONVERGED (-1)
#define OR_INVALID (-2)

int or_nparams(int model) { return model == OR_MODEL_ISO ? 3 : 4; }

/* Profile f_i(p) (Eq. 10; elliptic by analogy) and, if d != NULL, its partial
 * derivatives d[j*N + i] = df_i/dp_j (Eq. 11). */
void or_profile(int model, int W, int H, const double *p, double *f, double *d)
{
    const int N = W * H;
    for (int i = 0; i < N; ++i) {
        const double x = (double)(i % W), y = (double)(i / W);
        const double dx = x - p[0], dy = y - p[1];
        if (model == OR_MODEL_ISO) {
            const double s = p[2];
            const double q = dx * dx + dy * dy;
            const double fi = exp(-q / (2.0 * s * s));
            f[i] = fi;
            if (d) {
                d[0 * N + i] = dx / (s * s) * fi;
                d[1 * N + i] = dy / (s * s) * fi;
                d[2 * N + i] = q / (s * s * s) * fi;
            }
        } else {
            const double sx = p[2], sy = p[3];
            const double fi = exp(-dx * dx / (2.0 * sx * sx) - dy * dy / (2.0 * sy * sy));
            f[i] = fi;
            if (d) {
                d[0 * N + i] = dx / (sx * sx) * fi;
                d[1 * N + i] = dy / (sy * sy) * fi;
                d[2 * N + i] = dx * dx / (sx * sx * sx) * fi;
                d[3 * N + i] = dy * dy / (sy * sy * sy) * fi;
            }
        }
#ifdef OR_FP32_PROFILE
        /* the third build (see the header): the profile and its derivatives rounded to the
         * nearest FP32 value, everything after them in FP64 */
        f[i] = (double)(float)f[i];
        if (d)
            for (int j = 0; j < or_nparams(model); ++j) d[j * N + i] = (double)(float)d[j * N + i];
#endif
    }
}

/* Implicit amplitudes, Eq. 5 and Eq. 6. Returns 0, or -1 when N F(bold) - F^2 is not
 * positive and finite (no unique solution). */
int or_amplitudes(int N, const double *f, const double *g, double *alpha, double *beta)
{
    double F = 0.0, G = 0.0, FF = 0.0, FG = 0.0;
    for (int i = 0; i < N; ++i) {
        F += f[i];
        G += g[i];
        FF += f[i] * f[i];
        FG += f[i] * g[i];
    }
    const double D = (double)N * FF - F * F;
    if (!(D > 0.0) || !isfinite(D)) return -1;
    *alpha = ((double)N * FG - F * G) / D;
    *beta = (G * FF - F * FG) / D;
    return 0;
}

/* Squared error of Eq. 2 at given amplitudes; r (optional) receives g_i - h_i. */
double or_chi2(int N, const double *f, const double *g, double alpha, double beta, double *r)
{
#ifdef OR_PAPER_ARITHMETIC
    /* the second build (see the header): FP32 residuals, one per pixel thread, summed in
     * FP32 by a pairwise tree as the paper's per-fit Sum over threads would */
    float t[OR_MAX_PIXELS];
    int m = 1;
    while (m < N) m <<= 1;
    for (int i = 0; i < m; ++i) {
        if (i < N) {
            const float ri = (float)g[i] - ((float)alpha * (float)f[i] + (float)beta);
            if (r) r[i] = ri;
            t[i] = ri * ri;
        } else {
            t[i] = 0.0f;
        }
    }
    for (int h = m / 2; h > 0; h /= 2)
        for (int i = 0; i < h; ++i) t[i] += t[i + h];
    return (double)t[0];
#else
    double c2 = 0.0;
    for (int i = 0; i < N; ++i) {
        const double ri = g[i] - (alpha * f[i] + beta);
        if (r) r[i] = ri;
        c2 += ri * ri;
    }
    return c2;
#endif
}

/* Per-pixel Jacobian J[j*N + i] = dh_i/dp_j of the implicit-amplitude model
 * h_i = alpha^(p) f_i(p) + beta^(p): the second factor of Eq. 9, with the amplitude
 * derivatives of Eq. 8 built from the sums of Eq. 7. Also returns alpha^, beta^ and
 * their derivatives. Returns 0, or -1 if the amplitudes are undefined. */
int or_jacobian(int model, int W, int H, const double *g, const double *p, double *J,
                double *alpha, double *beta, double *dalpha, double *dbeta)
{
    const int N = W * H, P = or_nparams(model);
    double f[OR_MAX_PIXELS], d[4 * OR_MAX_PIXELS];
    or_profile(model, W, H, p, f, d);
    double a, b;
    if (or_amplitudes(N, f, g, &a, &b)) return -1;
    double F = 0.0, G = 0.0, FF = 0.0, FG = 0.0;
    for (int i = 0; i < N; ++i) {
        F += f[i];
        G += g[i];
        FF += f[i] * f[i];
        FG += f[i] * g[i];
    }
    const double D = (double)N * FF - F * F;
    for (int j = 0; j < P; ++j) {
        const double *dj = d + (size_t)j * N;
        double dF = 0.0, dFF = 0.0, dG = 0.0;           /* Eq. 7 */
        for (int i = 0; i < N; ++i) {
            dF += dj[i];
            dFF += 2.0 * f[i] * dj[i];
            dG += g[i] * dj[i];
        }
        const double gamma = (double)N * dFF - 2.0 * F * dF;
        const double da = ((double)N * dG - G * dF - a * gamma) / D;            /* Eq. 8 */
        const double db = (G * dFF - FG * dF - F * dG - b * gamma) / D;
        if (dalpha) dalpha[j] = da;
        if (dbeta) dbeta[j] = db;
        for (int i = 0; i < N; ++i) J[(size_t)j * N + i] = da * f[i] + a * dj[i] + db;
    }
    *alpha = a;
    *beta = b;
    return 0;
}

/* One evaluated point: alpha^, beta^, chi^2 and, if A != NULL, the normal equations
 * A = J^T J and b = J^T (g - h) of Eq. 12. Returns 0, or -1 (amplitudes undefined). */
static int evaluate(int model, int W, int H, const double *g, const double *p,
                    double *alpha, double *beta, double *chi2, double A[4][4], double b[4])
{
    const int N = W * H, P = or_nparams(model);
    double f[OR_MAX_PIXELS], r[OR_MAX_PIXELS];
    if (!A) {
        or_profile(model, W, H, p, f, NULL);
        if (or_amplitudes(N, f, g, alpha, beta)) return -1;
        *chi2 = or_chi2(N, f, g, *alpha, *beta, r);
        return 0;
    }
    double J[4 * OR_MAX_PIXELS];
    if (or_jacobian(model, W, H, g, p, J, alpha, beta, NULL, NULL)) return -1;
    or_profile(model, W, H, p, f, NULL);
    *chi2 = or_chi2(N, f, g, *alpha, *beta, r);
    for (int j = 0; j < P; ++j) {
        double bj = 0.0;
        for (int i = 0; i < N; ++i) bj += J[(size_t)j * N + i] * r[i];
        b[j] = bj;
        for (int k = 0; k < P; ++k) {
            double ajk = 0.0;
            for (int i = 0; i < N; ++i) ajk += J[(size_t)j * N + i] * J[(size_t)k * N + i];
            A[j][k] = ajk;
        }
    }
    return 0;
}

/* Reading R8: clamp a parameter vector to the spot's box. */
void or_limit(int model, int W, int H, double *p)
{
    const double smax = (double)(W > H ? W : H);
    if (p[0] < -0.5) p[0] = -0.5;
    if (p[0] > W - 0.5) p[0] = W - 0.5;
    if (p[1] < -0.5) p[1] = -0.5;
    if (p[1] > H - 0.5) p[1] = H - 0.5;
    const int ns = model == OR_MODEL_ISO ? 1 : 2;
    for (int j = 2; j < 2 + ns; ++j) {
        if (p[j] < 0.25) p[j] = 0.25;
        if (p[j] > smax) p[j] = smax;
    }
}

/* Eq. 14: delta = (A + lambda diag A)^-1 b by a plain Cholesky factorisation.
 * Returns 0, or -1 when the damped matrix is not positive definite. */
static int solve_damped(int P, double A[4][4], const double *b, double lambda, double *delta)
{
    double M[4][4], L[4][4] = {{0}}, y[4];
    for (int j = 0; j < P; ++j)
        for (int k = 0; k < P; ++k) M[j][k] = A[j][k] + (j == k ? lambda * A[j][j] : 0.0);
    for (int j = 0; j < P; ++j) {
        double s = M[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0) || !isfinite(s)) return -1;
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < P; ++i) {
            double t = M[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    for (int j = 0; j < P; ++j) {
        double t = b[j];
        for (int k = 0; k < j; ++k) t -= L[j][k] * y[k];
        y[j] = t / L[j][j];
    }
    for (int j = P - 1; j >= 0; --j) {
        double t = y[j];
        for (int k = j + 1; k < P; ++k) t -= L[k][j] * delta[k];
        delta[j] = t / L[j][j];
    }
    for (int j = 0; j < P; ++j)
        if (!isfinite(delta[j])) return -1;
    return 0;
}

/* An evaluated point: amplitudes, the objective and, if A != NULL, the normal equations;
 * returns 0, or -1 when the point cannot be evaluated. */
typedef int (*or_eval_fn)(int model, int W, int H, const double *g, const double *p,
                          double *alpha, double *beta, double *obj, double A[4][4], double b[4]);

/* The trial point limit(best + delta) and its objective; NaN if it cannot be evaluated. */
static double trial(or_eval_fn eval, int model, int W, int H, const double *g,
                    const double *best, const double *delta, double *pt, double *at, double *bt)
{
    const int P = or_nparams(model);
    pt[0] = best[0] + delta[0];
    pt[1] = best[1] + delta[1];
    pt[2] = best[2] + delta[2];
    pt[3] = P == 4 ? best[3] + delta[3] : pt[2];
    or_limit(model, W, H, pt);
    if (P == 3) pt[3] = pt[2];
    double c2;
    if (eval(model, W, H, g, pt, at, bt, &c2, NULL, NULL)) return NAN;
    return c2;
}

static int all_small(int P, int W, int H, const double *delta, const double *best,
                     double min_step)
{
    for (int j = 0; j < P; ++j) {
        double ref = best[j];
#ifdef OR_PAPER_ARITHMETIC
        if (j == 0) ref -= 0.5 * (W - 1);
        if (j == 1) ref -= 0.5 * (H - 1);
#else
        (void)W;
        (void)H;
#endif
        if (!(fabs(delta[j]) < min_step * fabs(ref))) return 0;
    }
    return 1;
}

/* A point of the search: parameters, the amplitudes of Eq. 6 there and the error of Eq. 2. */
typedef struct {
    double p[4], alpha, beta, chi2;
} or_point;

/* One spot under fit: model, size, data, the shape-parameter count, the tolerances and the
 * objective's evaluation. */
typedef struct {
    int model, W, H, P;
    const double *g;
    double max_error, min_delta, min_step;
    or_eval_fn eval;
} or_spot;

/* Outcomes of the damping search of one iteration. */
#define OR_SEARCH_DECREASED 0 /* a trial point lowered (or kept) the error          */
#define OR_SEARCH_STALLED 1   /* the step fell below minStep without a decrease     */
#define OR_SEARCH_FAILED 2    /* no solvable damped system, a NaN, or damping 10^4  */
/* Stop-test result meaning "take another iteration". */
#define OR_CONTINUE 100

/* One damped step from `from` (Eq. 14 with lambda = 10^k) and its trial point
 * limit(from + delta) with amplitudes and error (Eq. 6, Eq. 2). Returns -1 when the damped
 * normal matrix is not positive definite, else 0 (the trial error may be NaN). */
static int damped_trial(const or_spot *sp, double A[4][4], const double *b, int k,
                        const or_point *from, double *delta, or_point *to, int *evals)
{
    if (solve_damped(sp->P, A, b, pow(10.0, k), delta)) return -1;
    ++*evals;
    to->chi2 = trial(sp->eval, sp->model, sp->W, sp->H, sp->g, from->p, delta, to->p,
                     &to->alpha, &to->beta);
    return 0;
}

/* The damping search of one iteration (Sec. "Levenberg-Marquardt algorithm"): the first
 * trial uses the damping carried over from the last iteration, and a decrease there relaxes
 * the damping tenfold for the next one; while the trial error exceeds the current error, the
 * step is not yet below minStep and lambda < 10^4, the damping grows tenfold and the step is
 * solved again from the same normal equations (readings R3, R11). An equal error counts as a
 * decrease (R10). The last step is left in delta and the last trial point in `next`. */
static int damping_search(const or_spot *sp, double A[4][4], const double *b, int *k,
                          const or_point *cur, or_point *next, double *delta, int *evals)
{
    if (damped_trial(sp, A, b, *k, cur, delta, next, evals)) return OR_SEARCH_FAILED;
    if (next->chi2 < cur->chi2) --*k;
    while (cur->chi2 < next->chi2 && *k < 4 &&
           !all_small(sp->P, sp->W, sp->H, delta, cur->p, sp->min_step)) {
        ++*k;
        if (damped_trial(sp, A, b, *k, cur, delta, next, evals)) return OR_SEARCH_FAILED;
    }
    if (isnan(next->chi2)) return OR_SEARCH_FAILED;
    if (cur->chi2 < next->chi2)  /* R4: a step below minStep without decrease, or lambda 10^4 */
        return all_small(sp->P, sp->W, sp->H, delta, cur->p, sp->min_step) ? OR_SEARCH_STALLED
                                                                           : OR_SEARCH_FAILED;
    return OR_SEARCH_DECREASED;
}

/* Stop tests after an accepted step from `from` (error chi_from) to an error chi_to, in the
 * order of reading R10: maxError, minDelta (relative decrease), minStep (reading R6). */
static int stop_test(const or_spot *sp, const or_point *from, double chi_to, const double *delta)
{
    if (chi_to < sp->max_error) return OR_MAX_ERROR;
    if (from->chi2 * (1.0 - sp->min_delta) < chi_to) return OR_MIN_DELTA;
    if (all_small(sp->P, sp->W, sp->H, delta, from->p, sp->min_step)) return OR_MIN_STEP;
    return OR_CONTINUE;
}

/* One spot: the damped LM iteration of Sec. "Levenberg-Marquardt algorithm" with the stop
 * criteria of the Fit2DGaussian listing. Every iteration evaluates the current point with
 * its normal equations, runs the damping search and either moves to the trial point or
 * stops. p0 is the caller's start point (4 values; the isotropic model uses p0[2] as sigma).
 * Outputs p (4 values; isotropic writes sigma into both slots 2 and 3), alpha^, beta^,
 * normalised chi^2, outcome, iterations and the number of evaluated points. trace
 * (max_iter + 1 values, or NULL) receives the error at the start of every iteration followed
 * by the final error; unused slots are NaN. */
static int fit_one_with(or_eval_fn eval, int model, int W, int H, const double *g,
                        const double *p0, int max_iter, double max_error, double min_delta,
                        double min_step, double *p_out, double *alpha_out, double *beta_out,
                        double *chi2n_out, int *iters_out, int *evals_out, double *trace)
{
    const or_spot sp = {model, W, H, or_nparams(model), g, max_error, min_delta, min_step, eval};
    or_point cur = {{p0[0], p0[1], p0[2], sp.P == 4 ? p0[3] : p0[2]}, 0.0, 0.0, 0.0};
    or_limit(model, W, H, cur.p);
    if (sp.P == 3) cur.p[3] = cur.p[2];
    if (trace)
        for (int k = 0; k <= max_iter; ++k) trace[k] = NAN;

    int k_lambda = -2; /* lambda = 10^k, 0.01 at the start of every fit (R11) */
    int it = 0, evals = 0, state = OR_MAX_ITER;
    double A[4][4], b[4], delta[4];
    while (it < max_iter) {
        ++it;
        ++evals;
        if (eval(model, W, H, g, cur.p, &cur.alpha, &cur.beta, &cur.chi2, A, b))
            cur.chi2 = NAN;
        if (trace) trace[it - 1] = cur.chi2;
        if (isnan(cur.chi2)) { state = OR_NOT_CONVERGED; break; }
        if (cur.chi2 < max_error) { state = OR_MAX_ERROR; break; }

        or_point next;
        const int search = damping_search(&sp, A, b, &k_lambda, &cur, &next, delta, &evals);
        if (search == OR_SEARCH_FAILED) { state = OR_NOT_CONVERGED; break; }
        if (search == OR_SEARCH_STALLED) { state = OR_NO_DECREASE; break; }
        const int stop = stop_test(&sp, &cur, next.chi2, delta);
        cur = next; /* accepted: the search continues from the trial point */
        if (stop != OR_CONTINUE) { state = stop; break; }
    }

    /* final error at the reported parameters (the listing's NormalizedChi) */
    double a, bb, chi;
    if (eval(model, W, H, g, cur.p, &a, &bb, &chi, NULL, NULL)) { a = bb = chi = NAN; }
    if (trace) trace[it < max_iter ? it : max_iter] = chi;
    for (int j = 0; j < 4; ++j) p_out[j] = cur.p[j];
    *alpha_out = a;
    *beta_out = bb;
    *chi2n_out = chi / (double)(W * H - sp.P - 2);
    *iters_out = it;
    *evals_out = evals;
    return state;
}

int or_fit_one(int model, int W, int H, const double *g, const double *p0, int max_iter,
               double max_error, double min_delta, double min_step, double *p_out,
               double *alpha_out, double *beta_out, double *chi2n_out, int *iters_out,
               int *evals_out, double *trace)
{
    return fit_one_with(evaluate, model, W, H, g, p0, max_iter, max_error, min_delta, min_step,
                        p_out, alpha_out, beta_out, chi2n_out, iters_out, evals_out, trace);
}

/* Batch front end with the library's argument layout. images: element buffer of
 * `dtype`; spot s occupies elements [offsets[s], offsets[s] + W*H) row-major; dims holds
 * (W, H) per spot; init holds 4 floats per spot. Spots with W or H outside 3..32,
 * W*H <= P + 2, an unknown model or an out-of-range offset get OR_INVALID, their init
 * parameters back and NaN amplitudes. trace: NULL or n * (max_iter + 1) doubles. */
void or_fit_spots(const void *images, int dtype, int64_t image_elems, const int64_t *offsets,
                  const int32_t *dims, const float *init, const uint8_t *model, int64_t n,
                  int max_iter, double max_error, double min_delta, double min_step,
                  double *out_params, double *out_alpha, double *out_beta, double *out_chi2,
                  int32_t *out_state, int32_t *out_iters, int32_t *out_evals, double *trace,
                  int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n; ++s) {
        const int W = dims[2 * s], H = dims[2 * s + 1], m = model[s];
        const int64_t off = offsets[s];
        double p0[4] = {init[4 * s], init[4 * s + 1], init[4 * s + 2], init[4 * s + 3]};
        double *tr = trace ? trace + s * (int64_t)(max_iter + 1) : NULL;
        const int valid_model = (m == OR_MODEL_ISO || m == OR_MODEL_ELLIPTIC);
        const int sides_ok = W >= 3 && H >= 3 && W <= OR_MAX_PIXELS / 3 && H <= OR_MAX_PIXELS / 3;
        const int N = sides_ok ? W * H : 0;
        if (!valid_model || !sides_ok || N > OR_MAX_PIXELS || N <= or_nparams(m) + 2 || off < 0 ||
            off + N > image_elems) {
            for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p0[j];
            out_alpha[s] = out_beta[s] = out_chi2[s] = NAN;
            out_state[s] = OR_INVALID;
            out_iters[s] = 0;
            if (out_evals) out_evals[s] = 0;
            if (tr)
                for (int k = 0; k <= max_iter; ++k) tr[k] = NAN;
            continue;
        }
        double g[OR_MAX_PIXELS];
        for (int i = 0; i < N; ++i) {
            if (dtype == OR_U16) g[i] = (double)((const uint16_t *)images)[off + i];
            else if (dtype == OR_F32) g[i] = (double)((const float *)images)[off + i];
            else g[i] = ((const double *)images)[off + i];
        }
        double p[4], a, b, c2n;
        int it, ev;
        const int st = or_fit_one(m, W, H, g, p0, max_iter, max_error, min_delta, min_step, p,
                                  &a, &b, &c2n, &it, &ev, tr);
        for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p[j];
        out_alpha[s] = a;
        out_beta[s] = b;
        out_chi2[s] = c2n;
        out_state[s] = st;
        out_iters[s] = it;
        if (out_evals) out_evals[s] = ev;
    }
}

/* ------------------------------------------------------------------ explicit LM
 * The comparison method of the paper's claim that implicit amplitudes need fewer
 * iterations (Sec. "Results and Discussion"): plain LM over the full vector
 * q = (x, y, sigma[, sigma_y], alpha, beta) with the model h_i = alpha f_i + beta, the
 * per-pixel Jacobian (alpha df_i/dp_j, f_i, 1), the same damping schedule, limit() box on
 * the shape parameters and stop criteria as or_fit_one. Readings: alpha and beta are not
 * boxed; the minStep test covers the shape parameters (as for the implicit method, so both
 * stop on the same criteria); start amplitudes alpha0 = max g - min g, beta0 = min g. */
static int evaluate_explicit(int model, int W, int H, const double *g, const double *q,
                             double *chi2, double A[6][6], double b[6])
{
    const int N = W * H, P = or_nparams(model), Q = P + 2;
    double f[OR_MAX_PIXELS], d[4 * OR_MAX_PIXELS];
    const double p[4] = {q[0], q[1], q[2], P == 4 ? q[3] : q[2]};
    const double alpha = q[P], beta = q[P + 1];
    or_profile(model, W, H, p, f, A ? d : NULL);
    double c2 = 0.0;
    if (A)
        for (int j = 0; j < Q; ++j) {
            b[j] = 0.0;
            for (int k = 0; k < Q; ++k) A[j][k] = 0.0;
        }
    for (int i = 0; i < N; ++i) {
        const double r = g[i] - (alpha * f[i] + beta);
        c2 += r * r;
        if (!A) continue;
        double J[6];
        for (int j = 0; j < P; ++j) J[j] = alpha * d[(size_t)j * N + i];
        J[P] = f[i];
        J[P + 1] = 1.0;
        for (int j = 0; j < Q; ++j) {
            b[j] += J[j] * r;
            for (int k = 0; k < Q; ++k) A[j][k] += J[j] * J[k];
        }
    }
    *chi2 = c2;
    return isfinite(c2) ? 0 : -1;
}

/* Eq. 14 for up to 6 unknowns: (A + lambda diag A) delta = b by Cholesky. */
static int solve_damped6(int Q, double A[6][6], const double *b, double lambda, double *delta)
{
    double L[6][6] = {{0}}, y[6];
    for (int j = 0; j < Q; ++j) {
        double s = A[j][j] * (1.0 + lambda);
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0) || !isfinite(s)) return -1;
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < Q; ++i) {
            double t = A[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    for (int j = 0; j < Q; ++j) {
        double t = b[j];
        for (int k = 0; k < j; ++k) t -= L[j][k] * y[k];
        y[j] = t / L[j][j];
    }
    for (int j = Q - 1; j >= 0; --j) {
        double t = y[j];
        for (int k = j + 1; k < Q; ++k) t -= L[k][j] * delta[k];
        delta[j] = t / L[j][j];
    }
    for (int j = 0; j < Q; ++j)
        if (!isfinite(delta[j])) return -1;
    return 0;
}

static double trial_explicit(int model, int W, int H, const double *g, const double *best,
                             const double *delta, double *qt)
{
    const int P = or_nparams(model), Q = P + 2;
    double p[4];
    for (int j = 0; j < Q; ++j) qt[j] = best[j] + delta[j];
    p[0] = qt[0];
    p[1] = qt[1];
    p[2] = qt[2];
    p[3] = P == 4 ? qt[3] : qt[2];
    or_limit(model, W, H, p);
    for (int j = 0; j < P; ++j) qt[j] = p[j];
    double c2;
    if (evaluate_explicit(model, W, H, g, qt, &c2, NULL, NULL)) return NAN;
    return c2;
}

int or_fit_explicit_one(int model, int W, int H, const double *g, const double *p0,
                        int max_iter, double max_error, double min_delta, double min_step,
                        double *p_out, double *alpha_out, double *beta_out, double *chi2n_out,
                        int *iters_out, int *evals_out)
{
    const int P = or_nparams(model), Q = P + 2, N = W * H;
    double p[4] = {p0[0], p0[1], p0[2], P == 4 ? p0[3] : p0[2]};
    or_limit(model, W, H, p);
    double gmin = g[0], gmax = g[0];
    for (int i = 1; i < N; ++i) {
        if (g[i] < gmin) gmin = g[i];
        if (g[i] > gmax) gmax = g[i];
    }
    double q[6], best[6], delta[6], qt[6], A[6][6], b[6];
    for (int j = 0; j < P; ++j) q[j] = p[j];
    q[P] = gmax - gmin;
    q[P + 1] = gmin;

    int k_lambda = -2, it = 0, evals = 0, state = OR_MAX_ITER;
    while (it < max_iter) {
        ++it;
        double chi;
        ++evals;
        if (evaluate_explicit(model, W, H, g, q, &chi, A, b)) chi = NAN;
        if (isnan(chi)) { state = OR_NOT_CONVERGED; break; }
        if (chi < max_error) { state = OR_MAX_ERROR; break; }
        memcpy(best, q, sizeof best);
        double Chi;
        if (solve_damped6(Q, A, b, pow(10.0, k_lambda), delta)) { state = OR_NOT_CONVERGED; break; }
        ++evals;
        Chi = trial_explicit(model, W, H, g, best, delta, qt);
        if (chi > Chi) --k_lambda;
        int failed_solve = 0;
        while (!all_small(P, W, H, delta, best, min_step) && chi < Chi && k_lambda < 4) {
            ++k_lambda;
            if (solve_damped6(Q, A, b, pow(10.0, k_lambda), delta)) { failed_solve = 1; break; }
            ++evals;
            Chi = trial_explicit(model, W, H, g, best, delta, qt);
        }
        if (failed_solve) { state = OR_NOT_CONVERGED; break; }
        if (chi < Chi || isnan(Chi)) {
            state = (all_small(P, W, H, delta, best, min_step) && !isnan(Chi)) ? OR_NO_DECREASE
                                                                         : OR_NOT_CONVERGED;
            break;
        }
        memcpy(q, qt, sizeof q);
        if (Chi < max_error) { state = OR_MAX_ERROR; break; }
        if (chi * (1.0 - min_delta) < Chi) { state = OR_MIN_DELTA; break; }
        if (all_small(P, W, H, delta, best, min_step)) { state = OR_MIN_STEP; break; }
    }
    double chi;
    if (evaluate_explicit(model, W, H, g, q, &chi, NULL, NULL)) chi = NAN;
    for (int j = 0; j < 4; ++j) p_out[j] = j < P ? q[j] : q[2];
    *alpha_out = q[P];
    *beta_out = q[P + 1];
    *chi2n_out = chi / (double)(N - P - 2);
    *iters_out = it;
    *evals_out = evals;
    return state;
}

void or_fit_spots_explicit(const void *images, int dtype, int64_t image_elems,
                           const int64_t *offsets, const int32_t *dims, const float *init,
                           const uint8_t *model, int64_t n, int max_iter, double max_error,
                           double min_delta, double min_step, double *out_params,
                           double *out_alpha, double *out_beta, double *out_chi2,
                           int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                           int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n; ++s) {
        const int W = dims[2 * s], H = dims[2 * s + 1], m = model[s];
        const int64_t off = offsets[s];
        double p0[4] = {init[4 * s], init[4 * s + 1], init[4 * s + 2], init[4 * s + 3]};
        const int N = W * H;
        if (!(m == OR_MODEL_ISO || m == OR_MODEL_ELLIPTIC) || W < 3 || H < 3 ||
            W > OR_MAX_SIDE || H > OR_MAX_SIDE || N <= or_nparams(m) + 2 || off < 0 ||
            off + N > image_elems) {
            for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p0[j];
            out_alpha[s] = out_beta[s] = out_chi2[s] = NAN;
            out_state[s] = OR_INVALID;
            out_iters[s] = 0;
            if (out_evals) out_evals[s] = 0;
            continue;
        }
        double g[OR_MAX_PIXELS];
        for (int i = 0; i < N; ++i) {
            if (dtype == OR_U16) g[i] = (double)((const uint16_t *)images)[off + i];
            else if (dtype == OR_F32) g[i] = (double)((const float *)images)[off + i];
            else g[i] = ((const double *)images)[off + i];
        }
        double p[4], a, b, c2n;
        int it, ev;
        const int st = or_fit_explicit_one(m, W, H, g, p0, max_iter, max_error, min_delta,
                                           min_step, p, &a, &b, &c2n, &it, &ev);
        for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p[j];
        out_alpha[s] = a;
        out_beta[s] = b;
        out_chi2[s] = c2n;
        out_state[s] = st;
        out_iters[s] = it;
        if (out_evals) out_evals[s] = ev;
    }
}

/* ------------------------------------------------------------------ weighted fit
 * A variance-weighted variant (the paper notes that its residuals are unweighted and gives
 * no weighted method; readings): chi^2_w = sum w_i (g_i - h_i)^2 with w_i = 1 / max(g_i, 1),
 * the Poisson variance estimated from the data (Neyman's chi^2). The implicit amplitudes
 * solve the weighted normal equations of Eq. 5-6,
 *   [Sff Sf; Sf Sw] (alpha, beta) = (Sfg, Sg),  Sw = sum w, Sf = sum w f, Sff = sum w f^2,
 *   Sg = sum w g, Sfg = sum w f g,
 * their derivatives follow Eq. 7-8 with the same weights, J_ij = dh_i/dp_j as in Eq. 9, and
 * the LM step uses J^T W J and J^T W (g - h). Damping schedule, box and stop tests as
 * or_fit_one; with unit weights this is exactly the unweighted fit. */
static int weighted_jacobian(int model, int W, int H, const double *g, const double *w,
                             const double *p, double *f, double *J, double *alpha, double *beta)
{
    const int N = W * H, P = or_nparams(model);
    double d[4 * OR_MAX_PIXELS];
    or_profile(model, W, H, p, f, J ? d : NULL);
    double Sw = 0.0, Sf = 0.0, Sff = 0.0, Sg = 0.0, Sfg = 0.0;
    for (int i = 0; i < N; ++i) {
        Sw += w[i];
        Sf += w[i] * f[i];
        Sff += w[i] * f[i] * f[i];
        Sg += w[i] * g[i];
        Sfg += w[i] * f[i] * g[i];
    }
    const double D = Sw * Sff - Sf * Sf;
    if (!(D > 0.0) || !isfinite(D)) return -1;
    const double a = (Sw * Sfg - Sf * Sg) / D, b = (Sff * Sg - Sf * Sfg) / D;
    *alpha = a;
    *beta = b;
    if (!J) return 0;
    for (int j = 0; j < P; ++j) {
        const double *dj = d + (size_t)j * N;
        double dSf = 0.0, dSff = 0.0, dSfg = 0.0;
        for (int i = 0; i < N; ++i) {
            dSf += w[i] * dj[i];
            dSff += 2.0 * w[i] * f[i] * dj[i];
            dSfg += w[i] * g[i] * dj[i];
        }
        /* differentiate Sff a + Sf b = Sfg and Sf a + Sw b = Sg in p_j */
        const double r1 = dSfg - dSff * a - dSf * b, r2 = -dSf * a;
        const double da = (Sw * r1 - Sf * r2) / D, db = (Sff * r2 - Sf * r1) / D;
        for (int i = 0; i < N; ++i) J[(size_t)j * N + i] = da * f[i] + a * dj[i] + db;
    }
    return 0;
}

static int evaluate_weighted(int model, int W, int H, const double *g, const double *w,
                             const double *p, double *alpha, double *beta, double *chi2,
                             double A[4][4], double b[4])
{
    const int N = W * H, P = or_nparams(model);
    double f[OR_MAX_PIXELS], J[4 * OR_MAX_PIXELS];
    if (weighted_jacobian(model, W, H, g, w, p, f, A ? J : NULL, alpha, beta)) return -1;
    double c2 = 0.0, r[OR_MAX_PIXELS];
    for (int i = 0; i < N; ++i) {
        r[i] = g[i] - (*alpha * f[i] + *beta);
        c2 += w[i] * r[i] * r[i];
    }
    *chi2 = c2;
    if (!A) return 0;
    for (int j = 0; j < P; ++j) {
        double bj = 0.0;
        for (int i = 0; i < N; ++i) bj += J[(size_t)j * N + i] * w[i] * r[i];
        b[j] = bj;
        for (int k = 0; k < P; ++k) {
            double ajk = 0.0;
            for (int i = 0; i < N; ++i) ajk += J[(size_t)j * N + i] * w[i] * J[(size_t)k * N + i];
            A[j][k] = ajk;
        }
    }
    return 0;
}

static double trial_weighted(int model, int W, int H, const double *g, const double *w,
                             const double *best, const double *delta, double *pt)
{
    const int P = or_nparams(model);
    pt[0] = best[0] + delta[0];
    pt[1] = best[1] + delta[1];
    pt[2] = best[2] + delta[2];
    pt[3] = P == 4 ? best[3] + delta[3] : pt[2];
    or_limit(model, W, H, pt);
    if (P == 3) pt[3] = pt[2];
    double a, bb, c2;
    if (evaluate_weighted(model, W, H, g, w, pt, &a, &bb, &c2, NULL, NULL)) return NAN;
    return c2;
}

/* weights: NULL for 1 / max(g, 1), or one per pixel */
int or_fit_weighted_one(int model, int W, int H, const double *g, const double *weights,
                        const double *p0, int max_iter, double max_error, double min_delta,
                        double min_step, double *p_out, double *alpha_out, double *beta_out,
                        double *chi2n_out, int *iters_out, int *evals_out)
{
    const int P = or_nparams(model), N = W * H;
    double w[OR_MAX_PIXELS];
    for (int i = 0; i < N; ++i) w[i] = weights ? weights[i] : 1.0 / (g[i] > 1.0 ? g[i] : 1.0);
    double p[4] = {p0[0], p0[1], p0[2], P == 4 ? p0[3] : p0[2]};
    or_limit(model, W, H, p);
    if (P == 3) p[3] = p[2];
    int k_lambda = -2, it = 0, evals = 0, state = OR_MAX_ITER;
    double A[4][4], b[4], best[4], delta[4], pt[4];
    while (it < max_iter) {
        ++it;
        double a, bb, chi;
        ++evals;
        if (evaluate_weighted(model, W, H, g, w, p, &a, &bb, &chi, A, b)) chi = NAN;
        if (isnan(chi)) { state = OR_NOT_CONVERGED; break; }
        if (chi < max_error) { state = OR_MAX_ERROR; break; }
        memcpy(best, p, sizeof best);
        double Chi;
        if (solve_damped(P, A, b, pow(10.0, k_lambda), delta)) { state = OR_NOT_CONVERGED; break; }
        ++evals;
        Chi = trial_weighted(model, W, H, g, w, best, delta, pt);
        if (chi > Chi) --k_lambda;
        int failed_solve = 0;
        while (!all_small(P, W, H, delta, best, min_step) && chi < Chi && k_lambda < 4) {
            ++k_lambda;
            if (solve_damped(P, A, b, pow(10.0, k_lambda), delta)) { failed_solve = 1; break; }
            ++evals;
            Chi = trial_weighted(model, W, H, g, w, best, delta, pt);
        }
        if (failed_solve) { state = OR_NOT_CONVERGED; break; }
        if (chi < Chi || isnan(Chi)) {
            state = (all_small(P, W, H, delta, best, min_step) && !isnan(Chi)) ? OR_NO_DECREASE
                                                                         : OR_NOT_CONVERGED;
            break;
        }
        memcpy(p, pt, sizeof p);
        if (Chi < max_error) { state = OR_MAX_ERROR; break; }
        if (chi * (1.0 - min_delta) < Chi) { state = OR_MIN_DELTA; break; }
        if (all_small(P, W, H, delta, best, min_step)) { state = OR_MIN_STEP; break; }
    }
    double a, bb, chi;
    if (evaluate_weighted(model, W, H, g, w, p, &a, &bb, &chi, NULL, NULL)) { a = bb = chi = NAN; }
    for (int j = 0; j < 4; ++j) p_out[j] = p[j];
    *alpha_out = a;
    *beta_out = bb;
    *chi2n_out = chi / (double)(N - P - 2);
    *iters_out = it;
    *evals_out = evals;
    return state;
}

void or_fit_spots_weighted(const void *images, int dtype, int64_t image_elems,
                           const int64_t *offsets, const int32_t *dims, const float *init,
                           const uint8_t *model, int64_t n, int max_iter, double max_error,
                           double min_delta, double min_step, double *out_params,
                           double *out_alpha, double *out_beta, double *out_chi2,
                           int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                           int unit_weights, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n; ++s) {
        const int W = dims[2 * s], H = dims[2 * s + 1], m = model[s];
        const int64_t off = offsets[s];
        double p0[4] = {init[4 * s], init[4 * s + 1], init[4 * s + 2], init[4 * s + 3]};
        const int N = W * H;
        if (!(m == OR_MODEL_ISO || m == OR_MODEL_ELLIPTIC) || W < 3 || H < 3 ||
            W > OR_MAX_SIDE || H > OR_MAX_SIDE || N <= or_nparams(m) + 2 || off < 0 ||
            off + N > image_elems) {
            for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p0[j];
            out_alpha[s] = out_beta[s] = out_chi2[s] = NAN;
            out_state[s] = OR_INVALID;
            out_iters[s] = 0;
            if (out_evals) out_evals[s] = 0;
            continue;
        }
        double g[OR_MAX_PIXELS], ones[OR_MAX_PIXELS];
        for (int i = 0; i < N; ++i) {
            if (dtype == OR_U16) g[i] = (double)((const uint16_t *)images)[off + i];
            else if (dtype == OR_F32) g[i] = (double)((const float *)images)[off + i];
            else g[i] = ((const double *)images)[off + i];
            ones[i] = 1.0;
        }
        double p[4], a, b, c2n;
        int it, ev;
        const int st = or_fit_weighted_one(m, W, H, g, unit_weights ? ones : NULL, p0, max_iter,
                                           max_error, min_delta, min_step, p, &a, &b, &c2n,
                                           &it, &ev);
        for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p[j];
        out_alpha[s] = a;
        out_beta[s] = b;
        out_chi2[s] = c2n;
        out_state[s] = st;
        out_iters[s] = it;
        if (out_evals) out_evals[s] = ev;
    }
}

/* Pin helper: alpha^, beta^, chi^2 (Eq. 2, 6) and optionally J^T J, J^T (g-h) at p for
 * one spot given as doubles. Returns 0 or -1. */
int or_evaluate(int model, int W, int H, const double *g, const double *p, double *alpha,
                double *beta, double *chi2, double *A16, double *b4)
{
    double A[4][4], b[4];
    const int with_grad = A16 != NULL;
    if (evaluate(model, W, H, g, p, alpha, beta, chi2, with_grad ? A : NULL, b)) return -1;
    if (with_grad) {
        const int P = or_nparams(model);
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 4; ++k) A16[4 * j + k] = (j < P && k < P) ? A[j][k] : 0.0;
        for (int j = 0; j < 4; ++j) b4[j] = j < P ? b[j] : 0.0;
    }
    return 0;
}

/* Pin helper: the damped solve of Eq. 14 on a caller-given P x P system. */
int or_solve_damped(int P, const double *A16, const double *b, double lambda, double *delta)
{
    double A[4][4];
    for (int j = 0; j < 4; ++j)
        for (int k = 0; k < 4; ++k) A[j][k] = A16[4 * j + k];
    return solve_damped(P, A, b, lambda, delta);
}

/* ------------------------------------------------------------------------------------
 * Backward pass by the implicit-function theorem (not in the paper; derived from Eq. 2).
 * At a minimum of chi^2 over the full parameter vector q = (p, alpha, beta) the gradient
 * -sum_i r_i K_i vanishes, with K_i = dh_i/dq = (alpha df_i/dp, f_i, 1) and r = g - h.
 * Differentiating that condition in g_i gives dq/dg_i = M^-1 K_i with
 *   M = sum_i K_i K_i^T - sum_i r_i d^2 h_i / dq^2,
 * d^2 h/dp^2 = alpha d^2 f/dp^2, d^2 h/dp dalpha = df/dp, all other second derivatives 0.
 * A vector-Jacobian product with upstream u is then grad_g_i = (M^-1 u) . K_i; the
 * normalised chi^2 adds u_chi * 2 r_i / (N - P - 2) (its g-derivative at the minimum).
 * ------------------------------------------------------------------------------------ */

/* Second derivatives d2[(j*P+k)*N + i] = d^2 f_i / dp_j dp_k of the profile. */
void or_profile_second(int model, int W, int H, const double *p, double *d2)
{
    const int N = W * H, P = or_nparams(model);
    for (int i = 0; i < N; ++i) {
        const double x = (double)(i % W), y = (double)(i / W);
        const double dx = x - p[0], dy = y - p[1];
        double h[4][4];
        if (model == OR_MODEL_ISO) {
            const double s = p[2], s2 = s * s, q = dx * dx + dy * dy;
            const double f = exp(-q / (2.0 * s2));
            h[0][0] = (dx * dx / (s2 * s2) - 1.0 / s2) * f;
            h[1][1] = (dy * dy / (s2 * s2) - 1.0 / s2) * f;
            h[0][1] = h[1][0] = dx * dy / (s2 * s2) * f;
            h[0][2] = h[2][0] = (dx * q / (s2 * s2 * s) - 2.0 * dx / (s2 * s)) * f;
            h[1][2] = h[2][1] = (dy * q / (s2 * s2 * s) - 2.0 * dy / (s2 * s)) * f;
            h[2][2] = (q * q / (s2 * s2 * s2) - 3.0 * q / (s2 * s2)) * f;
        } else {
            const double sx = p[2], sy = p[3], sx2 = sx * sx, sy2 = sy * sy;
            const double f = exp(-dx * dx / (2.0 * sx2) - dy * dy / (2.0 * sy2));
            const double ax = dx / sx2, ay = dy / sy2;                 /* d ln f / d x0, y0 */
            const double bx = dx * dx / (sx2 * sx), by = dy * dy / (sy2 * sy); /* d ln f / d sx, sy */
            h[0][0] = (ax * ax - 1.0 / sx2) * f;
            h[1][1] = (ay * ay - 1.0 / sy2) * f;
            h[0][1] = h[1][0] = ax * ay * f;
            h[0][2] = h[2][0] = (ax * bx - 2.0 * dx / (sx2 * sx)) * f;
            h[1][3] = h[3][1] = (ay * by - 2.0 * dy / (sy2 * sy)) * f;
            h[0][3] = h[3][0] = ax * by * f;
            h[1][2] = h[2][1] = ay * bx * f;
            h[2][2] = (bx * bx - 3.0 * dx * dx / (sx2 * sx2)) * f;
            h[3][3] = (by * by - 3.0 * dy * dy / (sy2 * sy2)) * f;
            h[2][3] = h[3][2] = bx * by * f;
        }
        for (int j = 0; j < P; ++j)
            for (int k = 0; k < P; ++k) d2[((size_t)j * P + k) * N + i] = h[j][k];
    }
}

/* Solve A x = b (n <= 6) by Gaussian elimination with partial pivoting; -1 if singular. */
static int solve_dense(int n, double A[6][6], double *b)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (!(fabs(A[piv][c]) > 0.0) || !isfinite(A[piv][c])) return -1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            const double m = A[r][c] / A[c][c];
            for (int k = c; k < n; ++k) A[r][k] -= m * A[c][k];
            b[r] -= m * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double t = b[r];
        for (int k = r + 1; k < n; ++k) t -= A[r][k] * b[k];
        b[r] = t / A[r][r];
    }
    return 0;
}

/* Vector-Jacobian product of one fit. p (4 values; isotropic uses p[2]), alpha, beta:
 * the fitted point. upstream[7] = d loss / d (x0, y0, s_x, s_y, alpha, beta, chi2_norm);
 * for the isotropic model the fitted sigma is reported in slots 2 and 3, so its upstream
 * is upstream[2] + upstream[3]. grad_g receives N values. Returns 0, or -1 if M is
 * singular. */
int or_backward(int model, int W, int H, const double *g, const double *p, double alpha,
                double beta, const double *upstream, double *grad_g)
{
    const int N = W * H, P = or_nparams(model), Q = P + 2;
    double f[OR_MAX_PIXELS], d[4 * OR_MAX_PIXELS], d2[16 * OR_MAX_PIXELS];
    or_profile(model, W, H, p, f, d);
    or_profile_second(model, W, H, p, d2);
    double M[6][6] = {{0}}, v[6];
    for (int i = 0; i < N; ++i) {
        double K[6];
        for (int j = 0; j < P; ++j) K[j] = alpha * d[(size_t)j * N + i];
        K[P] = f[i];
        K[P + 1] = 1.0;
        const double r = g[i] - (alpha * f[i] + beta);
        for (int a = 0; a < Q; ++a)
            for (int b = 0; b < Q; ++b) M[a][b] += K[a] * K[b];
        for (int j = 0; j < P; ++j) {
            for (int k = 0; k < P; ++k) M[j][k] -= r * alpha * d2[((size_t)j * P + k) * N + i];
            M[j][P] -= r * d[(size_t)j * N + i];
            M[P][j] -= r * d[(size_t)j * N + i];
        }
    }
    if (model == OR_MODEL_ISO) {
        v[0] = upstream[0];
        v[1] = upstream[1];
        v[2] = upstream[2] + upstream[3];
    } else {
        for (int j = 0; j < 4; ++j) v[j] = upstream[j];
    }
    v[P] = upstream[4];
    v[P + 1] = upstream[5];
    if (solve_dense(Q, M, v)) return -1;
    const double cchi = 2.0 * upstream[6] / (double)(N - P - 2);
    for (int i = 0; i < N; ++i) {
        double t = v[P] * f[i] + v[P + 1];
        for (int j = 0; j < P; ++j) t += v[j] * alpha * d[(size_t)j * N + i];
        grad_g[i] = t + cchi * (g[i] - (alpha * f[i] + beta));
    }
    return 0;
}

/* ------------------------------------------------------------------ Poisson likelihood
 * The variant for Poisson-distributed pixel counts. The paper fits unweighted residuals and
 * says so (Sec. "Discussion"); the likelihood of the counts is the efficient objective for
 * photon-counting images. The objective is the Poisson deviance
 *     D(p) = 2 sum_i [h_i - g_i + g_i ln(g_i / h_i)]      (the last term is 0 where g_i = 0)
 * (each term evaluated as g (u - ln(1 + u)), u = h/g - 1, so that its rounding shrinks with
 * the residual and the deviance of a near-perfect model keeps its digits)
 * of the model h = alpha f(p) + beta, with the amplitudes at their Poisson maximum
 * likelihood for the profile at p: the implicit amplitudes of Eq. 5-6 with the likelihood in
 * place of chi^2. Readings:
 *   - the amplitudes solve the score equations sum (g/h - 1) (f, 1) = 0 by iteratively
 *     reweighted least squares (weighted Eq. 5-6 with weights 1/h of the current means),
 *     started from the least-squares amplitudes of Eq. 6, each step halved until every mean
 *     stays positive and the deviance does not grow; a point where no positive means are
 *     found is not evaluated (NaN);
 *   - pixel values below 0 count as 0 (the counts of a Poisson model are not negative);
 *   - the gradient for Eq. 12 is -1/2 dD/dp = sum (g/h - 1) alpha df/dp (the amplitude terms
 *     vanish at their optimum), the normal matrix the Fisher information sum J J^T / h of the
 *     shape parameters with J = alpha df/dp - (c f + e) the part of alpha df/dp that the
 *     amplitudes cannot absorb ((c, e): its least squares on (f, 1) with weights 1/h);
 *   - damping schedule, limit() box and stop tests are those of or_fit_one, on D;
 *   - the reported normalised objective is D / (N - P - 2).
 * ROIs of at most 32 x 32 pixels, as for the other comparison fits. */
#define OR_IRLS_MAX 200

static double poisson_deviance(int N, const double *f, const double *g, double a, double b)
{
    double D = 0.0;
    for (int i = 0; i < N; ++i) {
        const double h = a * f[i] + b;
        if (!(h > 0.0)) return NAN;
        if (g[i] > 0.0) { /* g (u - ln(1 + u)) with u = h/g - 1: small where h is close to g */
            const double u = (h - g[i]) / g[i];
            D += g[i] * (u - log1p(u));
        } else {
            D += h;
        }
    }
    return 2.0 * D;
}

/* Poisson maximum-likelihood amplitudes for the profile f; 0, or -1 if none is found. */
int or_poisson_amplitudes(int N, const double *f, const double *g, double *alpha, double *beta)
{
    double a, b, G = 0.0;
    for (int i = 0; i < N; ++i) G += g[i] > 0.0 ? g[i] : 0.0;
    if (or_amplitudes(N, f, g, &a, &b)) return -1;
    double D = poisson_deviance(N, f, g, a, b);
    if (isnan(D)) { /* a least-squares mean below zero: start from a flat positive model */
        a = 0.0;
        b = G / N > 1e-3 ? G / N : 1e-3;
        D = poisson_deviance(N, f, g, a, b);
        if (isnan(D)) return -1;
    }
    /* the deviance is a sum of terms of the size of the counts that cancel near the optimum:
     * a change below its rounding (about eps times the total count) is no increase */
    const double tolD = 1e-13 * (G + (double)N);
    for (int it = 0; it < OR_IRLS_MAX; ++it) {
        double Sw = 0.0, Sf = 0.0, Sff = 0.0, Sg = 0.0, Sfg = 0.0;
        for (int i = 0; i < N; ++i) {
            const double w = 1.0 / (a * f[i] + b), gi = g[i] > 0.0 ? g[i] : 0.0;
            Sw += w;
            Sf += w * f[i];
            Sff += w * f[i] * f[i];
            Sg += w * gi;
            Sfg += w * f[i] * gi;
        }
        const double Dt = Sff * Sw - Sf * Sf;
        if (!(Dt > 0.0)) return -1;
        const double a1 = (Sw * Sfg - Sf * Sg) / Dt, b1 = (Sff * Sg - Sf * Sfg) / Dt;
        double t = 1.0, an = a1, bn = b1, Dn = poisson_deviance(N, f, g, an, bn);
        while ((isnan(Dn) || Dn > D + tolD) && t > 1e-12) {
            t *= 0.5;
            an = a + t * (a1 - a);
            bn = b + t * (b1 - b);
            Dn = poisson_deviance(N, f, g, an, bn);
        }
        if (isnan(Dn) || Dn > D + tolD) break; /* no further decrease: at the optimum */
        const int done = fabs(an - a) <= 1e-14 * (fabs(a) + fabs(b)) &&
                         fabs(bn - b) <= 1e-14 * (fabs(a) + fabs(b));
        a = an;
        b = bn;
        D = Dn;
        if (done) break;
    }
    *alpha = a;
    *beta = b;
    return 0;
}

/* One evaluated point of the Poisson fit: amplitudes, deviance and, if A != NULL, the
 * Fisher normal equations of the shape parameters (see above). */
static int evaluate_poisson(int model, int W, int H, const double *g, const double *p,
                            double *alpha, double *beta, double *dev, double A[4][4],
                            double bvec[4])
{
    const int N = W * H, P = or_nparams(model);
    double f[OR_MAX_PIXELS], d[4 * OR_MAX_PIXELS];
    or_profile(model, W, H, p, f, A ? d : NULL);
    double a, b;
    if (or_poisson_amplitudes(N, f, g, &a, &b)) return -1;
    const double D = poisson_deviance(N, f, g, a, b);
    if (isnan(D)) return -1;
    *alpha = a;
    *beta = b;
    *dev = D;
    if (!A) return 0;
    double Sw = 0.0, Sf = 0.0, Sff = 0.0;
    for (int i = 0; i < N; ++i) {
        const double w = 1.0 / (a * f[i] + b);
        Sw += w;
        Sf += w * f[i];
        Sff += w * f[i] * f[i];
    }
    const double Dt = Sff * Sw - Sf * Sf;
    if (!(Dt > 0.0)) return -1;
    double c[4], e[4];
    for (int j = 0; j < P; ++j) {
        double vf = 0.0, v1 = 0.0;
        for (int i = 0; i < N; ++i) {
            const double w = 1.0 / (a * f[i] + b), ad = a * d[(size_t)j * N + i];
            vf += w * f[i] * ad;
            v1 += w * ad;
        }
        c[j] = (Sw * vf - Sf * v1) / Dt;
        e[j] = (Sff * v1 - Sf * vf) / Dt;
    }
    for (int j = 0; j < P; ++j) {
        bvec[j] = 0.0;
        for (int k = 0; k < P; ++k) A[j][k] = 0.0;
    }
    for (int i = 0; i < N; ++i) {
        const double h = a * f[i] + b, w = 1.0 / h, gi = g[i] > 0.0 ? g[i] : 0.0;
        double J[4];
        for (int j = 0; j < P; ++j) J[j] = a * d[(size_t)j * N + i] - c[j] * f[i] - e[j];
        for (int j = 0; j < P; ++j) {
            bvec[j] += (gi - h) * w * J[j];
            for (int k = 0; k < P; ++k) A[j][k] += w * J[j] * J[k];
        }
    }
    return 0;
}

int or_fit_poisson_one(int model, int W, int H, const double *g, const double *p0, int max_iter,
                       double max_error, double min_delta, double min_step, double *p_out,
                       double *alpha_out, double *beta_out, double *dn_out, int *iters_out,
                       int *evals_out)
{
    return fit_one_with(evaluate_poisson, model, W, H, g, p0, max_iter, max_error, min_delta,
                        min_step, p_out, alpha_out, beta_out, dn_out, iters_out, evals_out, NULL);
}

/* Batch front end of the Poisson fit, the library's argument layout (W, H in 3..32). */
void or_fit_spots_poisson(const void *images, int dtype, int64_t image_elems,
                          const int64_t *offsets, const int32_t *dims, const float *init,
                          const uint8_t *model, int64_t n, int max_iter, double max_error,
                          double min_delta, double min_step, double *out_params,
                          double *out_alpha, double *out_beta, double *out_chi2,
                          int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                          int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < n; ++s) {
        const int W = dims[2 * s], H = dims[2 * s + 1], m = model[s];
        const int64_t off = offsets[s];
        double p0[4] = {init[4 * s], init[4 * s + 1], init[4 * s + 2], init[4 * s + 3]};
        const int valid_model = (m == OR_MODEL_ISO || m == OR_MODEL_ELLIPTIC);
        const int sides_ok = W >= 3 && H >= 3 && W <= OR_MAX_SIDE && H <= OR_MAX_SIDE;
        const int N = sides_ok ? W * H : 0;
        if (!valid_model || !sides_ok || N <= or_nparams(m) + 2 || off < 0 || off + N > image_elems) {
            for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p0[j];
            out_alpha[s] = out_beta[s] = out_chi2[s] = NAN;
            out_state[s] = OR_INVALID;
            out_iters[s] = 0;
            if (out_evals) out_evals[s] = 0;
            continue;
        }
        double g[OR_MAX_PIXELS];
        for (int i = 0; i < N; ++i) {
            if (dtype == OR_U16) g[i] = (double)((const uint16_t *)images)[off + i];
            else if (dtype == OR_F32) g[i] = (double)((const float *)images)[off + i];
            else g[i] = ((const double *)images)[off + i];
        }
        double p[4], a, b, dn;
        int it, ev;
        const int st = or_fit_poisson_one(m, W, H, g, p0, max_iter, max_error, min_delta,
                                          min_step, p, &a, &b, &dn, &it, &ev);
        for (int j = 0; j < 4; ++j) out_params[4 * s + j] = p[j];
        out_alpha[s] = a;
        out_beta[s] = b;
        out_chi2[s] = dn;
        out_state[s] = st;
        out_iters[s] = it;
        if (out_evals) out_evals[s] = ev;
    }
}

/* ------------------------------------------------------------------ local background
 * The paper assumes a uniform background in the ROI and remarks (Sec. "Implicit-amplitudes
 * least-squares fitting") that a locally varying background may be estimated and
 * subtracted before the fit; it gives no method. Reading: a plane
 *     b(x, y) = c0 + cx (x - xc) + cy (y - yc),   xc = (W - 1) / 2, yc = (H - 1) / 2,
 * fitted by least squares to the ROI's border ring (the pixels within `border` of an edge,
 * where a spot centred in its ROI contributes nothing), and its tilt cx (x - xc) +
 * cy (y - yc) subtracted from every pixel of the ROI. The level c0 is kept: the uniform
 * beta of the fit takes it up, and the counts stay near their original scale.
 * Output images are double, same element layout; only the ROIs' pixels are written.
 * out_plane (n x 3: c0, cx, cy) may be NULL. An ROI with a side below 3, more than
 * OR_MAX_PIXELS pixels, a border outside 1..8 or an offset outside the image gets NaN
 * coefficients and no output pixels. */
void or_subtract_background(const void *images, int dtype, int64_t image_elems,
                            const int64_t *offsets, const int32_t *dims, int64_t n, int border,
                            double *out_images, double *out_plane)
{
    for (int64_t s = 0; s < n; ++s) {
        const int W = dims[2 * s], H = dims[2 * s + 1];
        const int64_t off = offsets[s];
        double *pl = out_plane ? out_plane + 3 * s : NULL;
        if (W < 3 || H < 3 || W > OR_MAX_PIXELS / 3 || H > OR_MAX_PIXELS / 3 ||
            W * H > OR_MAX_PIXELS || border < 1 || border > 8 || off < 0 ||
            off + (int64_t)W * H > image_elems) {
            if (pl) pl[0] = pl[1] = pl[2] = NAN;
            continue;
        }
        const double xc = 0.5 * (W - 1), yc = 0.5 * (H - 1);
        double M[6][6] = {{0}}, v[6] = {0};
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                if (x >= border && x < W - border && y >= border && y < H - border) continue;
                const int64_t i = off + (int64_t)y * W + x;
                const double gi = dtype == OR_U16 ? (double)((const uint16_t *)images)[i]
                                : dtype == OR_F32 ? (double)((const float *)images)[i]
                                                  : ((const double *)images)[i];
                const double a[3] = {1.0, x - xc, y - yc};
                for (int j = 0; j < 3; ++j) {
                    v[j] += a[j] * gi;
                    for (int k = 0; k < 3; ++k) M[j][k] += a[j] * a[k];
                }
            }
        if (solve_dense(3, M, v)) {
            if (pl) pl[0] = pl[1] = pl[2] = NAN;
            continue;
        }
        if (pl) {
            pl[0] = v[0];
            pl[1] = v[1];
            pl[2] = v[2];
        }
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t i = off + (int64_t)y * W + x;
                const double gi = dtype == OR_U16 ? (double)((const uint16_t *)images)[i]
                                : dtype == OR_F32 ? (double)((const float *)images)[i]
                                                  : ((const double *)images)[i];
                out_images[i] = gi - v[1] * (x - xc) - v[2] * (y - yc);
            }
    }
}
