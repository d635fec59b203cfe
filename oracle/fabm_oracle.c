/*
 * fabm_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * Plain, slow, CPU-only restatement of the fractional Adams-Bashforth-Moulton
 * (ABM) predictor-corrector for Caputo systems D^alpha y = f(t, y), as stated in
 * Section 2 of Bonchis, Kaslik, Rosu, "HPC optimal parallel communication
 * algorithm for the simulation of fractional-order systems" (arXiv:1710.01133):
 *
 *   grid            t_n = n h, n = 0..N, f_n = f(t_n, y_n)            (Sec. 2)
 *   Taylor part     T(t) = sum_{k < ceil(a)} t^k/k! y^(k)(0)  = y_0 (+ t y'_0 for 1 < a < 2)
 *   predictor       y^P_{n+1} = T(t_{n+1}) + h^a sum_{k=0}^{n} b_{n-k} f_k   (Eq. abm)
 *   corrector       y_{n+1}   = T(t_{n+1}) + h^a ( c_n f_0
 *                               + sum_{k=1}^{n} a_{n-k} f_k
 *                               + f(t_{n+1}, y^P_{n+1}) / Gamma(a+2) )  (Sec. 2)
 *   weights         b_n = ((n+1)^a - n^a) / Gamma(a+1)                  (Eq. abm)
 *                   a_n = ((n+2)^{a+1} - 2(n+1)^{a+1} + n^{a+1}) / Gamma(a+2)
 *                   c_n = (n^{a+1} - (n-a)(n+1)^a) / Gamma(a+2)         (Sec. 2)
 *   systems         componentwise                                      (Sec. 2)
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - b_n is printed with "+" between the two powers; the scheme the paper
 *     cites (Diethelm's fractional Adams method) has "-", which is also the only
 *     sign for which the weights telescope to (n+1)^a / Gamma(a+1) and the
 *     scheme reproduces constant right-hand sides.  "-" is used.
 *   - 0^p = 0 for p > 0, so b_0 = 1/Gamma(a+1) and c_0 = a/Gamma(a+2).
 *   - one predictor and one corrector evaluation per step (PECE); f_{n+1} is
 *     evaluated at the corrected value, as the grid definition says.
 *   - 0 < a < 2: the Taylor part is y_0 for a <= 1 and y_0 + t y'_0 for
 *     1 < a < 2 (the sum over k < ceil(a) of Sec. 2's formulas).
 *
 * Precision.  The weights are evaluated from the direct formulas above in
 * binary128 (_Float128) and rounded once to double: the second difference in
 * a_n cancels about 2 log2(n) bits, which binary128 absorbs for every n this
 * code is used with.  Every history sum is a compensated dot product (Dot2 of
 * Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
 * 26 (2005), Algorithm 5.3), i.e. as accurate as if it were evaluated in twice
 * the working precision and then rounded.  The sums run in the order the
 * formulas write them (k ascending); nothing is blocked or reordered.
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * load this file.  It shares no code with the CUDA library.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef _Float128 q128;

/* Right-hand sides known to the oracle (its own numbering; the Python wrapper
 * maps names to these). */
enum {
    ORC_CONST = 0,        /* f_i = p0                                       */
    ORC_TIME = 1,         /* f_i = t                                        */
    ORC_LINEAR = 2,       /* f_i = -p0 * y_i                                */
    ORC_LORENZ = 3,       /* fractional Lorenz-type system, dim 3           */
    ORC_DUFFING = 4,      /* forced oscillator with cubic capacitor, dim 2  */
    ORC_MANUFACTURED = 5, /* f = p0 t^p1 + t^p2 - y (solution t^p2), dim 1  */
    ORC_LCR = 6           /* the paper's forced series LCR system (Sec. 5)  */
};

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };

/* ---------------------------------------------------------------- RHS --- */

/* Piecewise-linear characteristic g of the LCR system (Sec. 5). */
static double orc_lcr_g(double x, double a, double b)
{
    if (x <= -1.0) return b * x - a + b;
    if (x >= 1.0) return b * x + a - b;
    return a * x;
}

/* f(t, y) for one state vector; params as documented per right-hand side. */
static void orc_rhs(int rhs, int dim, double t, const double *y, const double *p, double *out)
{
    switch (rhs) {
    case ORC_CONST:
        for (int i = 0; i < dim; ++i) out[i] = p[0];
        break;
    case ORC_TIME:
        for (int i = 0; i < dim; ++i) out[i] = t;
        break;
    case ORC_LINEAR:
        for (int i = 0; i < dim; ++i) out[i] = -p[0] * y[i];
        break;
    case ORC_LORENZ: /* p = (sigma, rho, beta) */
        out[0] = p[0] * (y[1] - y[0]);
        out[1] = y[0] * (p[1] - y[2]) - y[1];
        out[2] = y[0] * y[1] - p[2] * y[2];
        break;
    case ORC_DUFFING: /* p = (damping gamma, forcing frequency omega, amplitude F) */
        out[0] = y[1];
        out[1] = -p[0] * y[1] - y[0] - y[0] * y[0] * y[0] + p[2] * cos(p[1] * t);
        break;
    case ORC_MANUFACTURED: /* p = (kappa, q, r): f = kappa t^q + t^r - y */
        out[0] = p[0] * pow(t, p[1]) + pow(t, p[2]) - y[0];
        break;
    case ORC_LCR: /* p = (sigma, omega, a, b, f), Eq. sys.LRC */
        out[0] = y[1] - orc_lcr_g(y[0], p[2], p[3]);
        out[1] = -p[0] * y[1] - y[0] + p[4] * sin(p[1] * t);
        break;
    default:
        for (int i = 0; i < dim; ++i) out[i] = NAN;
    }
}

static int orc_rhs_dim_ok(int rhs, int dim, int np)
{
    switch (rhs) {
    case ORC_CONST: return dim >= 1 && np >= 1;
    case ORC_TIME: return dim >= 1;
    case ORC_LINEAR: return dim >= 1 && np >= 1;
    case ORC_LORENZ: return dim == 3 && np >= 3;
    case ORC_DUFFING: return dim == 2 && np >= 3;
    case ORC_MANUFACTURED: return dim == 1 && np >= 3;
    case ORC_LCR: return dim == 2 && np >= 5;
    default: return 0;
    }
}

int fabm_oracle_rhs(int rhs, int dim, double t, const double *y, const double *params,
                    int n_params, double *out)
{
    if (!orc_rhs_dim_ok(rhs, dim, n_params)) return ORC_EINVAL;
    orc_rhs(rhs, dim, t, y, params, out);
    return ORC_OK;
}

/* ------------------------------------------------------------ weights --- */

/* x^p in binary128 with the convention 0^p = 0 for p > 0. */
static q128 orc_powq(q128 x, q128 p)
{
    if (x == 0) return 0;
    return powf128(x, p);
}

/* b_j, a_j, c_j for j = 0..n-1 (Sec. 2), each rounded once from binary128.
 * Uses P[j] = j^alpha and j^{alpha+1} = j * P[j]. */
int fabm_oracle_weights(double alpha, int64_t n, double *b, double *a, double *c)
{
    if (!(alpha > 0.0 && alpha < 2.0) || n < 1) return ORC_EINVAL;
    q128 *P = (q128 *)malloc((size_t)(n + 2) * sizeof(q128));
    if (!P) return ORC_ENOMEM;
    const q128 al = (q128)alpha;
    for (int64_t j = 0; j < n + 2; ++j) P[j] = orc_powq((q128)j, al);
    const q128 g1 = tgammaf128(al + 1);
    const q128 g2 = tgammaf128(al + 2);
    for (int64_t j = 0; j < n; ++j) {
        const q128 j0 = (q128)j, j1 = (q128)(j + 1), j2 = (q128)(j + 2);
        if (b) b[j] = (double)((P[j + 1] - P[j]) / g1);
        if (a) a[j] = (double)((j2 * P[j + 2] - 2 * (j1 * P[j + 1]) + j0 * P[j]) / g2);
        if (c) c[j] = (double)((j0 * P[j] - (j0 - al) * P[j + 1]) / g2);
    }
    free(P);
    return ORC_OK;
}

/* h^alpha, 1/Gamma(alpha+2) rounded once from binary128. */
int fabm_oracle_constants(double alpha, double h, double *h_alpha, double *inv_gamma2)
{
    if (!(alpha > 0.0 && alpha < 2.0) || !(h > 0.0)) return ORC_EINVAL;
    if (h_alpha) *h_alpha = (double)powf128((q128)h, (q128)alpha);
    if (inv_gamma2) *inv_gamma2 = (double)(1 / tgammaf128((q128)alpha + 2));
    return ORC_OK;
}

/* --------------------------------------------------------------- sums --- */

/* Knuth's TwoSum: s + e == a + b exactly. */
static inline void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

/* sum_{k=k0}^{k1} w[n-k] * f[k*stride], compensated (Dot2, Ogita-Rump-Oishi)
 * or plain, k ascending. */
static double orc_hist_dot(const double *w, int64_t n, const double *f, int64_t stride,
                           int64_t k0, int64_t k1, int compensated)
{
    if (k1 < k0) return 0.0;
    if (!compensated) {
        double s = 0.0;
        for (int64_t k = k0; k <= k1; ++k) s += w[n - k] * f[k * stride];
        return s;
    }
    double p = w[n - k0] * f[k0 * stride];
    double s = fma(w[n - k0], f[k0 * stride], -p);
    for (int64_t k = k0 + 1; k <= k1; ++k) {
        double x = w[n - k], y = f[k * stride];
        double hp = x * y;
        double r = fma(x, y, -hp);
        double q;
        two_sum(p, hp, &p, &q);
        s += q + r;
    }
    return p + s;
}

/* --------------------------------------------------------------- solve --- */

/* One trajectory with caller-given weights (b, a, c of length >= N) and
 * constants; out holds (N+1) x dim values, row n = y_n. f_work holds
 * (N+1) x dim doubles of scratch.  y1 = y'(0) (dim values) enters the Taylor
 * part for 1 < a < 2; NULL means the Taylor part is y_0 alone. */
static int orc_solve_one_multi(int dim, double h, int64_t N, int rhs, const double *p,
                               const double *b, const double *a, const double *c,
                               int64_t wstride, const double *h_alpha, const double *inv_gamma2,
                               const int *taylor2, const double *y0, const double *y1,
                               double *out, double *fw, int compensated);

static int orc_solve_one(int dim, double h, int64_t N, int rhs, const double *p,
                         const double *b, const double *a, const double *c, double h_alpha,
                         double inv_gamma2, const double *y0, const double *y1, double *out,
                         double *fw, int compensated)
{
    double ha[8], ig[8];
    int t2[8];
    for (int i = 0; i < dim; ++i) ha[i] = h_alpha, ig[i] = inv_gamma2, t2[i] = y1 != NULL;
    return orc_solve_one_multi(dim, h, N, rhs, p, b, a, c, 0, ha, ig, t2, y0, y1, out, fw,
                               compensated);
}

/* The same with an order alpha_i per component (Sec. 5's systems carry one
 * order per equation): component i uses the weights b + i*wstride (a, c
 * likewise), h^alpha_i and 1/Gamma(alpha_i+2), and its Taylor part
 * y0_i + t y1_i when taylor2[i] (1 < alpha_i < 2), else y0_i. */
static int orc_solve_one_multi(int dim, double h, int64_t N, int rhs, const double *p,
                               const double *b, const double *a, const double *c,
                               int64_t wstride, const double *h_alpha, const double *inv_gamma2,
                               const int *taylor2, const double *y0, const double *y1,
                               double *out, double *fw, int compensated)
{
    double yp[8], fp[8], yc[8], T[8];
    for (int i = 0; i < dim; ++i) out[i] = y0[i];
    orc_rhs(rhs, dim, 0.0, y0, p, fw);
    for (int64_t n = 0; n < N; ++n) {
        const double t1 = (double)(n + 1) * h;
        for (int i = 0; i < dim; ++i) T[i] = (y1 && taylor2[i]) ? y0[i] + t1 * y1[i] : y0[i];
        /* predictor, Eq. abm */
        for (int i = 0; i < dim; ++i) {
            double sp = orc_hist_dot(b + i * wstride, n, fw + i, dim, 0, n, compensated);
            yp[i] = T[i] + h_alpha[i] * sp;
        }
        orc_rhs(rhs, dim, t1, yp, p, fp);
        /* corrector */
        for (int i = 0; i < dim; ++i) {
            const double *ai = a + i * wstride, *ci = c + i * wstride;
            double sc = orc_hist_dot(ai, n, fw + i, dim, 1, n, compensated);
            if (compensated) {
                double s, e, pr = ci[n] * fw[i], pe = fma(ci[n], fw[i], -pr);
                two_sum(pr, sc, &s, &e);
                sc = s + (e + pe);
            } else {
                sc = ci[n] * fw[i] + sc;
            }
            yc[i] = T[i] + h_alpha[i] * (sc + fp[i] * inv_gamma2[i]);
        }
        for (int i = 0; i < dim; ++i) out[(n + 1) * dim + i] = yc[i];
        orc_rhs(rhs, dim, t1, yc, p, fw + (n + 1) * dim);
    }
    return ORC_OK;
}

/* Solve with explicit weight vectors (b, a, c each of length >= N). */
int fabm_oracle_solve_w(int dim, double h, int64_t N, int rhs, const double *params, int n_params,
                        const double *b, const double *a, const double *c, double h_alpha,
                        double inv_gamma2, const double *y0, const double *y1, double *out,
                        int compensated)
{
    if (dim < 1 || dim > 8 || N < 1 || !(h > 0.0) || !orc_rhs_dim_ok(rhs, dim, n_params))
        return ORC_EINVAL;
    double *fw = (double *)malloc((size_t)(N + 1) * dim * sizeof(double));
    if (!fw) return ORC_ENOMEM;
    int st = orc_solve_one(dim, h, N, rhs, params, b, a, c, h_alpha, inv_gamma2, y0, y1, out, fw,
                           compensated);
    free(fw);
    return st;
}

/* y1 = y'(0) for 1 < alpha < 2 (NULL: zero); must be NULL for alpha <= 1. */
int fabm_oracle_solve(int dim, double alpha, double h, int64_t N, int rhs, const double *params,
                      int n_params, const double *y0, const double *y1, double *out,
                      int compensated)
{
    if (dim < 1 || dim > 8 || N < 1 || !(h > 0.0) || !(alpha > 0.0 && alpha < 2.0) ||
        (y1 && alpha <= 1.0) || !orc_rhs_dim_ok(rhs, dim, n_params))
        return ORC_EINVAL;
    double *w = (double *)malloc((size_t)3 * N * sizeof(double));
    if (!w) return ORC_ENOMEM;
    double ha, ig2;
    int st = fabm_oracle_weights(alpha, N, w, w + N, w + 2 * N);
    if (st == ORC_OK) st = fabm_oracle_constants(alpha, h, &ha, &ig2);
    if (st == ORC_OK)
        st = fabm_oracle_solve_w(dim, h, N, rhs, params, n_params, w, w + N, w + 2 * N, ha, ig2,
                                 y0, y1, out, compensated);
    free(w);
    return st;
}

/* ------------------------------------------- threaded k-reduction --- */

/* A timing reference only (the CPU baseline's "Alg. 2" leg): one trajectory
 * with the k-sums of every step split over T threads, as the paper's
 * MPI+OpenMP version splits the history index over the threads of a node
 * (Alg. 2).  Thread t sums the contiguous share t of k = 0..n (compensated),
 * thread 0 adds the T partial sums in thread order with TwoSum and takes the
 * step; two barriers per step.  The result equals fabm_oracle_solve's up to
 * the order of the additions (the tests check 1e-13 of the solution scale). */
typedef struct {
    int dim, rhs, tid, nthreads;
    double h, h_alpha, inv_gamma2;
    int64_t N;
    const double *p, *w, *y0;
    double *out, *fw, *part; /* part[tid][2][dim]: predictor then corrector partials */
    pthread_barrier_t *bar;
    /* start gate: the workers run only once every thread has been created */
    pthread_mutex_t *mu;
    pthread_cond_t *cv;
    int *go, *ok;
} orc_thr_job;

static void *orc_thr_worker(void *arg)
{
    orc_thr_job *j = (orc_thr_job *)arg;
    pthread_mutex_lock(j->mu);
    while (!*j->go) pthread_cond_wait(j->cv, j->mu);
    const int ok = *j->ok;
    pthread_mutex_unlock(j->mu);
    if (!ok) return NULL;
    const int dim = j->dim, T = j->nthreads;
    const double *b = j->w, *a = j->w + j->N, *c = j->w + 2 * j->N;
    double yp[8], fpv[8], yc[8];
    for (int64_t n = 0; n < j->N; ++n) {
        const int64_t k0 = (n + 1) * j->tid / T, k1 = (n + 1) * (j->tid + 1) / T - 1;
        double *mine = j->part + (size_t)j->tid * 2 * dim;
        for (int i = 0; i < dim; ++i) {
            mine[i] = orc_hist_dot(b, n, j->fw + i, dim, k0, k1, 1);
            /* corrector: k = 1..n (k = 0 carries c_n, added by thread 0) */
            mine[dim + i] = orc_hist_dot(a, n, j->fw + i, dim, k0 > 1 ? k0 : 1, k1, 1);
        }
        pthread_barrier_wait(j->bar);
        if (j->tid == 0) {
            const double t1 = (double)(n + 1) * j->h;
            for (int i = 0; i < dim; ++i) {
                double s = 0.0, e = 0.0;
                for (int t = 0; t < T; ++t) {
                    double q;
                    two_sum(s, j->part[(size_t)t * 2 * dim + i], &s, &q);
                    e += q;
                }
                yp[i] = j->y0[i] + j->h_alpha * (s + e);
            }
            orc_rhs(j->rhs, dim, t1, yp, j->p, fpv);
            for (int i = 0; i < dim; ++i) {
                double pr = c[n] * j->fw[i], s = pr, e = fma(c[n], j->fw[i], -pr);
                for (int t = 0; t < T; ++t) {
                    double q;
                    two_sum(s, j->part[(size_t)t * 2 * dim + dim + i], &s, &q);
                    e += q;
                }
                yc[i] = j->y0[i] + j->h_alpha * ((s + e) + fpv[i] * j->inv_gamma2);
                j->out[(n + 1) * dim + i] = yc[i];
            }
            orc_rhs(j->rhs, dim, t1, yc, j->p, j->fw + (n + 1) * dim);
        }
        pthread_barrier_wait(j->bar);
    }
    return NULL;
}

/* One trajectory (0 < alpha <= 1) with the k-sums split over n_threads threads;
 * the threads are started once and meet at two barriers per step. */
int fabm_oracle_solve_threaded(int dim, double alpha, double h, int64_t N, int rhs,
                               const double *params, int n_params, const double *y0, double *out,
                               int n_threads)
{
    if (dim < 1 || dim > 8 || N < 1 || !(h > 0.0) || !(alpha > 0.0 && alpha <= 1.0) ||
        n_threads < 1 || n_threads > 256 || !orc_rhs_dim_ok(rhs, dim, n_params))
        return ORC_EINVAL;
    double *w = (double *)malloc((size_t)3 * N * sizeof(double));
    double *fw = (double *)malloc((size_t)(N + 1) * dim * sizeof(double));
    double *part = (double *)malloc((size_t)n_threads * 2 * dim * sizeof(double));
    orc_thr_job *jobs = (orc_thr_job *)malloc(sizeof(orc_thr_job) * (size_t)n_threads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    int st = (w && fw && part && jobs && th) ? ORC_OK : ORC_ENOMEM;
    double ha = 0.0, ig2 = 0.0;
    if (st == ORC_OK) st = fabm_oracle_weights(alpha, N, w, w + N, w + 2 * N);
    if (st == ORC_OK) st = fabm_oracle_constants(alpha, h, &ha, &ig2);
    pthread_barrier_t bar;
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    pthread_cond_t cv = PTHREAD_COND_INITIALIZER;
    int go = 0, ok = 0;
    if (st == ORC_OK && pthread_barrier_init(&bar, NULL, (unsigned)n_threads) != 0) st = ORC_ENOMEM;
    if (st == ORC_OK) {
        for (int i = 0; i < dim; ++i) out[i] = y0[i];
        orc_rhs(rhs, dim, 0.0, y0, params, fw);
        int started = 0;
        for (int t = 0; t < n_threads; ++t) {
            jobs[t] = (orc_thr_job){dim, rhs, t, n_threads, h, ha, ig2, N, params, w, y0, out, fw,
                                    part, &bar, &mu, &cv, &go, &ok};
            if (t > 0) {
                if (pthread_create(&th[t], NULL, orc_thr_worker, &jobs[t]) != 0) break;
                ++started;
            }
        }
        /* open the gate: run if every thread exists, else let the started ones return */
        pthread_mutex_lock(&mu);
        ok = started == n_threads - 1;
        go = 1;
        pthread_cond_broadcast(&cv);
        pthread_mutex_unlock(&mu);
        if (ok) orc_thr_worker(&jobs[0]);
        else st = ORC_ENOMEM;
        for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
        pthread_barrier_destroy(&bar);
    }
    free(w), free(fw), free(part), free(jobs), free(th);
    return st;
}

/* ------------------------------------------------ binary128 self-check --- */

/* f(t, y) in binary128, the formulas of orc_rhs. */
static void orc_rhs_q(int rhs, int dim, q128 t, const q128 *y, const q128 *p, q128 *out)
{
    switch (rhs) {
    case ORC_CONST:
        for (int i = 0; i < dim; ++i) out[i] = p[0];
        break;
    case ORC_TIME:
        for (int i = 0; i < dim; ++i) out[i] = t;
        break;
    case ORC_LINEAR:
        for (int i = 0; i < dim; ++i) out[i] = -p[0] * y[i];
        break;
    case ORC_LORENZ:
        out[0] = p[0] * (y[1] - y[0]);
        out[1] = y[0] * (p[1] - y[2]) - y[1];
        out[2] = y[0] * y[1] - p[2] * y[2];
        break;
    case ORC_DUFFING:
        out[0] = y[1];
        out[1] = -p[0] * y[1] - y[0] - y[0] * y[0] * y[0] + p[2] * cosf128(p[1] * t);
        break;
    case ORC_MANUFACTURED:
        out[0] = p[0] * orc_powq(t, p[1]) + orc_powq(t, p[2]) - y[0];
        break;
    case ORC_LCR: {
        const q128 x = y[0], a = p[2], b = p[3];
        const q128 g = x <= -1 ? b * x - a + b : (x >= 1 ? b * x + a - b : a * x);
        out[0] = y[1] - g;
        out[1] = -p[0] * y[1] - y[0] + p[4] * sinf128(p[1] * t);
        break;
    }
    default:
        for (int i = 0; i < dim; ++i) out[i] = NAN;
    }
}

/* The scheme of orc_solve_one with every quantity in binary128: the weights
 * from the printed formulas without rounding them to double, the sums in plain
 * binary128 (113-bit significands, ~90 bits left after 2^20 additions), t_n =
 * n h and the right-hand side in binary128, y rounded to double once for out.
 * It estimates the rounding of the double-precision oracle and is the
 * reference of the double-double mode.  One order, 0 < alpha < 2 (y1 = y'(0)
 * for alpha > 1, NULL: zero), one trajectory; cost O(N^2) binary128
 * operations, meant for N of a few thousand. */
int fabm_oracle_solve_q(int dim, double alpha, double h, int64_t N, int rhs, const double *params,
                        int n_params, const double *y0, const double *y1, double *out)
{
    if (dim < 1 || dim > 8 || N < 1 || !(h > 0.0) || !(alpha > 0.0 && alpha < 2.0) ||
        (y1 && alpha <= 1.0) || !orc_rhs_dim_ok(rhs, dim, n_params) || n_params > 16)
        return ORC_EINVAL;
    q128 *w = (q128 *)malloc((size_t)3 * N * sizeof(q128));
    q128 *P = (q128 *)malloc((size_t)(N + 2) * sizeof(q128));
    q128 *F = (q128 *)malloc((size_t)(N + 1) * dim * sizeof(q128));
    if (!w || !P || !F) {
        free(w), free(P), free(F);
        return ORC_ENOMEM;
    }
    const q128 al = (q128)alpha, hq = (q128)h;
    for (int64_t j = 0; j < N + 2; ++j) P[j] = orc_powq((q128)j, al);
    const q128 g1 = tgammaf128(al + 1), g2 = tgammaf128(al + 2);
    q128 *b = w, *a = w + N, *c = w + 2 * N;
    for (int64_t j = 0; j < N; ++j) {
        const q128 j0 = (q128)j, j1 = (q128)(j + 1), j2 = (q128)(j + 2);
        b[j] = (P[j + 1] - P[j]) / g1;
        a[j] = (j2 * P[j + 2] - 2 * (j1 * P[j + 1]) + j0 * P[j]) / g2;
        c[j] = (j0 * P[j] - (j0 - al) * P[j + 1]) / g2;
    }
    const q128 ha = powf128(hq, al), ig2 = 1 / g2;
    q128 p[16], yq0[8], yq1[8], yp[8], fp[8], yc[8];
    for (int i = 0; i < n_params; ++i) p[i] = (q128)params[i];
    for (int i = 0; i < dim; ++i) {
        yq0[i] = (q128)y0[i];
        yq1[i] = y1 ? (q128)y1[i] : 0;
        out[i] = y0[i];
    }
    orc_rhs_q(rhs, dim, 0, yq0, p, F);
    for (int64_t n = 0; n < N; ++n) {
        const q128 t1 = (q128)(n + 1) * hq;
        for (int i = 0; i < dim; ++i) {
            q128 sp = 0;
            for (int64_t k = 0; k <= n; ++k) sp += b[n - k] * F[k * dim + i];
            yp[i] = yq0[i] + t1 * yq1[i] + ha * sp;
        }
        orc_rhs_q(rhs, dim, t1, yp, p, fp);
        for (int i = 0; i < dim; ++i) {
            q128 sc = c[n] * F[i];
            for (int64_t k = 1; k <= n; ++k) sc += a[n - k] * F[k * dim + i];
            yc[i] = yq0[i] + t1 * yq1[i] + ha * (sc + fp[i] * ig2);
            out[(n + 1) * dim + i] = (double)yc[i];
        }
        orc_rhs_q(rhs, dim, t1, yc, p, F + (n + 1) * dim);
    }
    free(w), free(P), free(F);
    return ORC_OK;
}

/* ------------------------------------------------------------- batches --- */

typedef struct {
    int dim, rhs, n_params, compensated, tid, nthreads;
    double h, h_alpha, inv_gamma2;
    int64_t N, B;
    const double *params, *traj_params, *y0, *y1, *w;
    const int64_t *N_each;
    double *out;
    int status;
} orc_batch_job;

static void *orc_batch_worker(void *arg)
{
    orc_batch_job *j = (orc_batch_job *)arg;
    double *fw = (double *)malloc((size_t)(j->N + 1) * j->dim * sizeof(double));
    if (!fw) {
        j->status = ORC_ENOMEM;
        return NULL;
    }
    for (int64_t t = j->tid; t < j->B; t += j->nthreads) {
        const int64_t Nt = j->N_each ? j->N_each[t] : j->N;
        const double *p = j->traj_params ? j->traj_params + t * j->n_params : j->params;
        orc_solve_one(j->dim, j->h, Nt, j->rhs, p, j->w, j->w + j->N, j->w + 2 * j->N, j->h_alpha,
                      j->inv_gamma2, j->y0 + t * j->dim, j->y1 ? j->y1 + t * j->dim : NULL,
                      j->out + t * (j->N + 1) * j->dim, fw, j->compensated);
    }
    free(fw);
    return NULL;
}

/* B independent trajectories sharing (dim, alpha, h, rhs) with initial values
 * y0 and, for 1 < alpha < 2, first derivatives y1 (B x dim each; y1 NULL:
 * zero); trajectory t runs
 * N_each[t] <= N steps (all N when N_each is NULL) with its own parameter row
 * traj_params[t*n_params ..] (params for all when NULL).  out is B x (N+1) x
 * dim; rows past N_each[t] are left untouched.  Trajectories are spread over
 * n_threads POSIX threads; each trajectory is computed exactly as a single
 * solve would compute it. */
int fabm_oracle_solve_batch(int dim, double alpha, double h, int64_t N, int rhs,
                            const double *params, int n_params, int64_t B, const double *y0,
                            const double *y1, const double *traj_params, const int64_t *N_each,
                            double *out, int n_threads, int compensated)
{
    if (dim < 1 || dim > 8 || N < 1 || B < 0 || !(h > 0.0) || !(alpha > 0.0 && alpha < 2.0) ||
        (y1 && alpha <= 1.0) || !orc_rhs_dim_ok(rhs, dim, n_params))
        return ORC_EINVAL;
    if (N_each)
        for (int64_t t = 0; t < B; ++t)
            if (N_each[t] < 1 || N_each[t] > N) return ORC_EINVAL;
    if (B == 0) return ORC_OK;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > B) n_threads = (int)B;
    double *w = (double *)malloc((size_t)3 * N * sizeof(double));
    if (!w) return ORC_ENOMEM;
    double ha, ig2;
    int st = fabm_oracle_weights(alpha, N, w, w + N, w + 2 * N);
    if (st == ORC_OK) st = fabm_oracle_constants(alpha, h, &ha, &ig2);
    if (st != ORC_OK) {
        free(w);
        return st;
    }
    orc_batch_job *jobs = (orc_batch_job *)calloc((size_t)n_threads, sizeof(orc_batch_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(w);
        free(jobs);
        free(th);
        return ORC_ENOMEM;
    }
    for (int i = 0; i < n_threads; ++i) {
        orc_batch_job *j = &jobs[i];
        j->dim = dim, j->rhs = rhs, j->n_params = n_params, j->compensated = compensated;
        j->tid = i, j->nthreads = n_threads, j->h = h, j->h_alpha = ha, j->inv_gamma2 = ig2;
        j->N = N, j->B = B, j->params = params, j->traj_params = traj_params, j->y0 = y0;
        j->y1 = y1;
        j->w = w, j->N_each = N_each, j->out = out, j->status = ORC_OK;
    }
    for (int i = 1; i < n_threads; ++i)
        if (pthread_create(&th[i], NULL, orc_batch_worker, &jobs[i]) != 0) jobs[i].status = -1;
    orc_batch_worker(&jobs[0]);
    for (int i = 1; i < n_threads; ++i) {
        if (jobs[i].status == -1) { /* thread could not start: run its share here */
            jobs[i].status = ORC_OK;
            orc_batch_worker(&jobs[i]);
        } else {
            pthread_join(th[i], NULL);
        }
    }
    for (int i = 0; i < n_threads; ++i)
        if (jobs[i].status != ORC_OK) st = jobs[i].status;
    free(w);
    free(jobs);
    free(th);
    return st;
}

/* --------------------------------------------------- per-component orders --- */

/* B trajectories of a system with one order alpha[i] per component, 0 < alpha[i]
 * < 2; y1 (B x dim or NULL) is used by the components with alpha[i] > 1.
 * Otherwise as fabm_oracle_solve_batch (single-threaded). */
int fabm_oracle_solve_batch_multi(int dim, const double *alpha, double h, int64_t N, int rhs,
                                  const double *params, int n_params, int64_t B,
                                  const double *y0, const double *y1,
                                  const double *traj_params, const int64_t *N_each, double *out,
                                  int compensated)
{
    if (dim < 1 || dim > 8 || N < 1 || B < 0 || !(h > 0.0) || !orc_rhs_dim_ok(rhs, dim, n_params))
        return ORC_EINVAL;
    double ha[8], ig[8];
    int t2[8];
    for (int i = 0; i < dim; ++i) {
        if (!(alpha[i] > 0.0 && alpha[i] < 2.0)) return ORC_EINVAL;
        t2[i] = alpha[i] > 1.0;
    }
    if (N_each)
        for (int64_t t = 0; t < B; ++t)
            if (N_each[t] < 1 || N_each[t] > N) return ORC_EINVAL;
    double *w = (double *)malloc((size_t)3 * N * dim * sizeof(double));
    double *fw = (double *)malloc((size_t)(N + 1) * dim * sizeof(double));
    if (!w || !fw) {
        free(w);
        free(fw);
        return ORC_ENOMEM;
    }
    int st = ORC_OK;
    /* layout: b for every component, then a, then c (stride N) */
    for (int i = 0; i < dim && st == ORC_OK; ++i) {
        st = fabm_oracle_weights(alpha[i], N, w + (int64_t)i * N, w + (int64_t)(dim + i) * N,
                                 w + (int64_t)(2 * dim + i) * N);
        if (st == ORC_OK) st = fabm_oracle_constants(alpha[i], h, &ha[i], &ig[i]);
    }
    for (int64_t t = 0; t < B && st == ORC_OK; ++t) {
        const int64_t Nt = N_each ? N_each[t] : N;
        const double *p = traj_params ? traj_params + t * n_params : params;
        st = orc_solve_one_multi(dim, h, Nt, rhs, p, w, w + (int64_t)dim * N,
                                 w + (int64_t)2 * dim * N, N, ha, ig, t2, y0 + t * dim,
                                 y1 ? y1 + t * dim : NULL, out + t * (N + 1) * dim, fw,
                                 compensated);
    }
    free(w);
    free(fw);
    return st;
}
