/* a1 in double-double for the FP64x2 precision: the weights of Sec. 2 of
 * arXiv:1710.01133 (the predictor weights b_n of Eq. abm, the corrector
 * weights a_n and c_n after it) in distance form,
 *   B(d) = b_{d-1},  A(d) = a_{d-1},  D(m) = C(m-1) - A(m) = c_{m-1} - a_{m-1},
 * evaluated in binary128 on the host and returned as pairs of doubles (hi, lo):
 * hi the double nearest the binary128 value, lo the rounded remainder.
 *
 * The printed differences cancel (b_n by ~log2 n bits, a_n and c_n by ~2 log2 n
 * bits), so they are rewritten with expm1 and log1p, each difference becoming
 * one small quantity times a power:
 *   B(d) = -d^a expm1(a log1p(-1/d)) / Gamma(a+1)                          d >= 2
 *   A(d) = d^(a+1) [expm1((a+1) log1p(1/d)) + expm1((a+1) log1p(-1/d))]
 *          / Gamma(a+2)                                                    d >= 2
 *   C(n) = n^(a+1) [(a/n - E) + (a/n) E] / Gamma(a+2),
 *          E = expm1(a log1p(1/n))                                         n >= 1
 * with B(1) = 1/Gamma(a+1), A(1) = (2^(a+1) - 2)/Gamma(a+2), C(0) = a/Gamma(a+2)
 * (0^p = 0), and B(0) = A(0) = D(0) = 0.  What still cancels (A: two terms of
 * size (a+1)/d whose sum is of size 1/d^2; C: likewise) costs at most ~log2 d
 * of binary128's 113 bits, so the pairs are good to ~1e-27 relative for
 * d <= 2^20.  Host code only; the work is spread over threads.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>

#include "../../include/fabm.h"

typedef _Float128 q_t;

typedef struct {
    q_t a, ig1, ig2;  /* order, 1/Gamma(a+1), 1/Gamma(a+2) */
    int64_t lo, hi;   /* index range [lo, hi) of this thread */
    double *Bh, *Bl, *Ah, *Al, *Dh, *Dl;
} job_t;

static void split(q_t v, double *h, double *l)
{
    const double vh = (double)v;
    *h = vh;
    *l = (double)(v - (q_t)vh);
}

static q_t wB(const job_t *j, int64_t d)
{
    if (d == 0) return 0;
    if (d == 1) return j->ig1;
    const q_t x = (q_t)d;
    return -powf128(x, j->a) * expm1f128(j->a * log1pf128(-1 / x)) * j->ig1;
}

static q_t wA(const job_t *j, int64_t d)
{
    if (d == 0) return 0;
    const q_t a1 = j->a + 1;
    if (d == 1) return (powf128(2, a1) - 2) * j->ig2;
    const q_t x = (q_t)d;
    return powf128(x, a1) * (expm1f128(a1 * log1pf128(1 / x)) + expm1f128(a1 * log1pf128(-1 / x))) *
           j->ig2;
}

static q_t wC(const job_t *j, int64_t n)
{
    if (n == 0) return j->a * j->ig2;
    const q_t x = (q_t)n, r = j->a / x;
    const q_t E = expm1f128(j->a * log1pf128(1 / x));
    return powf128(x, j->a + 1) * ((r - E) + r * E) * j->ig2;
}

static void *run(void *p)
{
    const job_t *j = (const job_t *)p;
    for (int64_t i = j->lo; i < j->hi; ++i) {
        split(wB(j, i), j->Bh + i, j->Bl + i);
        split(wA(j, i), j->Ah + i, j->Al + i);
        split(i == 0 ? (q_t)0 : wC(j, i - 1) - wA(j, i), j->Dh + i, j->Dl + i);
    }
    return 0;
}

/* 1/Gamma(a+1) and 1/Gamma(a+2) in binary128, as (hi, lo) pairs: out[0..1]
 * and out[2..3].  Internal: the device computes the FP64x2 weights (weights_dd.cu) and takes
 * these two constants from here. */
__attribute__((visibility("hidden"))) void fabm_x2_inv_gammas(double alpha, double out[4])
{
    const q_t a = (q_t)alpha;
    split(1 / tgammaf128(a + 1), &out[0], &out[1]);
    split(1 / tgammaf128(a + 2), &out[2], &out[3]);
}

fabm_status fabm_weights_x2(double alpha, int64_t n, double *Bh, double *Bl, double *Ah, double *Al,
                            double *Dh, double *Dl)
{
    if (!(alpha > 0 && alpha < 2) || n < 0 || !Bh || !Bl || !Ah || !Al || !Dh || !Dl)
        return FABM_EINVAL;
    enum { kMaxThreads = 16 };
    const q_t a = (q_t)alpha;
    job_t jobs[kMaxThreads];
    pthread_t th[kMaxThreads];
    int nt = n + 1 >= 4096 ? kMaxThreads : 1, started = 0;
    for (int t = 0; t < nt; ++t) {
        jobs[t] = (job_t){a, 1 / tgammaf128(a + 1), 1 / tgammaf128(a + 2),
                          (n + 1) * t / nt, (n + 1) * (t + 1) / nt, Bh, Bl, Ah, Al, Dh, Dl};
        if (t > 0 && pthread_create(&th[t], 0, run, &jobs[t]) == 0) {
            started |= 1 << t;
        } else if (t > 0) {
            run(&jobs[t]);  /* no thread: do it here */
        }
    }
    run(&jobs[0]);
    for (int t = 1; t < nt; ++t)
        if (started & (1 << t)) pthread_join(th[t], 0);
    return FABM_OK;
}
