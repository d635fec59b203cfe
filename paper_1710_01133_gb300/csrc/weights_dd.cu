// a1 in double-double on the device for the FP64x2 precision: the weights of
// Sec. 2 of arXiv:1710.01133 (b_n of Eq. abm, a_n and c_n after it) in the
// distance form of fabm_internal.cuh, B(d) = b_{d-1}, A(d) = a_{d-1},
// D(m) = c_{m-1} - a_{m-1}, as pairs of doubles (hi, lo) with |lo| <= ulp(hi)/2.
//
// Double-double arithmetic (about 106 significant bits) from the error-free
// transformations TwoSum and the FMA-based exact product (Dekker, Knuth).
// Powers: x^a = exp(a ln x), with exp from argument reduction by ln 2, a
// further division by 2^10, a Taylor series and ten squarings of (1 + s)
// written as s <- s (s + 2) on s = e^r - 1, and ln x from the double log by
// one Newton step on exp (which doubles its ~53 correct bits).
//
// The printed formulas cancel: B by ~log2 d bits, A and C by ~2 log2 d bits,
// which multiplies the pow errors.  Up to d = 4 they are evaluated as printed
// (at most 4 bits lost); beyond, from series in u = 1/d (u <= 1/5) whose terms
// do not cancel the result:
//   B(d) = d^a  sum_{k>=1} (-1)^(k+1) binom(a, k) u^k           / Gamma(a+1)
//   A(d) = 2 d^p sum_{k>=1} binom(p, 2k) u^(2k)                 / Gamma(a+2)
//   C(n) = n^p  sum_{k>=2} (a binom(a, k-1) - binom(a, k)) u^k  / Gamma(a+2)
// with p = a + 1 (the expansions of 1 - (1 - u)^a, (1+u)^p - 2 + (1-u)^p and
// 1 - (1 - a u)(1 + u)^a), summed until a term is below 2^-110 of the sum.
// p = a + 1 is not a double in general (a = 0.3 loses its last bits), so it is
// kept as an exact pair for the binomial coefficients and x^p is x x^a.
// 1/Gamma(a+1) and 1/Gamma(a+2) come from the host as double-double pairs.
#include "fabm_internal.cuh"

namespace fabm {
namespace {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd quick_two_sum(double a, double b)
{
    const double s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ dd two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ dd dd_add(dd x, dd y)
{
    dd s = two_sum(x.hi, y.hi);
    const dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

__device__ __forceinline__ dd dd_mul(dd x, dd y)
{
    const double p = x.hi * y.hi;
    double e = fma(x.hi, y.hi, -p);
    e = fma(x.hi, y.lo, e);
    e = fma(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ dd dd_mul_d(dd x, double y)
{
    const double p = x.hi * y;
    double e = fma(x.hi, y, -p);
    e = fma(x.lo, y, e);
    return quick_two_sum(p, e);
}

// x / y for a double y: the quotient of the high parts and two corrections
// from the exact remainders.
__device__ __forceinline__ dd dd_div_d(dd x, double y)
{
    const double q1 = x.hi / y;
    const dd r = dd_sub(x, dd_mul_d(dd{q1, 0.0}, y));
    const double q2 = r.hi / y;
    const dd r2 = dd_sub(r, dd_mul_d(dd{q2, 0.0}, y));
    const double q3 = r2.hi / y;
    return dd_add(quick_two_sum(q1, q2), dd{q3, 0.0});
}

__device__ __forceinline__ dd dd_ldexp(dd x, int e) { return {ldexp(x.hi, e), ldexp(x.lo, e)}; }

// ln 2 as a double-double (its value to 106 bits).
__device__ __forceinline__ dd ln2_dd() { return {0x1.62e42fefa39efp-1, 0x1.abc9e3b39803fp-56}; }

// e^x as a double-double: x = k ln 2 + r, s = e^(r/1024) - 1 by Taylor, ten
// squarings of 1 + s, then the exponent shift 2^k.
__device__ dd dd_exp(dd x)
{
    const double k = rint(x.hi / ln2_dd().hi);
    dd r = dd_sub(x, dd_mul_d(ln2_dd(), k));
    r = dd_ldexp(r, -10);  // |r| < 3.4e-4
    // s = e^r - 1 = r + r^2/2! + ... (r^14/14! < 2^-160 of r)
    dd term = r, s = r;
    for (int n = 2; n <= 14; ++n) {
        term = dd_div_d(dd_mul(term, r), (double)n);
        s = dd_add(s, term);
    }
    for (int i = 0; i < 10; ++i) s = dd_mul(s, dd_add(s, dd{2.0, 0.0}));  // e^{2r} - 1
    return dd_ldexp(dd_add(dd{1.0, 0.0}, s), (int)k);
}

// ln x for x > 0 given as a double: y0 = log(x), y = y0 + (x e^{-y0} - 1).
__device__ dd dd_log(double x)
{
    const double y0 = log(x);
    const dd e = dd_exp(dd{-y0, 0.0});
    const dd corr = dd_sub(dd_mul_d(e, x), dd{1.0, 0.0});
    return dd_add(dd{y0, 0.0}, corr);
}

// x^a for an integer x >= 1 (a double).
__device__ dd dd_pow(double x, double a)
{
    if (x == 1.0) return {1.0, 0.0};
    return dd_exp(dd_mul_d(dd_log(x), a));
}

// binom(a, k) from binom(a, k-1): times (a - k + 1) / k, with a - k + 1 a
// pair (a itself a pair: p = a + 1 does not fit a double).
__device__ __forceinline__ dd binom_next(dd c, dd a, int k)
{
    return dd_div_d(dd_mul(c, dd_add(a, dd{-(double)(k - 1), 0.0})), (double)k);
}

// x^(a+1) = x x^a for an integer x >= 1.
__device__ __forceinline__ dd dd_pow1(double x, double a) { return dd_mul_d(dd_pow(x, a), x); }

constexpr int kDirect = 4;  // distances up to here: the printed differences

__device__ dd weight_B(int64_t d, double a, dd ig1)
{
    if (d <= 0) return {0.0, 0.0};
    if (d == 1) return ig1;
    const double x = (double)d;
    if (d <= kDirect) return dd_mul(dd_sub(dd_pow(x, a), dd_pow(x - 1.0, a)), ig1);
    const dd u = dd_div_d(dd{1.0, 0.0}, x);
    const dd ad = {a, 0.0};
    dd c = ad, uk = u, sum = dd_mul(c, u);  // k = 1: binom(a, 1) u
    for (int k = 2; k < 80; ++k) {
        c = binom_next(c, ad, k);
        uk = dd_mul(uk, u);
        const dd t = dd_mul(c, uk);
        sum = (k & 1) ? dd_add(sum, t) : dd_sub(sum, t);  // (-1)^(k+1) binom(a, k) u^k
        if (fabs(t.hi) < 0x1p-110 * fabs(sum.hi)) break;
    }
    return dd_mul(dd_mul(dd_pow(x, a), sum), ig1);
}

__device__ dd weight_A(int64_t d, double a, dd ig2)
{
    if (d <= 0) return {0.0, 0.0};
    const dd p = two_sum(a, 1.0);  // a + 1 exactly
    // A(1) = (2^p - 2) / Gamma(a+2) = 2 (2^a - 1) / Gamma(a+2)
    if (d == 1) return dd_mul(dd_mul_d(dd_sub(dd_pow(2.0, a), dd{1.0, 0.0}), 2.0), ig2);
    const double x = (double)d;
    if (d <= kDirect) {
        const dd s = dd_add(dd_sub(dd_pow1(x + 1.0, a), dd_mul_d(dd_pow1(x, a), 2.0)),
                            dd_pow1(x - 1.0, a));
        return dd_mul(s, ig2);
    }
    const dd u = dd_div_d(dd{1.0, 0.0}, x);
    const dd u2 = dd_mul(u, u);
    dd c = p;  // binom(p, 1); each round advances it to binom(p, 2k), then 2k+1
    dd u2k = {1.0, 0.0}, sum = {0.0, 0.0};
    for (int k = 1; k < 60; ++k) {
        c = binom_next(c, p, 2 * k);
        u2k = dd_mul(u2k, u2);
        const dd t = dd_mul(c, u2k);
        sum = dd_add(sum, t);
        if (fabs(t.hi) < 0x1p-110 * fabs(sum.hi)) break;
        c = binom_next(c, p, 2 * k + 1);
    }
    return dd_mul(dd_mul_d(dd_mul(dd_pow1(x, a), sum), 2.0), ig2);
}

__device__ dd weight_C(int64_t n, double a, dd ig2)
{
    if (n <= 0) return dd_mul(dd{a, 0.0}, ig2);
    const double x = (double)n;
    if (n <= kDirect) {
        // n^p - (n - a) (n + 1)^a with n - a as an exact pair
        const dd s = dd_sub(dd_pow1(x, a), dd_mul(two_sum(x, -a), dd_pow(x + 1.0, a)));
        return dd_mul(s, ig2);
    }
    const dd u = dd_div_d(dd{1.0, 0.0}, x);
    const dd ad = {a, 0.0};
    dd cprev = ad, uk = u, sum = {0.0, 0.0};  // binom(a, 1), u^1
    for (int k = 2; k < 80; ++k) {
        const dd ck = binom_next(cprev, ad, k);
        uk = dd_mul(uk, u);
        const dd t = dd_mul(dd_sub(dd_mul_d(cprev, a), ck), uk);
        sum = dd_add(sum, t);
        if (fabs(t.hi) < 0x1p-110 * fabs(sum.hi)) break;
        cprev = ck;
    }
    return dd_mul(dd_mul(dd_pow1(x, a), sum), ig2);
}

__global__ void weights_x2_kernel(double a, int64_t n, dd ig1, dd ig2, double *Bh, double *Bl,
                                  double *Ah, double *Al, double *Dh, double *Dl)
{
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d <= n;
         d += (int64_t)gridDim.x * blockDim.x) {
        const dd b = weight_B(d, a, ig1);
        const dd A = weight_A(d, a, ig2);
        const dd D = d >= 1 ? dd_sub(weight_C(d - 1, a, ig2), A) : dd{0.0, 0.0};
        Bh[d] = b.hi, Bl[d] = b.lo;
        Ah[d] = A.hi, Al[d] = A.lo;
        Dh[d] = D.hi, Dl[d] = D.lo;
    }
}

}  // namespace

cudaError_t launch_weights_x2(double alpha, int64_t n, double ig1_hi, double ig1_lo,
                              double ig2_hi, double ig2_lo, double *Bh, double *Bl, double *Ah,
                              double *Al, double *Dh, double *Dl, cudaStream_t st)
{
    if (!(alpha > 0.0 && alpha < 2.0) || n < 0) return cudaErrorInvalidValue;
    int64_t blocks = (n + 1 + 127) / 128;
    if (blocks > 152 * 8) blocks = 152 * 8;
    weights_x2_kernel<<<(unsigned)blocks, 128, 0, st>>>(alpha, n, dd{ig1_hi, ig1_lo},
                                                        dd{ig2_hi, ig2_lo}, Bh, Bl, Ah, Al, Dh,
                                                        Dl);
    return cudaGetLastError();
}

}  // namespace fabm
