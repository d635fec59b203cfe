// a1: the ABM weights of Sec. 2 of arXiv:1710.01133 in double, from forms that
// do not cancel.
//
// The printed formulas are differences of nearly equal powers.  For the
// corrector weight the second difference (d+1)^p - 2 d^p + (d-1)^p, p = a+1,
// loses about 2 log2(d) bits in double (1e-4 relative at d ~ 2^20), so each
// weight is evaluated from an equivalent expression instead:
//   B(d) = d^a (1 - (1 - 1/d)^a) / G(a+1) = -d^a expm1(a log1p(-1/d)) / G(a+1)
//   A(d) = 2 d^p sum_{k>=1} binom(p, 2k) d^{-2k} / G(a+2)          (d >= 2)
//          all terms positive for 1 < p < 2, so the sum does not cancel;
//          A(1) = (2^p - 2)/G(a+2) = 2 expm1(a ln 2)/G(a+2)
//   c_n  = n^p sum_{k>=2} e_k n^{-k} / G(a+2),  e_k = a binom(a,k-1) - binom(a,k)
//          (the expansion of 1 - (1 - a/n)(1 + 1/n)^a; e_k alternate in sign and
//          fall off like 2^-k at n = 2, faster beyond); c_0 = a/G(a+2),
//          c_1 = (1 - (1-a) 2^a)/G(a+2).
// The series stop once a term is below 2^-56 of the partial sum.
#pragma once

#include "fabm_internal.cuh"

namespace fabm {


__device__ inline double weight_B(int64_t d, double alpha, double inv_g1)
{
    if (d <= 0) return 0.0;
    if (d == 1) return inv_g1;
    const double x = (double)d;
    return -pow(x, alpha) * expm1(alpha * log1p(-1.0 / x)) * inv_g1;
}

__device__ inline double weight_A(int64_t d, double alpha, double inv_g2)
{
    if (d <= 0) return 0.0;
    if (d == 1) return 2.0 * expm1(alpha * 0.69314718055994530942) * inv_g2;
    const double p = alpha + 1.0;
    const double x = (double)d;
    const double u2 = (1.0 / x) / x;
    double term = 0.5 * p * (p - 1.0) * u2;  // binom(p, 2) u^2
    double sum = term;
    for (int k = 1; k < 64; ++k) {
        const double tk = 2.0 * k;
        term *= u2 * (p - tk) * (p - tk - 1.0) / ((tk + 1.0) * (tk + 2.0));
        sum += term;
        if (fabs(term) < 0x1p-56 * sum) break;
    }
    return 2.0 * (x * pow(x, alpha)) * sum * inv_g2;
}

__device__ inline double weight_C(int64_t n, double alpha, double inv_g2)
{
    if (n <= 0) return alpha * inv_g2;
    if (n == 1) return (1.0 - (1.0 - alpha) * exp2(alpha)) * inv_g2;
    const double x = (double)n;
    const double u = 1.0 / x;
    double c_prev = alpha;  // binom(a, 1)
    double uk = u;
    double sum = 0.0;
    for (int k = 2; k < 128; ++k) {
        const double c_k = c_prev * (alpha - (k - 1)) / k;
        uk *= u;
        const double term = (alpha * c_prev - c_k) * uk;
        sum += term;
        if (fabs(term) < 0x1p-56 * fabs(sum)) break;
        c_prev = c_k;
    }
    return (x * pow(x, alpha)) * sum * inv_g2;
}

// B(d), A(d), D(d) = C(d-1) - A(d) for one distance d (index 0 holds 0).
__device__ inline void weights_at(int64_t d, double alpha, double inv_g1, double inv_g2, double *B,
                                  double *A, double *D)
{
    const double a = weight_A(d, alpha, inv_g2);
    B[d] = weight_B(d, alpha, inv_g1);
    A[d] = a;
    D[d] = d >= 1 ? weight_C(d - 1, alpha, inv_g2) - a : 0.0;
}

}  // namespace fabm
