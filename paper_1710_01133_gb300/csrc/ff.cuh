// Float-float ("double-single") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48
// significant bits.  The error-free transformations are Knuth's TwoSum,
// Dekker's Fast2Sum (|a| >= |b|) and the FMA-based exact product
// a*b = p + fma(a, b, -p); sums add the low parts and renormalise once
// ("sloppy" addition, relative error a few units of 2^-48 of the operands).
// GB300 issues fp32 at 64 times its FP64 rate with a short latency, so a
// chain of float-float operations completes sooner than the same chain in
// double.  Used by the split-precision recurrence.
#pragma once

#include <cuda_runtime.h>

namespace fabm {

struct FF {
    float hi, lo;
    FF() = default;
    __host__ __device__ constexpr FF(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr FF(int v) : hi((float)v), lo(0.f) {}
};

__device__ inline FF ff_from_double(double v)
{
    const float h = __double2float_rn(v);
    return FF(h, __double2float_rn(v - (double)h));
}

__device__ inline double ff_to_double(FF x) { return (double)x.hi + (double)x.lo; }

__device__ inline FF fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return FF(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ inline FF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return FF(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ inline FF operator+(FF x, FF y)
{
    const FF s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ inline FF operator-(FF x) { return FF(-x.hi, -x.lo); }
__device__ inline FF operator-(FF x, FF y) { return x + (-y); }

__device__ inline FF operator*(FF x, FF y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

// acc + w*f without normalising the product first
__device__ inline FF ff_fma(FF w, FF f, FF acc)
{
    const float p = __fmul_rn(w.hi, f.hi);
    float e = __fmaf_rn(w.hi, f.hi, -p);
    e = __fmaf_rn(w.hi, f.lo, e);
    e = __fmaf_rn(w.lo, f.hi, e);
    const FF s = two_sum(acc.hi, p);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, e)));
}

// acc += w*f for sums of many products (Ogita, Rump and Oishi's Dot2): acc.hi
// is the running sum, acc.lo collects the rounding errors of the additions
// and the low-order parts of the products; only one addition per term sits on
// the loop-carried chain.  The sum is accurate to about (n 2^-24)^2 of the sum
// of |terms| for n terms; ff_norm turns acc into a normalised value.
__device__ inline void dot2_acc(FF &acc, FF w, FF f)
{
    const float p = __fmul_rn(w.hi, f.hi);
    float e = __fmaf_rn(w.hi, f.hi, -p);
    e = __fmaf_rn(w.hi, f.lo, e);
    e = __fmaf_rn(w.lo, f.hi, e);
    const float s = __fadd_rn(acc.hi, p);
    const float z = __fsub_rn(s, acc.hi);
    const float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, z)), __fsub_rn(p, z));
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
    acc.hi = s;
}

__device__ inline FF ff_norm(FF a) { return two_sum(a.hi, a.lo); }

__device__ inline bool operator<=(FF x, FF y) { return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo); }
__device__ inline bool operator>=(FF x, FF y) { return y <= x; }

__device__ inline FF shfl_ff(FF x, int src)
{
    return FF(__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src));
}

}  // namespace fabm
