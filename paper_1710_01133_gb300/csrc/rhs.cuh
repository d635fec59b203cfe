// a5: right-hand sides f(t, y) of the FDE D^a y = f(t, y) (Sec. 2, Eq. fde),
// as device functors.  Each has the dimension and parameter layout documented
// for FABM_RHS_* in fabm.h.  aux() is double; one() runs in the scalar type T
// of y, p and aux: double on the FP64 path, float-float (FF, ff.cuh) in the
// split recurrence.
#pragma once

#include "fabm_internal.cuh"
#include "ff.cuh"

namespace fabm {

// Interface of a right-hand side functor:
//   aux(t, p)            the part of f that depends on t only (a forcing term,
//                        or 0); evaluated once per grid point, off the serial
//                        chain of the recurrence
//   kForcing             aux depends on t (the tensor path tabulates it ahead
//                        of the recurrence instead of evaluating it inline)
//   one<D>(i, y, p, aux) component i of f(t, y) given aux = aux(t, p)
// Component-wise evaluation lets the recurrence run the components of one
// trajectory on different warps.

struct RhsConst {  // f_i = p0
    static constexpr bool kForcing = false;
    __device__ static double aux(double, const double *p) { return p[0]; }
    template <int D, class T>
    __device__ static T one(int, const T *, const T *, T aux) { return aux; }
};

struct RhsTime {  // f_i = t
    static constexpr bool kForcing = true;
    __device__ static double aux(double t, const double *) { return t; }
    template <int D, class T>
    __device__ static T one(int, const T *, const T *, T aux) { return aux; }
};

struct RhsLinear {  // f_i = -p0 y_i
    static constexpr bool kForcing = false;
    __device__ static double aux(double, const double *) { return 0.0; }
    template <int D, class T>
    __device__ static T one(int i, const T *y, const T *p, T)
    {
        return -p[0] * y[i];
    }
};

struct RhsLorenz {  // p = (sigma, rho, beta)
    static constexpr bool kForcing = false;
    __device__ static double aux(double, const double *) { return 0.0; }
    template <int D, class T>
    __device__ static T one(int i, const T *y, const T *p, T)
    {
        if (i == 0) return p[0] * (y[1] - y[0]);
        if (i == 1) return y[0] * (p[1] - y[2]) - y[1];
        return y[0] * y[1] - p[2] * y[2];
    }
};

struct RhsDuffing {  // p = (gamma, omega, F): x' = y, y' = -gamma y - x - x^3 + F cos(omega t)
    static constexpr bool kForcing = true;
    __device__ static double aux(double t, const double *p) { return p[2] * cos(p[1] * t); }
    template <int D, class T>
    __device__ static T one(int i, const T *y, const T *p, T aux)
    {
        if (i == 0) return y[1];
        const T x = y[0];
        return aux - (p[0] * y[1] + x * (T(1) + x * x));
    }
};

struct RhsManufactured {  // f = p0 t^p1 + t^p2 - y
    static constexpr bool kForcing = true;
    __device__ static double aux(double t, const double *p) { return p[0] * pow(t, p[1]) + pow(t, p[2]); }
    template <int D, class T>
    __device__ static T one(int, const T *y, const T *, T aux)
    {
        return aux - y[0];
    }
};

struct RhsLcr {  // Sec. 5, Eq. sys.LRC; p = (sigma, omega, a, b, f)
    static constexpr bool kForcing = true;
    __device__ static double aux(double t, const double *p) { return p[4] * sin(p[1] * t); }
    template <int D, class T>
    __device__ static T one(int i, const T *y, const T *p, T aux)
    {
        const T x = y[0];
        if (i == 1) return aux - (p[0] * y[1] + x);
        const T a = p[2], b = p[3];
        T g;
        if (x <= T(-1))
            g = b * x - a + b;
        else if (x >= T(1))
            g = b * x + a - b;
        else
            g = a * x;
        return y[1] - g;
    }
};

// Calls fn.template operator()<Rhs, D>() for the (rhs, dim) pair; returns false
// if the pair is not supported.
template <class Fn>
bool dispatch_rhs(int rhs, int dim, Fn &&fn)
{
    switch (rhs) {
    case FABM_RHS_CONST:
    case FABM_RHS_TIME:
    case FABM_RHS_LINEAR:
        switch (dim) {
#define FABM_CASE_D(D)                                                                      \
    case D:                                                                                 \
        if (rhs == FABM_RHS_CONST) fn.template operator()<RhsConst, D>();                   \
        else if (rhs == FABM_RHS_TIME) fn.template operator()<RhsTime, D>();                \
        else fn.template operator()<RhsLinear, D>();                                        \
        return true;
            FABM_CASE_D(1)
            FABM_CASE_D(2)
            FABM_CASE_D(3)
            FABM_CASE_D(4)
#undef FABM_CASE_D
        default: return false;
        }
    case FABM_RHS_LORENZ:
        if (dim != 3) return false;
        fn.template operator()<RhsLorenz, 3>();
        return true;
    case FABM_RHS_DUFFING:
        if (dim != 2) return false;
        fn.template operator()<RhsDuffing, 2>();
        return true;
    case FABM_RHS_MANUFACTURED:
        if (dim != 1) return false;
        fn.template operator()<RhsManufactured, 1>();
        return true;
    case FABM_RHS_LCR:
        if (dim != 2) return false;
        fn.template operator()<RhsLcr, 2>();
        return true;
    default: return false;
    }
}

inline bool rhs_supports_dim(int rhs, int dim)
{
    switch (rhs) {
    case FABM_RHS_CONST:
    case FABM_RHS_TIME:
    case FABM_RHS_LINEAR: return dim >= 1 && dim <= 4;
    case FABM_RHS_LORENZ: return dim == 3;
    case FABM_RHS_DUFFING:
    case FABM_RHS_LCR: return dim == 2;
    case FABM_RHS_MANUFACTURED: return dim == 1;
    default: return false;
    }
}

inline int rhs_n_params(int rhs)
{
    switch (rhs) {
    case FABM_RHS_CONST: return 1;
    case FABM_RHS_TIME: return 0;
    case FABM_RHS_LINEAR: return 1;
    case FABM_RHS_LORENZ: return 3;
    case FABM_RHS_DUFFING: return 3;
    case FABM_RHS_MANUFACTURED: return 3;
    case FABM_RHS_LCR: return 5;
    default: return -1;
    }
}

}  // namespace fabm
