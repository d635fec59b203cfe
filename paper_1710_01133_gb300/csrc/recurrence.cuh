// a4 + a5 in double: the sequential predictor -> f -> corrector -> f chain of
// Sec. 2 of arXiv:1710.01133 (Eq. abm, the corrector after it) inside one
// block of L = 32*TPL targets.  One CTA per trajectory, one warp per
// component.
//
// Warp i keeps, in lane a + 32t, the running predictor and corrector sums of
// component i for target m = cL+1+a+32t:
//   start   far part from the history kernels (points k < (c-1)L) and the
//           k = 0 correction D(m) f_0;
//   lag 1   the L points of block c-1, all known when the block starts;
//   steps   for s = 0..L-1 the point k = cL+s becomes known; every pending
//           target adds its term, and the owner of target k+1 then has the
//           whole sum and runs the step: y^P_i, exchange of y^P across the
//           component warps, f_i(t, y^P), y_i, exchange of y, f_i(t, y).
// The accumulators hold y0 + h^alpha * (partial sum) and the weights are
// pre-multiplied by h^alpha, so the owner's accumulate of the newest point is
// already y^P (and y0 + h^alpha S^C): six dependent FP64 operations per step
// for a Lorenz-type component (accumulate, f, corrector, f).
// On GB300 a warp FP64 instruction takes the FP64 pipe for many cycles
// whatever the number of active lanes, so adding f_k to all pending targets
// of a warp costs one instruction per sum, and the components run on separate
// warps so that their chains overlap.  The time-only part of f (forcing) is
// evaluated for every target at block start, off the chain.
#pragma once

#include "rhs.cuh"

namespace fabm {


// v[q] for a runtime q < D without indexing the array dynamically (which
// would copy the kernel's parameter block to local memory).
template <int D>
__device__ inline double pick(const double (&v)[FABM_MAX_DIM], int q)
{
    double r = v[0];
#pragma unroll
    for (int k = 1; k < D; ++k)
        if (q == k) r = v[k];
    return r;
}

__device__ inline void report_nonfinite(unsigned long long *status, int64_t step, int traj)
{
    atomicMin(status, ((unsigned long long)step << 24) | (unsigned long long)traj);
}

// Finite test on the exponent bits (no floating-point compare).
__device__ inline bool finite_bits(double x)
{
    return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}

// y_0 and f_0 = f(0, y_0) of trajectory b; f_pairs: F holds float-float pairs.
template <class Rhs, int D>
__device__ inline void init_one(const DevBatch &bt, int b, bool f_pairs = false)
{
    double y[D], p[kMaxParams];
#pragma unroll
    for (int i = 0; i < kMaxParams; ++i) p[i] = bt.params[(int64_t)b * kMaxParams + i];
#pragma unroll
    for (int i = 0; i < D; ++i) y[i] = bt.y0[(int64_t)b * D + i];
    const double aux = Rhs::aux(0.0, p);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const double f = Rhs::template one<D>(i, y, p, aux);
        bt.Y[(int64_t)b * (bt.N + 1) * D + i] = y[i];
        if (f_pairs) {
            const float hi = __double2float_rn(f);
            reinterpret_cast<float2 *>(bt.F)[(int64_t)b * D + i] =
                make_float2(hi, __double2float_rn(f - (double)hi));
        } else {
            bt.F[(int64_t)b * D + i] = f;
        }
        if (bt.Ff) bt.Ff[(int64_t)b * D + i] = (float)f;
        ok = ok && finite_bits(y[i]) && finite_bits(f);
    }
    if (!ok) report_nonfinite(bt.status, 0, b);
}

// Shared-memory doubles recur_block<*, D, TPL, LAG> needs.
template <int D, int TPL, int LAG = 1>
__host__ __device__ constexpr int recur_smem_doubles()
{
    return 2 * ((LAG + 1) * kWarp * TPL + 1) * D + 2 * D + (LAG * kWarp * TPL + 1) * D;
}

// One block of steps for trajectory b of the batch, run by a CTA of at least D
// warps; smem holds recur_smem_doubles<D, TPL, LAG>() doubles.  The far part G
// covers the points k < (c - LAG) L; the LAG blocks before block c are summed
// here.
template <class Rhs, int D, int TPL, int LAG = 1>
__device__ void recur_block(const DevBatch &bt, int b, const DevWeights &w, const StepConsts &kc,
                            int64_t c, const double *G, double *smem)
{
    constexpr int L = kWarp * TPL;
    // weights pre-multiplied by h^alpha: the accumulators hold y0 + h^alpha * sum,
    // so adding the newest point to the owner's accumulator yields y^P directly
    constexpr int W = (LAG + 1) * L + 1;  // distances 0 .. (LAG+1) L
    double *sB = smem;                   // [D][W], per component (its own order)
    double *sA = sB + D * W;             // [D][W]
    double(*sy)[D] = reinterpret_cast<double(*)[D]>(sA + D * W);  // [2][D]
    double(*sF)[D] = sy + 2;             // [LAG L + 1][D]: f of the lag blocks and f_{m0}
    // component of this warp; warps beyond D (a CTA sized for a larger
    // dimension) mirror component 0 and write nothing
    const bool act = threadIdx.x / kWarp < D;
    const int i = act ? threadIdx.x / kWarp : 0;
    const int lane = threadIdx.x % kWarp;
    const int64_t Nb = bt.N_each[b];
    const int64_t m0 = c * L;  // f_{m0} is the newest known point
    if (m0 >= Nb) return;      // trajectory finished (uniform over the CTA)
    const int nW = w.stride ? D : 1;  // one weight set per order
    for (int j = threadIdx.x; j < nW * W; j += blockDim.x) {
        const int q = j / W, jj = j % W;
        const double hq = pick<D>(kc.h_alpha, q);
        sB[j] = hq * w.B[q * w.stride + jj];
        sA[j] = hq * w.A[q * w.stride + jj];
    }
    // rows m0-LAG*L .. m0 of this trajectory's history, all loads in flight at once
    for (int j = threadIdx.x; j < (LAG * L + 1) * D; j += blockDim.x) {
        const int64_t row = m0 - LAG * L + j / D;
        sF[j / D][j % D] = row >= 0 ? bt.F[row * bt.ldF + (int64_t)b * D + j % D] : 0.0;
    }
    __syncthreads();

    double p[kMaxParams];
#pragma unroll
    for (int q = 0; q < kMaxParams; ++q) p[q] = bt.params[(int64_t)b * kMaxParams + q];
    const double y0 = bt.y0[(int64_t)b * D + i];
    const int64_t col = (int64_t)b * D + i;
    const double ha = pick<D>(kc.h_alpha, i);
    const double ha_ig2 = ha * pick<D>(kc.inv_gamma2, i);
    const double *wD = w.D + i * w.stride;
    if (w.stride) sB += i * W, sA += i * W;  // this warp's component's order

    double accP[TPL], accC[TPL], aux[TPL];
    const double f0 = bt.F[col];
    const double y1 = bt.y1 ? bt.y1[col] : 0.0;
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int a = lane + kWarp * t;
        const int64_t m = m0 + 1 + a;
        aux[t] = Rhs::aux((double)m * kc.h, p);
        // Taylor part of the initial data at t_m: y0, or y0 + t_m y'(0) for 1 < alpha < 2
        const double Tm = bt.y1 ? fma((double)m * kc.h, y1, y0) : y0;
        const double gP = G ? G[(int64_t)a * bt.cols + col] : 0.0;
        const double gC = fma(wD[m], f0, G ? G[(int64_t)(L + a) * bt.cols + col] : 0.0);
        accP[t] = fma(ha, gP, Tm);
        accC[t] = fma(ha, gC, Tm);
    }
    if (c >= 1) {  // lag blocks: k = m0-LAG*L+j, d = m-k = LAG*L+1+a-j in [2, (LAG+1)L]
        for (int j = 0; j < LAG * L; ++j) {
            const double fk = sF[j][i];
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                const int d = LAG * L + 1 + lane + kWarp * t - j;
                accP[t] = fma(sB[d], fk, accP[t]);
                accC[t] = fma(sA[d], fk, accC[t]);
            }
        }
    }

    double fk = sF[LAG * L][i];
    const int steps = (int)(Nb - m0 < L ? Nb - m0 : L);
    double *Yb = bt.Y + (int64_t)b * (bt.N + 1) * D;
    for (int s = 0; s < steps; ++s) {
        // add the newest point k = m0+s; for the owner of target k+1 this
        // completes y^P (accP) and y0 + h^a S^C (accC)
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
            const int d = lane + kWarp * t - s + 1;
            const int dd = d > 0 ? d : 0;  // done targets add B(0) = A(0) = 0
            accP[t] = fma(sB[dd], fk, accP[t]);
            accC[t] = fma(sA[dd], fk, accC[t]);
        }
        const int owner = s % kWarp, slot = s / kWarp;  // uniform over the CTA
        double yp = 0.0, aC = 0.0, ax = 0.0;
#pragma unroll
        for (int t = 0; t < TPL; ++t)
            if (t == slot) yp = accP[t], aC = accC[t], ax = aux[t];
        double fn = 0.0, yc = 0.0;
        if constexpr (D == 1) {
            if (lane == owner) {
                const double fp = Rhs::template one<D>(0, &yp, p, ax);
                yc = fma(ha_ig2, fp, aC);
                fn = Rhs::template one<D>(0, &yc, p, ax);
            }
        } else {
            if (act && lane == owner) sy[0][i] = yp;
            __syncthreads();
            if (lane == owner) {
                double y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = sy[0][q];
                const double fp = Rhs::template one<D>(i, y, p, ax);
                yc = fma(ha_ig2, fp, aC);  // corrector
                if (act) sy[1][i] = yc;
            }
            __syncthreads();
            if (lane == owner) {
                double y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = sy[1][q];
                fn = Rhs::template one<D>(i, y, p, ax);
            }
        }
        if (act && lane == owner) {
            const int64_t mm = m0 + 1 + s;
            Yb[mm * D + i] = yc;
            bt.F[mm * bt.ldF + col] = fn;
            if (!(finite_bits(yc) && finite_bits(fn))) report_nonfinite(bt.status, mm, b);
        }
        fk = __shfl_sync(0xffffffffu, fn, owner);
    }
}

// ---- split precision ----
//
// The same block of steps for the split path with no FP64 operation on the
// serial chain of a step.  Per target (lane a, slot t):
//   base    y0 + h^alpha (far part + D(m) f_0), FP64, at block start;
//   near    the lag-1 block and the in-block points, h^alpha w(d) f_k summed
//           in float-float (ff.cuh, ~48 bits) as the points become known;
//   step    the owner forms, in float-float,
//             y^P = base_P + near_P,  inc = near_C + h^alpha/Gamma(alpha+2) f(t, y^P),
//           evaluates f(t, base_C + inc), and keeps inc and f;
//   end     y = base_C + inc (the FP64 corrector update) and f_k are written
//           as doubles, one target per lane, for the whole block at once.
// Float-float carries ~48 bits, so the recurrence adds rounding far below
// that of the split history; GB300 issues its fp32 at 64 times the FP64 rate
// and a float-float operation completes in fewer cycles than one FP64
// operation, so the chain is shorter and wide batches no longer saturate the
// FP64 pipe.
template <int D, int TPL, int LAG = 1>
__host__ __device__ constexpr int recur_split_smem_floats()
{
    return 4 * ((LAG + 1) * kWarp * TPL + 1) * D + 4 * D + 2 * (LAG * kWarp * TPL + 1) * D;
}

// smem: recur_split_smem_floats<D, TPL, LAG>() floats, 8-byte aligned; LAG as
// for recur_block
template <class Rhs, int D, int TPL, int LAG = 1>
__device__ void recur_block_split(const DevBatch &bt, int b, const DevWeights &w,
                                  const StepConsts &kc, int64_t c, const double *G, float *smem)
{
    constexpr int L = kWarp * TPL;
    constexpr int W = (LAG + 1) * L + 1;
    FF *sB = reinterpret_cast<FF *>(smem);  // [D][W]  h^alpha_i B_i(d)
    FF *sA = sB + D * W;                    // [D][W]  h^alpha_i A_i(d)
    FF(*sy)[D] = reinterpret_cast<FF(*)[D]>(sA + D * W);  // [2][D]
    FF(*sF)[D] = sy + 2;                    // [LAG L + 1][D]: f of the lag blocks and f_{m0}
    const bool act = threadIdx.x / kWarp < D;
    const int i = act ? threadIdx.x / kWarp : 0;
    const int lane = threadIdx.x % kWarp;
    const int64_t Nb = bt.N_each[b];
    const int64_t m0 = c * L;
    if (m0 >= Nb) return;
    const int nW = w.stride ? D : 1;  // one weight set per order
    for (int j = threadIdx.x; j < nW * W; j += blockDim.x) {
        const int q = j / W, jj = j % W;
        const double hq = pick<D>(kc.h_alpha, q);
        sB[j] = ff_from_double(hq * w.B[q * w.stride + jj]);
        sA[j] = ff_from_double(hq * w.A[q * w.stride + jj]);
    }
    for (int j = threadIdx.x; j < (LAG * L + 1) * D; j += blockDim.x) {
        const int64_t row = m0 - LAG * L + j / D;
        sF[j / D][j % D] =
            ff_from_double(row >= 0 ? bt.F[row * bt.ldF + (int64_t)b * D + j % D] : 0.0);
    }
    __syncthreads();

    double p[kMaxParams];
    FF pf[kMaxParams];
#pragma unroll
    for (int q = 0; q < kMaxParams; ++q) {
        p[q] = bt.params[(int64_t)b * kMaxParams + q];
        pf[q] = ff_from_double(p[q]);
    }
    const double y0 = bt.y0[(int64_t)b * D + i];
    const int64_t col = (int64_t)b * D + i;
    const double ha = pick<D>(kc.h_alpha, i);
    const FF ha_ig2 = ff_from_double(ha * pick<D>(kc.inv_gamma2, i));
    const double f0 = bt.F[col];
    const double *wD = w.D + i * w.stride;
    if (w.stride) sB += i * W, sA += i * W;  // this warp's component's order

    double baseC[TPL];
    FF bP[TPL], bC[TPL], aux[TPL], nP[TPL], nC[TPL], inc[TPL], fo[TPL];
    const double y1 = bt.y1 ? bt.y1[col] : 0.0;
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int a = lane + kWarp * t;
        const int64_t m = m0 + 1 + a;
        aux[t] = ff_from_double(Rhs::aux((double)m * kc.h, p));
        const double Tm = bt.y1 ? fma((double)m * kc.h, y1, y0) : y0;  // Taylor part at t_m
        const double gP = G ? G[(int64_t)a * bt.cols + col] : 0.0;
        const double gC = fma(wD[m], f0, G ? G[(int64_t)(L + a) * bt.cols + col] : 0.0);
        baseC[t] = fma(ha, gC, Tm);
        bP[t] = ff_from_double(fma(ha, gP, Tm));
        bC[t] = ff_from_double(baseC[t]);
        nP[t] = nC[t] = inc[t] = fo[t] = FF(0);
    }
    if (c >= 1) {  // lag blocks: k = m0-LAG*L+j, d = LAG*L+1+a-j in [2, (LAG+1)L]
        for (int j = 0; j < LAG * L; ++j) {
            const FF fk = sF[j][i];
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                const int d = LAG * L + 1 + lane + kWarp * t - j;
                nP[t] = ff_fma(sB[d], fk, nP[t]);
                nC[t] = ff_fma(sA[d], fk, nC[t]);
            }
        }
    }

    FF fk = sF[LAG * L][i];
    const int steps = (int)(Nb - m0 < L ? Nb - m0 : L);
    for (int s = 0; s < steps; ++s) {
        // add the newest point k = m0+s to every pending target
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
            const int d = lane + kWarp * t - s + 1;
            const int dd = d > 0 ? d : 0;  // done targets add B(0) = A(0) = 0
            nP[t] = ff_fma(sB[dd], fk, nP[t]);
            nC[t] = ff_fma(sA[dd], fk, nC[t]);
        }
        const int owner = s % kWarp, slot = s / kWarp;  // uniform over the CTA
        FF yp(0), nc(0), bc(0), ax(0);
#pragma unroll
        for (int t = 0; t < TPL; ++t)
            if (t == slot) yp = bP[t] + nP[t], nc = nC[t], bc = bC[t], ax = aux[t];
        FF fn(0), in(0);
        if constexpr (D == 1) {
            if (lane == owner) {
                const FF fp = Rhs::template one<D>(0, &yp, pf, ax);
                in = ha_ig2 * fp + nc;
                const FF yc = bc + in;
                fn = Rhs::template one<D>(0, &yc, pf, ax);
            }
        } else {
            if (act && lane == owner) sy[0][i] = yp;
            __syncthreads();
            if (lane == owner) {
                FF y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = sy[0][q];
                const FF fp = Rhs::template one<D>(i, y, pf, ax);
                in = ha_ig2 * fp + nc;  // corrector increment
                if (act) sy[1][i] = bc + in;
            }
            __syncthreads();
            if (lane == owner) {
                FF y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = sy[1][q];
                fn = Rhs::template one<D>(i, y, pf, ax);
            }
        }
#pragma unroll
        for (int t = 0; t < TPL; ++t)
            if (t == slot && lane == owner) inc[t] = in, fo[t] = fn;
        fk = shfl_ff(fn, owner);
    }

    // FP64 corrector update and f of the block's targets, one per lane
    if (act) {
        double *Yb = bt.Y + (int64_t)b * (bt.N + 1) * D;
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
            const int a = lane + kWarp * t;
            if (a < steps) {
                const int64_t mm = m0 + 1 + a;
                const double yc = baseC[t] + ff_to_double(inc[t]);
                const double fd = ff_to_double(fo[t]);
                Yb[mm * D + i] = yc;
                bt.F[mm * bt.ldF + col] = fd;
                if (bt.Ff) bt.Ff[mm * bt.ldF + col] = (float)fd;  // the fp32 history's input
                if (!(finite_bits(yc) && finite_bits(fd))) report_nonfinite(bt.status, mm, b);
            }
        }
    }
}

}  // namespace fabm
