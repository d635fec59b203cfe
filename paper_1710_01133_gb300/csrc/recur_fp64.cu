// a4 + a5 in double: the sequential predictor -> f -> corrector -> f chain of
// Sec. 2 of arXiv:1710.01133 inside one block of L = 32 targets, one warp per
// trajectory.
//
// Lane a owns target m = cL+1+a and keeps its two running sums (predictor and
// corrector, per component) in registers:
//   start   far part from the history kernels (points k < (c-1)L) and the
//           k = 0 correction D(m) f_0;
//   lag 1   the 32 points of block c-1, all known when the block starts;
//   steps   for s = 0..31 the point k = cL+s becomes known (f_k broadcast from
//           the lane that made it); every lane with a >= s adds its term, and
//           lane s then has the whole sum for m = k+1 and runs the step.
// Each FP64 instruction occupies a whole 64-cycle slot of the FP64 unit on
// GB300 regardless of active lanes, so accumulating f_k into all 32 pending
// targets costs the same as into one; the serial critical path per step is the
// lane-s update plus two evaluations of f.
#include "rhs.cuh"

namespace fabm {
namespace {

__device__ inline void report_nonfinite(unsigned long long *status, int64_t step, int traj)
{
    atomicMin(status, ((unsigned long long)step << 24) | (unsigned long long)traj);
}

template <class Rhs, int D>
__global__ void init_kernel(DevBatch bt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= bt.B) return;
    double y[D], f[D], p[kMaxParams];
#pragma unroll
    for (int i = 0; i < kMaxParams; ++i) p[i] = bt.params[(int64_t)b * kMaxParams + i];
#pragma unroll
    for (int i = 0; i < D; ++i) y[i] = bt.y0[(int64_t)b * D + i];
    Rhs::template eval<D>(0.0, y, p, f);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        bt.Y[(int64_t)b * (bt.N + 1) * D + i] = y[i];
        bt.F[(int64_t)b * D + i] = f[i];
        ok = ok && isfinite(y[i]) && isfinite(f[i]);
    }
    if (!ok) report_nonfinite(bt.status, 0, b);
}

template <class Rhs, int D>
__global__ void __launch_bounds__(128)
    recur_fp64_kernel(DevBatch bt, DevWeights w, StepConsts kc, int64_t c, const double *G)
{
    constexpr int L = kRecurL;
    __shared__ double sB[2 * L + 1], sA[2 * L + 1];
    for (int i = threadIdx.x; i <= 2 * L; i += blockDim.x) {
        sB[i] = w.B[i];
        sA[i] = w.A[i];
    }
    __syncthreads();

    const int lane = threadIdx.x % kWarp;
    const int b = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
    if (b >= bt.B) return;
    const int64_t Nb = bt.N_each[b];
    const int64_t m0 = c * L;  // f_{m0} is the newest known point
    if (m0 >= Nb) return;      // trajectory finished (warp-uniform)

    double p[kMaxParams], y0[D];
#pragma unroll
    for (int i = 0; i < kMaxParams; ++i) p[i] = bt.params[(int64_t)b * kMaxParams + i];
#pragma unroll
    for (int i = 0; i < D; ++i) y0[i] = bt.y0[(int64_t)b * D + i];

    const int64_t col0 = (int64_t)b * D;
    const int64_t ldF = bt.ldF;
    const double *F = bt.F;
    const int64_t m = m0 + 1 + lane;
    const double Dm = w.D[m];

    double accP[D], accC[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const double f0 = F[col0 + i];
        accP[i] = G ? G[(int64_t)lane * bt.cols + col0 + i] : 0.0;
        accC[i] = fma(Dm, f0, G ? G[(int64_t)(L + lane) * bt.cols + col0 + i] : 0.0);
    }
    if (c >= 1) {  // lag-1 block: k = m0-L+j, d = m-k = L+1+lane-j
        for (int j = 0; j < L; ++j) {
            const double *fr = F + (m0 - L + j) * ldF + col0;
            const int d = L + 1 + lane - j;
            const double wb = sB[d], wa = sA[d];
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const double fk = fr[i];
                accP[i] = fma(wb, fk, accP[i]);
                accC[i] = fma(wa, fk, accC[i]);
            }
        }
    }

    double fk[D];
#pragma unroll
    for (int i = 0; i < D; ++i) fk[i] = F[m0 * ldF + col0 + i];
    const int steps = (int)(Nb - m0 < L ? Nb - m0 : L);
    double *Yb = bt.Y + (int64_t)b * (bt.N + 1) * D;
    for (int s = 0; s < steps; ++s) {
        const int d = lane - s + 1;  // distance from k = m0+s to this lane's target
        const int dd = d > 0 ? d : 0;  // lanes already done add B(0) = A(0) = 0
        const double wb = sB[dd], wa = sA[dd];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            accP[i] = fma(wb, fk[i], accP[i]);
            accC[i] = fma(wa, fk[i], accC[i]);
        }
        double fn[D];
#pragma unroll
        for (int i = 0; i < D; ++i) fn[i] = 0.0;
        if (lane == s) {
            const int64_t mm = m0 + 1 + s;
            const double t = (double)mm * kc.h;
            double yp[D], fp[D], yc[D];
#pragma unroll
            for (int i = 0; i < D; ++i) yp[i] = fma(kc.h_alpha, accP[i], y0[i]);
            Rhs::template eval<D>(t, yp, p, fp);
#pragma unroll
            for (int i = 0; i < D; ++i) yc[i] = fma(kc.h_alpha, fma(fp[i], kc.inv_gamma2, accC[i]), y0[i]);
            Rhs::template eval<D>(t, yc, p, fn);
            bool ok = true;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                Yb[mm * D + i] = yc[i];
                bt.F[mm * ldF + col0 + i] = fn[i];
                ok = ok && isfinite(yc[i]) && isfinite(fn[i]);
            }
            if (!ok) report_nonfinite(bt.status, mm, b);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) fk[i] = __shfl_sync(0xffffffffu, fn[i], s);
    }
}

}  // namespace

cudaError_t launch_init(int rhs, const DevBatch &bt, cudaStream_t st)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((bt.B + threads - 1) / threads);
    bool ok = dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        init_kernel<R, D><<<blocks, threads, 0, st>>>(bt);
    });
    return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

cudaError_t launch_recur_fp64(int rhs, const DevBatch &bt, const DevWeights &w,
                              const StepConsts &k, int64_t c, const double *G, cudaStream_t st)
{
    const int warps = 4;
    const unsigned blocks = (unsigned)((bt.B + warps - 1) / warps);
    bool ok = dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        recur_fp64_kernel<R, D><<<blocks, warps * kWarp, 0, st>>>(bt, w, k, c, G);
    });
    return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

}  // namespace fabm
