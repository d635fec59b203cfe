// a4 + a5 for wide batches on the tensor-history path: the predictor -> f ->
// corrector -> f chain of Sec. 2 of arXiv:1710.01133 with one lane per column
// (trajectory b, component i) instead of one lane per target.
//
// On this path the history launches (far segments and the newest segment,
// history_split.cu) deliver every point k < cL of block c, so a step only adds
// the points of its own block.  Per lane, block c (targets m = cL+1+a, a < 64,
// points f_{cL+j}, j = 0..64):
//   bases   h^a (G_P(m)) and h^a (G_C(m) + D(m) f_0) from the combined history;
//   near    S(a) = sum_{j<=a} w(a+1-j) f_{cL+j}, float-float products summed
//           with separate error terms (dot2_acc), in sub-blocks of 8 targets:
//           the points before the sub-block at its start (independent
//           products, no chain), the sub-block's own points as they appear;
//   step    y^P = T + b_P + S_P, exchange of y^P between the lanes of the
//           trajectory (shuffles), f(t, y^P), y = T + b_C + S_C + h^a f^P /
//           Gamma(a+2), exchange, f(t, y);
//   output  the float-float increment h^a (...) in the double-sized slot of y
//           (finish_y_kernel adds the Taylor part in double after the last
//           block) and f as a float-float pair (the buffer the segment slicer
//           reads).
// A warp advances 32/D trajectories at once, so the serial part of a step is
// paid once per warp rather than once per column, and no step waits on a
// block-wide barrier.  GB300 runs FP64 at 1/64 of the fp32 rate with a long
// latency, so no FP64 operation is left in the kernel: the time-only part of f
// (forcing) comes from a table that aux_kernel fills blocks ahead on another
// stream, and y is converted to double once at the end.
#include "recurrence.cuh"

namespace fabm {
namespace {

constexpr int kColL = kSplitSeg;  // targets per block
constexpr int kSub = 8;           // targets per sub-block
constexpr int kMaxWarps = 12;     // warps per CTA at most (registers: <= 168 per thread)

// shared memory of a CTA of `warps` warps, in float-float pairs: h^a B and
// h^a A (65 each), then per warp f of the block's points [65][32]
constexpr int ff_per_warp(int) { return (kColL + 1) * kWarp; }
constexpr size_t cols_smem_bytes(int D, int warps)
{
    return sizeof(FF) * (2 * (kColL + 1) + (size_t)warps * ff_per_warp(D));
}

__device__ __forceinline__ bool finite_f(float x)
{
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

__device__ __forceinline__ FF ld_ff(const float2 *p)
{
    const float2 v = *p;
    return FF(v.x, v.y);
}

// History of every point before block c for target a of column col, kind k
// (0 predictor, 1 corrector): the far value plus the near partials (at most
// kMaxNear), all loads issued before the additions.
constexpr int kMaxNear = 3;
__device__ __forceinline__ FF hist_in(const HistIn &h, int k, int a, int64_t col, int cols)
{
    float2 v[kMaxNear + 1];
    v[0] = h.G ? h.G[((int64_t)k * h.g_rows + h.g_off + a) * cols + col] : make_float2(0.f, 0.f);
#pragma unroll
    for (int ch = 0; ch < kMaxNear; ++ch)
        v[ch + 1] = ch < h.n_near ? h.near[(((int64_t)ch * 2 + k) * kColL + a) * cols + col]
                                  : make_float2(0.f, 0.f);
    FF s(v[0].x, v[0].y);
#pragma unroll
    for (int ch = 1; ch <= kMaxNear; ++ch) s = s + FF(v[ch].x, v[ch].y);
    return s;
}

// Time-only part of f for the 64 targets of block c: X[a][b] = aux(t_m, p_b),
// m = 64c+1+a, as float-float pairs.
template <class Rhs>
__global__ void aux_kernel(DevBatch bt, double h, int64_t c, float2 *__restrict__ X)
{
    const int64_t n = (int64_t)kColL * bt.B;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / bt.B);
        const int64_t b = e % bt.B;
        double p[kMaxParams];
#pragma unroll
        for (int q = 0; q < kMaxParams; ++q) p[q] = bt.params[b * kMaxParams + q];
        const FF v = ff_from_double(Rhs::aux((double)(c * kColL + 1 + a) * h, p));
        X[e] = make_float2(v.hi, v.lo);
    }
}

// y_m = T(t_m) + (hi + lo) in double for m = m_lo .. min(m_hi, N_each[b])
// (m_lo >= 1), where the recurrence left the float-float increment (hi, lo) in
// y's slot; T = y0, or y0 + t y'(0) for 1 < alpha < 2.
__global__ void finish_y_kernel(DevBatch bt, double h, int64_t m_lo, int64_t m_hi)
{
    const int64_t per_traj = (m_hi - m_lo + 1) * bt.dim;
    const int64_t n = (int64_t)bt.B * per_traj;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / per_traj, r = e % per_traj;
        const int64_t m = m_lo + r / bt.dim;
        const int i = (int)(r % bt.dim);
        if (m > bt.N_each[b]) continue;
        double *slot = bt.Y + (b * (bt.N + 1) + m) * bt.dim + i;
        const float2 v = *reinterpret_cast<const float2 *>(slot);
        const double y0 = bt.y0[b * bt.dim + i];
        const double T = bt.y1 ? fma((double)m * h, bt.y1[b * bt.dim + i], y0) : y0;
        *slot = T + ((double)v.x + (double)v.y);
    }
}

// Warp w of CTA x advances the trajectories 32/D * (x * warps + w) ...; the
// CTA size is chosen by the host so that the CTAs fill the SMs the tensor
// history leaves free (a tensor CTA and a recurrence CTA never share an SM).
// WB, WA: h^a B(d), h^a A(d) for d = 0..64 as float-float pairs; WD: h^a D(m);
// F: float-float pairs in the double-sized slots of bt.F; hin: the history of
// block c (a far value and near partials, float-float pairs); X: the
// forcing table of block c ([64][B] pairs, aux_kernel) when Rhs::kForcing.
// Y1: bt.y1 is set (1 < alpha < 2, Taylor part y0 + t y'(0)); a template
// parameter so that the solves without it carry no FP64 work per step.
template <class Rhs, int D, bool Y1>
__global__ void __launch_bounds__(kMaxWarps *kWarp)
    recur_cols_kernel(DevBatch bt, const float2 *__restrict__ WB, const float2 *__restrict__ WA,
                      const float2 *__restrict__ WD, StepConsts kc, int64_t c,
                      const HistIn hin, const float2 *__restrict__ X)
{
    constexpr int TPW = kWarp / D;  // trajectories per warp
    extern __shared__ __align__(16) FF smem_ff[];
    FF *sB = smem_ff, *sA = smem_ff + (kColL + 1);
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    FF *wbase = smem_ff + 2 * (kColL + 1) + warp * ff_per_warp(D);
    FF(*sF)[kWarp] = reinterpret_cast<FF(*)[kWarp]>(wbase);  // f_{cL+j} of the warp's columns

    for (int d = threadIdx.x; d <= kColL; d += blockDim.x) sB[d] = ld_ff(WB + d), sA[d] = ld_ff(WA + d);
    __syncthreads();  // the only CTA-wide barrier: warps run independently from here

    const int g = lane / D, i = lane % D;
    const int64_t b = ((int64_t)blockIdx.x * (blockDim.x / kWarp) + warp) * TPW + g;
    const bool act = g < TPW && b < bt.B;
    const int64_t bb = act ? b : 0;  // in-range index for the loads of idle lanes
    const int64_t col = bb * D + i;
    const int64_t m0 = c * kColL;
    const int64_t Nb = act ? bt.N_each[bb] : 0;
    const int steps = (int)(Nb - m0 < 0 ? 0 : (Nb - m0 < kColL ? Nb - m0 : kColL));
    const int wsteps = (int)__reduce_max_sync(0xffffffffu, (unsigned)steps);
    if (wsteps == 0) return;  // every trajectory of the warp has finished (uniform)

    const float2 *F2 = reinterpret_cast<const float2 *>(bt.F);
    float2 *Fw = reinterpret_cast<float2 *>(bt.F);
    sF[0][lane] = ld_ff(F2 + m0 * bt.ldF + col);
    const FF f0 = ld_ff(F2 + col);

    double p[kMaxParams];
    FF pf[kMaxParams];
#pragma unroll
    for (int q = 0; q < kMaxParams; ++q) {
        p[q] = bt.params[bb * kMaxParams + q];
        pf[q] = ff_from_double(p[q]);
    }
    // time-independent aux (a constant, or 0) once per lane
    const FF aux0 = Rhs::kForcing ? FF(0) : ff_from_double(Rhs::aux(0.0, p));
    const double y0 = bt.y0[bb * D + i];
    const double y1 = Y1 ? bt.y1[bb * D + i] : 0.0;
    const FF T0 = ff_from_double(y0);
    const FF ha = ff_from_double(kc.h_alpha[0]);
    const FF ha_ig2 = ff_from_double(kc.h_alpha[0] * kc.inv_gamma2[0]);
    float2 *Yb = reinterpret_cast<float2 *>(bt.Y + bb * (bt.N + 1) * D);
    const int cols = bt.cols;
    __syncwarp();

    FF accP[kSub], accC[kSub], bP[kSub], bC[kSub], rcs[kSub], axs[kSub];
    for (int a0 = 0; a0 < wsteps; a0 += kSub) {
        // the sub-block's forcing values, loaded before the work that does not
        // need them (rows a0 .. a0+7 < 64 of the [64][B] table: in range even
        // past the last step), so the steps do not wait on them
#pragma unroll
        for (int r = 0; r < kSub; ++r)
            axs[r] = Rhs::kForcing ? ld_ff(X + (int64_t)(a0 + r) * bt.B + bb) : aux0;
        // bases from the history of the points k < cL
#pragma unroll
        for (int r = 0; r < kSub; ++r) {
            const int a = a0 + r;
            const FF gP = hist_in(hin, 0, a, col, cols);
            const FF gC = hist_in(hin, 1, a, col, cols);
            bP[r] = ha * gP;
            bC[r] = ff_fma(ld_ff(WD + (m0 + 1 + a)), f0, ha * gC);
            accP[r] = accC[r] = FF(0);
        }
        // points of the block before the sub-block: j = 0 .. a0
        for (int j = 0; j <= a0; ++j) {
            const FF fj = sF[j][lane];
#pragma unroll
            for (int r = 0; r < kSub; ++r) {
                const int d = a0 + r + 1 - j;
                dot2_acc(accP[r], sB[d], fj);
                dot2_acc(accC[r], sA[d], fj);
            }
        }
        __syncwarp();
        // the serial chain of the sub-block's steps
#pragma unroll
        for (int r = 0; r < kSub; ++r) {
            if (a0 + r < wsteps) {  // uniform over the warp
                const FF ax = axs[r];
                // Taylor part of the initial data: y0, or y0 + t y'(0) for 1 < alpha < 2
                FF T = T0;
                if constexpr (Y1) T = ff_from_double(fma((double)(m0 + 1 + a0 + r) * kc.h, y1, y0));
                const FF yp = T + (bP[r] + ff_norm(accP[r]));
                FF y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = shfl_ff(yp, g * D + q);
                const FF fp = Rhs::template one<D>(i, y, pf, ax);
                rcs[r] = bC[r] + ff_fma(ha_ig2, fp, ff_norm(accC[r]));  // h^a (history + f^P / Gamma(a+2))
                const FF yc = T + rcs[r];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = shfl_ff(yc, g * D + q);
                const FF fn = Rhs::template one<D>(i, y, pf, ax);
                sF[a0 + r + 1][lane] = fn;
                // the sub-block's later targets take the new point now
#pragma unroll
                for (int r2 = r + 1; r2 < kSub; ++r2) {
                    dot2_acc(accP[r2], sB[r2 - r], fn);
                    dot2_acc(accC[r2], sA[r2 - r], fn);
                }
            }
        }
        // outputs of the sub-block, off the chain: the increment of y and f, as pairs
#pragma unroll
        for (int r = 0; r < kSub; ++r) {
            const int a = a0 + r;
            if (act && a < steps) {
                const int64_t m = m0 + 1 + a;
                const FF fn = sF[a + 1][lane];
                Yb[m * D + i] = make_float2(rcs[r].hi, rcs[r].lo);
                Fw[m * bt.ldF + col] = make_float2(fn.hi, fn.lo);
                if (!(finite_f(rcs[r].hi) && finite_f(fn.hi))) report_nonfinite(bt.status, m, (int)bb);
            }
        }
        __syncwarp();
    }
}

// The same block with one lane per target (targets a and a+32 on lane a), one
// CTA of D warps per trajectory: for narrow batches, where one lane per column
// leaves the GPU mostly idle.  Every pending target adds the newest point as
// it appears; the owner of the next target runs the step, the components
// exchange y through shared memory.  Same inputs and outputs as
// recur_cols_kernel.
template <class Rhs, int D>
__global__ void __launch_bounds__(D *kWarp)
    recur_targets_kernel(DevBatch bt, const float2 *__restrict__ WB, const float2 *__restrict__ WA,
                         const float2 *__restrict__ WD, StepConsts kc, int64_t c,
                         const HistIn hin, const float2 *__restrict__ X)
{
    constexpr int TPL = kColL / kWarp;
    __shared__ FF sB[kColL + 1], sA[kColL + 1];
    __shared__ FF sy[2][D];
    const int b = blockIdx.x;
    const int i = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    const int64_t Nb = bt.N_each[b];
    const int64_t m0 = c * kColL;
    if (m0 >= Nb) return;  // trajectory finished (uniform over the CTA)
    for (int d = threadIdx.x; d <= kColL; d += blockDim.x) sB[d] = ld_ff(WB + d), sA[d] = ld_ff(WA + d);

    double p[kMaxParams];
    FF pf[kMaxParams];
#pragma unroll
    for (int q = 0; q < kMaxParams; ++q) {
        p[q] = bt.params[(int64_t)b * kMaxParams + q];
        pf[q] = ff_from_double(p[q]);
    }
    const int64_t col = (int64_t)b * D + i;
    const float2 *F2 = reinterpret_cast<const float2 *>(bt.F);
    const double y0 = bt.y0[col];
    const double y1 = bt.y1 ? bt.y1[col] : 0.0;
    const FF ha = ff_from_double(kc.h_alpha[0]);
    const FF ha_ig2 = ff_from_double(kc.h_alpha[0] * kc.inv_gamma2[0]);
    const FF f0 = ld_ff(F2 + col);
    const FF aux0 = Rhs::kForcing ? FF(0) : ff_from_double(Rhs::aux(0.0, p));

    FF T[TPL], bP[TPL], bC[TPL], ax[TPL], nP[TPL], nC[TPL], rc[TPL], fo[TPL];
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int a = lane + kWarp * t;
        const int64_t m = m0 + 1 + a;
        T[t] = bt.y1 ? ff_from_double(fma((double)m * kc.h, y1, y0)) : ff_from_double(y0);
        const FF gP = hist_in(hin, 0, a, col, bt.cols);
        const FF gC = hist_in(hin, 1, a, col, bt.cols);
        bP[t] = ha * gP;
        bC[t] = ff_fma(ld_ff(WD + m), f0, ha * gC);
        ax[t] = Rhs::kForcing ? ld_ff(X + (int64_t)a * bt.B + b) : aux0;
        nP[t] = nC[t] = rc[t] = fo[t] = FF(0);
    }
    FF fk = ld_ff(F2 + m0 * bt.ldF + col);  // the newest known point, f_{cL}
    __syncthreads();

    const int steps = (int)(Nb - m0 < kColL ? Nb - m0 : kColL);
    for (int s = 0; s < steps; ++s) {
        // every pending target adds the point cL+s; targets already done add
        // the weight of distance 0, which is 0
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
            const int d = lane + kWarp * t - s + 1;
            const int dd = d > 0 ? d : 0;
            dot2_acc(nP[t], sB[dd], fk);
            dot2_acc(nC[t], sA[dd], fk);
        }
        const int owner = s % kWarp, slot = s / kWarp;  // uniform over the CTA
        FF yp(0), ncor(0), tt(0), bc(0), axs(0);
#pragma unroll
        for (int t = 0; t < TPL; ++t)
            if (t == slot) yp = T[t] + (bP[t] + ff_norm(nP[t])), ncor = ff_norm(nC[t]), tt = T[t],
                           bc = bC[t], axs = ax[t];
        FF fn(0), r(0);
        if constexpr (D == 1) {
            if (lane == owner) {
                const FF fp = Rhs::template one<D>(0, &yp, pf, axs);
                r = bc + ff_fma(ha_ig2, fp, ncor);
                const FF yc = tt + r;
                fn = Rhs::template one<D>(0, &yc, pf, axs);
            }
        } else {
            if (lane == owner) sy[0][i] = yp;
            __syncthreads();
            if (lane == owner) {
                FF y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = sy[0][q];
                const FF fp = Rhs::template one<D>(i, y, pf, axs);
                r = bc + ff_fma(ha_ig2, fp, ncor);
                sy[1][i] = tt + r;
            }
            __syncthreads();
            if (lane == owner) {
                FF y[D];
#pragma unroll
                for (int q = 0; q < D; ++q) y[q] = sy[1][q];
                fn = Rhs::template one<D>(i, y, pf, axs);
            }
        }
#pragma unroll
        for (int t = 0; t < TPL; ++t)
            if (t == slot && lane == owner) rc[t] = r, fo[t] = fn;
        fk = shfl_ff(fn, owner);
    }

    // the block's increments of y and f, one target per lane
    float2 *Yb = reinterpret_cast<float2 *>(bt.Y + (int64_t)b * (bt.N + 1) * D);
    float2 *Fw = reinterpret_cast<float2 *>(bt.F);
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int a = lane + kWarp * t;
        if (a < steps) {
            const int64_t m = m0 + 1 + a;
            Yb[m * D + i] = make_float2(rc[t].hi, rc[t].lo);
            Fw[m * bt.ldF + col] = make_float2(fo[t].hi, fo[t].lo);
            if (!(finite_f(rc[t].hi) && finite_f(fo[t].hi))) report_nonfinite(bt.status, m, b);
        }
    }
}

}  // namespace

cudaError_t prepare_recur_cols(int rhs, int dim)
{
    cudaError_t e = cudaSuccess;
    const bool ok = dispatch_rhs(rhs, dim, [&]<class R, int D>() {
        auto prep = [&](auto kernel) {
            cudaFuncAttributes fa;
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
            if (e == cudaSuccess && fa.numRegs * kMaxWarps * kWarp > 65536)
                e = cudaErrorInvalidConfiguration;
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cols_smem_bytes(D, kMaxWarps));
        };
        prep(recur_cols_kernel<R, D, false>);
        prep(recur_cols_kernel<R, D, true>);
    });
    return ok ? e : cudaErrorInvalidValue;
}

int recur_cols_warps(int dim, int64_t B) { return (int)((B + kWarp / dim - 1) / (kWarp / dim)); }

cudaError_t launch_recur_cols(int rhs, const DevBatch &bt, const float2 *WB, const float2 *WA,
                              const float2 *WD, const StepConsts &k, int64_t c, const HistIn &hin,
                              const float2 *X, int warps_per_cta, cudaStream_t st)
{
    if (warps_per_cta < 0 || warps_per_cta > kMaxWarps) return cudaErrorInvalidValue;
    if (hin.n_near < 0 || hin.n_near > kMaxNear) return cudaErrorInvalidValue;
    bool need_x = false;
    const bool ok = dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        need_x = R::kForcing;
        if (need_x && !X) return;
        if (warps_per_cta == 0) {  // one lane per target
            recur_targets_kernel<R, D><<<(unsigned)bt.B, D * kWarp, 0, st>>>(bt, WB, WA, WD, k, c,
                                                                             hin, X);
            return;
        }
        const int warps = recur_cols_warps(D, bt.B);
        const unsigned blocks = (unsigned)((warps + warps_per_cta - 1) / warps_per_cta);
        const size_t smem = cols_smem_bytes(D, warps_per_cta);
        if (bt.y1)
            recur_cols_kernel<R, D, true><<<blocks, warps_per_cta * kWarp, smem, st>>>(
                bt, WB, WA, WD, k, c, hin, X);
        else
            recur_cols_kernel<R, D, false><<<blocks, warps_per_cta * kWarp, smem, st>>>(
                bt, WB, WA, WD, k, c, hin, X);
    });
    return ok && !(need_x && !X) ? cudaGetLastError() : cudaErrorInvalidValue;
}

bool rhs_has_forcing(int rhs, int dim)
{
    bool f = false;
    dispatch_rhs(rhs, dim, [&]<class R, int D>() { f = R::kForcing; });
    return f;
}

cudaError_t launch_aux_table(int rhs, const DevBatch &bt, double h, int64_t c, float2 *X,
                             cudaStream_t st)
{
    const int64_t n = (int64_t)kColL * bt.B;
    int64_t blocks = (n + 127) / 128;
    if (blocks > 152 * 8) blocks = 152 * 8;
    const bool ok = dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        aux_kernel<R><<<(unsigned)blocks, 128, 0, st>>>(bt, h, c, X);
    });
    return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

cudaError_t launch_finish_y(const DevBatch &bt, double h, int64_t m_lo, int64_t m_hi,
                            cudaStream_t st)
{
    if (m_lo < 1 || m_hi > bt.N) return cudaErrorInvalidValue;
    if (m_hi < m_lo) return cudaSuccess;
    const int64_t n = (int64_t)bt.B * (m_hi - m_lo + 1) * bt.dim;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    finish_y_kernel<<<(unsigned)blocks, 256, 0, st>>>(bt, h, m_lo, m_hi);
    return cudaGetLastError();
}

}  // namespace fabm
