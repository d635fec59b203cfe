// CTA-level bodies of the far-history kernels (a2), shared by the batch
// kernels and the serving kernels.
#pragma once

#include "fabm_internal.cuh"

namespace fabm {
namespace hist {

constexpr int kColsPerCta = 4;  // one warp per column
constexpr int kL = kRecurL;     // targets per block (one per lane)

namespace f64 {
constexpr int kTile = 256;      // points staged in shared memory at a time

// The points k in [k0, k1) of the far history of block c for the columns
// col0 .. col0+3, by 32 * kColsPerCta threads (tid = 0 .. 127 among them) that
// share the tiles sF[kTile * kColsPerCta], sB, sA[NW][kTile + kL] and
// synchronise with sync(); the sums go to out[(kind * kL + a) * out_ld + w],
// kind 0 predictor, 1 corrector, a the target, w < 4 the column after col0.
// MULTI: one order per component, column col's weights at WB + (col % dim)
// * wstride (WA likewise), one staged window per warp.  CG: read F around L1
// (ld.global.cg), for callers whose F rows are written by other CTAs of the
// same launch while it runs.
template <bool MULTI, bool CG, class Sync>
__device__ inline void hist_fp64_chunk(const double *__restrict__ F, int64_t ldF, int cols,
                                       const double *__restrict__ WB,
                                       const double *__restrict__ WA, int64_t c, int64_t k0,
                                       int64_t k1, double *__restrict__ out, int64_t out_ld,
                                       int col0, int64_t wstride, int dim, int tid, double *sF,
                                       double (*sB)[kTile + kL], double (*sA)[kTile + kL],
                                       Sync sync)
{
    constexpr int NW = MULTI ? kColsPerCta : 1;  // weight windows
    constexpr int nthr = kWarp * kColsPerCta;
    const int ncol = min(kColsPerCta, cols - col0);
    const int w = tid / kWarp;
    const int a = tid % kWarp;  // target m = cL+1+a
    double sp = 0.0, sc = 0.0;

    for (int64_t t0 = k0; t0 < k1; t0 += kTile) {
        const int64_t t1 = t0 + kTile < k1 ? t0 + kTile : k1;
        const int nk = (int)(t1 - t0);
        // weights for d = m - k, m in [cL+1, cL+L], k in [t0, t1):
        // window index i <-> d = cL+2-t1 + i, i < nk+L-1
        const int64_t d_min = c * kL + 2 - t1;
        const int nwin = nk + kL - 1;
        if constexpr (MULTI) {
            for (int i = tid; i < NW * nwin; i += nthr) {
                const int v = i / nwin, ii = i % nwin;
                const int64_t o = (int64_t)((col0 + v) % dim) * wstride;
                sB[v][ii] = WB[o + d_min + ii];
                sA[v][ii] = WA[o + d_min + ii];
            }
        } else {
            for (int i = tid; i < nwin; i += nthr) {
                sB[0][i] = WB[d_min + i];
                sA[0][i] = WA[d_min + i];
            }
        }
        for (int i = tid; i < nk * kColsPerCta; i += nthr) {
            const int k = i / kColsPerCta, j = i % kColsPerCta;
            const double *src = F + (t0 + k) * ldF + col0 + j;
            sF[i] = j < ncol ? (CG ? __ldcg(src) : *src) : 0.0;
        }
        sync();
        if (w < ncol) {
            // d - d_min = (cL+1+a - (t0+j)) - (cL+2-t1) = a + nk-1-j
            const double *fb = sF + w;
            const double *wb = sB[MULTI ? w : 0], *wa = sA[MULTI ? w : 0];
            const int base = a + nk - 1;
#pragma unroll 4
            for (int j = 0; j < nk; ++j) {
                const double f = fb[j * kColsPerCta];
                sp = fma(wb[base - j], f, sp);
                sc = fma(wa[base - j], f, sc);
            }
        }
        sync();
    }
    if (w < ncol) {
        out[(int64_t)a * out_ld + w] = sp;
        out[(int64_t)(kL + a) * out_ld + w] = sc;
    }
}

// One CTA of 32 * kColsPerCta threads: chunk `chunk` (points k in
// [chunk*kc, min((chunk+1)*kc, k_end))) of the far history of block c for the
// columns col0 .. col0+3 into part[chunk][2][kL][cols] (hist_fp64_chunk with
// the CTA's own tiles and barrier).
template <bool MULTI = false>
__device__ inline void hist_fp64_block(const double *__restrict__ F, int64_t ldF, int cols,
                                       const double *__restrict__ WB,
                                       const double *__restrict__ WA, int64_t c, int64_t kc,
                                       int64_t k_end, double *__restrict__ part, int64_t chunk,
                                       int col0, int64_t wstride = 0, int dim = 1)
{
    constexpr int NW = MULTI ? kColsPerCta : 1;
    __shared__ double sF[kTile * kColsPerCta];
    __shared__ double sB[NW][kTile + kL], sA[NW][kTile + kL];
    const int64_t k0 = chunk * kc;
    const int64_t k1 = k0 + kc < k_end ? k0 + kc : k_end;
    hist_fp64_chunk<MULTI, false>(F, ldF, cols, WB, WA, c, k0, k1,
                                  part + (chunk * 2) * kL * (int64_t)cols + col0, cols, col0,
                                  wstride, dim, threadIdx.x, sF, sB, sA, [] { __syncthreads(); });
}

}  // namespace f64

namespace f32c {
constexpr int kTile = 512;      // points staged in shared memory at a time
constexpr int kGroup = 16;      // products added in plain fp32 before a Kahan step

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v)
{
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// One CTA of 32 * kHistCols threads: chunk `chunk` of the far history of
// block c for the columns col0 .. col0+3, in compensated fp32.  Ff: f rounded
// to float (same layout as F), read instead of converting F when not NULL.
// The next tile's f and weights are loaded into registers while the current
// tile is summed, so the staging latency hides behind the arithmetic.
// MULTI as for hist_fp64_block.
template <bool MULTI = false>
__device__ inline void hist_fp32c_block(const double *__restrict__ F, const float *__restrict__ Ff,
                                        int64_t ldF, int cols, const float *__restrict__ WB,
                                        const float *__restrict__ WA, int64_t c, int64_t kc,
                                        int64_t k_end, float2 *__restrict__ part, int64_t chunk,
                                        int col0, int64_t wstride = 0, int dim = 1)
{
    constexpr int NW = MULTI ? kColsPerCta : 1;  // weight windows
    constexpr int kThreads = kWarp * kColsPerCta;
    constexpr int kRF = kTile * kColsPerCta / kThreads;            // f values per thread
    constexpr int kRW = (NW * (kTile + kL) + kThreads - 1) / kThreads;  // weights per thread and kind
    __shared__ float sF[kTile * kColsPerCta];
    __shared__ float sB[NW][kTile + kL], sA[NW][kTile + kL];
    const int64_t k0 = chunk * kc;
    const int64_t k1 = k0 + kc < k_end ? k0 + kc : k_end;
    const int ncol = min(kColsPerCta, cols - col0);
    const int w = threadIdx.x / kWarp;
    const int a = threadIdx.x % kWarp;  // target m = cL+1+a
    float sp = 0.f, cp = 0.f, sc = 0.f, cc = 0.f;
    float rf[kRF], rb[kRW], ra[kRW];

    // the tile starting at t0 into registers: window index i <-> d = cL+2-t1 + i
    auto fetch = [&](int64_t t0) {
        const int64_t t1 = t0 + kTile < k1 ? t0 + kTile : k1;
        const int nk = (int)(t1 - t0), nwin = nk + kL - 1;
        const int64_t d_min = c * kL + 2 - t1;
#pragma unroll
        for (int u = 0; u < kRW; ++u) {
            const int i = threadIdx.x + u * kThreads;
            const int v = MULTI ? i / nwin : 0, ii = MULTI ? i % nwin : i;
            const bool in = MULTI ? i < NW * nwin : i < nwin;
            const int64_t o = MULTI ? (int64_t)((col0 + v) % dim) * wstride : 0;
            rb[u] = in ? WB[o + d_min + ii] : 0.f;
            ra[u] = in ? WA[o + d_min + ii] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kRF; ++u) {
            const int i = threadIdx.x + u * kThreads;
            const int k = i / kColsPerCta, j = i % kColsPerCta;
            float f = 0.f;
            if (k < nk && j < ncol)
                f = Ff ? Ff[(t0 + k) * ldF + col0 + j] : (float)F[(t0 + k) * ldF + col0 + j];
            rf[u] = f;
        }
    };

    if (k0 < k1) fetch(k0);
    for (int64_t t0 = k0; t0 < k1; t0 += kTile) {
        const int64_t t1 = t0 + kTile < k1 ? t0 + kTile : k1;
        const int nk = (int)(t1 - t0), nwin = nk + kL - 1;
#pragma unroll
        for (int u = 0; u < kRW; ++u) {
            const int i = threadIdx.x + u * kThreads;
            if (MULTI ? i < NW * nwin : i < nwin) {
                const int v = MULTI ? i / nwin : 0, ii = MULTI ? i % nwin : i;
                sB[v][ii] = rb[u];
                sA[v][ii] = ra[u];
            }
        }
#pragma unroll
        for (int u = 0; u < kRF; ++u) sF[threadIdx.x + u * kThreads] = rf[u];
        __syncthreads();
        if (t1 < k1) fetch(t1);  // next tile in flight during the sums below
        if (w < ncol) {
            const float *fb = sF + w;
            const float *wb = sB[MULTI ? w : 0], *wa = sA[MULTI ? w : 0];
            const int base = a + nk - 1;
            int j = 0;
            for (; j + kGroup <= nk; j += kGroup) {
                float gp = 0.f, gc = 0.f;
#pragma unroll
                for (int u = 0; u < kGroup; ++u) {
                    const float f = fb[(j + u) * kColsPerCta];
                    gp = fmaf(wb[base - j - u], f, gp);
                    gc = fmaf(wa[base - j - u], f, gc);
                }
                kahan_add(sp, cp, gp);
                kahan_add(sc, cc, gc);
            }
            float gp = 0.f, gc = 0.f;
            for (; j < nk; ++j) {
                const float f = fb[j * kColsPerCta];
                gp = fmaf(wb[base - j], f, gp);
                gc = fmaf(wa[base - j], f, gc);
            }
            kahan_add(sp, cp, gp);
            kahan_add(sc, cc, gc);
        }
        __syncthreads();
    }
    if (w < ncol) {
        float2 *out = part + ((chunk * 2) * kL + a) * (int64_t)cols + col0 + w;
        out[0] = make_float2(sp, -cp);
        out[(int64_t)kL * cols] = make_float2(sc, -cc);
    }
}

}  // namespace f32c

}  // namespace hist
}  // namespace fabm
