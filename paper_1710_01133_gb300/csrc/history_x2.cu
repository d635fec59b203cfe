// a2 + a3 in double-double (FP64X2 precision): the far part of the hereditary
// sums of Sec. 2 of arXiv:1710.01133, as hist_fp64_kernel computes it, with
// the weights as double-double pairs (wh + wl) and every product and sum kept
// to about twice double precision:
//   product  w f = p + e exactly for the high part (p = wh f rounded,
//            e = fma(wh, f, -p)), plus wl f folded into e;
//   sum      Ogita-Rump-Oishi Dot2: s = acc + p with its rounding error t
//            (TwoSum), acc_lo += t + e.
// Ten FP64 operations per multiply-add instead of one FMA; this is the mode
// the paper keeps for precise runs (long double), not the fast one.  Chunk
// partials are double-double pairs, combined in a fixed order in double-double
// and rounded once to double.
#include "fabm_internal.cuh"

namespace fabm {
namespace {

constexpr int kCols = 4;   // one warp per column
constexpr int kL = kRecurL;
constexpr int kTile = 256;  // points staged in shared memory at a time

// (hi, lo) += (p, e): the running sum and its error term
__device__ __forceinline__ void dot2_step(double &hi, double &lo, double p, double e)
{
    const double s = hi + p;
    const double z = s - hi;
    const double t = (hi - (s - z)) + (p - z);
    lo += t + e;
    hi = s;
}

// grid = (n_chunks, ceil(cols / 4)); block = 128.  Chunk `chunk` covers the
// points [chunk*kc, min((chunk+1)*kc, k_end)) of target block c (targets
// m = cL+1+a, lane a); part[chunk][kind][a][col] = (hi, lo).  wstride > 0: one
// order per component (column col's weights at offset (col % dim) * wstride).
__global__ void __launch_bounds__(kWarp *kCols)
    hist_x2_kernel(const double *__restrict__ F, int64_t ldF, int cols, const double *__restrict__ WBh,
                   const double *__restrict__ WBl, const double *__restrict__ WAh,
                   const double *__restrict__ WAl, int64_t c, int64_t kc, int64_t k_end,
                   double2 *__restrict__ part, int64_t wstride, int dim)
{
    __shared__ double sF[kTile * kCols];
    __shared__ double sBh[kCols][kTile + kL], sBl[kCols][kTile + kL];
    __shared__ double sAh[kCols][kTile + kL], sAl[kCols][kTile + kL];
    const int64_t chunk = blockIdx.x;
    const int col0 = blockIdx.y * kCols;
    const int64_t k0 = chunk * kc;
    const int64_t k1 = k0 + kc < k_end ? k0 + kc : k_end;
    const int ncol = min(kCols, cols - col0);
    const int w = threadIdx.x / kWarp;
    const int a = threadIdx.x % kWarp;
    // weight windows: one per warp when the orders differ, else warp 0's
    const int nwv = wstride ? kCols : 1;
    double ph = 0, pl = 0, ch = 0, cl = 0;

    for (int64_t t0 = k0; t0 < k1; t0 += kTile) {
        const int64_t t1 = t0 + kTile < k1 ? t0 + kTile : k1;
        const int nk = (int)(t1 - t0);
        // window index i <-> d = cL+2-t1 + i, i < nk+L-1 (as hist_fp64_block)
        const int64_t d_min = c * kL + 2 - t1;
        const int nwin = nk + kL - 1;
        for (int i = threadIdx.x; i < nwv * nwin; i += blockDim.x) {
            const int v = i / nwin, ii = i % nwin;
            const int64_t o = wstride ? (int64_t)((col0 + v) % dim) * wstride : 0;
            sBh[v][ii] = WBh[o + d_min + ii];
            sBl[v][ii] = WBl[o + d_min + ii];
            sAh[v][ii] = WAh[o + d_min + ii];
            sAl[v][ii] = WAl[o + d_min + ii];
        }
        for (int i = threadIdx.x; i < nk * kCols; i += blockDim.x) {
            const int k = i / kCols, j = i % kCols;
            sF[i] = j < ncol ? F[(t0 + k) * ldF + col0 + j] : 0.0;
        }
        __syncthreads();
        if (w < ncol) {
            const int v = wstride ? w : 0;
            const int base = a + nk - 1;  // d - d_min for point t0+j: a + nk-1-j
            for (int j = 0; j < nk; ++j) {
                const double f = sF[j * kCols + w];
                const double bh = sBh[v][base - j], ah = sAh[v][base - j];
                const double pp = bh * f, pc = ah * f;
                const double ep = fma(sBl[v][base - j], f, fma(bh, f, -pp));
                const double ec = fma(sAl[v][base - j], f, fma(ah, f, -pc));
                dot2_step(ph, pl, pp, ep);
                dot2_step(ch, cl, pc, ec);
            }
        }
        __syncthreads();
    }
    if (w < ncol) {
        double2 *out = part + ((chunk * 2) * kL + a) * (int64_t)cols + col0 + w;
        out[0] = make_double2(ph, pl);
        out[(int64_t)kL * cols] = make_double2(ch, cl);
    }
}

// double-double (hi, lo) += (x, y), renormalised
__device__ __forceinline__ void dd_add(double &hi, double &lo, double x, double y)
{
    const double s = hi + x;
    const double bb = s - hi;
    const double e = (hi - (s - bb)) + (x - bb);
    lo += e + y;
    hi = s + lo;
    lo = lo - (hi - s);
}

// a3: G[kind][a][col] = sum over chunks of (hi + lo) in double-double, R lanes
// per output summing chunks r, r+R, ... in ascending order, then a fixed xor
// tree; rounded once to double.  Every thread runs the same number of rounds,
// so the shuffles always see full warps.
template <int R>
__global__ void reduce_x2_kernel(const double2 *__restrict__ part, int n_chunks, int64_t n_out,
                                 double *__restrict__ G)
{
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = (int)(gtid % R);
    const int64_t groups = (int64_t)gridDim.x * blockDim.x / R;
    for (int64_t base = 0; base < n_out; base += groups) {
        const int64_t o = base + gtid / R;
        double hi = 0, lo = 0;
        if (o < n_out)
            for (int ch = r; ch < n_chunks; ch += R) {
                const double2 v = part[(int64_t)ch * n_out + o];
                dd_add(hi, lo, v.x, v.y);
            }
#pragma unroll
        for (int off = R / 2; off > 0; off >>= 1) {
            const double ohi = __shfl_xor_sync(0xffffffffu, hi, off);
            const double olo = __shfl_xor_sync(0xffffffffu, lo, off);
            dd_add(hi, lo, ohi, olo);
        }
        if (r == 0 && o < n_out) G[o] = hi + lo;
    }
}

}  // namespace

cudaError_t launch_hist_x2(const DevBatch &bt, const DevWeights &w, const DevWeightsLo &wl,
                           int64_t c, int lag, int n_chunks, int64_t kc, double2 *part,
                           cudaStream_t st)
{
    const int64_t k_end = (c - lag) * kL;
    if (lag < 1) return cudaErrorInvalidValue;
    if (k_end <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_chunks, (unsigned)((bt.cols + kCols - 1) / kCols));
    hist_x2_kernel<<<grid, kWarp * kCols, 0, st>>>(bt.F, bt.ldF, bt.cols, w.B, wl.B, w.A, wl.A, c,
                                                   kc, k_end, part, w.stride, bt.dim);
    return cudaGetLastError();
}

cudaError_t launch_reduce_x2(const double2 *part, int n_chunks, int cols, double *G, cudaStream_t st)
{
    const int64_t n_out = 2LL * kL * cols;
    const int threads = 256;
    auto blocks_for = [&](int R) {
        const int64_t b = (n_out * R + threads - 1) / threads;
        return (unsigned)(b > 152 * 16 ? 152 * 16 : b);
    };
    if (n_chunks >= 32)
        reduce_x2_kernel<8><<<blocks_for(8), threads, 0, st>>>(part, n_chunks, n_out, G);
    else
        reduce_x2_kernel<1><<<blocks_for(1), threads, 0, st>>>(part, n_chunks, n_out, G);
    return cudaGetLastError();
}

}  // namespace fabm
