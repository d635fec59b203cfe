// a2 + a3 in double: the far part of the hereditary sums of Sec. 2 of
// arXiv:1710.01133 (the k-loop of Algorithm 1, which is all of the O(N^2)
// work), for one block of L targets, split over the points k in chunks.
//
// For target block c (targets m = cL+1+a, a < L) and the points k < (c-1)L:
//   GP[a][col] = sum_k B(m-k) F[k][col],   GC[a][col] = sum_k A(m-k) F[k][col].
// The weights depend on m-k only (Toeplitz), so a chunk of kc points needs
// kc+L-1 consecutive weights, staged in shared memory with the chunk of F.
//
// GB300's FP64 pipe retires two double FMA lanes per clock per SM (measured
// 1.19 TFLOP/s at 1.96 GHz), and a warp FP64 instruction costs the same pipe
// time however many of its lanes are active, so this kernel keeps all 32
// lanes of every DFMA busy (lane = target, warp = column).  The chunks are
// summed afterwards in a fixed order with compensation (a3), so results do
// not depend on scheduling.  In isolation it reaches ~0.8 of the FP64 peak at one wave of
// ~600 CTAs; staging each tile before computing it costs most of the rest.
#include "history_blocks.cuh"

namespace fabm {
namespace {

// grid = (n_chunks, ceil(cols / kColsPerCta)); block = 32 * kColsPerCta.
// MULTI: one order per component (weights of component i at WB + i*wstride).
template <bool MULTI>
__global__ void __launch_bounds__(kWarp *hist::kColsPerCta)
    hist_fp64_kernel(const double *__restrict__ F, int64_t ldF, int cols,
                     const double *__restrict__ WB, const double *__restrict__ WA, int64_t c,
                     int64_t kc, int64_t k_end, double *__restrict__ part, int64_t wstride,
                     int dim)
{
    hist::f64::hist_fp64_block<MULTI>(F, ldF, cols, WB, WA, c, kc, k_end, part, blockIdx.x,
                                      blockIdx.y * hist::kColsPerCta, wstride, dim);
}

// Error-free sum of two doubles (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// (s, c) += v with compensation: the rounding error of every addition is
// collected in c (Neumaier's compensated summation, written with TwoSum so
// that it needs no branch on the magnitudes).
__device__ __forceinline__ void comp_add(double &s, double &c, double v)
{
    double e;
    two_sum(s, v, s, e);
    c += e;
}

// a3: G[pc][a][col] = sum_{chunk} part[chunk][pc][a][col], chunk ascending
// within each lane's strided subset, then a fixed xor tree over the R lanes of
// a group; every addition compensated (running sum s and error term c, added
// once at the end), so the combined history carries the rounding of one
// addition rather than of n_chunks.  grid-stride over the 2*L*cols outputs.
template <int R>
__global__ void hist_reduce_kernel(const double *__restrict__ part, int n_chunks, int64_t n_out,
                                   double *__restrict__ G)
{
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = (int)(gtid % R);
    const int64_t groups = (int64_t)gridDim.x * blockDim.x / R;
    // every thread runs the same number of rounds, so the shuffles below
    // always see full warps
    for (int64_t base = 0; base < n_out; base += groups) {
        const int64_t o = base + gtid / R;
        double s = 0.0, c = 0.0;
        if (o < n_out) {
            // independent loads in flight, summed in chunk order
            int ch = r;
            for (; ch + 3 * R < n_chunks; ch += 4 * R) {
                const double v0 = part[(int64_t)ch * n_out + o];
                const double v1 = part[(int64_t)(ch + R) * n_out + o];
                const double v2 = part[(int64_t)(ch + 2 * R) * n_out + o];
                const double v3 = part[(int64_t)(ch + 3 * R) * n_out + o];
                comp_add(s, c, v0);
                comp_add(s, c, v1);
                comp_add(s, c, v2);
                comp_add(s, c, v3);
            }
            for (; ch < n_chunks; ch += R) comp_add(s, c, part[(int64_t)ch * n_out + o]);
        }
#pragma unroll
        for (int off = R / 2; off > 0; off >>= 1) {
            const double os = __shfl_xor_sync(0xffffffffu, s, off);
            const double oc = __shfl_xor_sync(0xffffffffu, c, off);
            comp_add(s, c, os);
            c += oc;
        }
        if (r == 0 && o < n_out) G[o] = s + c;
    }
}

}  // namespace

cudaError_t launch_hist_fp64(const DevBatch &bt, const DevWeights &w, int64_t c, int L, int lag,
                             int n_chunks, int64_t kc, double *part, cudaStream_t st)
{
    const int64_t k_end = (c - lag) * L;
    if (L != hist::kL || lag < 1) return cudaErrorInvalidValue;
    if (k_end <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_chunks, (unsigned)((bt.cols + hist::kColsPerCta - 1) / hist::kColsPerCta));
    if (w.stride)
        hist_fp64_kernel<true><<<grid, kWarp * hist::kColsPerCta, 0, st>>>(
            bt.F, bt.ldF, bt.cols, w.B, w.A, c, kc, k_end, part, w.stride, bt.dim);
    else
        hist_fp64_kernel<false><<<grid, kWarp * hist::kColsPerCta, 0, st>>>(
            bt.F, bt.ldF, bt.cols, w.B, w.A, c, kc, k_end, part, 0, 1);
    return cudaGetLastError();
}

cudaError_t launch_hist_reduce(const double *part, int n_chunks, int L, int cols, double *G,
                               cudaStream_t st)
{
    const int64_t n_out = 2LL * L * cols;
    const int threads = 256;
    auto blocks_for = [&](int R) {
        int64_t b = (n_out * R + threads - 1) / threads;
        return (unsigned)(b > 152 * 16 ? 152 * 16 : b);
    };
    if (n_chunks >= 256) {
        hist_reduce_kernel<32><<<blocks_for(32), threads, 0, st>>>(part, n_chunks, n_out, G);
    } else if (n_chunks >= 32) {
        hist_reduce_kernel<8><<<blocks_for(8), threads, 0, st>>>(part, n_chunks, n_out, G);
    } else {
        hist_reduce_kernel<1><<<blocks_for(1), threads, 0, st>>>(part, n_chunks, n_out, G);
    }
    return cudaGetLastError();
}

}  // namespace fabm
