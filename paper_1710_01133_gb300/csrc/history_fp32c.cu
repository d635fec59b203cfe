// a2 on CUDA cores in compensated single precision ("split" precision for
// narrow batches): the far part of the hereditary sums of Sec. 2 of
// arXiv:1710.01133 for one block of 32 targets, split over the points k in
// chunks, like the double-precision kernel but in fp32, which GB300 runs at
// 64 times the double rate.
//
// f (the recurrence's float copy of the double history) and the weights are
// in fp32 (2^-24 relative); each thread adds 16 products in plain fp32 and folds the
// group into a Kahan-compensated fp32 sum, so the rounding of a chunk's sum
// stays within a few units of 2^-24 of its magnitude.  Each chunk writes
// (sum, -compensation) pairs that the float-float combine adds up in a fixed
// order and rounds once to double.  This suits batches with few columns,
// where a 128-column tensor tile would be mostly padding; wide batches use
// the tensor-core kernel.
#include "history_blocks.cuh"

namespace fabm {
namespace {

// grid = (n_chunks, ceil(cols / kColsPerCta)); block = 32 * kColsPerCta.
template <bool MULTI>
__global__ void __launch_bounds__(kWarp *hist::kColsPerCta)
    hist_fp32c_kernel(const double *__restrict__ F, const float *__restrict__ Ff, int64_t ldF,
                      int cols, const float *__restrict__ WB, const float *__restrict__ WA,
                      int64_t c, int64_t kc, int64_t k_end, float2 *__restrict__ part,
                      int64_t wstride, int dim)
{
    hist::f32c::hist_fp32c_block<MULTI>(F, Ff, ldF, cols, WB, WA, c, kc, k_end, part, blockIdx.x,
                                        blockIdx.y * hist::kColsPerCta, wstride, dim);
}

__global__ void to_float_kernel(const double *__restrict__ x, int64_t n, float *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

}  // namespace

cudaError_t launch_to_float(const double *x, int64_t n, float *y, cudaStream_t st)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    to_float_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, y);
    return cudaGetLastError();
}

cudaError_t launch_hist_fp32c(const DevBatch &bt, const float *WBf, const float *WAf,
                              int64_t wstride, int64_t c, int lag, int n_chunks, int64_t kc,
                              float2 *part, cudaStream_t st)
{
    const int64_t k_end = (c - lag) * hist::kL;
    if (lag < 1) return cudaErrorInvalidValue;
    if (k_end <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_chunks, (unsigned)((bt.cols + hist::kColsPerCta - 1) / hist::kColsPerCta));
    if (wstride)
        hist_fp32c_kernel<true><<<grid, kWarp * hist::kColsPerCta, 0, st>>>(
            bt.F, bt.Ff, bt.ldF, bt.cols, WBf, WAf, c, kc, k_end, part, wstride, bt.dim);
    else
        hist_fp32c_kernel<false><<<grid, kWarp * hist::kColsPerCta, 0, st>>>(
            bt.F, bt.Ff, bt.ldF, bt.cols, WBf, WAf, c, kc, k_end, part, 0, 1);
    return cudaGetLastError();
}

}  // namespace fabm
