// a1: the ABM weights of Sec. 2 of arXiv:1710.01133 in double (the
// cancellation-free forms are in weights.cuh).
#include "weights.cuh"

namespace fabm {
namespace {

__global__ void weights_kernel(double alpha, int64_t N, double inv_g1, double inv_g2, double *B,
                               double *A, double *D)
{
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d <= N;
         d += (int64_t)gridDim.x * blockDim.x)
        weights_at(d, alpha, inv_g1, inv_g2, B, A, D);
}

}  // namespace
cudaError_t launch_weights(double alpha, int64_t N, double inv_g1, double inv_g2, double *B,
                           double *A, double *D, cudaStream_t st)
{
    const int threads = 256;
    int64_t blocks = (N + 1 + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    weights_kernel<<<(unsigned)blocks, threads, 0, st>>>(alpha, N, inv_g1, inv_g2, B, A, D);
    return cudaGetLastError();
}

}  // namespace fabm
