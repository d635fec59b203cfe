// a4 + a5: kernels around recur_block / init_one (recurrence.cuh).
#include "recurrence.cuh"

namespace fabm {
namespace {

template <class Rhs, int D>
__global__ void init_kernel(DevBatch bt)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < bt.B) init_one<Rhs, D>(bt, b);
}

template <class Rhs, int D, int TPL>
__global__ void __launch_bounds__(D *kWarp)
    recur_kernel(DevBatch bt, DevWeights w, StepConsts kc, int64_t c, const double *G)
{
    __shared__ double smem[recur_smem_doubles<D, TPL>()];
    recur_block<Rhs, D, TPL>(bt, blockIdx.x, w, kc, c, G, smem);
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

cudaError_t launch_recur(int rhs, const DevBatch &bt, const DevWeights &w, const StepConsts &k,
                         int64_t c, int L, const double *G, cudaStream_t st)
{
    const unsigned blocks = (unsigned)bt.B;
    bool ok = false;
    if (L == kWarp) {
        ok = dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
            recur_kernel<R, D, 1><<<blocks, D * kWarp, 0, st>>>(bt, w, k, c, G);
        });
    } else if (L == 2 * kWarp) {
        ok = dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
            recur_kernel<R, D, 2><<<blocks, D * kWarp, 0, st>>>(bt, w, k, c, G);
        });
    }
    return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

}  // namespace fabm
