// a4 + a5: kernels around recur_block / init_one (recurrence.cuh).
#include "recurrence.cuh"

namespace fabm {
namespace {

template <class Rhs, int D>
__global__ void init_kernel(DevBatch bt, bool f_pairs)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < bt.B) init_one<Rhs, D>(bt, b, f_pairs);
}

template <class Rhs, int D, int TPL, bool SPLIT, int LAG>
__global__ void __launch_bounds__(D *kWarp)
    recur_kernel(DevBatch bt, DevWeights w, StepConsts kc, int64_t c, const double *G)
{
    if constexpr (SPLIT) {
        __shared__ __align__(16) float smem_f[recur_split_smem_floats<D, TPL, LAG>()];
        recur_block_split<Rhs, D, TPL, LAG>(bt, blockIdx.x, w, kc, c, G, smem_f);
    } else {
        __shared__ double smem[recur_smem_doubles<D, TPL, LAG>()];
        recur_block<Rhs, D, TPL, LAG>(bt, blockIdx.x, w, kc, c, G, smem);
    }
}

template <int TPL, bool SPLIT, int LAG>
bool launch_recur_t(int rhs, const DevBatch &bt, const DevWeights &w, const StepConsts &k,
                    int64_t c, const double *G, cudaStream_t st)
{
    return dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        recur_kernel<R, D, TPL, SPLIT, LAG><<<(unsigned)bt.B, D * kWarp, 0, st>>>(bt, w, k, c, G);
    });
}

}  // namespace

cudaError_t launch_init(int rhs, const DevBatch &bt, cudaStream_t st, bool f_pairs)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((bt.B + threads - 1) / threads);
    bool ok = dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        init_kernel<R, D><<<blocks, threads, 0, st>>>(bt, f_pairs);
    });
    return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

cudaError_t launch_recur(int rhs, const DevBatch &bt, const DevWeights &w, const StepConsts &k,
                         int64_t c, int L, int lag, bool split, const double *G, cudaStream_t st)
{
    bool ok = false;
    if (L == kWarp && lag == 1)
        ok = split ? launch_recur_t<1, true, 1>(rhs, bt, w, k, c, G, st)
                   : launch_recur_t<1, false, 1>(rhs, bt, w, k, c, G, st);
    else if (L == kWarp && lag == 2)
        ok = split ? launch_recur_t<1, true, 2>(rhs, bt, w, k, c, G, st)
                   : launch_recur_t<1, false, 2>(rhs, bt, w, k, c, G, st);
    return ok ? cudaGetLastError() : cudaErrorInvalidValue;
}

}  // namespace fabm
