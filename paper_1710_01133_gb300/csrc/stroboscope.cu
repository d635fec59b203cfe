// Stroboscopic sampling of solved trajectories (Sec. 5 of arXiv:1710.01133:
// the bifurcation diagram of the forced LCR system plots the attractor once
// per forcing period 2 pi / omega against the forcing amplitude f).
//
// samples[b][j] = component `comp` of trajectory b at t_j = t0 + j * period,
// linearly interpolated between the grid points t_n = n h around t_j; NaN
// where t_j lies outside [0, N_b h].  One thread per (trajectory, sample);
// the output is trajectory-major, the reads are a gather of two rows.
#include <cmath>

#include "fabm_internal.cuh"

namespace fabm {
namespace {

__global__ void stroboscope_kernel(const double *__restrict__ Y, int64_t B, int64_t N, int dim,
                                   const int64_t *__restrict__ N_each, double h, double t0,
                                   double period, int64_t n_samples, int comp,
                                   double *__restrict__ samples)
{
    const int64_t total = B * n_samples;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / n_samples, j = i % n_samples;
        const int64_t nb = N_each ? N_each[b] : N;  // rows 0..nb of trajectory b hold data
        const double u = (t0 + (double)j * period) / h;
        double v = nan("");
        if (nb >= 1 && nb <= N && u >= 0.0 && u <= (double)nb) {
            int64_t n = (int64_t)floor(u);
            if (n > nb - 1) n = nb - 1;  // u == nb: the last interval, weight 1
            const double w = u - (double)n;
            const double *row = Y + (b * (N + 1) + n) * dim + comp;
            v = fma(w, row[dim] - row[0], row[0]);
        }
        samples[i] = v;
    }
}

}  // namespace
}  // namespace fabm

extern "C" fabm_status fabm_stroboscope(const double *Y, int64_t B, int64_t N, int dim,
                                        const int64_t *N_each, double h, double t0,
                                        double period, int64_t n_samples, int comp,
                                        double *samples)
{
    using namespace fabm;
    if (!Y || !samples) {
        set_last_error("fabm_stroboscope: Y and samples must be device pointers");
        return FABM_EINVAL;
    }
    if (B < 0 || N < 1 || dim < 1 || dim > FABM_MAX_DIM || comp < 0 || comp >= dim ||
        n_samples < 0 || !(h > 0.0) || !(period > 0.0) || !std::isfinite(t0)) {
        set_last_error("fabm_stroboscope: invalid sizes, component, h, period or t0");
        return FABM_EINVAL;
    }
    if (B == 0 || n_samples == 0) return FABM_OK;
    const int64_t total = B * n_samples;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    stroboscope_kernel<<<(unsigned)blocks, 256>>>(Y, B, N, dim, N_each, h, t0, period, n_samples,
                                                  comp, samples);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return FABM_ECUDA;
    }
    return FABM_OK;
}
