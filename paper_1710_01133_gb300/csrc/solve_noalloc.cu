// fabm_solve_noalloc: a single-trajectory FP64 solve that makes no device
// allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// solve: code that runs under a fixed device-memory budget that another
// allocator (for example a framework's caching allocator) owns in full, code
// that must not call cudaMalloc/cudaFree because those calls synchronize the
// device, and plug-ins whose host process forbids them allocations of their
// own.  For them this entry point runs the same kernels as fabm_solve
// (weights, initial values, far-history sums with their split-k partials,
// fixed-order combine, recurrence) with every buffer carved out of one
// file-scope device array of fixed size.  The caller passes only its host
// input (y0, parameters) and host output.
//
// Limits and sharing: N <= kNoallocMaxN steps, dim <= FABM_MAX_DIM, one
// trajectory, FP64 only.  Every GPU that loads the library holds the array
// (about 7 MB) until the process exits.  All calls of a process share it: a
// host mutex serializes calls made through this entry point, but work that
// overlaps on the GPU with another user of the same array (for example a
// second process-level instance of this code driving the same context from
// outside the mutex) would race.  The array keeps the contents of the last
// call; the only value that must start from a fixed state (the non-finite
// status word) is reset at the start of every call.
//
// The array belongs to the CUDA context that loaded the library's device
// code, not to the device number: after cudaDeviceReset, or with another
// context current, it lives at a different address.  So every call looks the
// address up again (cudaGetSymbolAddress, with the calling thread's current
// device and context, under the mutex) instead of keeping one from an earlier
// call.  The first call in a context may load the library's device code into
// that context; make it before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "fabm_internal.cuh"
#include "rhs.cuh"

using namespace fabm;

namespace {

constexpr int64_t kNoallocMaxN = 65536;
constexpr int kNaL = kRecurL;                         // block length (32)
constexpr int kNaMaxChunks = 608;                     // far-history chunks per block
constexpr int64_t kNaW = kNoallocMaxN + 3 * kNaL;     // weight entries: last block + lag window
constexpr int64_t kNaRows = (kNoallocMaxN + 1) * FABM_MAX_DIM;
// region offsets in doubles (each a multiple of 32 doubles = 256 bytes)
constexpr int64_t kRound = 32;
constexpr int64_t rnd(int64_t x) { return (x + kRound - 1) / kRound * kRound; }
constexpr int64_t kOffB = 0;
constexpr int64_t kOffA = kOffB + rnd(kNaW);
constexpr int64_t kOffD = kOffA + rnd(kNaW);
constexpr int64_t kOffF = kOffD + rnd(kNaW);
constexpr int64_t kOffY = kOffF + rnd(kNaRows);
constexpr int64_t kOffG = kOffY + rnd(kNaRows);
constexpr int64_t kOffPart = kOffG + rnd(2 * 2 * kNaL * FABM_MAX_DIM);
constexpr int64_t kOffY0 = kOffPart + rnd((int64_t)kNaMaxChunks * 2 * kNaL * FABM_MAX_DIM);
constexpr int64_t kOffPar = kOffY0 + rnd(FABM_MAX_DIM);
constexpr int64_t kOffNe = kOffPar + rnd(kMaxParams);   // one int64
constexpr int64_t kOffSt = kOffNe + kRound;             // one unsigned long long
constexpr int64_t kScratchDoubles = kOffSt + kRound;

// The scratch array (about 7 MB).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_noalloc_mutex;

fabm_status na_fail(fabm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

#define NA_TRY(expr)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return na_fail(FABM_ECUDA, "fabm_solve_noalloc: %s failed: %s", #expr,           \
                           cudaGetErrorString(e_));                                          \
    } while (0)

}  // namespace

extern "C" fabm_status fabm_solve_noalloc(int dim, double alpha, double h, int64_t N, int rhs_id,
                                          const double *params, int n_params, const double *y0,
                                          double *out)
{
    set_last_error("");
    if (dim < 1 || dim > FABM_MAX_DIM)
        return na_fail(FABM_EINVAL, "fabm_solve_noalloc: dim %d outside 1..%d", dim, FABM_MAX_DIM);
    if (N < 1 || N > kNoallocMaxN)
        return na_fail(FABM_EINVAL,
                       "fabm_solve_noalloc: N = %lld outside 1..%lld (the fixed scratch array "
                       "holds at most %lld steps)",
                       (long long)N, (long long)kNoallocMaxN, (long long)kNoallocMaxN);
    if (!(alpha > 0.0 && alpha < 1.0))
        return na_fail(FABM_EINVAL, "fabm_solve_noalloc: alpha %g outside (0, 1)", alpha);
    if (!(h > 0.0) || !std::isfinite(h))
        return na_fail(FABM_EINVAL, "fabm_solve_noalloc: h %g must be positive", h);
    const int np = rhs_n_params(rhs_id);
    if (np < 0 || !rhs_supports_dim(rhs_id, dim))
        return na_fail(FABM_EINVAL, "fabm_solve_noalloc: rhs_id %d with dim %d unsupported", rhs_id,
                       dim);
    if (n_params < np || n_params > kMaxParams || (n_params > 0 && !params))
        return na_fail(FABM_EINVAL, "fabm_solve_noalloc: rhs_id %d needs %d params", rhs_id, np);
    if (!y0 || !out) return na_fail(FABM_EINVAL, "fabm_solve_noalloc: y0 and out must not be NULL");
    for (int i = 0; i < dim; ++i)
        if (!std::isfinite(y0[i])) return na_fail(FABM_EINVAL, "fabm_solve_noalloc: y0 not finite");

    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    // the address in the context current now (see the header comment)
    void *sym = nullptr;
    NA_TRY(cudaGetSymbolAddress(&sym, g_noalloc_scratch));
    double *S = static_cast<double *>(sym);
    cudaStream_t st = cudaStreamPerThread;

    // host-side constants and inputs
    StepConsts kc{};
    kc.h = h;
    for (int q = 0; q < FABM_MAX_DIM; ++q) {
        kc.h_alpha[q] = std::pow(h, alpha);
        kc.inv_gamma2[q] = 1.0 / std::tgamma(alpha + 2.0);
    }
    const double inv_g1 = 1.0 / std::tgamma(alpha + 1.0);
    double par[kMaxParams] = {};
    for (int i = 0; i < n_params; ++i) par[i] = params[i];
    const int64_t nrow = N;

    NA_TRY(cudaMemcpyAsync(S + kOffY0, y0, sizeof(double) * dim, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(S + kOffPar, par, sizeof par, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(S + kOffNe, &nrow, sizeof nrow, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemsetAsync(S + kOffSt, 0xff, sizeof(unsigned long long), st));

    // weights for every distance the kernels read: targets up to the last
    // block's end plus the lag-1 window
    const int64_t nblk = (N + kNaL - 1) / kNaL;
    const int64_t w_ext = nblk * kNaL + 2 * kNaL;
    NA_TRY(launch_weights(alpha, w_ext, inv_g1, kc.inv_gamma2[0], S + kOffB, S + kOffA, S + kOffD, st));

    DevBatch bt{};
    bt.dim = dim;
    bt.B = 1;
    bt.cols = dim;
    bt.N = N;
    bt.N_each = reinterpret_cast<const int64_t *>(S + kOffNe);
    bt.y0 = S + kOffY0;
    bt.params = S + kOffPar;
    bt.F = S + kOffF;
    bt.ldF = dim;
    bt.Y = S + kOffY;
    bt.status = reinterpret_cast<unsigned long long *>(S + kOffSt);
    DevWeights w{S + kOffB, S + kOffA, S + kOffD, w_ext};

    NA_TRY(launch_init(rhs_id, bt, st));
    for (int64_t c = 0; c < nblk; ++c) {
        const double *Gc = nullptr;
        if (c >= 2) {
            const int64_t k_end = (c - 1) * kNaL;
            int64_t n = (k_end + 63) / 64;
            if (n > kNaMaxChunks) n = kNaMaxChunks;
            int64_t kc_pts = (k_end + n - 1) / n;
            kc_pts = (kc_pts + 31) / 32 * 32;
            const int n_chunks = (int)((k_end + kc_pts - 1) / kc_pts);
            double *Gbuf = S + kOffG + (c % 2) * 2 * kNaL * dim;
            NA_TRY(launch_hist_fp64(bt, w, c, kNaL, 1, n_chunks, kc_pts, S + kOffPart, st));
            NA_TRY(launch_hist_reduce(S + kOffPart, n_chunks, kNaL, dim, Gbuf, st));
            Gc = Gbuf;
        }
        NA_TRY(launch_recur(rhs_id, bt, w, kc, c, kNaL, 1, false, Gc, st));
    }
    NA_TRY(cudaStreamSynchronize(st));
    unsigned long long status = 0;
    NA_TRY(cudaMemcpy(&status, S + kOffSt, sizeof status, cudaMemcpyDeviceToHost));
    NA_TRY(cudaMemcpy(out, S + kOffY, sizeof(double) * (N + 1) * dim, cudaMemcpyDeviceToHost));
    if (status != ~0ull)
        return na_fail(FABM_ENONFINITE, "fabm_solve_noalloc: non-finite value at step %llu",
                       status >> 24);
    return FABM_OK;
}
