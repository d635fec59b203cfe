// C ABI (include/fabm.h): solver state, argument checks, device memory, and
// the block-by-block schedule of the kernels.
//
// Schedule of one solve (Sec. 2 of arXiv:1710.01133 evaluated block by block):
//   init                      y_0, f_0
//   for each block c of L targets (CUDA-core history kernels, L = 32):
//     stream G:  wait R(c-2); history(c) over k < (c-1)L; combine -> G[c%2]
//     stream R:  wait G(c);   recurrence(c), which adds the lag-1 block itself
//   (long FP64 solves: lag 2, the history of consecutive blocks on two streams)
//   tensor history, L = 64:
//     stream G:  wait R(c-2); far history(c) over segments 0..c-2; wait N(c);
//                combine of far and newest partials -> G[c%2] (float-float)
//     stream R:  slice segment c-1; N(c): newest segment c-1; wait G(c);
//                recurrence(c) over its own triangle only
//     stream G2: forcing tables up to three blocks ahead
//     stream C:  finished rows of y to pinned host memory (large outputs)
// The history of block c+1 therefore runs while the recurrence of block c
// runs.  This replaces the per-step MPI_Allreduce of the paper's Algorithm 1
// by one hand-off per block.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fabm_internal.cuh"
#include "rhs.cuh"
#include "trace.h"

using namespace fabm;

namespace {

thread_local std::string g_last_error;

fabm_status fail(fabm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define FABM_CUDA_TRY(expr)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? FABM_ENOMEM : FABM_ECUDA,          \
                        "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,    \
                        __LINE__);                                                           \
    } while (0)

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t want)
    {
        if (want <= n) return cudaSuccess;
        release();
        cudaError_t e = take_injected_alloc_failure() ? cudaErrorMemoryAllocation
                                                      : cudaMalloc(&p, want * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            return e;
        }
        n = want;
        return cudaSuccess;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

constexpr int kMaxBlockL = 1024;
constexpr int kEvRing = 4;
constexpr int kAuxRing = 4;  // forcing tables computed up to 3 blocks ahead

}  // namespace

void fabm::set_last_error(const char *msg) { g_last_error = msg; }

namespace {
std::atomic<int> g_alloc_failures{0};  // injected device-allocation failures left
}  // namespace

bool fabm::take_injected_alloc_failure()
{
    int n = g_alloc_failures.load(std::memory_order_relaxed);
    while (n > 0)
        if (g_alloc_failures.compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) return true;
    return false;
}

struct fabm_solver {
    int device = 0;
    int dim = 0;
    double alpha = 0, h = 0;            // alpha: the largest order of the components
    double alpha_c[FABM_MAX_DIM] = {};  // order of each component
    bool multi = false;                 // components have different orders
    int64_t N = 0;
    int rhs = 0;
    int n_params = 0;
    double params[kMaxParams] = {};
    int precision = FABM_FP64;
    int hist_kernel = FABM_HIST_AUTO;  // requested
    int last_hk = -1;                  // run by the last solve (fabm_last_history_kernel)
    int chunk_ctas = 0;                // split-k CTA target of the CUDA-core history kernels (0: auto)
    int sm_reserve = -1;               // SMs kept free of tensor-history CTAs (-1: automatic)
    long long wait_cycles = 0;         // tensor kernel's wait limit (0: its default)
    bool wide = false;                 // the solve being set up uses the 128-target far history
    int near_chunks = 1;               // wide path: CTAs per column tile of a near launch
    int persist_ctas = 0;              // FP64: CTAs of the persistent kernel resident at once
    int L = kRecurL;                   // block length of the last solve
    int rec_layout = FABM_REC_AUTO;    // recurrence layout on the tensor path (requested)
    int rec_warps = 0;                 // column recurrence: warps per CTA (0: automatic)
    int64_t plan_N = 0;                // > 0: schedule choices (lag, layout) as for this many
                                       // steps (the autotuner's truncated probes of a longer solve)
    int cols_warps = 1;                // tensor path: warps per CTA of the column recurrence,
                                       // or 0 for the lane-per-target layout
    StepConsts k{};
    int64_t w_ext = 0;  // weights valid for index 0..w_ext
    DevBuf<double> wB, wA, wD;
    DevBuf<double> wBl, wAl, wDl;  // FP64X2: low parts of the double-double weights
    // split path: fp32 weights (narrow kernel), Hankel weight tiles per lag and
    // their exponents (tensor kernel), float-float h^a B(d), h^a A(d) for
    // d <= 64 and h^a D(m) (column recurrence)
    DevBuf<float> wBf, wAf;
    DevBuf<float2> wBff, wAff, wDff;
    DevBuf<__nv_bfloat16> wH;
    DevBuf<int> wHe;
    int64_t g_max = 0;
    // wide far history: Hankel tiles per group lag (128-point groups) and exponents
    DevBuf<__nv_bfloat16> wH2;
    DevBuf<int> wHe2;
    int64_t G_max = 0;
    // per-batch workspace
    DevBuf<double> F, Ystage, G, part, y0, par;
    DevBuf<float> Ff;          // compensated-fp32 history: f rounded to float
    DevBuf<__nv_bfloat16> Fs;  // split: f slices
    DevBuf<int> Fe;            // split: f exponents
    DevBuf<float2> spart;      // split: float-float partials
    DevBuf<__nv_bfloat16> Fs2; // wide far history: f slices per 128-point group
    DevBuf<int> Fe2;           // wide far history: exponents per group
    DevBuf<float2> fpart;      // wide far history: partials of two target groups
    DevBuf<float2> fsum;       // wide far history: their chunk sums, [C % 2][2][128][cols]
    DevBuf<double> ppart, pspart;  // persistent FP64 solve: chunk and super-group partial slots
    DevBuf<int> psg, pdone, prdone; // persistent FP64 solve: chunks done per super-group,
                                    // super-groups done per block, blocks done per trajectory
    DevBuf<float2> auxb;       // tensor path: forcing tables of kAuxRing blocks
    DevBuf<unsigned int> err;  // split: timeout flag
    DevBuf<int64_t> nEach;
    DevBuf<unsigned long long> status;
    // sR: recurrence; sG, sG2: far history (the CUDA-core history of odd blocks
    // runs on sG2, so that consecutive blocks' history launches overlap)
    // sC: device-to-host copies of finished rows while the solve goes on
    // sG3: far history of odd target groups (wide tensor path); sS: the sums of
    // their chunks, at the recurrence's priority so that they are not queued
    // behind the next far launch's CTAs
    cudaStream_t sR = nullptr, sG = nullptr, sG2 = nullptr, sC = nullptr, sG3 = nullptr, sS = nullptr;
    double *out_stream = nullptr;  // pinned host output of the solve being enqueued, or NULL
    int64_t out_group = 1;         // blocks per streamed copy
    // evN: the newest-segment history launch of the tensor path (on sR); evA:
    // the forcing tables (tensor path, on sG2)
    cudaEvent_t evR[kEvRing] = {}, evG[3] = {}, evN[3] = {}, evA[kAuxRing] = {};
    cudaEvent_t evF[2] = {};  // wide far history of target group C summed, slot C % 2
    cudaEvent_t evFK[2] = {}; // wide far kernel of target group C done, slot C % 2
    cudaEvent_t evFork = nullptr, evJoin = nullptr, evJoinC = nullptr, evJoin3 = nullptr,
                evJoinS = nullptr;
    std::mutex busy;
    int64_t launches = 0;
    // per-launch timing (fabm_set_timing)
    bool timing = false;
    int timing_period = 1;    // time the launches of every k-th block
    bool sample_now = true;   // the block being enqueued is timed
    bool capturing = false;
    std::vector<cudaEvent_t> ev_pool;  // pairs (start, stop)
    struct Rec {
        int kind;
        double flops;
    };
    std::vector<Rec> recs;             // one per timed launch, pair i = ev_pool[2i], [2i+1]
    // CUDA graph of the last solve's launch sequence (fabm_set_graphs)
    bool use_graphs = true;
    cudaGraphExec_t gexec = nullptr;
    std::vector<uintptr_t> gkey;
    std::vector<Rec> grecs;
    int64_t glaunches = 0;
    int64_t k_launches[FABM_KERNEL_KINDS] = {};
    double k_ms[FABM_KERNEL_KINDS] = {};
    double k_flops[FABM_KERNEL_KINDS] = {};
    double k_busy[FABM_KERNEL_KINDS] = {};  // union of the timed launches' intervals

    ~fabm_solver()
    {
        wB.release(), wA.release(), wD.release(), wH.release(), wHe.release();
        wH2.release(), wHe2.release(), Fs2.release(), Fe2.release(), fpart.release(), fsum.release();
        ppart.release(), pdone.release(), prdone.release();
        wBl.release(), wAl.release(), wDl.release();
        wBf.release(), wAf.release(), wBff.release(), wAff.release(), wDff.release();
        F.release(), Ff.release(), Ystage.release(), G.release(), part.release();
        Fs.release(), Fe.release(), spart.release(), auxb.release(), err.release();
        y0.release(), par.release(), nEach.release(), status.release();
        for (auto &e : evR)
            if (e) cudaEventDestroy(e);
        for (auto &e : evG)
            if (e) cudaEventDestroy(e);
        for (auto &e : evN)
            if (e) cudaEventDestroy(e);
        for (auto &e : evA)
            if (e) cudaEventDestroy(e);
        for (auto &e : evF)
            if (e) cudaEventDestroy(e);
        for (auto &e : evFK)
            if (e) cudaEventDestroy(e);
        if (evJoinS) cudaEventDestroy(evJoinS);
        if (evJoin3) cudaEventDestroy(evJoin3);
        if (evFork) cudaEventDestroy(evFork);
        if (evJoin) cudaEventDestroy(evJoin);
        if (evJoinC) cudaEventDestroy(evJoinC);
        if (gexec) cudaGraphExecDestroy(gexec);
        for (auto &e : ev_pool) cudaEventDestroy(e);
        if (sR) cudaStreamDestroy(sR);
        if (sG) cudaStreamDestroy(sG);
        if (sG2) cudaStreamDestroy(sG2);
        if (sC) cudaStreamDestroy(sC);
        if (sG3) cudaStreamDestroy(sG3);
        if (sS) cudaStreamDestroy(sS);
    }
};

namespace {

// Chunking of the far history of block c over the points k < (c-1)L.
// Automatic split-k CTA target of the CUDA-core history kernels: more CTAs
// (warps to hide the FP64 latency) the more column groups of 4 there are.
// Measured with the autotuner (predicted full solves, ms for 152/304/608/1216
// CTAs): Lorenz 2^18 FP64, 3 columns: 499/381/419/710; 4 trajectories x 2^16,
// 12 columns: 117/103/108/122; 16 x 2^15, 48 columns: 115/114/109/99; Duffing
// 64 x 2^14, 128 columns: 106/106/94/83; LCR 256 x 2^13, 512 columns:
// 256/173/107/68.  FP64X2 (10 FP64 operations per term) is best at 608 for 3
// columns.
int auto_chunk_ctas(int hk, int64_t cols)
{
    if (hk == FABM_HIST_X2) return 152 * 4;
    const int64_t col_tiles = (cols + 3) / 4;
    return col_tiles <= 4 ? 152 * 2 : (col_tiles >= 8 ? 152 * 8 : 152 * 4);
}

void plan_chunks(int64_t k_end, int cols, int64_t max_chunks, int want_ctas, int *n_chunks,
                 int64_t *kc)
{
    const int col_tiles = (cols + 3) / 4;
    int64_t n = (want_ctas + col_tiles - 1) / col_tiles;
    const int64_t min_kc = 64;
    n = std::min<int64_t>(n, (k_end + min_kc - 1) / min_kc);
    n = std::min<int64_t>(n, max_chunks);
    n = std::max<int64_t>(n, 1);
    int64_t c = (k_end + n - 1) / n;
    c = (c + 7) / 8 * 8;  // near n chunks of equal size (one wave of want_ctas CTAs)
    *kc = c;
    *n_chunks = (int)((k_end + c - 1) / c);
}

fabm_status check_rhs(int rhs, int dim, int n_params)
{
    const int np = rhs_n_params(rhs);
    if (np < 0) return fail(FABM_EINVAL, "unknown rhs_id %d", rhs);
    if (!rhs_supports_dim(rhs, dim)) return fail(FABM_EINVAL, "rhs_id %d does not support dim %d", rhs, dim);
    if (n_params < np || n_params > kMaxParams)
        return fail(FABM_EINVAL, "rhs_id %d needs %d params (got %d, max %d)", rhs, np, n_params,
                    kMaxParams);
    return FABM_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Runs launch() on stream st; counts it, and with timing on brackets it with a
// pair of CUDA events on st (captured as event nodes when a graph is being
// recorded).
template <class Fn>
cudaError_t timed_launch(fabm_solver *s, int kind, cudaStream_t st, double flops, Fn &&launch)
{
    ++s->launches;
    if (!s->timing || !s->sample_now) return launch();
    const size_t pair = s->recs.size();
    while (s->ev_pool.size() < 2 * (pair + 1)) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        s->ev_pool.push_back(e);
    }
    const unsigned flags = s->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaError_t err = cudaEventRecordWithFlags(s->ev_pool[2 * pair], st, flags);
    if (err != cudaSuccess) return err;
    err = launch();
    if (err != cudaSuccess) return err;
    err = cudaEventRecordWithFlags(s->ev_pool[2 * pair + 1], st, flags);
    if (err != cudaSuccess) return err;
    s->recs.push_back({kind, flops});
    return cudaSuccess;
}

// After the streams are idle: add up the event pairs of the given records.
cudaError_t collect_timing(fabm_solver *s, const std::vector<fabm_solver::Rec> &recs)
{
    // per launch: duration, and start relative to the first timed launch, so
    // that the time during which launches of a kind ran (overlapping launches
    // counted once) can be formed as well
    std::vector<std::pair<double, double>> iv[FABM_KERNEL_KINDS];
    for (size_t i = 0; i < recs.size(); ++i) {
        float ms = 0.f, t0 = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, s->ev_pool[2 * i], s->ev_pool[2 * i + 1]);
        if (e == cudaSuccess && i > 0) e = cudaEventElapsedTime(&t0, s->ev_pool[0], s->ev_pool[2 * i]);
        if (e != cudaSuccess) return e;
        s->k_ms[recs[i].kind] += ms;
        s->k_launches[recs[i].kind] += 1;
        s->k_flops[recs[i].kind] += recs[i].flops;
        iv[recs[i].kind].push_back({(double)t0, (double)t0 + ms});
    }
    for (int k = 0; k < FABM_KERNEL_KINDS; ++k) {
        std::sort(iv[k].begin(), iv[k].end());
        double busy = 0.0, lo = 0.0, hi = -1.0;
        for (const auto &p : iv[k]) {
            if (p.first > hi) {
                if (hi > lo) busy += hi - lo;
                lo = p.first, hi = p.second;
            } else {
                hi = std::max(hi, p.second);
            }
        }
        if (hi > lo) busy += hi - lo;
        s->k_busy[k] += busy;
    }
    return cudaSuccess;
}

// History kernel for a batch of `cols` columns.
int resolve_hist_kernel(const fabm_solver *s, int64_t cols)
{
    if (s->precision == FABM_FP64) {
        // one persistent launch per solve on request (narrow single-order
        // batches): the recurrence CTAs take B SMs, the rest sum the history
        const int64_t B = cols / s->dim;
        const bool fits = !s->multi && s->persist_ctas >= B + 8 && B <= 64;
        if (s->hist_kernel == FABM_HIST_FP64_PERSIST) return fits ? FABM_HIST_FP64_PERSIST : FABM_HIST_FP64;
        return FABM_HIST_FP64;
    }
    if (s->precision == FABM_FP64X2) return FABM_HIST_X2;
    // one order per component: every column tile would need its own weight
    // operand, so the tensor kernel (one weight operand per tile) is not used
    if (s->multi) return FABM_HIST_FP32C;
    if (s->hist_kernel == FABM_HIST_TENSOR || s->hist_kernel == FABM_HIST_TENSOR_WIDE)
        return FABM_HIST_TENSOR;
    if (s->hist_kernel == FABM_HIST_FP32C) return s->hist_kernel;
    return cols >= 64 ? FABM_HIST_TENSOR : FABM_HIST_FP32C;
}

// Enqueues one solve on the solver's two streams (or records it into the
// graph being captured): init, then per block the far history on stream G and
// the recurrence (and, split path, the slicing of the finished segment) on
// stream R.
// Lag of the history launches: the history of block c covers the points
// k < (c - lag) L and the recurrence sums the lag blocks before c.  With lag 2
// (CUDA-core history kernels, long histories) the history of block c waits
// only for the recurrence of block c-3, and the launches of consecutive blocks,
// on two streams, overlap each other's tails and reductions; the tensor kernel
// uses lag 1 (a 64-point segment is sliced once its block is done).
// Lag 2 pays where the history bounds the solve: N x cols at least 2^19 for
// the FP64 kernel (its per-block work then exceeds the recurrence's ~30 us),
// 2^25 for the compensated-fp32 kernel (64x the FP64 rate).  Below that the
// extra lag block only lengthens the recurrence.
int history_lag(int hk, int64_t N, int64_t cols)
{
    if (hk == FABM_HIST_FP64 || hk == FABM_HIST_X2) return N * cols >= (1LL << 19) ? 2 : 1;
    if (hk == FABM_HIST_FP32C) return N * cols >= (1LL << 25) ? 2 : 1;
    return 1;
}

// Enqueues one solve on the solver's streams (or records it into the graph
// being captured): init, then per block the far history on sG / sG2 and the
// recurrence (and, tensor path, the newest segment's history and the slicing
// of the finished segment) on sR.
fabm_status enqueue_solve(fabm_solver *s, const DevBatch &bt, const DevWeights &w, int64_t nblk,
                          int64_t Nmax, int64_t max_chunks, int n_ct, int split_chunks, int hk,
                          int far_chunks)
{
    const int L = s->L;
    const int64_t cols = bt.cols;
    const bool split = hk == FABM_HIST_TENSOR;
    const int lag = history_lag(hk, s->plan_N > 0 ? s->plan_N : Nmax, cols);
    const int n_gbuf = lag + 1;  // G of block c is read by R(c) until H(c + lag + 1) starts
    s->sample_now = true;
    FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_INIT, s->sR, 0.0,
                               [&] { return launch_init(s->rhs, bt, s->sR, split); }));
    // tensor path with forcing: the tables of the time-only part of f, on sG2,
    // up to kAuxRing - 1 blocks ahead of the recurrence
    const bool tables = split && rhs_has_forcing(s->rhs, bt.dim);
    auto enqueue_aux = [&](int64_t c) -> fabm_status {
        float2 *X = s->auxb.p + (size_t)(c % kAuxRing) * kSplitSeg * bt.B;
        if (c >= kAuxRing) FABM_CUDA_TRY(cudaStreamWaitEvent(s->sG2, s->evR[(c - kAuxRing) % kEvRing], 0));
        FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_RECURRENCE, s->sG2, 0.0, [&] {
            return launch_aux_table(s->rhs, bt, s->h, c, X, s->sG2);
        }));
        FABM_CUDA_TRY(cudaEventRecord(s->evA[c % kAuxRing], s->sG2));
        return FABM_OK;
    };
    if (tables)
        for (int64_t c = 0; c < std::min<int64_t>(nblk, kAuxRing); ++c) {
            const fabm_status st = enqueue_aux(c);
            if (st != FABM_OK) return st;
        }
    for (int64_t c = 0; c < nblk; ++c) {
        // timed blocks; with two history streams, runs of 8 consecutive blocks,
        // so that the overlap of their history launches is measured
        const int64_t ph = c % s->timing_period;
        s->sample_now = ph == 0 || (lag == 2 && ph < 8);
        const void *Gc = nullptr;
        HistIn hin;  // tensor path: the history the recurrence starts from
        if (split && c >= 1 && s->wide) {
            // pairs of blocks: the far history of target group C = c/2 over
            // the point groups 0 .. C-2 (128 points each) on sG / sG3, started
            // once R(2C-3) has finished group C-2 and due by R(2C), so it runs
            // beside the recurrences of blocks 2C-2 and 2C-1, its chunks summed
            // on the same stream; the segments of 64 points from 2C-2 up to c-1
            // as a near launch on sR; the recurrence adds the two
            const int64_t C = c / 2;
            const int t = (int)(c % 2);
            const size_t fstride = far_part_elems(far_chunks, (int)cols);
            const size_t sstride = far_part_elems(1, (int)cols);
            if (C >= 2 && t == 0) {
                const int n_far = (int)std::min<int64_t>(far_chunks, C - 1);
                cudaStream_t fs = (C & 1) ? s->sG3 : s->sG;
                float2 *fw = s->fpart.p + (size_t)(C & 1) * fstride;
                float2 *fsw = s->fsum.p + (size_t)(C & 1) * sstride;
                const double flops = 4.0 * 128.0 * (double)((C - 1) * 128) * (double)cols;
                FABM_CUDA_TRY(cudaStreamWaitEvent(fs, s->evR[(c - 3) % kEvRing], 0));
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_SLICE, fs, 0.0, [&] {
                    return launch_slice_group(bt, n_ct, C - 2, s->Fs2.p, s->Fe2.p, fs);
                }));
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, fs, flops, [&] {
                    return launch_hist_far(s->Fs2.p, s->Fe2.p, s->wH2.p, s->wHe2.p, C,
                                           (int)(C - 1), n_far, n_ct, (int)cols, fw, s->err.p,
                                           s->wait_cycles, fs);
                }));
                FABM_CUDA_TRY(cudaEventRecord(s->evFK[C & 1], fs));
                FABM_CUDA_TRY(cudaStreamWaitEvent(s->sS, s->evFK[C & 1], 0));
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_COMBINE, s->sS, 0.0, [&] {
                    return launch_sum_far(fw, n_far, (int)cols, fsw, s->sS);
                }));
                FABM_CUDA_TRY(cudaEventRecord(s->evF[C & 1], s->sS));
            }
            const int64_t lo = std::max<int64_t>(0, 2 * C - 2);
            const int n_near = (int)(c - lo);
            const double nflops = 4.0 * L * (double)(n_near * L) * (double)cols;
            const int n_nc = std::min(n_near, s->near_chunks);
            FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, s->sR, nflops, [&] {
                return launch_hist_split(s->Fs.p, s->Fe.p, s->wH.p, s->wHe.p, c, (int)lo, n_near,
                                         0, n_nc, n_ct, (int)cols, s->spart.p, s->err.p,
                                         s->wait_cycles, s->sR);
            }));
            if (C >= 2) {
                FABM_CUDA_TRY(cudaStreamWaitEvent(s->sR, s->evF[C & 1], 0));
                hin.G = s->fsum.p + (size_t)(C & 1) * sstride;
                hin.g_rows = 128;
                hin.g_off = 64 * t;
            }
            hin.near = s->spart.p;
            hin.n_near = n_nc;
        } else if (split && c >= 1) {
            // far part (segments 0 .. c-2) on sG beside the recurrence of block
            // c-1; the newest segment c-1 on sR once it is sliced; the combine
            // on sG after both
            float2 *Gbuf = reinterpret_cast<float2 *>(s->G.p) + (size_t)(c % n_gbuf) * 2 * L * cols;
            const int n_far = (int)std::min<int64_t>(c - 1, split_chunks);
            if (n_far > 0) {
                const double flops = 4.0 * L * (double)((c - 1) * L) * (double)cols;
                FABM_CUDA_TRY(cudaStreamWaitEvent(s->sG, s->evR[(c - 2) % kEvRing], 0));
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, s->sG, flops, [&] {
                    return launch_hist_split(s->Fs.p, s->Fe.p, s->wH.p, s->wHe.p, c, 0, (int)(c - 1),
                                             0, n_far, n_ct, (int)cols, s->spart.p, s->err.p,
                                             s->wait_cycles, s->sG);
                }));
            }
            const double nflops = 4.0 * L * (double)L * (double)cols;
            FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, s->sR, nflops, [&] {
                return launch_hist_split(s->Fs.p, s->Fe.p, s->wH.p, s->wHe.p, c, (int)(c - 1), 1,
                                         n_far, 1, n_ct, (int)cols, s->spart.p, s->err.p,
                                         s->wait_cycles, s->sR);
            }));
            FABM_CUDA_TRY(cudaEventRecord(s->evN[c % 3], s->sR));
            FABM_CUDA_TRY(cudaStreamWaitEvent(s->sG, s->evN[c % 3], 0));
            FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_COMBINE, s->sG, 0.0, [&] {
                return launch_combine_split_ff(s->spart.p, n_far + 1, (int)cols, L, Gbuf, s->sG);
            }));
            FABM_CUDA_TRY(cudaEventRecord(s->evG[c % 3], s->sG));
            FABM_CUDA_TRY(cudaStreamWaitEvent(s->sR, s->evG[c % 3], 0));
            hin.G = Gbuf;
        } else if (!split && (c - lag) * L > 0) {
            const int64_t k_end = (c - lag) * L;
            double *Gbuf = s->G.p + (size_t)(c % n_gbuf) * 2 * L * cols;
            const bool two = lag == 2;  // alternate history streams
            cudaStream_t gs = (two && (c & 1)) ? s->sG2 : s->sG;
            const size_t poff = two ? (size_t)(c & 1) * max_chunks * 2 * L * cols : 0;
            int n_chunks;
            int64_t kc;
            // algorithmic work: 2 sums x L targets x k_end points x cols, 2 flops each
            const double flops = 4.0 * L * (double)k_end * (double)cols;
            FABM_CUDA_TRY(cudaStreamWaitEvent(gs, s->evR[(c - lag - 1) % kEvRing], 0));
            plan_chunks(k_end, (int)cols, max_chunks,
                        s->chunk_ctas > 0 ? s->chunk_ctas : auto_chunk_ctas(hk, cols), &n_chunks,
                        &kc);
            if (hk == FABM_HIST_X2) {
                double2 *xp = reinterpret_cast<double2 *>(s->part.p) + poff;
                const DevWeightsLo wl{s->wBl.p, s->wAl.p, s->wDl.p};
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, gs, flops, [&] {
                    return launch_hist_x2(bt, w, wl, c, lag, n_chunks, kc, xp, gs);
                }));
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_COMBINE, gs, 0.0, [&] {
                    return launch_reduce_x2(xp, n_chunks, (int)cols, Gbuf, gs);
                }));
            } else if (hk == FABM_HIST_FP32C) {
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, gs, flops, [&] {
                    return launch_hist_fp32c(bt, s->wBf.p, s->wAf.p, w.stride, c, lag, n_chunks,
                                             kc, s->spart.p + poff, gs);
                }));
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_COMBINE, gs, 0.0, [&] {
                    return launch_combine_split(s->spart.p + poff, n_chunks, (int)cols, L, Gbuf, gs);
                }));
            } else {
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, gs, flops, [&] {
                    return launch_hist_fp64(bt, w, c, L, lag, n_chunks, kc, s->part.p + poff, gs);
                }));
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_COMBINE, gs, 0.0, [&] {
                    return launch_hist_reduce(s->part.p + poff, n_chunks, L, (int)cols, Gbuf, gs);
                }));
            }
            FABM_CUDA_TRY(cudaEventRecord(s->evG[c % 3], gs));
            FABM_CUDA_TRY(cudaStreamWaitEvent(s->sR, s->evG[c % 3], 0));
            Gc = Gbuf;
        }
        // lag blocks (CUDA-core paths) and the in-block triangle: per target up
        // to (rlag + 1) L points
        const int rlag = split ? 0 : lag;
        const int64_t lo = c * L, hi = std::min<int64_t>((c + 1) * L, Nmax);
        const double rflops = 4.0 * (double)cols * (double)(hi - lo) *
                              ((double)std::min<int64_t>(c, rlag) * L + 0.5 * (double)(hi - lo + 1));
        const float2 *X = nullptr;
        if (tables) {
            X = s->auxb.p + (size_t)(c % kAuxRing) * kSplitSeg * bt.B;
            FABM_CUDA_TRY(cudaStreamWaitEvent(s->sR, s->evA[c % kAuxRing], 0));
        }
        FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_RECURRENCE, s->sR, rflops, [&] {
            if (split)
                return launch_recur_cols(s->rhs, bt, s->wBff.p, s->wAff.p, s->wDff.p, s->k, c, hin,
                                         X, s->cols_warps, s->sR);
            return launch_recur(s->rhs, bt, w, s->k, c, L, lag, s->precision == FABM_SPLIT,
                                static_cast<const double *>(Gc), s->sR);
        }));
        if (split && c + 1 < nblk) {  // segment c is read by the blocks c+1 ..
            FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_SLICE, s->sR, 0.0, [&] {
                return launch_slice_f(bt, n_ct, c, s->Fs.p, s->Fe.p, s->sR);
            }));
        }
        FABM_CUDA_TRY(cudaEventRecord(s->evR[c % kEvRing], s->sR));
        if (s->out_stream && ((c + 1) % s->out_group == 0 || c + 1 == nblk)) {
            // rows of the blocks c0 .. c are final: (tensor path: to double, then)
            // to the host, beside the next blocks
            const int64_t c0 = c / s->out_group * s->out_group;
            const int64_t r_lo = c0 == 0 ? 0 : c0 * L + 1, r_hi = std::min<int64_t>((c + 1) * L, bt.N);
            FABM_CUDA_TRY(cudaStreamWaitEvent(s->sC, s->evR[c % kEvRing], 0));
            if (split)
                FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_SLICE, s->sC, 0.0, [&] {
                    return launch_finish_y(bt, s->h, std::max<int64_t>(r_lo, 1), r_hi, s->sC);
                }));
            const size_t pitch = sizeof(double) * (size_t)(bt.N + 1) * bt.dim;
            FABM_CUDA_TRY(cudaMemcpy2DAsync(s->out_stream + r_lo * bt.dim, pitch, bt.Y + r_lo * bt.dim,
                                            pitch, sizeof(double) * (size_t)(r_hi - r_lo + 1) * bt.dim,
                                            (size_t)bt.B, cudaMemcpyDeviceToHost, s->sC));
        }
        if (tables && c + kAuxRing < nblk) {
            const fabm_status st = enqueue_aux(c + kAuxRing);
            if (st != FABM_OK) return st;
        }
    }
    s->sample_now = true;
    if (split && !s->out_stream)  // y = Taylor part + the float-float increments, in double
        FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_SLICE, s->sR, 0.0,
                                   [&] { return launch_finish_y(bt, s->h, 1, bt.N, s->sR); }));
    return FABM_OK;
}

fabm_status run_batch(fabm_solver *s, int64_t B, const double *y0, const double *y1,
                      const double *traj_params, const int64_t *N_each, double *out,
                      int out_on_device)
{
    const int dim = s->dim;
    const int64_t cols = B * dim;
    const int64_t N = s->N;
    const int hk = resolve_hist_kernel(s, cols);
    const int L = hk == FABM_HIST_TENSOR ? kSplitSeg : kRecurL;
    s->last_hk = hk;
    s->L = L;
    s->launches = 0;

    // host-side inputs: per-trajectory steps and parameter rows
    std::vector<int64_t> ne(B);
    int64_t Nmax = 0;
    bool all_full = true;
    for (int64_t b = 0; b < B; ++b) {
        ne[b] = N_each ? N_each[b] : N;
        if (ne[b] < 1 || ne[b] > N)
            return fail(FABM_EINVAL, "N_each[%lld] = %lld outside 1..N=%lld", (long long)b,
                        (long long)ne[b], (long long)N);
        Nmax = std::max(Nmax, ne[b]);
        all_full = all_full && ne[b] == N;
    }
    std::vector<double> par((size_t)B * kMaxParams, 0.0);
    for (int64_t b = 0; b < B; ++b)
        for (int i = 0; i < s->n_params; ++i)
            par[b * kMaxParams + i] = traj_params ? traj_params[b * s->n_params + i] : s->params[i];
    for (int64_t i = 0; i < B * dim; ++i)
        if (!std::isfinite(y0[i]) || (y1 && !std::isfinite(y1[i])))
            return fail(FABM_EINVAL, "y0[%lld] or y1[%lld] is not finite", (long long)i, (long long)i);

    const bool split = hk == FABM_HIST_TENSOR;
    // workspace
    const int64_t nblk = (Nmax + L - 1) / L;
    const size_t f_elems = (size_t)(N + 1) * cols;
    const int64_t part_per_chunk = 2LL * L * cols;
    int64_t max_chunks = std::max<int64_t>(1, (int64_t)(64ull << 20) / (part_per_chunk * 8));
    max_chunks = std::min<int64_t>(max_chunks, 4096);
    FABM_CUDA_TRY(s->F.ensure(f_elems));
    FABM_CUDA_TRY(s->G.ensure((size_t)3 * 2 * L * cols));
    // two partial buffers: the history launches of blocks c and c+1 may overlap
    if (hk == FABM_HIST_FP64) FABM_CUDA_TRY(s->part.ensure((size_t)2 * max_chunks * part_per_chunk));
    if (hk == FABM_HIST_X2) FABM_CUDA_TRY(s->part.ensure((size_t)4 * max_chunks * part_per_chunk));
    if (hk == FABM_HIST_FP32C) {
        FABM_CUDA_TRY(s->spart.ensure((size_t)2 * max_chunks * part_per_chunk));
        FABM_CUDA_TRY(s->Ff.ensure(f_elems));
    }
    FABM_CUDA_TRY(s->y0.ensure((size_t)B * dim * 2));  // y0, then y1
    FABM_CUDA_TRY(s->par.ensure((size_t)B * kMaxParams));
    FABM_CUDA_TRY(s->nEach.ensure((size_t)B));
    FABM_CUDA_TRY(s->status.ensure(1));
    const int n_ct = (int)((cols + 127) / 128);
    int split_chunks = 1, far_chunks = 1;
    s->wide = false;
    if (split) {
        // recurrence layout: one lane per column for wide batches, and where
        // the history dominates (its SMs matter more than the recurrence's
        // latency); one lane per target for short, narrow runs (more
        // parallelism, more instructions)
        const int cwarps = recur_cols_warps(dim, B);
        const bool columns =
            s->rec_layout == FABM_REC_COLUMNS ||
            (s->rec_layout == FABM_REC_AUTO &&
             (cwarps >= 96 || (double)(s->plan_N > 0 ? s->plan_N : Nmax) * cols >= 0x1p28));
        // leave SMs for the recurrence that runs beside the tensor kernel (one
        // tensor CTA fills an SM's register file), only where the column tiles
        // do not need every SM: one SM per 8 column warps, or per 12
        // trajectories of the lane-per-target layout up to 16 SMs (LCR 1024 x
        // 2^14: reserves of 40, 16 and 0 SMs predicted 25.3, 23.5, 23.1 ms)
        int reserve = s->sm_reserve;
        if (reserve < 0) {
            const int64_t want = columns ? std::clamp<int64_t>((cwarps + 7) / 8, 4, 40)
                                         : std::min<int64_t>((B + 11) / 12, 16);
            reserve = n_ct <= 16 ? (int)want : 0;
        }
        split_chunks = std::max(1, (148 - reserve) / n_ct);
        // far history with 128 targets per MMA (pairs of blocks): requested,
        // or automatic where the far history is large enough to pay for its
        // extra launches: N^2 x columns >= 2^40 (measured: the 64-target
        // tiling is faster up to 2^39, e.g. LCR 1024 x 2^14 25.4 vs 27.0 ms;
        // the wide one from 2^41, Duffing 1024 x 2^15 57.6 vs 71.2 ms)
        const double nplan = (double)(s->plan_N > 0 ? s->plan_N : Nmax);
        s->wide = s->G_max >= 2 &&
                  (s->hist_kernel == FABM_HIST_TENSOR_WIDE ||
                   (s->hist_kernel == FABM_HIST_AUTO && nplan * nplan * (double)cols >= 0x1p40));
        far_chunks = std::max(1, (148 - reserve) / (2 * n_ct));
        if (s->wide) s->last_hk = FABM_HIST_TENSOR_WIDE;
        // a near launch (on the serial chain) takes whole SMs: as many CTAs per
        // column tile as the SMs the far kernel leaves free allow, so that it
        // does not wait for far CTAs to retire (one CTA sums its segments in turn)
        const int far_free = 152 - 2 * n_ct * far_chunks;
        s->near_chunks = std::clamp(far_free / n_ct, 1, 3);
        // column layout: CTAs sized to fill the SMs the tensor CTAs leave free,
        // at most 4 warps each, so that a CTA fits beside others on an SM that
        // is partly free (Duffing 4096 x 2^16: 4 warps 323 ms, 11 warps 340)
        const int free_sms = std::max(4, 152 - n_ct * split_chunks);
        s->cols_warps = !columns        ? 0
                        : s->rec_warps > 0 ? s->rec_warps
                                           : std::clamp((cwarps + free_sms - 1) / free_sms, 1, 4);
        FABM_CUDA_TRY(s->Fs.ensure((size_t)nblk * n_ct * 3 * 128 * 64));
        FABM_CUDA_TRY(s->Fe.ensure((size_t)nblk * n_ct * 128));
        // far chunks and one chunk for the newest segment; with the wide far
        // history, up to three near segments
        FABM_CUDA_TRY(s->spart.ensure(split_part_elems(std::max(split_chunks + 1, 3), (int)cols)));
        if (s->wide) {
            const int64_t n_grp = (N + 127) / 128;
            FABM_CUDA_TRY(s->Fs2.ensure((size_t)n_grp * n_ct * far_group_slice_elems()));
            FABM_CUDA_TRY(s->Fe2.ensure((size_t)n_grp * n_ct * 128));
            FABM_CUDA_TRY(s->fpart.ensure(2 * far_part_elems(far_chunks, (int)cols)));
            FABM_CUDA_TRY(s->fsum.ensure(2 * far_part_elems(1, (int)cols)));
        }
        if (rhs_has_forcing(s->rhs, dim))
            FABM_CUDA_TRY(s->auxb.ensure((size_t)kAuxRing * kSplitSeg * B));
        FABM_CUDA_TRY(s->err.ensure(1));
        FABM_CUDA_TRY(cudaMemsetAsync(s->err.p, 0, sizeof(unsigned int), s->sR));
    }
    double *Y = out;
    if (!out_on_device) {
        FABM_CUDA_TRY(s->Ystage.ensure((size_t)B * (N + 1) * dim));
        Y = s->Ystage.p;
    }
    // a large output into pinned host memory, every trajectory to N: copied
    // block group by block group on sC while the solve goes on (a group is at
    // least 8 MB), instead of once at the end
    s->out_stream = nullptr;
    const size_t out_bytes = sizeof(double) * (size_t)B * (N + 1) * dim;
    if (!out_on_device && all_full && out_bytes >= (64u << 20) && hk != FABM_HIST_FP64_PERSIST) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost) {
            s->out_stream = out;
            const size_t block_bytes = sizeof(double) * (size_t)B * L * dim;
            s->out_group = (int64_t)std::max<size_t>(1, ((8u << 20) + block_bytes - 1) / block_bytes);
        }
        cudaGetLastError();  // an unregistered pointer is not an error here
    }
    FABM_CUDA_TRY(cudaMemcpyAsync(s->y0.p, y0, sizeof(double) * B * dim, cudaMemcpyHostToDevice, s->sR));
    // y'(0) (1 < alpha < 2): zeros when not given, so that one cached graph
    // serves solves with and without it
    std::vector<double> y1m;
    if (y1 && s->multi) {  // components of order <= 1 have no y'(0) term
        y1m.assign(y1, y1 + B * dim);
        for (int64_t i = 0; i < B * dim; ++i)
            if (s->alpha_c[i % dim] <= 1.0) y1m[i] = 0.0;
        y1 = y1m.data();
    }
    if (y1)
        FABM_CUDA_TRY(cudaMemcpyAsync(s->y0.p + B * dim, y1, sizeof(double) * B * dim,
                                      cudaMemcpyHostToDevice, s->sR));
    else
        FABM_CUDA_TRY(cudaMemsetAsync(s->y0.p + B * dim, 0, sizeof(double) * B * dim, s->sR));
    FABM_CUDA_TRY(cudaMemcpyAsync(s->par.p, par.data(), sizeof(double) * par.size(),
                                  cudaMemcpyHostToDevice, s->sR));
    FABM_CUDA_TRY(cudaMemcpyAsync(s->nEach.p, ne.data(), sizeof(int64_t) * B,
                                  cudaMemcpyHostToDevice, s->sR));
    FABM_CUDA_TRY(cudaMemsetAsync(s->status.p, 0xff, sizeof(unsigned long long), s->sR));

    DevBatch bt{};
    bt.dim = dim;
    bt.B = (int)B;
    bt.cols = (int)cols;
    bt.N = N;
    bt.N_each = s->nEach.p;
    bt.y0 = s->y0.p;
    bt.y1 = s->alpha > 1.0 ? s->y0.p + B * dim : nullptr;
    bt.params = s->par.p;
    bt.F = s->F.p;
    bt.Ff = hk == FABM_HIST_FP32C ? s->Ff.p : nullptr;
    bt.ldF = cols;
    bt.Y = Y;
    bt.status = s->status.p;
    DevWeights w{s->wB.p, s->wA.p, s->wD.p, s->w_ext, s->multi ? s->w_ext + 1 : 0};

    const std::vector<uintptr_t> key = {
        (uintptr_t)B, (uintptr_t)nblk, (uintptr_t)L, (uintptr_t)s->timing,
        (uintptr_t)s->timing_period, (uintptr_t)hk, (uintptr_t)s->chunk_ctas,
        (uintptr_t)(s->sm_reserve + 1), (uintptr_t)s->cols_warps, (uintptr_t)Y,
        (uintptr_t)s->F.p, (uintptr_t)s->Ff.p, (uintptr_t)s->G.p, (uintptr_t)s->part.p, (uintptr_t)s->Fs.p,
        (uintptr_t)s->Fe.p, (uintptr_t)s->spart.p, (uintptr_t)s->y0.p, (uintptr_t)s->par.p,
        (uintptr_t)s->nEach.p, (uintptr_t)s->status.p, (uintptr_t)s->err.p, (uintptr_t)s->auxb.p,
        (uintptr_t)s->out_stream, (uintptr_t)s->out_group, (uintptr_t)s->wait_cycles,
        (uintptr_t)s->wide, (uintptr_t)far_chunks, (uintptr_t)s->Fs2.p, (uintptr_t)s->Fe2.p,
        (uintptr_t)s->fpart.p, (uintptr_t)s->fsum.p, (uintptr_t)s->near_chunks,
        (uintptr_t)s->plan_N};
    auto enqueue = [&]() -> fabm_status {
        return enqueue_solve(s, bt, w, nblk, Nmax, max_chunks, n_ct, split_chunks, hk, far_chunks);
    };
    if (hk == FABM_HIST_FP64_PERSIST) {
        // one cooperative launch runs every block (after the initial values);
        // its flags start at zero
        const int grid = s->persist_ctas;
        const int pchunks = persist_workers(grid, (int)B);
        const int ncg = (int)((cols + 3) / 4);
        const size_t n_sg = (size_t)nblk * ncg * persist_max_sg(pchunks);
        FABM_CUDA_TRY(s->ppart.ensure(persist_part_elems(pchunks, (int)cols)));
        FABM_CUDA_TRY(s->pspart.ensure(persist_spart_elems(pchunks, (int)cols)));
        FABM_CUDA_TRY(s->psg.ensure(n_sg));
        FABM_CUDA_TRY(s->pdone.ensure((size_t)nblk * ncg));
        FABM_CUDA_TRY(s->prdone.ensure((size_t)B));
        FABM_CUDA_TRY(s->err.ensure(1));
        s->recs.clear();
        FABM_CUDA_TRY(cudaMemsetAsync(s->psg.p, 0, sizeof(int) * n_sg, s->sR));
        FABM_CUDA_TRY(cudaMemsetAsync(s->pdone.p, 0, sizeof(int) * nblk * ncg, s->sR));
        FABM_CUDA_TRY(cudaMemsetAsync(s->prdone.p, 0, sizeof(int) * B, s->sR));
        FABM_CUDA_TRY(cudaMemsetAsync(s->err.p, 0, sizeof(unsigned int), s->sR));
        s->sample_now = true;
        FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_INIT, s->sR, 0.0,
                                   [&] { return launch_init(s->rhs, bt, s->sR); }));
        const double flops = 2.0 * (double)Nmax * (double)Nmax * (double)cols;
        FABM_CUDA_TRY(timed_launch(s, FABM_KERNEL_HISTORY, s->sR, flops, [&] {
            return launch_persist_fp64(s->rhs, bt, w, s->k, nblk, grid, pchunks, s->ppart.p,
                                       s->pspart.p, s->psg.p, s->pdone.p, s->prdone.p, s->err.p,
                                       s->wait_cycles, s->sR);
        }));
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sR));
        FABM_CUDA_TRY(collect_timing(s, s->recs));
        unsigned int tout = 0;
        FABM_CUDA_TRY(cudaMemcpy(&tout, s->err.p, sizeof tout, cudaMemcpyDeviceToHost));
        if (tout) return fail(FABM_ETIMEOUT, "the persistent solve gave up waiting on a flag");
    } else if (!s->use_graphs) {
        s->recs.clear();
        // the side streams start after this solve's inputs are on the device
        FABM_CUDA_TRY(cudaEventRecord(s->evFork, s->sR));
        FABM_CUDA_TRY(cudaStreamWaitEvent(s->sG, s->evFork, 0));
        FABM_CUDA_TRY(cudaStreamWaitEvent(s->sG2, s->evFork, 0));
        FABM_CUDA_TRY(cudaStreamWaitEvent(s->sC, s->evFork, 0));
        FABM_CUDA_TRY(cudaStreamWaitEvent(s->sG3, s->evFork, 0));
        FABM_CUDA_TRY(cudaStreamWaitEvent(s->sS, s->evFork, 0));
        fabm_status est = enqueue();
        if (est != FABM_OK) return est;
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sG3));
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sS));
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sR));
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sG));
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sG2));
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sC));
        FABM_CUDA_TRY(collect_timing(s, s->recs));
    } else {
        if (!s->gexec || s->gkey != key) {
            if (s->gexec) cudaGraphExecDestroy(s->gexec);
            s->gexec = nullptr;
            s->recs.clear();
            cudaGraph_t graph = nullptr;
            FABM_CUDA_TRY(cudaStreamBeginCapture(s->sR, cudaStreamCaptureModeThreadLocal));
            s->capturing = true;
            cudaError_t e = cudaEventRecord(s->evFork, s->sR);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sG, s->evFork, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sG2, s->evFork, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sC, s->evFork, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sG3, s->evFork, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sS, s->evFork, 0);
            fabm_status est = e == cudaSuccess ? enqueue() : FABM_ECUDA;
            if (est == FABM_OK) {
                e = cudaEventRecord(s->evFork, s->sG);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sR, s->evFork, 0);
                if (e == cudaSuccess) e = cudaEventRecord(s->evJoin, s->sG2);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sR, s->evJoin, 0);
                if (e == cudaSuccess) e = cudaEventRecord(s->evJoinC, s->sC);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sR, s->evJoinC, 0);
                if (e == cudaSuccess) e = cudaEventRecord(s->evJoin3, s->sG3);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sR, s->evJoin3, 0);
                if (e == cudaSuccess) e = cudaEventRecord(s->evJoinS, s->sS);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s->sR, s->evJoinS, 0);
            }
            cudaError_t e2 = cudaStreamEndCapture(s->sR, &graph);
            s->capturing = false;
            if (est != FABM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return est;
            }
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&s->gexec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                s->gexec = nullptr;
                return fail(FABM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
            }
            s->gkey = key;
            s->grecs = s->recs;
            s->glaunches = s->launches;
        }
        FABM_CUDA_TRY(cudaGraphLaunch(s->gexec, s->sR));
        FABM_CUDA_TRY(cudaStreamSynchronize(s->sR));
        s->launches = s->glaunches;
        FABM_CUDA_TRY(collect_timing(s, s->grecs));
    }


    unsigned long long st = 0;
    FABM_CUDA_TRY(cudaMemcpy(&st, s->status.p, sizeof st, cudaMemcpyDeviceToHost));
    if (split) {  // tensor kernel's bounded waits
        unsigned int tout = 0;
        FABM_CUDA_TRY(cudaMemcpy(&tout, s->err.p, sizeof tout, cudaMemcpyDeviceToHost));
        if (tout) return fail(FABM_ETIMEOUT, "a history kernel gave up waiting on a barrier");
    }

    if (!out_on_device && !s->out_stream) {
        const size_t row = (size_t)(N + 1) * dim;
        if (all_full) {
            FABM_CUDA_TRY(cudaMemcpy(out, Y, sizeof(double) * row * B, cudaMemcpyDeviceToHost));
        } else {
            // copy only the rows each trajectory owns; runs of full-length
            // trajectories go in one copy
            int64_t b = 0;
            while (b < B) {
                if (ne[b] == N) {
                    int64_t e = b;
                    while (e < B && ne[e] == N) ++e;
                    FABM_CUDA_TRY(cudaMemcpy(out + b * row, Y + b * row,
                                             sizeof(double) * row * (e - b),
                                             cudaMemcpyDeviceToHost));
                    b = e;
                } else {
                    FABM_CUDA_TRY(cudaMemcpy(out + b * row, Y + b * row,
                                             sizeof(double) * (ne[b] + 1) * dim,
                                             cudaMemcpyDeviceToHost));
                    ++b;
                }
            }
        }
    }
    if (st != ~0ull)
        return fail(FABM_ENONFINITE, "non-finite value at trajectory %llu, step %llu",
                    st & 0xffffffull, st >> 24);
    return FABM_OK;
}

}  // namespace

extern "C" {

const char *fabm_last_error(void) { return g_last_error.c_str(); }

namespace {

fabm_status create_solver(int dim, const double *alpha_c, double h, int64_t N, int rhs_id,
                          const double *params, int n_params, int precision, fabm_solver **out)
{
    g_last_error.clear();
    if (!out) return fail(FABM_EINVAL, "out is NULL");
    *out = nullptr;
    if (dim < 1 || dim > FABM_MAX_DIM) return fail(FABM_EINVAL, "dim %d outside 1..%d", dim, FABM_MAX_DIM);
    if (!alpha_c) return fail(FABM_EINVAL, "alpha is NULL");
    double alpha = 0.0;
    bool multi = false;
    for (int i = 0; i < dim; ++i) {
        if (!(alpha_c[i] > 0.0 && alpha_c[i] < 2.0))
            return fail(FABM_EINVAL, "alpha %g outside (0, 2)", alpha_c[i]);
        alpha = std::max(alpha, alpha_c[i]);
        multi = multi || alpha_c[i] != alpha_c[0];
    }
    if (!(h > 0.0) || !std::isfinite(h)) return fail(FABM_EINVAL, "h %g must be positive", h);
    if (N < 1 || N > (1LL << 31)) return fail(FABM_EINVAL, "N %lld outside 1..2^31", (long long)N);
    if (precision != FABM_FP64 && precision != FABM_SPLIT && precision != FABM_FP64X2)
        return fail(FABM_EINVAL, "precision %d unknown", precision);
    fabm_status st = check_rhs(rhs_id, dim, n_params);
    if (st != FABM_OK) return st;
    if (n_params > 0 && !params) return fail(FABM_EINVAL, "params is NULL");
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) return fail(FABM_EINVAL, "params[%d] is not finite", i);

    fabm_solver *s = new (std::nothrow) fabm_solver();
    if (!s) return fail(FABM_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return fail(FABM_ECUDA, "no CUDA device");
    }
    s->dim = dim, s->alpha = alpha, s->h = h, s->N = N, s->rhs = rhs_id;
    s->n_params = n_params, s->precision = precision, s->multi = multi;
    for (int i = 0; i < n_params; ++i) s->params[i] = params[i];
    s->k.h = h;
    for (int q = 0; q < FABM_MAX_DIM; ++q) {
        const double a = alpha_c[q < dim ? q : 0];
        if (q < dim) s->alpha_c[q] = a;
        s->k.h_alpha[q] = std::pow(h, a);
        s->k.inv_gamma2[q] = 1.0 / std::tgamma(a + 2.0);
    }
    const int n_sets = multi ? dim : 1;  // weight sets

    auto cleanup = [&](fabm_status e) {
        delete s;
        return e;
    };
    // weights for every distance a history kernel can ask for: block padding
    // beyond N plus the lag-1 window
    s->w_ext = (N + kMaxBlockL - 1) / kMaxBlockL * kMaxBlockL + 2 * kMaxBlockL;
    cudaError_t e = cudaSuccess;
    const size_t wlen = (size_t)n_sets * (s->w_ext + 1);
    if (e == cudaSuccess) e = s->wB.ensure(wlen);
    if (e == cudaSuccess) e = s->wA.ensure(wlen);
    if (e == cudaSuccess) e = s->wD.ensure(wlen);
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    // the recurrence is the serial chain: its CTAs are scheduled first
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->sR, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->sG, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->sG2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->sC, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->sG3, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->sS, cudaStreamNonBlocking, prio_hi);
    for (auto &ev : s->evF)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (auto &ev : s->evFK)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->evJoinS, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->evJoin3, cudaEventDisableTiming);
    for (auto &ev : s->evR)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (auto &ev : s->evG)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (auto &ev : s->evN)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (auto &ev : s->evA)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->evFork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->evJoin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->evJoinC, cudaEventDisableTiming);
    if (e == cudaSuccess && precision == FABM_FP64X2) {
        // double-double weights on the device (weights_dd.cu): high parts into
        // wB, wA, wD, low parts into wBl, wAl, wDl
        e = s->wBl.ensure(wlen);
        if (e == cudaSuccess) e = s->wAl.ensure(wlen);
        if (e == cudaSuccess) e = s->wDl.ensure(wlen);
        s->timing = true;  // the weight launch is always timed
        s->recs.clear();
        for (int q = 0; q < n_sets && e == cudaSuccess; ++q) {
            const size_t o = (size_t)q * (s->w_ext + 1);
            double g[4];
            fabm_x2_inv_gammas(alpha_c[q], g);
            e = timed_launch(s, FABM_KERNEL_WEIGHTS, s->sR, 0.0, [&] {
                return launch_weights_x2(alpha_c[q], s->w_ext, g[0], g[1], g[2], g[3], s->wB.p + o,
                                         s->wBl.p + o, s->wA.p + o, s->wAl.p + o, s->wD.p + o,
                                         s->wDl.p + o, s->sR);
            });
        }
        s->timing = false;
    } else if (e == cudaSuccess) {
        s->timing = true;  // the weight launch is always timed
        s->recs.clear();
        for (int q = 0; q < n_sets && e == cudaSuccess; ++q) {
            const size_t o = (size_t)q * (s->w_ext + 1);
            const double a = alpha_c[q];
            e = timed_launch(s, FABM_KERNEL_WEIGHTS, s->sR, 0.0, [&] {
                return launch_weights(a, s->w_ext, 1.0 / std::tgamma(a + 1.0),
                                      s->k.inv_gamma2[q], s->wB.p + o, s->wA.p + o, s->wD.p + o,
                                      s->sR);
            });
        }
        s->timing = false;
    }
    if (e == cudaSuccess && precision == FABM_SPLIT) {
        s->L = kSplitSeg;
        e = s->wBf.ensure(wlen);
        if (e == cudaSuccess) e = s->wAf.ensure(wlen);
        if (e == cudaSuccess) e = launch_to_float(s->wB.p, (int64_t)wlen, s->wBf.p, s->sR);
        if (e == cudaSuccess) e = launch_to_float(s->wA.p, (int64_t)wlen, s->wAf.p, s->sR);
        if (e == cudaSuccess) e = prepare_hist_split();
        s->g_max = multi ? 0 : (N + kSplitSeg - 1) / kSplitSeg - 1;  // no tensor tiles when multi
        if (e == cudaSuccess && s->g_max >= 1) {
            e = s->wH.ensure((size_t)(s->g_max + 1) * 2 * 3 * 15 * 64);
            if (e == cudaSuccess) e = s->wHe.ensure((size_t)(s->g_max + 1) * 2);
            if (e == cudaSuccess)
                e = launch_hankel_weights(s->wB.p, s->wA.p, s->g_max, s->wH.p, s->wHe.p, s->sR);
        }
        // wide far history: 128-point groups, lags 2 .. G_max
        s->G_max = multi ? 0 : (N + 127) / 128 - 1;
        if (e == cudaSuccess && s->G_max >= 2) {
            e = prepare_hist_far();
            if (e == cudaSuccess) e = s->wH2.ensure((size_t)(s->G_max + 1) * far_group_tile_elems());
            if (e == cudaSuccess) e = s->wHe2.ensure((size_t)(s->G_max + 1) * 2);
            if (e == cudaSuccess)
                e = launch_hankel_group(s->wB.p, s->wA.p, s->G_max, s->wH2.p, s->wHe2.p, s->sR);
        }
        if (e == cudaSuccess && !multi) {
            const double ha = s->k.h_alpha[0];
            e = prepare_recur_cols(rhs_id, dim);
            if (e == cudaSuccess) e = s->wBff.ensure(kSplitSeg + 1);
            if (e == cudaSuccess) e = s->wAff.ensure(kSplitSeg + 1);
            if (e == cudaSuccess) e = s->wDff.ensure((size_t)s->w_ext + 1);
            if (e == cudaSuccess) e = launch_ff_weights(s->wB.p, ha, kSplitSeg + 1, s->wBff.p, s->sR);
            if (e == cudaSuccess) e = launch_ff_weights(s->wA.p, ha, kSplitSeg + 1, s->wAff.p, s->sR);
            if (e == cudaSuccess) e = launch_ff_weights(s->wD.p, ha, s->w_ext + 1, s->wDff.p, s->sR);
        }
    }
    if (e == cudaSuccess && precision == FABM_FP64 && !multi) {
        int coop = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device) == cudaSuccess && coop)
            s->persist_ctas = std::min(persist_max_ctas(rhs_id, dim), 152);
        cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->sR);
    if (e == cudaSuccess) e = collect_timing(s, s->recs);
    s->recs.clear();
    if (e != cudaSuccess)
        return cleanup(fail(e == cudaErrorMemoryAllocation ? FABM_ENOMEM : FABM_ECUDA,
                            "fabm_create: %s", cudaGetErrorString(e)));
    *out = s;
    return FABM_OK;
}

}  // namespace

fabm_status fabm_create(int dim, double alpha, double h, int64_t N, int rhs_id,
                        const double *params, int n_params, int precision, fabm_solver **out)
{
    TraceRange tr("fabm_create");
    double a[FABM_MAX_DIM] = {alpha, alpha, alpha, alpha};
    return create_solver(dim, a, h, N, rhs_id, params, n_params, precision, out);
}

fabm_status fabm_create_multi(int dim, const double *alpha, double h, int64_t N, int rhs_id,
                              const double *params, int n_params, int precision,
                              fabm_solver **out)
{
    TraceRange tr("fabm_create_multi");
    return create_solver(dim, alpha, h, N, rhs_id, params, n_params, precision, out);
}

fabm_status fabm_solve_batch(fabm_solver *s, int64_t B, const double *y0, const double *traj_params,
                             const int64_t *N_each, double *out, int out_on_device)
{
    return fabm_solve_batch_ic(s, B, y0, nullptr, traj_params, N_each, out, out_on_device);
}

fabm_status fabm_solve_batch_ic(fabm_solver *s, int64_t B, const double *y0, const double *y1,
                                const double *traj_params, const int64_t *N_each, double *out,
                                int out_on_device)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (y1 && s->alpha <= 1.0)
        return fail(FABM_EINVAL, "y1 given for alpha %g <= 1 (its Taylor part is y0 alone)", s->alpha);
    if (B < 0 || B > (1LL << 24)) return fail(FABM_EINVAL, "B %lld outside 0..2^24", (long long)B);
    if (B == 0) return FABM_OK;
    if (!y0 || !out) return fail(FABM_EINVAL, "y0 and out must not be NULL");
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    if (traj_params)
        for (int64_t i = 0; i < B * s->n_params; ++i)
            if (!std::isfinite(traj_params[i]))
                return fail(FABM_EINVAL, "traj_params[%lld] is not finite", (long long)i);
    DeviceGuard g(s->device);
    TraceRange tr("fabm_solve_batch");
    return run_batch(s, B, y0, y1, traj_params, N_each, out, out_on_device);
}

fabm_status fabm_solve(fabm_solver *s, const double *y0, double *out)
{
    return fabm_solve_batch(s, 1, y0, nullptr, nullptr, out, 0);
}

fabm_status fabm_destroy(fabm_solver *s)
{
    g_last_error.clear();
    if (!s) return FABM_OK;
    {
        std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
        if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    }
    DeviceGuard g(s->device);
    delete s;
    return FABM_OK;
}

fabm_status fabm_set_block(fabm_solver *s, int L)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    int hk;
    if (L == kSplitSeg && s->precision == FABM_SPLIT)
        hk = FABM_HIST_TENSOR;
    else if (L == kRecurL)
        hk = s->precision == FABM_SPLIT ? FABM_HIST_FP32C
                                        : (s->precision == FABM_FP64X2 ? FABM_HIST_X2 : FABM_HIST_FP64);
    else
        return fail(FABM_EINVAL,
                    "block length %d: 32 (fp64 or fp32c history) or 64 (tensor history, split "
                    "precision) are available",
                    L);
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    s->hist_kernel = hk;
    s->L = L;
    return FABM_OK;
}

fabm_status fabm_set_history_kernel(fabm_solver *s, int kernel)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    const bool ok = kernel == FABM_HIST_AUTO ||
                    (s->precision == FABM_FP64 &&
                     (kernel == FABM_HIST_FP64 || kernel == FABM_HIST_FP64_PERSIST)) ||
                    (s->precision == FABM_FP64X2 && kernel == FABM_HIST_X2) ||
                    (s->precision == FABM_SPLIT &&
                     (kernel == FABM_HIST_TENSOR || kernel == FABM_HIST_TENSOR_WIDE ||
                      kernel == FABM_HIST_FP32C));
    if (!ok) return fail(FABM_EINVAL, "history kernel %d does not fit precision %d", kernel, s->precision);
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    s->hist_kernel = kernel;
    s->L = (kernel == FABM_HIST_TENSOR || kernel == FABM_HIST_TENSOR_WIDE ||
            (kernel == FABM_HIST_AUTO && s->precision == FABM_SPLIT))
               ? kSplitSeg
               : kRecurL;
    return FABM_OK;
}

int fabm_get_history_kernel(const fabm_solver *s) { return s ? s->hist_kernel : -1; }

int fabm_last_history_kernel(const fabm_solver *s) { return s ? s->last_hk : -1; }

fabm_status fabm_set_recurrence_layout(fabm_solver *s, int layout)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (layout != FABM_REC_AUTO && layout != FABM_REC_COLUMNS && layout != FABM_REC_TARGETS)
        return fail(FABM_EINVAL, "recurrence layout %d: 0 (auto), 1 (columns) or 2 (targets)", layout);
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    s->rec_layout = layout;
    return FABM_OK;
}

int fabm_get_recurrence_layout(const fabm_solver *s) { return s ? s->rec_layout : -1; }

fabm_status fabm_set_recurrence_warps(fabm_solver *s, int warps)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (warps < 0 || warps > 12) return fail(FABM_EINVAL, "recurrence warps %d: 0 (automatic) or 1..12", warps);
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    s->rec_warps = warps;
    return FABM_OK;
}

int fabm_get_recurrence_warps(const fabm_solver *s) { return s ? s->rec_warps : -1; }

int fabm_get_block(const fabm_solver *s) { return s ? s->L : 0; }

fabm_status fabm_copy_weights(fabm_solver *s, int64_t n, double *B, double *A, double *D)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (n < 0 || n > s->N + 1) return fail(FABM_EINVAL, "n %lld outside 0..N+1", (long long)n);
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    DeviceGuard g(s->device);
    if (B) FABM_CUDA_TRY(cudaMemcpy(B, s->wB.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (A) FABM_CUDA_TRY(cudaMemcpy(A, s->wA.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (D) FABM_CUDA_TRY(cudaMemcpy(D, s->wD.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return FABM_OK;
}

fabm_status fabm_copy_weights_lo(fabm_solver *s, int64_t n, double *Bl, double *Al, double *Dl)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (s->precision != FABM_FP64X2) return fail(FABM_EINVAL, "low weight parts exist for FP64X2 only");
    if (n < 0 || n > s->N + 1) return fail(FABM_EINVAL, "n %lld outside 0..N+1", (long long)n);
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    DeviceGuard g(s->device);
    if (Bl) FABM_CUDA_TRY(cudaMemcpy(Bl, s->wBl.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (Al) FABM_CUDA_TRY(cudaMemcpy(Al, s->wAl.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (Dl) FABM_CUDA_TRY(cudaMemcpy(Dl, s->wDl.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
    return FABM_OK;
}

int64_t fabm_last_launch_count(const fabm_solver *s) { return s ? s->launches : 0; }

fabm_status fabm_autotune(fabm_solver *s, int64_t B, const double *y0, const double *traj_params,
                          int64_t n_probe, int max_report, double *ms_report, int *kernel_report,
                          int *ctas_report, int *n_report)
{
    g_last_error.clear();
    TraceRange tr("fabm_autotune");
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (B < 1 || !y0) return fail(FABM_EINVAL, "autotune needs B >= 1 and y0");
    if (n_probe < 1) return fail(FABM_EINVAL, "n_probe %lld < 1", (long long)n_probe);
    // probe lengths n_probe, 2 n_probe, 4 n_probe (at most N): a solve takes
    // about c + alpha n + beta n^2 (fixed costs, the per-step chain, the
    // history), so three truncated solves predict the full one
    const int64_t n1 = std::min<int64_t>(n_probe, s->N);
    struct Cand {
        int kernel, ctas;
    };
    std::vector<Cand> cands;
    const int ctas_opts[] = {152, 152 * 2, 152 * 4, 152 * 8};
    // at most 8 candidates are reported
    if (s->precision == FABM_FP64 || s->precision == FABM_FP64X2) {
        const int k = s->precision == FABM_FP64 ? FABM_HIST_FP64 : FABM_HIST_X2;
        for (int c : ctas_opts) cands.push_back({k, c});
        if (s->precision == FABM_FP64 && s->persist_ctas >= B + 8 && !s->multi)
            cands.push_back({FABM_HIST_FP64_PERSIST, s->persist_ctas});
    } else {
        // tensor kernels (far history of pairs of blocks with 128 targets per
        // MMA, or of single blocks with 64): "ctas" carries the SM reserve
        // (-1 automatic, 0, 16); the compensated-fp32 kernel at two CTA targets
        for (int k : {FABM_HIST_TENSOR_WIDE, FABM_HIST_TENSOR})
            for (int r : {-1, 0, 16}) cands.push_back({k, r});
        for (int c : {152 * 2, 152 * 4}) cands.push_back({FABM_HIST_FP32C, c});
    }
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    DeviceGuard g(s->device);
    double *dout = nullptr;
    {
        cudaError_t e = cudaMalloc(&dout, sizeof(double) * (size_t)B * (s->N + 1) * s->dim);
        if (e != cudaSuccess) return fail(FABM_ENOMEM, "autotune output: %s", cudaGetErrorString(e));
    }
    std::vector<int64_t> ne((size_t)B, n1);
    const int keep_kernel = s->hist_kernel, keep_ctas = s->chunk_ctas, keep_res = s->sm_reserve;
    const int keep_L = s->L;
    const bool keep_timing = s->timing;
    s->timing = false;
    s->plan_N = s->N;  // the probes take the full solve's lag and recurrence layout
    double best = 1e300;
    Cand pick{keep_kernel, keep_ctas};
    int nr = 0;
    fabm_status st = FABM_OK;
    // milliseconds of a solve of n steps (second of two runs: the first
    // records the graph), and the prediction for all N steps
    auto time_n = [&](int64_t n) {
        std::fill(ne.begin(), ne.end(), n);
        double ms = 1e300;
        for (int rep = 0; rep < 2 && st == FABM_OK; ++rep) {
            const auto t0 = std::chrono::steady_clock::now();
            st = run_batch(s, B, y0, nullptr, traj_params, ne.data(), dout, 1);
            const auto t1 = std::chrono::steady_clock::now();
            ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        }
        return ms;
    };
    auto predict = [&]() {
        double x[3], t[3];
        for (int i = 0; i < 3; ++i) {
            const int64_t n = std::min<int64_t>(n1 << i, s->N);
            x[i] = (double)n;
            t[i] = time_n(n);
            if (st != FABM_OK || n == s->N) return t[i];  // the full solve was timed
        }
        // the quadratic through the three points (Newton's divided
        // differences), evaluated at N; a negative n^2 coefficient (noise)
        // falls back to the line through the two longer probes
        const double N = (double)s->N;
        const double d01 = (t[1] - t[0]) / (x[1] - x[0]), d12 = (t[2] - t[1]) / (x[2] - x[1]);
        const double beta = (d12 - d01) / (x[2] - x[0]);
        if (beta < 0.0) return t[2] + d12 * (N - x[2]);
        return t[0] + d01 * (N - x[0]) + beta * (N - x[0]) * (N - x[1]);
    };
    for (const Cand &cd : cands) {
        s->hist_kernel = cd.kernel;
        if (cd.kernel == FABM_HIST_TENSOR || cd.kernel == FABM_HIST_TENSOR_WIDE)
            s->sm_reserve = cd.ctas, s->chunk_ctas = keep_ctas;
        else if (cd.kernel == FABM_HIST_FP64_PERSIST)
            s->chunk_ctas = keep_ctas, s->sm_reserve = keep_res;
        else
            s->chunk_ctas = cd.ctas, s->sm_reserve = keep_res;
        const double ms = predict();
        if (st != FABM_OK) break;
        if (nr < max_report) {
            if (ms_report) ms_report[nr] = ms;
            if (kernel_report) kernel_report[nr] = cd.kernel;
            if (ctas_report) ctas_report[nr] = cd.ctas;
        }
        ++nr;
        if (ms < best) best = ms, pick = cd;
    }
    auto apply = [&](const Cand &cd) {
        s->hist_kernel = cd.kernel;
        const bool tensor = cd.kernel == FABM_HIST_TENSOR || cd.kernel == FABM_HIST_TENSOR_WIDE;
        if (tensor || cd.kernel == FABM_HIST_FP64_PERSIST)
            s->sm_reserve = tensor ? cd.ctas : keep_res, s->chunk_ctas = keep_ctas;
        else
            s->chunk_ctas = cd.ctas, s->sm_reserve = keep_res;
        s->L = tensor ? kSplitSeg : kRecurL;
    };
    cudaFree(dout);
    s->timing = keep_timing;
    s->plan_N = 0;
    if (st != FABM_OK) {
        s->hist_kernel = keep_kernel, s->chunk_ctas = keep_ctas, s->sm_reserve = keep_res;
        s->L = keep_L;
        return st;
    }
    apply(pick);
    if (n_report) *n_report = nr;
    return FABM_OK;
}

fabm_status fabm_set_wait_limit(fabm_solver *s, int64_t cycles)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (cycles < 0) return fail(FABM_EINVAL, "wait limit %lld < 0", (long long)cycles);
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    s->wait_cycles = (long long)cycles;
    return FABM_OK;
}

fabm_status fabm_inject_alloc_failures(int n)
{
    g_last_error.clear();
    if (n < 0) return fail(FABM_EINVAL, "n %d < 0", n);
    g_alloc_failures.store(n, std::memory_order_relaxed);
    return FABM_OK;
}

fabm_status fabm_set_graphs(fabm_solver *s, int enable)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    s->use_graphs = enable != 0;
    return FABM_OK;
}

fabm_status fabm_set_timing(fabm_solver *s, int enable)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    std::unique_lock<std::mutex> lk(s->busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(FABM_EBUSY, "solver in use by another thread");
    s->timing = enable > 0;
    s->timing_period = enable > 0 ? enable : 1;
    if (s->timing)
        for (int k = 0; k < FABM_KERNEL_KINDS; ++k)
            if (k != FABM_KERNEL_WEIGHTS)
                s->k_launches[k] = 0, s->k_ms[k] = 0, s->k_flops[k] = 0, s->k_busy[k] = 0;
    return FABM_OK;
}

fabm_status fabm_kernel_busy(const fabm_solver *s, int kind, double *busy_ms)
{
    g_last_error.clear();
    if (!s || !busy_ms) return fail(FABM_EINVAL, "NULL argument");
    if (kind < 0 || kind >= FABM_KERNEL_KINDS) return fail(FABM_EINVAL, "kind %d unknown", kind);
    *busy_ms = s->k_busy[kind];
    return FABM_OK;
}

fabm_status fabm_kernel_stats(const fabm_solver *s, int kind, int64_t *launches, double *total_ms,
                              double *flops)
{
    g_last_error.clear();
    if (!s) return fail(FABM_EINVAL, "solver is NULL");
    if (kind < 0 || kind >= FABM_KERNEL_KINDS) return fail(FABM_EINVAL, "kind %d unknown", kind);
    if (launches) *launches = s->k_launches[kind];
    if (total_ms) *total_ms = s->k_ms[kind];
    if (flops) *flops = s->k_flops[kind];
    return FABM_OK;
}

}  // extern "C"
