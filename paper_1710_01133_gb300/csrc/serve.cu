// a7: continuous-batching server.  Requests (each an independent Caputo
// problem of Sec. 2 of arXiv:1710.01133 with its own right-hand side, dim,
// alpha, h and N) wait in a host queue and are admitted as "slots" while the
// device memory they need (weights, history, output, partials) fits in the
// server's HBM budget.  Each fabm_server_step advances every admitted slot by
// one block of 32 steps with shared launches over tables of slots:
//   stream G: far history of block c+1 of every slot (one launch whose CTAs
//             derive their (slot, chunk, column) items from each slot's block
//             index, so the host builds no work list), then the fixed-order
//             combine
//   stream R: the recurrence of block c of every slot (one CTA per slot,
//             the right-hand side dispatched at run time)
//   stream W: weights and initial values of newly admitted slots, beside the
//             step's launches; new slots run their first block at the next step
// which is the two-stream schedule of a single solve, run for all slots at
// once.  Finished slots are copied to host memory and their device memory is
// returned to the stream-ordered pool; the freed budget admits waiting
// requests at the next step.  Per step the host uploads one block index per
// slot, and the slot table only when slots were admitted or retired.  A slot's chunking depends on its own block index
// only, so its result does not depend on the other requests in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "history_blocks.cuh"
#include "trace.h"
#include "recurrence.cuh"
#include "weights.cuh"

using namespace fabm;

namespace {

constexpr int kSL = kRecurL;        // block length of served solves (32)
constexpr int kMaxChunksSlot = 16;  // far-history chunks per slot and block
constexpr int kMinChunkPts = 1024;  // points per chunk at least

struct SlotDev {
    int rhs, dim, hk;
    int pad;
    int64_t N, w_ext;
    int64_t *Nb;  // device copy of N (read by the recurrence)
    double *F, *Y, *y0, *params, *WB, *WA, *WD, *G;
    double *y1;  // y'(0) (dim doubles) for 1 < alpha < 2, or NULL: Taylor part y0
    float *WBf, *WAf, *Ff;  // split slots: fp32 weights and f rounded to float
    void *part;  // double (FP64) or float2 (split) partials
    StepConsts kc;
    double alpha, inv_g1;
    unsigned long long *status;
};

// Chunking of block c's far history for one slot: depends on c only, so a
// request's partial sums do not depend on the other requests in flight.
__host__ __device__ inline void slot_chunks(int64_t c, int64_t *kc, int *n)
{
    const int64_t k_end = (c - 1) * kSL;
    int64_t pts = (k_end + kMaxChunksSlot - 1) / kMaxChunksSlot;
    if (pts < kMinChunkPts) pts = kMinChunkPts;
    pts = (pts + 31) / 32 * 32;
    *kc = pts;
    *n = (int)((k_end + pts - 1) / pts);
}

__host__ __device__ inline int64_t slot_blocks(int64_t N) { return (N + kSL - 1) / kSL; }

__device__ inline DevBatch slot_batch(const SlotDev &s)
{
    DevBatch bt{};
    bt.dim = s.dim;
    bt.B = 1;
    bt.cols = s.dim;
    bt.N = s.N;
    bt.N_each = s.Nb;
    bt.y0 = s.y0;
    bt.y1 = s.y1;
    bt.params = s.params;
    bt.F = s.F;
    bt.Ff = s.Ff;
    bt.ldF = s.dim;
    bt.Y = s.Y;
    bt.status = s.status;
    return bt;
}

// Runs fn.template operator()<Rhs, D>() for the slot's right-hand side.
template <class Fn>
__device__ inline void slot_dispatch(int rhs, int dim, Fn &&fn)
{
    switch (rhs) {
    case FABM_RHS_CONST:
        if (dim == 1) fn.template operator()<RhsConst, 1>();
        else if (dim == 2) fn.template operator()<RhsConst, 2>();
        else if (dim == 3) fn.template operator()<RhsConst, 3>();
        else fn.template operator()<RhsConst, 4>();
        break;
    case FABM_RHS_TIME:
        if (dim == 1) fn.template operator()<RhsTime, 1>();
        else if (dim == 2) fn.template operator()<RhsTime, 2>();
        else if (dim == 3) fn.template operator()<RhsTime, 3>();
        else fn.template operator()<RhsTime, 4>();
        break;
    case FABM_RHS_LINEAR:
        if (dim == 1) fn.template operator()<RhsLinear, 1>();
        else if (dim == 2) fn.template operator()<RhsLinear, 2>();
        else if (dim == 3) fn.template operator()<RhsLinear, 3>();
        else fn.template operator()<RhsLinear, 4>();
        break;
    case FABM_RHS_LORENZ: fn.template operator()<RhsLorenz, 3>(); break;
    case FABM_RHS_DUFFING: fn.template operator()<RhsDuffing, 2>(); break;
    case FABM_RHS_MANUFACTURED: fn.template operator()<RhsManufactured, 1>(); break;
    case FABM_RHS_LCR: fn.template operator()<RhsLcr, 2>(); break;
    default: break;
    }
}

// Weights (double, and fp32 copies for split slots) of new slots:
// blockIdx.y = new slot, grid-stride over the distances.
__global__ void weights_slots_kernel(const SlotDev *__restrict__ slots, const int *__restrict__ idx)
{
    const SlotDev s = slots[idx[blockIdx.y]];
    const double inv_g2 = s.kc.inv_gamma2[0];
    for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d <= s.w_ext;
         d += (int64_t)gridDim.x * blockDim.x) {
        weights_at(d, s.alpha, s.inv_g1, inv_g2, s.WB, s.WA, s.WD);
        if (s.WBf) {
            s.WBf[d] = (float)s.WB[d];
            s.WAf[d] = (float)s.WA[d];
        }
    }
}

__global__ void init_slots_kernel(const SlotDev *__restrict__ slots, const int *__restrict__ idx,
                                  int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const SlotDev s = slots[idx[j]];
    const DevBatch bt = slot_batch(s);
    slot_dispatch(s.rhs, s.dim, [&]<class R, int D>() { init_one<R, D>(bt, 0); });
}

// Far history, one warp per (slot, chunk, column) item: requests have one to
// three columns, so a CTA of four warps takes four items (of one request or
// several) and no warp idles.  Each warp stages its own tiles of f and of the
// weights and runs the same per-column arithmetic as the batch kernels
// (hist_fp64_block / hist_fp32c_block), so a request's partial sums do not
// depend on which items share its CTA.
constexpr int kWarpsPerHistCta = 4;

__device__ void hist_warp_f64(const SlotDev &s, int64_t c, int chunk, int64_t kc, int q,
                              double *sF, double *sB, double *sA)
{
    using hist::kL;
    constexpr int kT = hist::f64::kTile;
    const int a = threadIdx.x % kWarp, dim = s.dim;
    const int64_t k_end = (c - 1) * kSL;
    const int64_t k0 = (int64_t)chunk * kc;
    const int64_t k1 = k0 + kc < k_end ? k0 + kc : k_end;
    double sp = 0.0, sc = 0.0;
    for (int64_t t0 = k0; t0 < k1; t0 += kT) {
        const int64_t t1 = t0 + kT < k1 ? t0 + kT : k1;
        const int nk = (int)(t1 - t0);
        const int64_t d_min = c * kL + 2 - t1;
        for (int i = a; i < nk + kL - 1; i += kWarp) sB[i] = s.WB[d_min + i], sA[i] = s.WA[d_min + i];
        for (int i = a; i < nk; i += kWarp) sF[i] = s.F[(t0 + i) * dim + q];
        __syncwarp();
        const int base = a + nk - 1;
#pragma unroll 4
        for (int j = 0; j < nk; ++j) {
            const double f = sF[j];
            sp = fma(sB[base - j], f, sp);
            sc = fma(sA[base - j], f, sc);
        }
        __syncwarp();
    }
    double *out = static_cast<double *>(s.part) + ((int64_t)(chunk * 2) * kL + a) * dim + q;
    out[0] = sp;
    out[(int64_t)kL * dim] = sc;
}

__device__ void hist_warp_f32c(const SlotDev &s, int64_t c, int chunk, int64_t kc, int q,
                               float *sF, float *sB, float *sA)
{
    using hist::kL;
    constexpr int kT = hist::f32c::kTile, kG = hist::f32c::kGroup;
    constexpr int kRF = kT / kWarp, kRW = (kT + kL + kWarp - 1) / kWarp;
    const int a = threadIdx.x % kWarp, dim = s.dim;
    const int64_t k_end = (c - 1) * kSL;
    const int64_t k0 = (int64_t)chunk * kc;
    const int64_t k1 = k0 + kc < k_end ? k0 + kc : k_end;
    float sp = 0.f, cp = 0.f, sc = 0.f, cc = 0.f;
    // the next tile's f (the recurrence's float copy) and weights are loaded
    // into registers while the current tile is summed
    float rf[kRF], rb[kRW], ra[kRW];
    auto fetch = [&](int64_t t0) {
        const int64_t t1 = t0 + kT < k1 ? t0 + kT : k1;
        const int nk = (int)(t1 - t0);
        const int64_t d_min = c * kL + 2 - t1;
#pragma unroll
        for (int u = 0; u < kRW; ++u) {
            const int i = a + u * kWarp;
            rb[u] = i < nk + kL - 1 ? s.WBf[d_min + i] : 0.f;
            ra[u] = i < nk + kL - 1 ? s.WAf[d_min + i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kRF; ++u) {
            const int i = a + u * kWarp;
            rf[u] = i < nk ? s.Ff[(t0 + i) * dim + q] : 0.f;
        }
    };
    if (k0 < k1) fetch(k0);
    for (int64_t t0 = k0; t0 < k1; t0 += kT) {
        const int64_t t1 = t0 + kT < k1 ? t0 + kT : k1;
        const int nk = (int)(t1 - t0);
#pragma unroll
        for (int u = 0; u < kRW; ++u) {
            const int i = a + u * kWarp;
            if (i < nk + kL - 1) sB[i] = rb[u], sA[i] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < kRF; ++u) sF[a + u * kWarp] = rf[u];
        __syncwarp();
        if (t1 < k1) fetch(t1);
        const int base = a + nk - 1;
        int j = 0;
        for (; j + kG <= nk; j += kG) {
            float gp = 0.f, gc = 0.f;
#pragma unroll
            for (int u = 0; u < kG; ++u) {
                const float f = sF[j + u];
                gp = fmaf(sB[base - j - u], f, gp);
                gc = fmaf(sA[base - j - u], f, gc);
            }
            hist::f32c::kahan_add(sp, cp, gp);
            hist::f32c::kahan_add(sc, cc, gc);
        }
        float gp = 0.f, gc = 0.f;
        for (; j < nk; ++j) {
            const float f = sF[j];
            gp = fmaf(sB[base - j], f, gp);
            gc = fmaf(sA[base - j], f, gc);
        }
        hist::f32c::kahan_add(sp, cp, gp);
        hist::f32c::kahan_add(sc, cc, gc);
        __syncwarp();
    }
    float2 *out = static_cast<float2 *>(s.part) + ((int64_t)(chunk * 2) * kL + a) * dim + q;
    out[0] = make_float2(sp, -cp);
    out[(int64_t)kL * dim] = make_float2(sc, -cc);
}

// Slots blockIdx.y, blockIdx.y + gridDim.y, ...: the slot's items are
// (chunk, column) pairs in chunk-major order, warp w of CTA x taking item
// 4x + w; the item list is derived here from the slot's block index cs[slot],
// so the host uploads no work list.
__global__ void __launch_bounds__(kWarp *kWarpsPerHistCta)
    hist_slots_kernel(const SlotDev *__restrict__ slots, const int64_t *__restrict__ cs, int ns)
{
    constexpr int kBytesF64 = (hist::f64::kTile + 2 * (hist::f64::kTile + hist::kL)) * 8;
    constexpr int kBytesF32 = (hist::f32c::kTile + 2 * (hist::f32c::kTile + hist::kL)) * 4;
    constexpr int kWarpBytes = kBytesF64 > kBytesF32 ? kBytesF64 : kBytesF32;
    __shared__ __align__(16) unsigned char smem[kWarpsPerHistCta][kWarpBytes];
    const int w = threadIdx.x / kWarp;
    for (int slot = blockIdx.y; slot < ns; slot += gridDim.y) {
        const SlotDev s = slots[slot];
        const int64_t cn = cs[slot] + 1;  // far history of the slot's next block
        if (cn < 2 || cn >= slot_blocks(s.N)) continue;
        int64_t kc;
        int n;
        slot_chunks(cn, &kc, &n);
        const int g = (int)blockIdx.x * kWarpsPerHistCta + w;
        if (g >= n * s.dim) continue;  // uniform over the warp; warps never synchronize
        const int chunk = g / s.dim, q = g % s.dim;
        if (s.hk == FABM_HIST_FP32C) {
            float *sF = reinterpret_cast<float *>(smem[w]);
            float *sB = sF + hist::f32c::kTile;
            hist_warp_f32c(s, cn, chunk, kc, q, sF, sB, sB + hist::f32c::kTile + hist::kL);
        } else {
            double *sF = reinterpret_cast<double *>(smem[w]);
            double *sB = sF + hist::f64::kTile;
            hist_warp_f64(s, cn, chunk, kc, q, sF, sB, sB + hist::f64::kTile + hist::kL);
        }
    }
}

// One CTA per slot: G[gbuf][kind][t][col] = sum over the chunks in ascending
// order (compensated double, or float-float rounded once to double).
__global__ void combine_slots_kernel(const SlotDev *__restrict__ slots, const int64_t *__restrict__ cs)
{
    const SlotDev s = slots[blockIdx.x];
    const int64_t cn = cs[blockIdx.x] + 1;
    if (cn < 2 || cn >= slot_blocks(s.N)) return;  // no far history this step (uniform)
    int64_t kc;
    int n_chunks;
    slot_chunks(cn, &kc, &n_chunks);
    const int n_out = 2 * kSL * s.dim;
    double *G = s.G + (int64_t)(cn % 2) * n_out;
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
        if (s.hk == FABM_HIST_FP32C) {
            const float2 *p = static_cast<const float2 *>(s.part);
            float hi = 0.f, lo = 0.f;
            for (int ch = 0; ch < n_chunks; ++ch) {
                const float2 v = p[(int64_t)ch * n_out + o];
                const float t = hi + v.x;
                const float bb = t - hi;
                const float e = (hi - (t - bb)) + (v.x - bb);
                lo += e + v.y;
                hi = t + lo;
                lo = lo - (hi - t);
            }
            G[o] = (double)hi + (double)lo;
        } else {
            // Neumaier: the rounding error of every addition (TwoSum) is kept
            // in a second sum, added once at the end; chunk order fixed
            const double *p = static_cast<const double *>(s.part);
            double acc = 0.0, err = 0.0;
            for (int ch = 0; ch < n_chunks; ++ch) {
                const double v = p[(int64_t)ch * n_out + o];
                const double t = acc + v;
                const double bv = t - acc;
                err += (acc - (t - bv)) + (v - bv);
                acc = t;
            }
            G[o] = acc + err;
        }
    }
}

// One CTA of 4 warps per slot: block cs[slot] of the recurrence (the split
// recurrence for split slots).
__global__ void __launch_bounds__(kWarp *FABM_MAX_DIM)
    recur_slots_kernel(const SlotDev *__restrict__ slots, const int64_t *__restrict__ cs)
{
    static_assert(recur_split_smem_floats<FABM_MAX_DIM, 1>() <=
                  2 * recur_smem_doubles<FABM_MAX_DIM, 1>());
    __shared__ double smem[recur_smem_doubles<FABM_MAX_DIM, 1>()];
    const SlotDev s = slots[blockIdx.x];
    const int64_t c = cs[blockIdx.x];  // the block this step runs; -1: none (new slot)
    if (c < 0) return;
    const DevBatch bt = slot_batch(s);
    const DevWeights w{s.WB, s.WA, s.WD, s.w_ext};
    const double *G = c >= 2 ? s.G + (c % 2) * 2 * kSL * s.dim : nullptr;
    const bool split = s.hk == FABM_HIST_FP32C;
    slot_dispatch(s.rhs, s.dim, [&]<class R, int D>() {
        if (split)
            recur_block_split<R, D, 1>(bt, 0, w, s.kc, c, G, reinterpret_cast<float *>(smem));
        else
            recur_block<R, D, 1>(bt, 0, w, s.kc, c, G, smem);
    });
}

// ------------------------------------------------------------------- host ---

fabm_status srv_fail(fabm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

#define SRV_TRY(expr)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return srv_fail(e_ == cudaErrorMemoryAllocation ? FABM_ENOMEM : FABM_ECUDA,      \
                            "%s failed: %s", #expr, cudaGetErrorString(e_));                 \
    } while (0)

// State of a request taken at a block boundary (fabm_server_checkpoint): the
// next block to run, the history f and the solution rows known so far, both
// far-history buffers and the non-finite status word.
struct Ckpt {
    int64_t c = 0;
    unsigned long long status = ~0ull;
    std::vector<double> F, Y, G;  // rows x dim, rows x dim, 2 x 2 x kSL x dim
};

// Layout of a serialized checkpoint: this header, then F and Y (rows x dim
// each) and G (2 x 2 x kSL x dim), doubles in the host's byte order.
constexpr char kCkptMagic[8] = {'F', 'A', 'B', 'M', 'C', 'K', 'P', '2'};
struct CkptHead {
    char magic[8];
    int32_t precision, dim, rhs, n_params;
    double alpha, h;
    int64_t N, c, rows;
    unsigned long long status;
    double params[kMaxParams];
    double y0[FABM_MAX_DIM];
    int32_t has_y1, pad;
    double y1[FABM_MAX_DIM];  // y'(0) when has_y1 (1 < alpha < 2)
};

struct Req {
    int64_t ticket;
    int dim, rhs;
    double alpha, h;
    int64_t N;
    double params[kMaxParams];
    int n_params;
    double y0[FABM_MAX_DIM];
    double y1[FABM_MAX_DIM];  // y'(0), used when has_y1 (1 < alpha < 2)
    int has_y1;
    std::shared_ptr<const Ckpt> ckpt;  // set for a resumed request
};

struct Slot {
    Req req;
    int64_t c = 0, nblk = 0;
    size_t bytes = 0;
    void *mem = nullptr;
    SlotDev dev{};
    bool pending = false;  // admitted at this step: weights being computed, no block run yet
};

struct Result {
    int state;  // FABM_REQ_*
    fabm_status status;
    std::vector<double> y;
};

size_t slot_bytes(const Req &r, int hk, int64_t *w_ext_out)
{
    const int64_t nblk = (r.N + kSL - 1) / kSL;
    const int64_t w_ext = nblk * kSL + 2 * kSL;
    *w_ext_out = w_ext;
    const int64_t n_chunks = kMaxChunksSlot;
    size_t b = 0;
    auto add = [&](size_t n) { b += (n + 255) / 256 * 256; };
    add(sizeof(int64_t));                                   // Nb
    add(sizeof(unsigned long long));                        // status
    add(sizeof(double) * FABM_MAX_DIM);                     // y0
    add(sizeof(double) * FABM_MAX_DIM);                     // y1
    add(sizeof(double) * kMaxParams);                       // params
    for (int i = 0; i < 3; ++i) add(sizeof(double) * (w_ext + 1));  // WB WA WD
    if (hk == FABM_HIST_FP32C) {
        for (int i = 0; i < 2; ++i) add(sizeof(float) * (w_ext + 1));
        add(sizeof(float) * (r.N + 1) * r.dim);             // Ff
    }
    add(sizeof(double) * (r.N + 1) * r.dim);                // F
    add(sizeof(double) * (r.N + 1) * r.dim);                // Y
    add(sizeof(double) * 2 * 2 * kSL * r.dim);              // G
    add((size_t)8 * n_chunks * 2 * kSL * r.dim);            // partials
    return b;
}

// Carves a slot's device block into its buffers.
void slot_layout(Slot &s, int hk, int64_t w_ext)
{
    uint8_t *p = static_cast<uint8_t *>(s.mem);
    auto take = [&](size_t n) {
        uint8_t *q = p;
        p += (n + 255) / 256 * 256;
        return q;
    };
    const Req &r = s.req;
    SlotDev &d = s.dev;
    d.rhs = r.rhs, d.dim = r.dim, d.hk = hk, d.N = r.N, d.w_ext = w_ext;
    d.Nb = reinterpret_cast<int64_t *>(take(sizeof(int64_t)));
    d.status = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long)));
    d.y0 = reinterpret_cast<double *>(take(sizeof(double) * FABM_MAX_DIM));
    double *y1 = reinterpret_cast<double *>(take(sizeof(double) * FABM_MAX_DIM));
    d.y1 = r.has_y1 ? y1 : nullptr;
    d.params = reinterpret_cast<double *>(take(sizeof(double) * kMaxParams));
    d.WB = reinterpret_cast<double *>(take(sizeof(double) * (w_ext + 1)));
    d.WA = reinterpret_cast<double *>(take(sizeof(double) * (w_ext + 1)));
    d.WD = reinterpret_cast<double *>(take(sizeof(double) * (w_ext + 1)));
    d.WBf = d.WAf = d.Ff = nullptr;
    if (hk == FABM_HIST_FP32C) {
        d.WBf = reinterpret_cast<float *>(take(sizeof(float) * (w_ext + 1)));
        d.WAf = reinterpret_cast<float *>(take(sizeof(float) * (w_ext + 1)));
        d.Ff = reinterpret_cast<float *>(take(sizeof(float) * (r.N + 1) * r.dim));
    }
    d.F = reinterpret_cast<double *>(take(sizeof(double) * (r.N + 1) * r.dim));
    d.Y = reinterpret_cast<double *>(take(sizeof(double) * (r.N + 1) * r.dim));
    d.G = reinterpret_cast<double *>(take(sizeof(double) * 2 * 2 * kSL * r.dim));
    d.part = take((size_t)8 * kMaxChunksSlot * 2 * kSL * r.dim);
    d.kc.h = r.h;
    for (int q = 0; q < FABM_MAX_DIM; ++q) {
        d.kc.h_alpha[q] = std::pow(r.h, r.alpha);
        d.kc.inv_gamma2[q] = 1.0 / std::tgamma(r.alpha + 2.0);
    }
    d.alpha = r.alpha;
    d.inv_g1 = 1.0 / std::tgamma(r.alpha + 1.0);
}


}  // namespace

struct fabm_server {
    int device = 0;
    int precision = FABM_FP64;
    size_t budget = 0, in_use = 0;
    int max_slots = 0;
    std::deque<Req> queue;
    std::vector<Slot> slots;
    std::unordered_map<int64_t, Result> results;
    std::unordered_map<int64_t, std::pair<int64_t, int>> shapes;  // ticket -> (N, dim)
    std::vector<int64_t> finished;  // finished since the last fabm_server_finished
    int64_t next_ticket = 1;
    cudaStream_t sR = nullptr, sG = nullptr, sW = nullptr;
    cudaEvent_t evUp = nullptr, evIn = nullptr;
    SlotDev *d_slots = nullptr;  // device tables: the slots, uploaded when they change,
    int64_t *d_c = nullptr;      // each slot's block index, uploaded every step,
    int *d_idx = nullptr;        // and the indices of newly admitted slots
    SlotDev *h_slots = nullptr;  // pinned staging
    int64_t *h_c = nullptr;
    int *h_idx = nullptr;
    bool table_dirty = true;     // the slot table changed since its last upload
    int64_t steps_done = 0, launches = 0;
    std::mutex mu;

    ~fabm_server()
    {
        for (auto &s : slots)
            if (s.mem) cudaFreeAsync(s.mem, sR);
        if (sR) cudaStreamSynchronize(sR);
        if (d_slots) cudaFree(d_slots);
        if (d_c) cudaFree(d_c);
        if (d_idx) cudaFree(d_idx);
        if (h_slots) cudaFreeHost(h_slots);
        if (h_c) cudaFreeHost(h_c);
        if (h_idx) cudaFreeHost(h_idx);
        if (sW) cudaStreamSynchronize(sW);
        if (evUp) cudaEventDestroy(evUp);
        if (evIn) cudaEventDestroy(evIn);
        if (sR) cudaStreamDestroy(sR);
        if (sG) cudaStreamDestroy(sG);
        if (sW) cudaStreamDestroy(sW);
    }
};

namespace {

fabm_status server_step(fabm_server *S, int *n_active, int *n_waiting)
{
    const int hk = S->precision == FABM_SPLIT ? FABM_HIST_FP32C : FABM_HIST_FP64;
    // 1. admission: waiting requests in arrival order while the budget allows
    std::vector<int> fresh;
    while (!S->queue.empty() && (int)S->slots.size() < S->max_slots) {
        Req r = S->queue.front();
        int64_t w_ext;
        const size_t bytes = slot_bytes(r, hk, &w_ext);
        if (S->in_use + bytes > S->budget) {
            if (S->slots.empty()) {  // can never fit
                S->queue.pop_front();
                S->results[r.ticket] = {FABM_REQ_FAILED, FABM_ENOMEM, {}};
                S->finished.push_back(r.ticket);
                continue;
            }
            break;
        }
        Slot s;
        s.req = r;
        s.bytes = bytes;
        s.nblk = (r.N + kSL - 1) / kSL;
        cudaError_t e = take_injected_alloc_failure() ? cudaErrorMemoryAllocation
                                                      : cudaMallocAsync(&s.mem, bytes, S->sR);
        if (e != cudaSuccess) {
            if (S->slots.empty()) {
                S->queue.pop_front();
                S->results[r.ticket] = {FABM_REQ_FAILED, FABM_ENOMEM, {}};
                S->finished.push_back(r.ticket);
                continue;
            }
            break;  // retry when memory frees up
        }
        slot_layout(s, hk, w_ext);
        if (r.ckpt) s.c = r.ckpt->c;
        S->queue.pop_front();
        S->in_use += bytes;
        S->results[r.ticket] = {FABM_REQ_RUNNING, FABM_OK, {}};
        s.pending = true;
        fresh.push_back((int)S->slots.size());
        S->slots.push_back(s);
    }
    // new slots needing initial values first, resumed ones after them
    std::stable_partition(fresh.begin(), fresh.end(),
                          [&](int i) { return !S->slots[i].req.ckpt; });
    int n_init = 0;
    for (int i : fresh) n_init += S->slots[i].req.ckpt ? 0 : 1;
    const int ns = (int)S->slots.size();
    *n_waiting = (int)S->queue.size();
    *n_active = ns;
    if (ns == 0) return FABM_OK;

    // 2. tables: the slots (when they changed), each slot's block index (its
    // history, combine and recurrence items follow from it on the device) and
    // the indices of new slots
    if (!fresh.empty()) S->table_dirty = true;
    if (S->table_dirty) {
        for (int i = 0; i < ns; ++i) S->h_slots[i] = S->slots[i].dev;
        SRV_TRY(cudaMemcpyAsync(S->d_slots, S->h_slots, sizeof(SlotDev) * ns, cudaMemcpyHostToDevice, S->sR));
        S->table_dirty = false;
    }
    int max_items = 0;  // history items of the busiest slot
    for (int i = 0; i < ns; ++i) {
        const Slot &s = S->slots[i];
        S->h_c[i] = s.pending ? -1 : s.c;  // -1: the device skips the slot this step
        if (s.pending) continue;
        const int64_t cn = s.c + 1;
        if (cn >= 2 && cn < s.nblk) {
            int64_t kc;
            int n;
            slot_chunks(cn, &kc, &n);
            max_items = std::max(max_items, n * s.req.dim);
        }
    }
    for (size_t j = 0; j < fresh.size(); ++j) S->h_idx[j] = fresh[j];
    SRV_TRY(cudaMemcpyAsync(S->d_c, S->h_c, sizeof(int64_t) * ns, cudaMemcpyHostToDevice, S->sR));
    // 3. new slots: inputs (stream R), then weights and initial values on
    // stream W beside this step's launches (they take ~0.1-0.2 ms of FP64
    // work, which had delayed the whole step whenever requests arrived); the
    // new slots run their first block at the next step
    if (!fresh.empty()) {
        SRV_TRY(cudaMemcpyAsync(S->d_idx, S->h_idx, sizeof(int) * fresh.size(), cudaMemcpyHostToDevice, S->sR));
        for (int i : fresh) {
            Slot &s = S->slots[i];
            double par[kMaxParams] = {};
            for (int q = 0; q < s.req.n_params; ++q) par[q] = s.req.params[q];
            SRV_TRY(cudaMemcpyAsync(s.dev.y0, s.req.y0, sizeof(double) * s.req.dim, cudaMemcpyHostToDevice, S->sR));
            if (s.dev.y1)
                SRV_TRY(cudaMemcpyAsync(s.dev.y1, s.req.y1, sizeof(double) * s.req.dim, cudaMemcpyHostToDevice, S->sR));
            SRV_TRY(cudaMemcpyAsync(s.dev.params, par, sizeof par, cudaMemcpyHostToDevice, S->sR));
            SRV_TRY(cudaMemcpyAsync(s.dev.Nb, &s.req.N, sizeof(int64_t), cudaMemcpyHostToDevice, S->sR));
            if (const Ckpt *k = s.req.ckpt.get()) {  // resumed: the saved state
                const size_t rows = k->F.size() / s.req.dim;
                SRV_TRY(cudaMemcpyAsync(s.dev.F, k->F.data(), sizeof(double) * rows * s.req.dim, cudaMemcpyHostToDevice, S->sR));
                if (s.dev.Ff)  // the float copy the fp32 history reads
                    SRV_TRY(launch_to_float(s.dev.F, (int64_t)(rows * s.req.dim), s.dev.Ff, S->sR));
                SRV_TRY(cudaMemcpyAsync(s.dev.Y, k->Y.data(), sizeof(double) * rows * s.req.dim, cudaMemcpyHostToDevice, S->sR));
                SRV_TRY(cudaMemcpyAsync(s.dev.G, k->G.data(), sizeof(double) * k->G.size(), cudaMemcpyHostToDevice, S->sR));
                SRV_TRY(cudaMemcpyAsync(s.dev.status, &k->status, sizeof k->status, cudaMemcpyHostToDevice, S->sR));
            } else {
                SRV_TRY(cudaMemsetAsync(s.dev.status, 0xff, sizeof(unsigned long long), S->sR));
            }
        }
        SRV_TRY(cudaEventRecord(S->evIn, S->sR));
        SRV_TRY(cudaStreamWaitEvent(S->sW, S->evIn, 0));
        int64_t wmax = 0;
        for (int i : fresh) wmax = std::max(wmax, S->slots[i].dev.w_ext);
        const unsigned gx = (unsigned)std::min<int64_t>((wmax + 256) / 256, 64);
        weights_slots_kernel<<<dim3(gx, (unsigned)fresh.size()), 256, 0, S->sW>>>(S->d_slots, S->d_idx);
        SRV_TRY(cudaGetLastError());
        S->launches += 1;
        if (n_init > 0) {
            init_slots_kernel<<<(unsigned)((n_init + 127) / 128), 128, 0, S->sW>>>(
                S->d_slots, S->d_idx, n_init);
            SRV_TRY(cudaGetLastError());
            S->launches += 1;
        }
    }
    SRV_TRY(cudaEventRecord(S->evUp, S->sR));
    SRV_TRY(cudaStreamWaitEvent(S->sG, S->evUp, 0));
    // 4. shared launches
    if (max_items > 0) {
        const unsigned hx = (unsigned)((max_items + kWarpsPerHistCta - 1) / kWarpsPerHistCta);
        const unsigned hy = (unsigned)std::min(ns, 65535);
        hist_slots_kernel<<<dim3(hx, hy), kWarp * kWarpsPerHistCta, 0, S->sG>>>(S->d_slots, S->d_c, ns);
        SRV_TRY(cudaGetLastError());
        combine_slots_kernel<<<(unsigned)ns, 256, 0, S->sG>>>(S->d_slots, S->d_c);
        SRV_TRY(cudaGetLastError());
        S->launches += 2;
    }
    recur_slots_kernel<<<(unsigned)ns, kWarp * FABM_MAX_DIM, 0, S->sR>>>(S->d_slots, S->d_c);
    SRV_TRY(cudaGetLastError());
    ++S->launches;
    SRV_TRY(cudaStreamSynchronize(S->sG));
    SRV_TRY(cudaStreamSynchronize(S->sR));
    SRV_TRY(cudaStreamSynchronize(S->sW));
    ++S->steps_done;

    // 5. advance; finished slots to host, memory back to the pool; the table
    // is compacted (and uploaded at the next step) only when a slot finished
    bool retired = false;
    for (int i = 0; i < ns; ++i) {
        Slot &s = S->slots[i];
        s.req.ckpt.reset();  // restored on the device by now
        if (s.pending) {  // weights and initial values are in place: run from the next step
            s.pending = false;
            continue;
        }
        s.c += 1;
        if (s.c < s.nblk) continue;
        retired = true;
        Result &res = S->results[s.req.ticket];
        res.y.resize((size_t)(s.req.N + 1) * s.req.dim);
        unsigned long long st = 0;
        SRV_TRY(cudaMemcpy(res.y.data(), s.dev.Y, sizeof(double) * res.y.size(), cudaMemcpyDeviceToHost));
        SRV_TRY(cudaMemcpy(&st, s.dev.status, sizeof st, cudaMemcpyDeviceToHost));
        res.state = st == ~0ull ? FABM_REQ_DONE : FABM_REQ_FAILED;
        res.status = st == ~0ull ? FABM_OK : FABM_ENONFINITE;
        S->finished.push_back(s.req.ticket);
        SRV_TRY(cudaFreeAsync(s.mem, S->sR));
        S->in_use -= s.bytes;
    }
    if (retired) {
        S->slots.erase(std::remove_if(S->slots.begin(), S->slots.end(),
                                      [](const Slot &s) { return s.c >= s.nblk; }),
                       S->slots.end());
        S->table_dirty = true;
    }
    *n_active = (int)S->slots.size();
    return FABM_OK;
}

}  // namespace

extern "C" {

fabm_status fabm_server_create(size_t budget_bytes, int precision, int max_slots, fabm_server **out)
{
    set_last_error("");
    if (!out) return srv_fail(FABM_EINVAL, "out is NULL");
    *out = nullptr;
    if (precision != FABM_FP64 && precision != FABM_SPLIT)
        return srv_fail(FABM_EINVAL, "precision %d unknown", precision);
    if (max_slots < 1 || max_slots > (1 << 20)) return srv_fail(FABM_EINVAL, "max_slots %d", max_slots);
    if (budget_bytes == 0) return srv_fail(FABM_EINVAL, "budget is 0");
    fabm_server *S = new (std::nothrow) fabm_server();
    if (!S) return srv_fail(FABM_ENOMEM, "host allocation failed");
    S->budget = budget_bytes, S->precision = precision, S->max_slots = max_slots;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->sR, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->sG, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->sW, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->evUp, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->evIn, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_slots, sizeof(SlotDev) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_idx, sizeof(int) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_c, sizeof(int64_t) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_c, sizeof(int64_t) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_slots, sizeof(SlotDev) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_idx, sizeof(int) * max_slots);
    if (e != cudaSuccess) {
        delete S;
        return srv_fail(FABM_ECUDA, "fabm_server_create: %s", cudaGetErrorString(e));
    }
    *out = S;
    return FABM_OK;
}

static fabm_status server_submit(fabm_server *S, const fabm_request *q, const double *y1,
                                 int64_t *ticket)
{
    set_last_error("");
    if (!S || !q || !ticket) return srv_fail(FABM_EINVAL, "NULL argument");
    if (q->dim < 1 || q->dim > FABM_MAX_DIM) return srv_fail(FABM_EINVAL, "dim %d", q->dim);
    if (!(q->alpha > 0.0 && q->alpha < 2.0)) return srv_fail(FABM_EINVAL, "alpha %g", q->alpha);
    if (y1 && !(q->alpha > 1.0))
        return srv_fail(FABM_EINVAL, "y'(0) given for alpha %g <= 1", q->alpha);
    if (!(q->h > 0.0) || !std::isfinite(q->h)) return srv_fail(FABM_EINVAL, "h %g", q->h);
    if (q->N < 1 || q->N > (1LL << 31)) return srv_fail(FABM_EINVAL, "N %lld", (long long)q->N);
    const int np = rhs_n_params(q->rhs_id);
    if (np < 0 || !rhs_supports_dim(q->rhs_id, q->dim))
        return srv_fail(FABM_EINVAL, "rhs_id %d with dim %d unsupported", q->rhs_id, q->dim);
    if (q->n_params < np || q->n_params > kMaxParams || (q->n_params > 0 && !q->params))
        return srv_fail(FABM_EINVAL, "rhs_id %d needs %d params", q->rhs_id, np);
    if (!q->y0) return srv_fail(FABM_EINVAL, "y0 is NULL");
    Req r{};
    r.dim = q->dim, r.rhs = q->rhs_id, r.alpha = q->alpha, r.h = q->h, r.N = q->N;
    r.n_params = q->n_params;
    for (int i = 0; i < q->n_params; ++i) r.params[i] = q->params[i];
    for (int i = 0; i < q->dim; ++i) {
        if (!std::isfinite(q->y0[i])) return srv_fail(FABM_EINVAL, "y0 not finite");
        r.y0[i] = q->y0[i];
    }
    if (y1) {
        r.has_y1 = 1;
        for (int i = 0; i < q->dim; ++i) {
            if (!std::isfinite(y1[i])) return srv_fail(FABM_EINVAL, "y'(0) not finite");
            r.y1[i] = y1[i];
        }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    r.ticket = S->next_ticket++;
    S->queue.push_back(r);
    S->results[r.ticket] = {FABM_REQ_WAITING, FABM_OK, {}};
    S->shapes[r.ticket] = {r.N, r.dim};
    *ticket = r.ticket;
    return FABM_OK;
}

fabm_status fabm_server_submit(fabm_server *S, const fabm_request *q, int64_t *ticket)
{
    return server_submit(S, q, nullptr, ticket);
}

fabm_status fabm_server_submit_ic(fabm_server *S, const fabm_request *q, const double *y1,
                                  int64_t *ticket)
{
    return server_submit(S, q, y1, ticket);
}

fabm_status fabm_server_step(fabm_server *S, int *n_active, int *n_waiting)
{
    set_last_error("");
    TraceRange tr("fabm_server_step");
    if (!S) return srv_fail(FABM_EINVAL, "server is NULL");
    int a = 0, w = 0;
    std::lock_guard<std::mutex> lk(S->mu);
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != S->device) cudaSetDevice(S->device);
    fabm_status st = server_step(S, &a, &w);
    if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
    if (n_active) *n_active = a;
    if (n_waiting) *n_waiting = w;
    return st;
}

fabm_status fabm_server_poll(fabm_server *S, int64_t ticket, int *state)
{
    set_last_error("");
    if (!S || !state) return srv_fail(FABM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return srv_fail(FABM_EINVAL, "unknown ticket %lld", (long long)ticket);
    *state = it->second.state;
    return FABM_OK;
}

fabm_status fabm_server_result(fabm_server *S, int64_t ticket, double *out)
{
    set_last_error("");
    if (!S || !out) return srv_fail(FABM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return srv_fail(FABM_EINVAL, "unknown ticket %lld", (long long)ticket);
    Result &r = it->second;
    if (r.state == FABM_REQ_WAITING || r.state == FABM_REQ_RUNNING)
        return srv_fail(FABM_EBUSY, "request %lld not finished", (long long)ticket);
    const fabm_status st = r.status;
    if (!r.y.empty()) std::memcpy(out, r.y.data(), sizeof(double) * r.y.size());
    S->results.erase(it);
    S->shapes.erase(ticket);
    if (st != FABM_OK)
        return srv_fail(st, "request %lld failed (%s)", (long long)ticket,
                        st == FABM_ENONFINITE ? "non-finite value" : "does not fit the budget");
    return FABM_OK;
}

fabm_status fabm_server_wait(fabm_server *S, int64_t ticket, double *out)
{
    set_last_error("");
    if (!S || !out) return srv_fail(FABM_EINVAL, "NULL argument");
    for (;;) {
        int state = 0;
        const fabm_status st = fabm_server_poll(S, ticket, &state);
        if (st != FABM_OK) return st;
        if (state == FABM_REQ_DONE || state == FABM_REQ_FAILED) break;
        const fabm_status ss = fabm_server_step(S, nullptr, nullptr);
        if (ss != FABM_OK) return ss;
    }
    return fabm_server_result(S, ticket, out);
}

fabm_status fabm_server_checkpoint(fabm_server *S, int64_t ticket, void *buf, size_t cap,
                                   size_t *size)
{
    set_last_error("");
    if (!S || !size) return srv_fail(FABM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    const Req *r = nullptr;
    const Slot *slot = nullptr;
    for (const Slot &sl : S->slots)
        if (sl.req.ticket == ticket) slot = &sl, r = &sl.req;
    if (!r)
        for (const Req &q : S->queue)
            if (q.ticket == ticket) r = &q;
    if (!r) return srv_fail(FABM_EINVAL, "request %lld is not waiting or running", (long long)ticket);
    const int64_t c = slot ? slot->c : (r->ckpt ? r->ckpt->c : 0);
    const int64_t rows = c == 0 ? 0 : std::min<int64_t>(r->N, c * kSL) + 1;
    const size_t n_g = (size_t)4 * kSL * r->dim;
    const size_t need = sizeof(CkptHead) + sizeof(double) * ((size_t)2 * rows * r->dim + n_g);
    *size = need;
    if (!buf) return FABM_OK;
    if (cap < need) return srv_fail(FABM_EINVAL, "checkpoint needs %zu bytes, buffer has %zu", need, cap);
    CkptHead hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.precision = S->precision, hd.dim = r->dim, hd.rhs = r->rhs, hd.n_params = r->n_params;
    hd.alpha = r->alpha, hd.h = r->h, hd.N = r->N, hd.c = c, hd.rows = rows;
    hd.status = ~0ull;
    for (int i = 0; i < kMaxParams; ++i) hd.params[i] = r->params[i];
    for (int i = 0; i < FABM_MAX_DIM; ++i) hd.y0[i] = r->y0[i], hd.y1[i] = r->y1[i];
    hd.has_y1 = r->has_y1;
    uint8_t *p = static_cast<uint8_t *>(buf);
    double *F = reinterpret_cast<double *>(p + sizeof hd);
    double *Y = F + rows * r->dim;
    double *G = Y + rows * r->dim;
    if (slot) {  // between steps both streams are idle: plain copies
        const size_t n = sizeof(double) * rows * r->dim;
        SRV_TRY(cudaMemcpy(F, slot->dev.F, n, cudaMemcpyDeviceToHost));
        SRV_TRY(cudaMemcpy(Y, slot->dev.Y, n, cudaMemcpyDeviceToHost));
        SRV_TRY(cudaMemcpy(G, slot->dev.G, sizeof(double) * n_g, cudaMemcpyDeviceToHost));
        SRV_TRY(cudaMemcpy(&hd.status, slot->dev.status, sizeof hd.status, cudaMemcpyDeviceToHost));
    } else if (r->ckpt) {
        std::memcpy(F, r->ckpt->F.data(), sizeof(double) * r->ckpt->F.size());
        std::memcpy(Y, r->ckpt->Y.data(), sizeof(double) * r->ckpt->Y.size());
        std::memcpy(G, r->ckpt->G.data(), sizeof(double) * n_g);
        hd.status = r->ckpt->status;
    } else {
        std::memset(G, 0, sizeof(double) * n_g);
    }
    std::memcpy(p, &hd, sizeof hd);
    return FABM_OK;
}

fabm_status fabm_server_resume(fabm_server *S, const void *buf, size_t size, int64_t *ticket)
{
    set_last_error("");
    if (!S || !buf || !ticket) return srv_fail(FABM_EINVAL, "NULL argument");
    if (size < sizeof(CkptHead)) return srv_fail(FABM_EINVAL, "checkpoint of %zu bytes is truncated", size);
    CkptHead hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0) return srv_fail(FABM_EINVAL, "not a checkpoint");
    if (hd.precision != S->precision)
        return srv_fail(FABM_EINVAL, "checkpoint of precision %d on a server of precision %d",
                        hd.precision, S->precision);
    if (hd.dim < 1 || hd.dim > FABM_MAX_DIM || !rhs_supports_dim(hd.rhs, hd.dim) ||
        hd.n_params < rhs_n_params(hd.rhs) || hd.n_params > kMaxParams ||
        !(hd.alpha > 0.0 && hd.alpha < 2.0) || !(hd.h > 0.0) || hd.N < 1 || hd.N > (1LL << 31) ||
        (hd.has_y1 != 0 && hd.has_y1 != 1) || (hd.has_y1 && !(hd.alpha > 1.0)))
        return srv_fail(FABM_EINVAL, "checkpoint header is invalid");
    const int64_t nblk = (hd.N + kSL - 1) / kSL;
    const int64_t rows = hd.c == 0 ? 0 : std::min<int64_t>(hd.N, hd.c * kSL) + 1;
    const size_t n_g = (size_t)4 * kSL * hd.dim;
    if (hd.c < 0 || hd.c >= nblk || hd.rows != rows ||
        size != sizeof hd + sizeof(double) * ((size_t)2 * rows * hd.dim + n_g))
        return srv_fail(FABM_EINVAL, "checkpoint sizes are inconsistent");
    Req r{};
    r.dim = hd.dim, r.rhs = hd.rhs, r.alpha = hd.alpha, r.h = hd.h, r.N = hd.N;
    r.n_params = hd.n_params;
    for (int i = 0; i < kMaxParams; ++i) r.params[i] = hd.params[i];
    for (int i = 0; i < FABM_MAX_DIM; ++i) r.y0[i] = hd.y0[i], r.y1[i] = hd.y1[i];
    r.has_y1 = hd.has_y1;
    if (hd.c > 0) {
        auto k = std::make_shared<Ckpt>();
        const double *F = reinterpret_cast<const double *>(static_cast<const uint8_t *>(buf) + sizeof hd);
        k->c = hd.c;
        k->status = hd.status;
        k->F.assign(F, F + rows * hd.dim);
        k->Y.assign(F + rows * hd.dim, F + 2 * rows * hd.dim);
        k->G.assign(F + 2 * rows * hd.dim, F + 2 * rows * hd.dim + n_g);
        r.ckpt = std::move(k);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    r.ticket = S->next_ticket++;
    S->queue.push_back(r);
    S->results[r.ticket] = {FABM_REQ_WAITING, FABM_OK, {}};
    S->shapes[r.ticket] = {r.N, r.dim};
    *ticket = r.ticket;
    return FABM_OK;
}

fabm_status fabm_server_shape(fabm_server *S, int64_t ticket, int64_t *N, int *dim)
{
    set_last_error("");
    if (!S || !N || !dim) return srv_fail(FABM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->shapes.find(ticket);
    if (it == S->shapes.end()) return srv_fail(FABM_EINVAL, "unknown ticket %lld", (long long)ticket);
    *N = it->second.first;
    *dim = it->second.second;
    return FABM_OK;
}

fabm_status fabm_server_cancel(fabm_server *S, int64_t ticket)
{
    set_last_error("");
    if (!S) return srv_fail(FABM_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return srv_fail(FABM_EINVAL, "unknown ticket %lld", (long long)ticket);
    S->results.erase(it);
    S->shapes.erase(ticket);
    S->finished.erase(std::remove(S->finished.begin(), S->finished.end(), ticket), S->finished.end());
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
        if (q->ticket == ticket) {
            S->queue.erase(q);
            return FABM_OK;
        }
    for (size_t i = 0; i < S->slots.size(); ++i)
        if (S->slots[i].req.ticket == ticket) {
            SRV_TRY(cudaFreeAsync(S->slots[i].mem, S->sR));
            S->in_use -= S->slots[i].bytes;
            S->slots.erase(S->slots.begin() + (std::ptrdiff_t)i);
            S->table_dirty = true;
            return FABM_OK;
        }
    return FABM_OK;  // finished: its result is dropped
}

fabm_status fabm_server_finished(fabm_server *S, int64_t *tickets, int max, int *n)
{
    set_last_error("");
    if (!S || !n || max < 0 || (max > 0 && !tickets)) return srv_fail(FABM_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    const int k = (int)std::min<size_t>((size_t)max, S->finished.size());
    for (int i = 0; i < k; ++i) tickets[i] = S->finished[i];
    S->finished.erase(S->finished.begin(), S->finished.begin() + k);
    *n = k;
    return FABM_OK;
}

fabm_status fabm_server_stats(const fabm_server *S, int64_t *steps, int64_t *launches,
                              size_t *bytes_in_use)
{
    set_last_error("");
    if (!S) return srv_fail(FABM_EINVAL, "server is NULL");
    if (steps) *steps = S->steps_done;
    if (launches) *launches = S->launches;
    if (bytes_in_use) *bytes_in_use = S->in_use;
    return FABM_OK;
}

fabm_status fabm_server_destroy(fabm_server *S)
{
    set_last_error("");
    if (!S) return FABM_OK;
    const int dev = S->device;
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    delete S;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return FABM_OK;
}

}  // extern "C"
