// a2 + a3 on tensor cores for pairs of blocks ("wide" far history): the
// hereditary sums of Sec. 2 of arXiv:1710.01133 over every point before a
// group of 128 targets (two 64-step blocks of the recurrence), with 128
// targets per MMA and one weight kind per CTA.
//
// Why 128 targets.  Per 64-point slice of f (48 KB for 128 columns) the
// 64-target kernel (history_split.cu) does 6 products x 2 kinds x 64 x 64 x
// 128 multiply-adds: 256 bf16 flops per HBM byte, under the 279 flop/byte at
// which HBM and the tensor pipe balance on this part, so it cannot exceed
// ~0.7 of the tensor peak however it is scheduled.  With 128 targets every
// byte of f feeds twice the products.  TMEM then holds one kind only (level-0
// and level-1/2 accumulators of 128 columns each, double-buffered: 512
// columns), so the two kinds go to two CTAs that read the same slices (the
// second read hits L2).
//
// Number format (as history_split.cu, over 128 points).  A "group" is 128
// consecutive points (two blocks of the recurrence); per group and column, f
// is written on a fixed-point grid x = f 2^(8-E) with |x| < 256 and split into
// three bf16 terms s0 + s1 + s2 (integer, multiples of 2^-8 and of 2^-16);
// the weight tile of a group gets the same treatment with one exponent per
// kind.  Level-0 products are integers below 2^16, so their sum over the 128
// points of a group (< 2^23) is exact in the fp32 accumulator; the five other
// products go to a second accumulator.  Per group each value is L0 + L12,
// scaled by 2^(E_f + E_w - 16) and added with Kahan compensation.
// Representation error: at most 2^-25 of the group's largest |f| and weight.
//
// Toeplitz weights.  For the target group C (m = 128C+1 .. 128C+128) and the
// point group S <= C-2, with the points in reverse order j' = 127 - j, the
// weights form the Hankel tile W(128 (C-S) - 126 + n + j'), n, j' < 128, whose
// 8x8 core matrices (n1, k1) depend on n1 + k1 only: 31 per kind and slice,
// read with LBO = SBO = 128 bytes (11.6 KB per kind and lag instead of 96 KB).
//
// CTA (1 per SM, 384 threads): warp 0 streams half-groups (64 points: 48 KB of
// slices plus the 11.6 KB weight tile) into a 3-stage ring with bulk copies;
// warp 1 issues the MMAs (M = 128 columns, N = 128 targets, K = 16) into one
// of two accumulator buffers; warps 2..9 drain the other buffer, warp w
// reading the TMEM lanes of its sub-partition (columns 32 (w % 4) ..) for 64
// of the 128 targets; on the MMA warp's sub-partition (quadrant 1) warps 5 and
// 9 only scale their values into shared memory and warps 10 and 11 keep the
// Kahan sums.  Shared memory delivers 128 bytes per clock per SM: an MMA of
// this shape reads 8 KB of operands in its 64 compute clocks, exactly that
// rate (measured: 64 clocks per MMA, dependent MMAs pipelined), and the bulk
// copies write ~39 bytes per clock of MMA time into the same memory, so the
// kernel is bound by shared-memory bandwidth at ~0.8 of the tensor pipe.
// Every wait on another warp is bounded by a launch parameter; on timeout the
// CTA sets the error word, waits for its own copies and MMAs, frees TMEM and
// returns.
#include <cuda_bf16.h>

#include "fabm_internal.cuh"
#include "sm100_ptx.cuh"

namespace fabm {
namespace {

using namespace ptx;

constexpr int kGrp = 128;           // points per group = targets per launch row
constexpr int kHalf = 64;           // points per pipeline stage
constexpr int kMC = 128;            // columns per CTA (TMEM lanes)
constexpr int kStages = 3;
constexpr int kHk = 31;             // Hankel core matrices per (kind, slice)
constexpr int kFHalfBytes = 3 * kMC * kHalf * 2;     // 49152: 3 slices x 128 cols x 64 points
constexpr int kWTileBytes = 3 * kHk * 128;           // 11904: one kind's tile, 3 slices
constexpr int kStageStride = 61440;                  // F half + W tile, padded to 1 KB
constexpr int kThreads = 384;
constexpr int kEpiT = 64;                            // targets per drain thread
constexpr int kStashBytes = 2 * 2 * kEpiT * 32 * 4;  // [buffer][target half][target][lane]
constexpr size_t kSmemBytes = (size_t)kStages * kStageStride + 1024 + kStashBytes;
constexpr long long kWaitCycles = 4000000000LL;      // default wait limit (~2 s at 2 GHz)

static_assert(kFHalfBytes + kWTileBytes <= kStageStride, "stage layout");
static_assert(kWTileBytes % 16 == 0 && kFHalfBytes % 16 == 0, "bulk copies move 16-byte units");

__device__ __forceinline__ int exp_clamp(int e) { return e < -126 ? -126 : (e > 127 ? 127 : e); }
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((exp_clamp(e) + 127) << 23); }

// x (|x| < 256 after scaling) -> the three bf16-exact terms of the split.
__device__ __forceinline__ void split3(float xh, float xl, float &t0, float &t1, float &t2)
{
    t0 = rintf(xh);
    const float r = ((xh - t0) + xl) * 256.f;
    const float u1 = rintf(r);
    t1 = u1 * 0x1p-8f;
    t2 = rintf((r - u1) * 256.f) * 0x1p-16f;
}

// f of group S (points 128S .. 128S+127, float-float pairs) -> slices in the
// layout [S][ct][half][slice][k1 8][col 128][k0 8] with j' = 127 - j =
// 64 half + 8 k1 + k0, and the exponent per column in Ef[S][ct][col].
// grid = cols_pad/32, block = 256 = 32 columns x 8 groups of 16 points.
__global__ void __launch_bounds__(256) slice_group_kernel(const float2 *__restrict__ F, int64_t ldF,
                                                          int64_t n_rows, int cols, int n_ct,
                                                          int64_t S,
                                                          __nv_bfloat16 *__restrict__ Fs,
                                                          int *__restrict__ Ef)
{
    __shared__ float smax[8][32];
    const int cl = threadIdx.x % 32, k1 = threadIdx.x / 32;
    const int col = blockIdx.x * 32 + cl;
    float hi[2][8], lo[2][8];
    float m = 0.f;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)
#pragma unroll
        for (int k0 = 0; k0 < 8; ++k0) {
            const int j = 127 - (64 * hf + 8 * k1 + k0);
            const int64_t row = S * kGrp + j;
            const float2 f = (col < cols && row < n_rows) ? F[row * ldF + col] : make_float2(0.f, 0.f);
            hi[hf][k0] = f.x;
            lo[hf][k0] = f.y;
            m = fmaxf(m, fabsf(f.x));
        }
    smax[k1][cl] = m;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) m = fmaxf(m, smax[i][cl]);
    int E = 0;
    if (m > 0.f && m <= 3.0e38f) E = ilogbf(m) + 1;
    if (E < -100) E = -100;
    const float sc = pow2f(8 - E);
    const int ct = col / kMC, cloc = col % kMC;
    if (col >= n_ct * kMC) return;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
        uint32_t w[3][4];
#pragma unroll
        for (int k0 = 0; k0 < 8; k0 += 2) {
            float t[3][2];
#pragma unroll
            for (int u = 0; u < 2; ++u)
                split3(hi[hf][k0 + u] * sc, lo[hf][k0 + u] * sc, t[0][u], t[1][u], t[2][u]);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                __nv_bfloat162 p = __floats2bfloat162_rn(t[q][0], t[q][1]);
                w[q][k0 / 2] = *reinterpret_cast<uint32_t *>(&p);
            }
        }
        __nv_bfloat16 *base = Fs + (((S * n_ct + ct) * 2 + hf) * 3) * (int64_t)(kMC * kHalf);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            *reinterpret_cast<uint4 *>(base + q * (kMC * kHalf) + k1 * (kMC * 8) + cloc * 8) =
                make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
    if (k1 == 0) Ef[(S * n_ct + ct) * kMC + cloc] = E;
}

// For every group lag G in [2, G_max]: D0 = 128 G - 126 (the tile spans the
// distances D0 .. D0 + 254), exponent E_w per kind from the tile's largest
// weight (weights are monotone in the distance, so at one end), and the
// Hankel core matrices of the three slices of W(D0 + t), t = 8h + r0 + c0.
// Layout WH[G][kind][slice][h 31][r0 8][c0 8]; Ew[G][kind].  One thread per
// (G, kind, h, r0) row.
__global__ void hankel_group_kernel(const double *__restrict__ WB, const double *__restrict__ WA,
                                    int64_t G_max, __nv_bfloat16 *__restrict__ WH,
                                    int *__restrict__ Ew)
{
    const int64_t rows = (G_max + 1) * 2 * kHk * 8;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int r0 = (int)(r % 8), h = (int)((r / 8) % kHk), kind = (int)((r / (8 * kHk)) % 2);
        const int64_t G = r / (8 * kHk * 2);
        if (G < 2) continue;
        const double *W = kind ? WA : WB;
        const int64_t D0 = 128 * G - 126;
        const int E = ilogb(fmax(W[D0], W[D0 + 254])) + 1;
        if (h == 0 && r0 == 0) Ew[G * 2 + kind] = E;
        const double sc = ldexp(1.0, 8 - E);
        uint32_t w[3][4];
#pragma unroll
        for (int c0 = 0; c0 < 8; c0 += 2) {
            float t[3][2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const double x = W[D0 + 8 * h + r0 + c0 + u] * sc;
                const double t0 = rint(x);
                const double rr = (x - t0) * 256.0;
                const double t1 = rint(rr);
                const double t2 = rint((rr - t1) * 256.0);
                t[0][u] = (float)t0, t[1][u] = (float)(t1 * 0x1p-8), t[2][u] = (float)(t2 * 0x1p-16);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                __nv_bfloat162 p = __floats2bfloat162_rn(t[q][0], t[q][1]);
                w[q][c0 / 2] = *reinterpret_cast<uint32_t *>(&p);
            }
        }
        __nv_bfloat16 *base = WH + (G * 2 + kind) * (int64_t)(kWTileBytes / 2);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            *reinterpret_cast<uint4 *>(base + q * kHk * 64 + h * 64 + r0 * 8) =
                make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

struct FarArgs {
    const __nv_bfloat16 *Fs;  // [S][ct][2][3][8][128][8]
    const int *Ef;            // [S][ct][128]
    const __nv_bfloat16 *WH;  // [G][2][3][31][8][8]
    const int *Ew;            // [G][2]
    int64_t C;                // target group: m = 128C+1 .. 128C+128
    int n_ct;
    int cols;
    int n_grp;                // point groups 0 .. n_grp-1 (n_grp <= C-1)
    int n_chunks;             // gridDim.y
    float2 *part;             // [chunk][2][128][cols] (sum, -compensation)
    unsigned int *err;
    long long wait;           // clock cycles a wait on another warp may take
};

// One MMA K step of one kind: a0*b0 into d0 (accumulating unless `first`);
// a0*b1, a1*b0, a0*b2, a1*b1, a2*b0 into d12.
__device__ __forceinline__ void mma_split6(uint32_t d0, uint32_t d12, uint64_t a0, uint64_t a1,
                                           uint64_t a2, uint64_t b0, uint64_t b1, uint64_t b2,
                                           uint32_t idesc, uint32_t first)
{
    asm volatile(
        "{\n .reg .pred pa, pt;\n"
        " setp.eq.b32 pa, %9, 0;\n"
        " setp.eq.b32 pt, %9, %9;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %5, %8, pa;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %6, %8, pa;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %3, %5, %8, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %7, %8, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %3, %6, %8, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %5, %8, pt;\n}\n" ::"r"(d0),
        "r"(d12), "l"(a0), "l"(a1), "l"(a2), "l"(b0), "l"(b1), "l"(b2), "r"(idesc), "r"(first)
        : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) hist_far_kernel(const FarArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageStride);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;  // [buffer]
    uint64_t *acc_empty = acc_full + 2;    // [buffer]
    uint64_t *done = acc_empty + 2;
    uint64_t *stash_full = done + 1;         // [buffer][target half]
    uint64_t *stash_empty = stash_full + 4;  // [buffer][target half]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(stash_empty + 4);
    float *stash = reinterpret_cast<float *>(smem + kStages * kStageStride + 1024);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int kind = blockIdx.x & 1, ct = blockIdx.x >> 1, ch = blockIdx.y;
    const int g_lo = (int)((int64_t)ch * a.n_grp / a.n_chunks);
    const int g_hi = (int)((int64_t)(ch + 1) * a.n_grp / a.n_chunks);
    const int ngrp = g_hi - g_lo;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1), mbar_init(&empty[i], 1);
        // acc_empty: the 6 drain warps of the buffer's targets (2 x 3: the
        // quadrants 0, 2, 3 per target half) plus the 2 light drain warps
        for (int i = 0; i < 2; ++i) mbar_init(&acc_full[i], 1), mbar_init(&acc_empty[i], 8);
        mbar_init(done, 1);
        for (int i = 0; i < 4; ++i) mbar_init(&stash_full[i], 1), mbar_init(&stash_empty[i], 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            // stage t = 2 i + half of group g_lo + i
            const int n_st = 2 * ngrp;
            int issued = 0;
            for (int t = 0; t < n_st && ok; ++t) {
                const int st = t % kStages;
                const uint32_t ph = (t / kStages) & 1;
                if (!mbar_wait(&empty[st], ph ^ 1, a.wait)) {
                    ok = false;
                    break;
                }
                const int64_t S = g_lo + t / 2;
                const int hf = t & 1;
                const int64_t G = a.C - S;
                uint8_t *dst = smem + st * kStageStride;
                mbar_arrive_expect_tx(&full[st], kFHalfBytes + kWTileBytes);
                bulk_g2s(dst, a.Fs + ((S * a.n_ct + ct) * 2 + hf) * (int64_t)(kFHalfBytes / 2),
                         kFHalfBytes, &full[st]);
                bulk_g2s(dst + kFHalfBytes, a.WH + (G * 2 + kind) * (int64_t)(kWTileBytes / 2),
                         kWTileBytes, &full[st]);
                issued = t + 1;
            }
            // copies still in flight complete their stage's phase: wait for them
            for (int t = (issued > kStages ? issued - kStages : 0); t < issued; ++t)
                mbar_wait(&full[t % kStages], (t / kStages) & 1, kWaitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kMC, kGrp);
            for (int i = 0; i < ngrp && ok; ++i) {
                const int b = i & 1;
                const uint32_t bph = (i >> 1) & 1;
                if (!mbar_wait(&acc_empty[b], bph ^ 1, a.wait)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + b * 256;  // level 0
                const uint32_t d12 = d0 + 128;       // levels 1 and 2
                for (int hf = 0; hf < 2; ++hf) {
                    const int t = 2 * i + hf;
                    const int st = t % kStages;
                    if (!mbar_wait(&full[st], (t / kStages) & 1, a.wait)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sF = smem_u32(smem + st * kStageStride);
                    const uint32_t sW = sF + kFHalfBytes;
                    // A: no-swizzle K-major, core matrix (col1, k1) at
                    // 128 col1 + 2048 k1 within a slice; B: the Hankel tile,
                    // (n1, k1) at 128 (n1 + k1), k1 counted over the group
                    const uint32_t a_lo = smem_desc_lo(sF, 2048);
                    const uint32_t b_lo = smem_desc_lo(sW + hf * 8 * 128, 128);
                    constexpr uint32_t a_hi = smem_desc_hi(128), b_hi = smem_desc_hi(128);
                    constexpr uint32_t fq = (kFHalfBytes / 3) >> 4, wq = (kHk * 128) >> 4;
#pragma unroll
                    for (int s = 0; s < kHalf / 16; ++s) {
                        const uint32_t ao = a_lo + s * (4096 >> 4), bo = b_lo + s * (256 >> 4);
                        mma_split6(d0, d12, desc_join(ao, a_hi), desc_join(ao + fq, a_hi),
                                   desc_join(ao + 2 * fq, a_hi), desc_join(bo, b_hi),
                                   desc_join(bo + wq, b_hi), desc_join(bo + 2 * wq, b_hi), idesc,
                                   hf == 0 && s == 0);
                    }
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                mma_commit(&acc_full[b]);
            }
            mma_commit(done);
            if (!mbar_wait(done, 0, kWaitCycles)) ok = false;
        }
    } else if (warp < 10 && warp % 4 == 1) {
        // light drain of TMEM quadrant 1 (the MMA warp's sub-partition): scale
        // the values and hand them to warp 10 or 11 through shared memory
        const int th = (warp - 2) / 4;  // target half
        const int cloc = 32 + lane;
        int ef_next = a.Ef[((int64_t)g_lo * a.n_ct + ct) * kMC + cloc];
        int ew_next = a.Ew[(a.C - g_lo) * 2 + kind];
        for (int i = 0; i < ngrp; ++i) {
            const int b = i & 1;
            const uint32_t bph = (i >> 1) & 1;
            const float scale = pow2f(ef_next + ew_next - 16);
            if (i + 1 < ngrp) {
                const int64_t sn = g_lo + i + 1;
                ef_next = a.Ef[(sn * a.n_ct + ct) * kMC + cloc];
                ew_next = a.Ew[(a.C - sn) * 2 + kind];
            }
            if (!mbar_wait(&acc_full[b], bph, a.wait) ||
                !mbar_wait(&stash_empty[b * 2 + th], bph ^ 1, a.wait)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t base = tmem + (32u << 16) + b * 256 + th * 64;
            float *st = stash + (b * 2 + th) * kEpiT * 32 + lane;
            uint32_t ra[16], rb[16];
            tmem_ld8x2_issue(base, base + 128, ra);
            tmem_wait16(ra);
#pragma unroll
            for (int p = 0; p < kEpiT / 8; ++p) {
                uint32_t(&cur)[16] = (p % 2 == 0) ? ra : rb;
                uint32_t(&nxt)[16] = (p % 2 == 0) ? rb : ra;
                if (p + 1 < kEpiT / 8) tmem_ld8x2_issue(base + (p + 1) * 8, base + 128 + (p + 1) * 8, nxt);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    st[(p * 8 + j) * 32] = (__uint_as_float(cur[j]) + __uint_as_float(cur[8 + j])) * scale;
                if (p + 1 < kEpiT / 8) tmem_wait16(nxt);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&acc_empty[b]);
                mbar_arrive(&stash_full[b * 2 + th]);
            }
        }
    } else {
        // drain: warps 2..9 read TMEM lanes 32 (w % 4) .. (their columns) and
        // the 64 targets of half (w - 2) / 4; warps 10 and 11 take quadrant 1's
        // values from shared memory.  Kahan sums in fp32, compensation terms as
        // packed bf16 pairs.
        const bool helper = warp >= 10;
        const int q = helper ? 1 : warp % 4, th = helper ? warp - 10 : (warp - 2) / 4;
        const int cloc = q * 32 + lane;
        const int64_t col = (int64_t)ct * kMC + cloc;
        float sum[kEpiT];
        uint32_t cmp2[kEpiT / 2];
#pragma unroll
        for (int t = 0; t < kEpiT; ++t) sum[t] = 0.f;
#pragma unroll
        for (int t = 0; t < kEpiT / 2; ++t) cmp2[t] = 0u;
        auto add2 = [&](int t, float v0, float v1) {
            const uint32_t cw = cmp2[t / 2];
            float cnew[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float c = __uint_as_float(u ? (cw & 0xffff0000u) : (cw << 16));
                const float y = (u ? v1 : v0) - c;
                const float s2 = sum[t + u] + y;
                cnew[u] = (s2 - sum[t + u]) - y;
                sum[t + u] = s2;
            }
            __nv_bfloat162 pk = __floats2bfloat162_rn(cnew[0], cnew[1]);
            cmp2[t / 2] = *reinterpret_cast<uint32_t *>(&pk);
        };
        if (helper) {
            for (int i = 0; i < ngrp; ++i) {
                const int b = i & 1;
                const uint32_t bph = (i >> 1) & 1;
                if (!mbar_wait(&stash_full[b * 2 + th], bph, a.wait)) {
                    ok = false;
                    break;
                }
                const float *st = stash + (b * 2 + th) * kEpiT * 32 + lane;
#pragma unroll
                for (int t = 0; t < kEpiT; t += 2) add2(t, st[t * 32], st[(t + 1) * 32]);
                __syncwarp();
                if (lane == 0) mbar_arrive(&stash_empty[b * 2 + th]);
            }
        } else {
            int ef_next = a.Ef[((int64_t)g_lo * a.n_ct + ct) * kMC + cloc];
            int ew_next = a.Ew[(a.C - g_lo) * 2 + kind];
            for (int i = 0; i < ngrp; ++i) {
                const int b = i & 1;
                const uint32_t bph = (i >> 1) & 1;
                const float scale = pow2f(ef_next + ew_next - 16);
                if (i + 1 < ngrp) {
                    const int64_t sn = g_lo + i + 1;
                    ef_next = a.Ef[(sn * a.n_ct + ct) * kMC + cloc];
                    ew_next = a.Ew[(a.C - sn) * 2 + kind];
                }
                if (!mbar_wait(&acc_full[b], bph, a.wait)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + b * 256 + th * 64;
                uint32_t ra[16], rb[16];
                tmem_ld8x2_issue(base, base + 128, ra);
                tmem_wait16(ra);
#pragma unroll
                for (int p = 0; p < kEpiT / 8; ++p) {
                    uint32_t(&cur)[16] = (p % 2 == 0) ? ra : rb;
                    uint32_t(&nxt)[16] = (p % 2 == 0) ? rb : ra;
                    if (p + 1 < kEpiT / 8) tmem_ld8x2_issue(base + (p + 1) * 8, base + 128 + (p + 1) * 8, nxt);
#pragma unroll
                    for (int j = 0; j < 8; j += 2)
                        add2(p * 8 + j,
                             (__uint_as_float(cur[j]) + __uint_as_float(cur[8 + j])) * scale,
                             (__uint_as_float(cur[j + 1]) + __uint_as_float(cur[8 + j + 1])) * scale);
                    if (p + 1 < kEpiT / 8) tmem_wait16(nxt);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[b]);
            }
        }
        if (ok && col < a.cols) {
            float2 *out = a.part + ((int64_t)(ch * 2 + kind) * kGrp + th * kEpiT) * a.cols + col;
#pragma unroll
            for (int t = 0; t < kEpiT; ++t) {
                const uint32_t cw = cmp2[t / 2];
                const float c = __uint_as_float((t & 1) ? (cw & 0xffff0000u) : (cw << 16));
                out[(int64_t)t * a.cols] = make_float2(sum[t], -c);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (!ok) atomicOr(a.err, 1u);
}

// float-float (hi, lo) += (x, y), as history_split.cu.
__device__ __forceinline__ void ff_acc(float &hi, float &lo, float x, float y)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (x - bb);
    lo += e + y;
    hi = s + lo;
    lo = lo - (hi - s);
}

// Sum of the far chunks of one target group: out[kind][t][col] (128 targets)
// = far[.][kind][t][col] over n_far chunks in float-float, chunk order fixed.
// Runs after the far kernel on its stream, so that the recurrence of each of
// the pair's blocks reads one far value per target plus its near partials.
__global__ void sum_far_kernel(const float2 *__restrict__ far, int n_far, int64_t n_out,
                               float2 *__restrict__ out)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out;
         o += (int64_t)gridDim.x * blockDim.x) {
        float hi = 0.f, lo = 0.f;
        for (int ch = 0; ch < n_far; ++ch) {
            const float2 v = far[(int64_t)ch * n_out + o];
            ff_acc(hi, lo, v.x, v.y);
        }
        out[o] = make_float2(hi, lo);
    }
}

}  // namespace

cudaError_t launch_slice_group(const DevBatch &bt, int n_ct, int64_t S, __nv_bfloat16 *Fs, int *Ef,
                               cudaStream_t st)
{
    const unsigned blocks = (unsigned)(n_ct * kMC / 32);
    slice_group_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(bt.F), bt.ldF,
                                               bt.N + 1, bt.cols, n_ct, S, Fs, Ef);
    return cudaGetLastError();
}

cudaError_t launch_hankel_group(const double *WB, const double *WA, int64_t G_max,
                                __nv_bfloat16 *WH, int *Ew, cudaStream_t st)
{
    if (G_max < 2) return cudaSuccess;
    const int64_t rows = (G_max + 1) * 2 * kHk * 8;
    int64_t blocks = (rows + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    hankel_group_kernel<<<(unsigned)blocks, 256, 0, st>>>(WB, WA, G_max, WH, Ew);
    return cudaGetLastError();
}

size_t far_group_tile_elems() { return (size_t)kWTileBytes / 2 * 2; }
size_t far_group_slice_elems() { return (size_t)2 * kFHalfBytes / 2; }

cudaError_t prepare_hist_far()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, hist_far_kernel);
    if (e != cudaSuccess) return e;
    if (fa.numRegs * kThreads > 65536) return cudaErrorInvalidConfiguration;
    return cudaFuncSetAttribute(hist_far_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemBytes);
}

size_t far_part_elems(int n_chunks, int cols) { return (size_t)n_chunks * 2 * kGrp * cols; }

cudaError_t launch_hist_far(const __nv_bfloat16 *Fs, const int *Ef, const __nv_bfloat16 *WH,
                            const int *Ew, int64_t C, int n_grp, int n_chunks, int n_ct, int cols,
                            float2 *part, unsigned int *err, long long wait_cycles,
                            cudaStream_t st)
{
    if (n_grp < 1) return cudaSuccess;
    // point groups lie at least two groups before the target group: lag >= 2
    if (n_grp > C - 1 || n_chunks < 1 || n_chunks > n_grp) return cudaErrorInvalidValue;
    if (wait_cycles <= 0) wait_cycles = kWaitCycles;
    FarArgs a{Fs, Ef, WH, Ew, C, n_ct, cols, n_grp, n_chunks, part, err, wait_cycles};
    hist_far_kernel<<<dim3((unsigned)(2 * n_ct), (unsigned)n_chunks), kThreads, kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sum_far(const float2 *far, int n_far, int cols, float2 *out, cudaStream_t st)
{
    const int64_t n_out = 2LL * kGrp * cols;
    int64_t blocks = (n_out + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    sum_far_kernel<<<(unsigned)blocks, 256, 0, st>>>(far, n_far, n_out, out);
    return cudaGetLastError();
}

}  // namespace fabm
