// a2 + a3 on tensor cores ("split" precision): the hereditary sums of Sec. 2
// of arXiv:1710.01133 over every point before a 64-target block, as bf16
// tcgen05 MMAs that are exact per 64-point segment, accumulated across
// segments in compensated fp32 and combined across CTAs in compensated
// float-float (kept as float-float pairs for the recurrence).  Per block the kernel runs twice:
// over the far segments beside the previous block's recurrence, and over the
// newest segment once that recurrence has finished.
//
// Number format.  Time is cut into segments of kSeg = 64 points (one
// recurrence block each).  For a segment and a column, f is written on a
// fixed-point grid: x = f 2^(8-E) with |x| < 256 (E from the segment's largest
// |f|), then x = s0 + s1 + s2 with s0 an integer, s1 a multiple of 2^-8 and s2
// of 2^-16, each with at most 8 significant bits, i.e. each an exact bf16.
// The weight rows of a segment get the same treatment with one exponent per
// weight kind (the weights are monotone in the distance, so the largest is at
// one end of the tile).  Dropping the products of order >= 3 and the rounding of the
// last slice leave a representation error of at most 2^-25 of the segment's
// largest |f| (and weight).
//
// Exactness.  Level-0 products s0*t0 are integers below 2^16 in magnitude, so
// their sum over the 64 points of a segment (< 2^22) is exact in the fp32
// accumulator whatever order or truncation the tensor core uses.  The other
// five products (levels 1 and 2) go to a second accumulator whose rounding is
// below 2^-32 of the result.  Per segment each value is then v = L0 + L12
// (one fp32 rounding), scaled by 2^(E_f + E_w - 16) (exact) and added with
// Kahan compensation.
//
// Toeplitz weights without an N x N matrix.  Inside a segment the points are
// taken in reverse order j' = 63 - j, which turns the weight tile into a Hankel
// matrix W(D0 + n + j'), D0 = (c - seg) 64 - 62.  A no-swizzle K-major operand
// is a grid of 8x8 core matrices addressed as base + LBO*k1 + SBO*n1; with
// LBO = SBO = 128 bytes, core matrix (n1, k1) is stored once at index n1 + k1,
// so a 64 x 64 weight tile needs 15 core matrices (1920 bytes) per kind and
// slice instead of 8 KB.  These tiles depend only on the lag c - seg and are
// built once per solver.
//
// CTA layout (1 CTA per SM, 384 threads): warp 0 streams segments into a
// 3-stage shared-memory ring with bulk copies; warp 1 issues the MMAs into one
// of two TMEM accumulator sets (512 columns), both weight kinds at once with
// their MMAs interleaved; warps 2..9 drain the other set, each warp one TMEM lane
// quadrant (its columns) and the 64 targets of one kind, with
// Kahan-compensated fp32 sums held in registers.  A warp can only read the
// TMEM lanes of its own sub-partition, so quadrant 1 is drained on the MMA
// warp's sub-partition; there warps 5 and 9 only scale their values into
// shared memory and warps 10 and 11 (other sub-partitions) keep the sums, so
// that the MMA thread keeps its issue slots.  Measured in isolation: the copy
// ring alone streams at the HBM peak, the MMAs alone reach ~0.6 of the bf16
// peak (N = 64 per MMA), the full kernel 0.47-0.53 (0.43-0.49 with the whole
// drain on the MMA warp's sub-partition).  An M = 128, N = 64, K = 16 MMA
// reads 6 KB of operands from shared memory, which at the 128 B per clock an
// SM delivers takes 48 clocks against 32 of compute (measured: N = 128 takes
// its 64 compute clocks), so this shape caps at ~0.67 of the tensor pipe; the
// 128-target kernel (history_far.cu) is the fast path for long histories.
// Every wait is bounded; on timeout the CTA sets an error flag, waits for its
// own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>


#include "fabm_internal.cuh"
#include "sm100_ptx.cuh"

namespace fabm {
namespace {

using namespace ptx;

constexpr int kSeg = kSplitSeg;      // 64 points per segment = targets per block
constexpr int kMC = 128;             // columns per CTA (TMEM lanes)
constexpr int kStages = 3;
constexpr int kHk = 15;              // Hankel core matrices per (kind, slice)
constexpr int kFBytes = 3 * kMC * kSeg * 2;          // 49152: 3 slices of 128 x 64 bf16
constexpr int kWBytes = 2 * 3 * kHk * 128;           // 11520
constexpr int kStageStride = 61440;                  // F + W, padded to 1 KB
// warp 0: copies, warp 1: MMAs, warps 2..9: drain (warps 5 and 9, on the MMA
// warp's sub-partition, only move their values to shared memory), warps 10 and
// 11: the Kahan sums of warps 5 and 9
constexpr int kThreads = 384;
constexpr int kEpiWarps = 8;
constexpr int kEpiT = 64;         // targets per drain thread
constexpr int kStashBytes = 2 * 2 * kEpiT * 32 * 4;  // [buffer][kind][target][column]
constexpr size_t kSmemBytes = (size_t)kStages * kStageStride + 1024 + kStashBytes;
// limit of the waits that wait for the rest of the CTA (launch parameter,
// default ~2 s at 2 GHz); waits for the CTA's own copies and MMAs to land,
// which always complete, keep the default
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ int exp_clamp(int e) { return e < -126 ? -126 : (e > 127 ? 127 : e); }
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((exp_clamp(e) + 127) << 23); }

// --------------------------------------------------------- f slicing ---

// f of segment `seg` (points seg*64 .. seg*64+63) -> three bf16 slices in the
// operand layout [seg][ct][slice][k1 = j'/8][col 128][j'%8], j' = 63 - j, and
// the exponent E per column in Ef[seg][ct][col].  On this path the recurrence
// stores f as float-float pairs (hi, lo).  grid = cols_pad/32, block = 256 =
// 32 columns x 8 groups of 8 points.
__global__ void __launch_bounds__(256) slice_f_kernel(const float2 *__restrict__ F, int64_t ldF,
                                                      int64_t n_rows, int cols, int n_ct,
                                                      int64_t seg,
                                                      __nv_bfloat16 *__restrict__ Fs,
                                                      int *__restrict__ Ef)
{
    __shared__ float smax[8][32];
    const int cl = threadIdx.x % 32, k1 = threadIdx.x / 32;
    const int col = blockIdx.x * 32 + cl;
    float hi[8], lo[8];
    float m = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < 8; ++k0) {
        const int j = 63 - (8 * k1 + k0);
        const int64_t row = seg * kSeg + j;
        const float2 f = (col < cols && row < n_rows) ? F[row * ldF + col] : make_float2(0.f, 0.f);
        hi[k0] = f.x;
        lo[k0] = f.y;
        m = fmaxf(m, fabsf(hi[k0]));
    }
    smax[k1][cl] = m;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) m = fmaxf(m, smax[i][cl]);
    int E = 0;
    if (m > 0.f && m <= 3.0e38f) E = ilogbf(m) + 1;
    if (E < -100) E = -100;
    const float sc = pow2f(8 - E);
    uint32_t w[3][4];
#pragma unroll
    for (int k0 = 0; k0 < 8; k0 += 2) {
        float t[3][2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float xh = hi[k0 + u] * sc, xl = lo[k0 + u] * sc;
            const float t0 = rintf(xh);
            const float r = ((xh - t0) + xl) * 256.f;
            const float t1 = rintf(r);
            const float t2 = rintf((r - t1) * 256.f);
            t[0][u] = t0, t[1][u] = t1 * 0x1p-8f, t[2][u] = t2 * 0x1p-16f;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            __nv_bfloat162 p = __floats2bfloat162_rn(t[q][0], t[q][1]);
            w[q][k0 / 2] = *reinterpret_cast<uint32_t *>(&p);
        }
    }
    const int ct = col / kMC, cloc = col % kMC;
    if (col < n_ct * kMC) {
        __nv_bfloat16 *base = Fs + ((seg * n_ct + ct) * 3) * (int64_t)(kMC * kSeg);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            *reinterpret_cast<uint4 *>(base + q * (kMC * kSeg) + k1 * (kMC * 8) + cloc * 8) =
                make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
        if (k1 == 0) Ef[(seg * n_ct + ct) * kMC + cloc] = E;
    }
}

// ------------------------------------------------- Hankel weight tiles ---

// For every lag g in [1, g_max]: D0 = 64 g - 62, exponent E_w = ilogb of the
// tile's largest weight + 1 per kind, and the Hankel core matrices of the three
// slices of W(D0 + t), t = 8h + r0 + c0.  WH[g][kind][slice][h][r0][c0];
// Ew[g][kind].  Lag 1 (distances 2..128) serves the newest segment.
// One thread per (g, kind, h, r0) row.
__global__ void hankel_weights_kernel(const double *__restrict__ WB, const double *__restrict__ WA,
                                      int64_t g_max, __nv_bfloat16 *__restrict__ WH,
                                      int *__restrict__ Ew)
{
    const int64_t rows = (g_max + 1) * 2 * kHk * 8;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int r0 = (int)(r % 8), h = (int)((r / 8) % kHk), kind = (int)((r / (8 * kHk)) % 2);
        const int64_t g = r / (8 * kHk * 2);
        if (g < 1) continue;
        const double *W = kind ? WA : WB;
        const int64_t D0 = 64 * g - 62;
        // the tile spans the distances D0 .. D0+126; the weights are monotone in
        // the distance (decreasing for alpha < 1, increasing for alpha > 1), so
        // the largest sits at one end
        const int E = ilogb(fmax(W[D0], W[D0 + 126])) + 1;
        if (h == 0 && r0 == 0) Ew[g * 2 + kind] = E;
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
        __nv_bfloat16 *base = WH + g * (kWBytes / 2) + (int64_t)kind * 3 * kHk * 64;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            *reinterpret_cast<uint4 *>(base + q * kHk * 64 + h * 64 + r0 * 8) =
                make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

// --------------------------------------------------- the tensor kernel ---

struct SplitArgs {
    const __nv_bfloat16 *Fs;  // [seg][ct][3][8][128][8]
    const int *Ef;            // [seg][ct][128]
    const __nv_bfloat16 *WH;  // [g][2][3][15][8][8]
    const int *Ew;            // [g][2]
    int64_t c;                // target block: m = 64c+1 .. 64c+64
    int n_ct;
    int cols;
    int seg0;                 // segments seg0 .. seg0+n_seg-1
    int n_seg;
    int chunk0;               // CTA row y writes partial chunk chunk0 + y
    int n_chunks;             // gridDim.y
    float2 *part;             // [chunk][2][64][cols] (sum, -compensation)
    unsigned int *err;
    long long wait;           // clock cycles a wait on another warp may take
};

__global__ void __launch_bounds__(kThreads, 1) hist_split_kernel(const SplitArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageStride);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;  // [buffer][kind]
    uint64_t *acc_empty = acc_full + 4;    // [buffer][kind]
    uint64_t *done = acc_empty + 4;
    uint64_t *stash_full = done + 1;         // [buffer][kind]
    uint64_t *stash_empty = stash_full + 4;  // [buffer][kind]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(stash_empty + 4);
    float *stash = reinterpret_cast<float *>(smem + kStages * kStageStride + 1024);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int ct = blockIdx.x, ch = blockIdx.y;
    const int s_lo = a.seg0 + (int)((int64_t)ch * a.n_seg / a.n_chunks);
    const int s_hi = a.seg0 + (int)((int64_t)(ch + 1) * a.n_seg / a.n_chunks);
    const int nseg = s_hi - s_lo;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1), mbar_init(&empty[i], 1);
        for (int i = 0; i < 4; ++i) mbar_init(&acc_full[i], 1), mbar_init(&acc_empty[i], kEpiWarps / 2);
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
            int issued = 0;
            for (int i = 0; i < nseg && ok; ++i) {
                const int st = i % kStages;
                const uint32_t ph = (i / kStages) & 1;
                if (!mbar_wait(&empty[st], ph ^ 1, a.wait)) {
                    ok = false;
                    break;
                }
                const int64_t seg = s_lo + i;
                const int64_t g = a.c - seg;
                uint8_t *dst = smem + st * kStageStride;
                mbar_arrive_expect_tx(&full[st], kFBytes + kWBytes);
                bulk_g2s(dst, a.Fs + (seg * a.n_ct + ct) * (int64_t)(kFBytes / 2), kFBytes, &full[st]);
                bulk_g2s(dst + kFBytes, a.WH + g * (int64_t)(kWBytes / 2), kWBytes, &full[st]);
                issued = i + 1;
            }
            // copies still in flight complete their stage's phase: wait for them
            for (int i = (issued > kStages ? issued - kStages : 0); i < issued; ++i)
                mbar_wait(&full[i % kStages], (i / kStages) & 1, kWaitCycles);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kMC, kSeg);
            for (int i = 0; i < nseg && ok; ++i) {
                const int st = i % kStages;
                const uint32_t ph = (i / kStages) & 1;
                const int b = i & 1;
                const uint32_t bph = (i >> 1) & 1;
                if (!mbar_wait(&full[st], ph, a.wait)) {
                    ok = false;
                    break;
                }
                const uint32_t sF = smem_u32(smem + st * kStageStride);
                const uint32_t sW = sF + kFBytes;
                // both kinds at once, their dependent MMAs interleaved (see
                // mma_bf16_split6x2); the drain of this buffer runs during the
                // next segment's MMAs, which use the other buffer
                if (!mbar_wait(&acc_empty[b * 2], bph ^ 1, a.wait) ||
                    !mbar_wait(&acc_empty[b * 2 + 1], bph ^ 1, a.wait)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + b * 256;  // level 0, kind 0 (kind 1: +64)
                const uint32_t d12 = d0 + 128;       // levels 1 and 2
                // descriptors as base word + offset/16: few instructions per
                // MMA, since this thread shares its issue slots with two drain
                // warps
                const uint32_t a_lo = smem_desc_lo(sF, 2048);
                const uint32_t b_lo = smem_desc_lo(sW, 128);
                constexpr uint32_t a_hi = smem_desc_hi(128), b_hi = smem_desc_hi(128);
                constexpr uint32_t fq = (kFBytes / 3) >> 4, wq = (kHk * 128) >> 4;
                constexpr uint32_t kq = (3 * kHk * 128) >> 4;  // kind 1's weight tiles
#pragma unroll
                for (int s = 0; s < kSeg / 16; ++s) {
                    const uint32_t ao = a_lo + s * (4096 >> 4), bo = b_lo + s * (256 >> 4);
                    mma_bf16_split6x2(d0, d12, d0 + 64, d12 + 64, desc_join(ao, a_hi),
                                      desc_join(ao + fq, a_hi), desc_join(ao + 2 * fq, a_hi),
                                      desc_join(bo, b_hi), desc_join(bo + wq, b_hi),
                                      desc_join(bo + 2 * wq, b_hi), desc_join(bo + kq, b_hi),
                                      desc_join(bo + kq + wq, b_hi),
                                      desc_join(bo + kq + 2 * wq, b_hi), idesc, s == 0);
                }
                mma_commit(&acc_full[b * 2]);
                mma_commit(&acc_full[b * 2 + 1]);
                mma_commit(&empty[st]);
            }
            mma_commit(done);
            if (!mbar_wait(done, 0, kWaitCycles)) ok = false;
        }
    } else if (warp < 10 && warp % 4 == 1) {
        // light drain of TMEM quadrant 1 (the MMA warp's sub-partition): scale
        // the values and hand them to warp 10 or 11 through shared memory
        const int kind = (warp - 2) / 4;
        const int cloc = 32 + lane;
        int ef_next = a.Ef[((int64_t)s_lo * a.n_ct + ct) * kMC + cloc];
        int ew_next = a.Ew[(a.c - s_lo) * 2 + kind];
        for (int i = 0; i < nseg; ++i) {
            const int b = i & 1;
            const uint32_t bph = (i >> 1) & 1;
            const float scale = pow2f(ef_next + ew_next - 16);
            if (i + 1 < nseg) {
                const int64_t sn = s_lo + i + 1;
                ef_next = a.Ef[(sn * a.n_ct + ct) * kMC + cloc];
                ew_next = a.Ew[(a.c - sn) * 2 + kind];
            }
            if (!mbar_wait(&acc_full[b * 2 + kind], bph, a.wait) ||
                !mbar_wait(&stash_empty[b * 2 + kind], bph ^ 1, a.wait)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t base = tmem + (32u << 16) + b * 256 + kind * 64;
            float *st = stash + (b * 2 + kind) * kEpiT * 32 + lane;
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
                mbar_arrive(&acc_empty[b * 2 + kind]);
                mbar_arrive(&stash_full[b * 2 + kind]);
            }
        }
    } else {
        // drain: warps 2..9 read TMEM lanes 32*(w%4).. (their columns) and the
        // 64 targets of one kind; warps 10 and 11 take quadrant 1's values from
        // shared memory.  Kahan sums in fp32; the compensation terms are kept as
        // packed bf16 pairs (fp32's exponent range, 2^-9 relative error on a term
        // that is itself below half an ulp of the sum).
        const bool helper = warp >= 10;
        const int q = helper ? 1 : warp % 4, kind = helper ? warp - 10 : (warp - 2) / 4;
        const int cloc = q * 32 + lane;
        const int64_t col = (int64_t)ct * kMC + cloc;
        float sum[kEpiT];
        uint32_t cmp2[kEpiT / 2];
#pragma unroll
        for (int t = 0; t < kEpiT; ++t) sum[t] = 0.f;
#pragma unroll
        for (int t = 0; t < kEpiT / 2; ++t) cmp2[t] = 0u;
        // Kahan step for targets t, t+1 with the scaled values v0, v1
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
            for (int i = 0; i < nseg; ++i) {
                const int b = i & 1;
                const uint32_t bph = (i >> 1) & 1;
                if (!mbar_wait(&stash_full[b * 2 + kind], bph, a.wait)) {
                    ok = false;
                    break;
                }
                const float *st = stash + (b * 2 + kind) * kEpiT * 32 + lane;
#pragma unroll
                for (int t = 0; t < kEpiT; t += 2) add2(t, st[t * 32], st[(t + 1) * 32]);
                __syncwarp();
                if (lane == 0) mbar_arrive(&stash_empty[b * 2 + kind]);
            }
        } else {
            // exponents of the first segment; later ones are fetched a segment ahead
            int ef_next = a.Ef[((int64_t)s_lo * a.n_ct + ct) * kMC + cloc];
            int ew_next = a.Ew[(a.c - s_lo) * 2 + kind];
            for (int i = 0; i < nseg; ++i) {
                const int b = i & 1;
                const uint32_t bph = (i >> 1) & 1;
                const float scale = pow2f(ef_next + ew_next - 16);
                if (i + 1 < nseg) {
                    const int64_t sn = s_lo + i + 1;
                    ef_next = a.Ef[(sn * a.n_ct + ct) * kMC + cloc];
                    ew_next = a.Ew[(a.c - sn) * 2 + kind];
                }
                if (!mbar_wait(&acc_full[b * 2 + kind], bph, a.wait)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + b * 256 + kind * 64;
                // software pipeline over 8 pieces of 8 targets: the load of piece
                // p+1 is in flight while piece p is added
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
                if (lane == 0) mbar_arrive(&acc_empty[b * 2 + kind]);
            }
        }
        if (ok && col < a.cols) {
            float2 *out = a.part + ((int64_t)((a.chunk0 + ch) * 2 + kind) * kSeg) * a.cols + col;
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

// float-float (hi, lo) += (x, y): two-sum of the high parts, low parts folded
// in, renormalized.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float x, float y)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (x - bb);
    lo += e + y;
    hi = s + lo;
    lo = lo - (hi - s);
}

// a3: G[kind][t][col] = sum over chunks of the float-float partials, R lanes
// per output, each summing chunks r, r+R, ... in ascending order (four loads
// in flight), then a fixed xor tree, in compensated float-float (~48 bits,
// 2^24 finer than the fp32 partials).  Out = float2 (tensor path) keeps the
// pair; Out = double (compensated-fp32 history) rounds hi + lo once.  The
// combine sits on the serial chain of every block and FP64 issues at 1/64 of
// the fp32 rate on this part, so the accumulation stays in fp32 pairs.  Every
// thread runs the same number of rounds, so the shuffles always see full warps.
template <int R, class Out>
__global__ void combine_split_kernel(const float2 *__restrict__ part, int n_chunks, int64_t n_out,
                                     Out *__restrict__ G)
{
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = (int)(gtid % R);
    const int64_t groups = (int64_t)gridDim.x * blockDim.x / R;
    for (int64_t base = 0; base < n_out; base += groups) {
        const int64_t o = base + gtid / R;
        float hi = 0.f, lo = 0.f;
        if (o < n_out) {
            int ch = r;
            for (; ch + 3 * R < n_chunks; ch += 4 * R) {
                const float2 v0 = part[(int64_t)ch * n_out + o];
                const float2 v1 = part[(int64_t)(ch + R) * n_out + o];
                const float2 v2 = part[(int64_t)(ch + 2 * R) * n_out + o];
                const float2 v3 = part[(int64_t)(ch + 3 * R) * n_out + o];
                ff_add(hi, lo, v0.x, v0.y);
                ff_add(hi, lo, v1.x, v1.y);
                ff_add(hi, lo, v2.x, v2.y);
                ff_add(hi, lo, v3.x, v3.y);
            }
            for (; ch < n_chunks; ch += R) {
                const float2 v = part[(int64_t)ch * n_out + o];
                ff_add(hi, lo, v.x, v.y);
            }
        }
#pragma unroll
        for (int off = R / 2; off > 0; off >>= 1) {
            const float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
            const float olo = __shfl_xor_sync(0xffffffffu, lo, off);
            ff_add(hi, lo, ohi, olo);
        }
        if (r == 0 && o < n_out) {
            if constexpr (std::is_same_v<Out, double>)
                G[o] = (double)hi + (double)lo;
            else
                G[o] = make_float2(hi, lo);  // normalised by ff_add
        }
    }
}

}  // namespace

cudaError_t launch_slice_f(const DevBatch &bt, int n_ct, int64_t seg, __nv_bfloat16 *Fs, int *Ef,
                           cudaStream_t st)
{
    const unsigned blocks = (unsigned)(n_ct * kMC / 32);
    slice_f_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const float2 *>(bt.F), bt.ldF,
                                           bt.N + 1, bt.cols, n_ct, seg, Fs, Ef);
    return cudaGetLastError();
}

cudaError_t launch_hankel_weights(const double *WB, const double *WA, int64_t g_max,
                                  __nv_bfloat16 *WH, int *Ew, cudaStream_t st)
{
    const int64_t rows = (g_max + 1) * 2 * kHk * 8;
    int64_t blocks = (rows + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    hankel_weights_kernel<<<(unsigned)blocks, 256, 0, st>>>(WB, WA, g_max, WH, Ew);
    return cudaGetLastError();
}

cudaError_t prepare_hist_split()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, hist_split_kernel);
    if (e != cudaSuccess) return e;
    if (fa.numRegs * kThreads > 65536) return cudaErrorInvalidConfiguration;
    return cudaFuncSetAttribute(hist_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemBytes);
}

size_t split_part_elems(int n_chunks, int cols) { return (size_t)n_chunks * 2 * kSeg * cols; }

cudaError_t launch_hist_split(const __nv_bfloat16 *Fs, const int *Ef, const __nv_bfloat16 *WH,
                              const int *Ew, int64_t c, int seg0, int n_seg, int chunk0,
                              int n_chunks, int n_ct, int cols, float2 *part, unsigned int *err,
                              long long wait_cycles, cudaStream_t st)
{
    if (n_seg < 1) return cudaSuccess;
    if (wait_cycles <= 0) wait_cycles = kWaitCycles;
    // segments lie before block c: lag g = c - seg >= 1
    if (seg0 < 0 || seg0 + n_seg > c || n_chunks < 1 || n_chunks > n_seg || chunk0 < 0)
        return cudaErrorInvalidValue;
    SplitArgs a{Fs, Ef, WH, Ew, c, n_ct, cols, seg0, n_seg, chunk0, n_chunks, part, err, wait_cycles};
    hist_split_kernel<<<dim3((unsigned)n_ct, (unsigned)n_chunks), kThreads, kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

template <class Out>
cudaError_t launch_combine_t(const float2 *part, int n_chunks, int cols, int L, Out *G,
                             cudaStream_t st)
{
    const int64_t n_out = 2LL * L * cols;
    const int threads = 128;
    auto blocks_for = [&](int R) {
        int64_t b = (n_out * R + threads - 1) / threads;
        return (unsigned)(b > 152 * 16 ? 152 * 16 : b);
    };
    if (n_chunks >= 256)
        combine_split_kernel<32, Out><<<blocks_for(32), threads, 0, st>>>(part, n_chunks, n_out, G);
    else if (n_chunks >= 32)
        combine_split_kernel<8, Out><<<blocks_for(8), threads, 0, st>>>(part, n_chunks, n_out, G);
    else
        combine_split_kernel<1, Out><<<blocks_for(1), threads, 0, st>>>(part, n_chunks, n_out, G);
    return cudaGetLastError();
}

cudaError_t launch_combine_split(const float2 *part, int n_chunks, int cols, int L, double *G,
                                 cudaStream_t st)
{
    return launch_combine_t(part, n_chunks, cols, L, G, st);
}

cudaError_t launch_combine_split_ff(const float2 *part, int n_chunks, int cols, int L,
                                    float2 *G, cudaStream_t st)
{
    return launch_combine_t(part, n_chunks, cols, L, G, st);
}

namespace {
__global__ void ff_weights_kernel(const double *__restrict__ W, double scale, int64_t n,
                                  float2 *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = scale * W[i];
        const float hi = __double2float_rn(v);
        out[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}
}  // namespace

cudaError_t launch_ff_weights(const double *W, double scale, int64_t n, float2 *out,
                              cudaStream_t st)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) return cudaSuccess;
    ff_weights_kernel<<<(unsigned)blocks, 256, 0, st>>>(W, scale, n, out);
    return cudaGetLastError();
}

}  // namespace fabm
