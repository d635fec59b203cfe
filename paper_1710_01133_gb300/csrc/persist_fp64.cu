// a2 + a3 + a4 + a5 in double as one persistent launch per solve: the whole
// predictor-corrector of Sec. 2 of arXiv:1710.01133 for a narrow batch (a few
// trajectories), with the recurrence of every trajectory and the far history
// sums running side by side in one cooperative launch instead of ~3 launches
// per 32-step block.
//
// Roles (every CTA on its own SM: the dynamic shared-memory request keeps one
// CTA per SM, and a cooperative launch keeps all of them resident, so the
// CTAs can wait on one another; CTAs of 16 warps):
//   CTA b < B          the recurrence of trajectory b, block after block:
//                      all 16 warps add the far history's chunk partials of
//                      the block (several lanes per value, compensated FP64,
//                      loads in flight together), then four warps step it
//                      (predictor -> f -> corrector -> f, one warp per
//                      component as recurrence.cuh) with the h^alpha-scaled
//                      weights and the recent window of f (the two lag
//                      blocks and the block being stepped) resident in
//                      shared memory for the whole solve; after each block
//                      it publishes how many blocks it has finished.
//   CTA B + w          history worker w: for every block c, the chunks of
//                      the far sums over k < (c-2) L (Sec. 2's k-loop, the
//                      O(N^2) part) assigned to it; it waits until the
//                      trajectories of its four columns have finished block
//                      c-3, whose last rows those chunks read, splits the
//                      chunk's points over four groups of four warps
//                      (hist_fp64_chunk, f read around L1 since other SMs
//                      write it during the launch; several chunks' warps in
//                      flight hide the FP64 pipe's latency), adds the four
//                      sums in a fixed order and counts the chunk done in
//                      its super-group (16 consecutive chunks); the worker
//                      that finishes a super-group's last chunk adds the
//                      group's chunk partials in chunk order, compensated,
//                      and counts the super-group done.
// The recurrence of block c waits for every super-group of its block and adds
// their ~10 partials, not the ~150 chunk partials: on GB300 a warp FP64
// instruction costs ~16 cycles of an SM's FP64 pipe, and the chunk-level sum
// on the recurrence's one SM had put ~35 us on the serial chain of every
// block.  Lag 2: block c's far history starts once block c-3 is finished, so
// the recurrences of blocks c-2 and c-1 hide it.
//
// Every wait polls a flag for at most the launch's wait limit; on timeout the
// CTA sets the error word and leaves its loop, and the CTAs waiting on it
// time out in turn: the launch always ends, and the host reports
// FABM_ETIMEOUT.
#include "history_blocks.cuh"
#include "recurrence.cuh"

namespace fabm {
namespace {

constexpr int kPL = kRecurL;                       // targets per block (32)
constexpr int kLag = 2;                            // far history of block c: k < (c - kLag) L
constexpr int kSG = 16;                            // chunks per super-group
constexpr int kSlots = kLag + 2;                   // blocks whose partials are in flight
constexpr int kSubThreads = kWarp * hist::kColsPerCta;  // 128: the stepping warps, a point group
constexpr int kSubs = 4;                                // point groups per history CTA
constexpr int kThreads = kSubThreads * kSubs;           // 512
constexpr int kBarStep = 1;   // named barrier of the four stepping warps
constexpr int kBarAll = 7;    // named barrier of all 512 threads
constexpr int kW = (kLag + 1) * kPL + 1;           // weight distances 0 .. (kLag+1) L
constexpr int kRing = (kLag + 1) * kPL + 1;        // rows of f a recurrence CTA keeps
// doubles of one history worker's tiles (f of 4 columns, two weight windows)
constexpr size_t kTileDoubles = hist::f64::kTile * hist::kColsPerCta + 2 * (hist::f64::kTile + kPL);
constexpr size_t kPadSmem = 116 * 1024;            // one CTA per SM

struct PersistArgs {
    DevBatch bt;
    DevWeights w;
    StepConsts kc;
    int64_t nblk;     // blocks of the longest trajectory
    int n_rec;        // recurrence CTAs (= trajectories)
    int n_hist;       // history CTAs
    int ncg;          // column groups of hist::kColsPerCta
    int max_chunks;   // chunks per (block, column group) at most
    int max_sg;       // super-groups per (block, column group) at most
    double *part;     // [kSlots][max_chunks][2][32][cols] chunk partials
    double *spart;    // [kSlots][max_sg][2][32][cols] super-group partials
    int *sg_cnt;      // [nblk][ncg][max_sg] chunks finished, zero at launch
    int *done;        // [nblk][ncg] super-groups finished, zero at launch
    int *r_done;      // [B] blocks finished per trajectory, zero at launch
    unsigned *err;
    long long wait;   // clock cycles a wait may take
};

// Barrier `id` over `n` threads (128: the stepping warps or a point group;
// 512: the whole CTA).
__device__ __forceinline__ void bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void sub_sync(int id) { bar_sync(id, kSubThreads); }
__device__ __forceinline__ void all_sync() { bar_sync(kBarAll, kThreads); }

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// *p >= v within `budget` clock cycles.
__device__ bool wait_geq(const int *p, int v, long long budget)
{
    if (ld_acquire(p) >= v) return true;
    const long long t0 = clock64();
    while (ld_acquire(p) < v) {
        if (clock64() - t0 > budget) return false;
        __nanosleep(100);
    }
    return true;
}

// Chunking of block c's far history (k < (c - kLag) L) per column group: about
// one chunk per history CTA, chunks of a multiple of 32 points (8 per point
// group).
__device__ __forceinline__ void plan(const PersistArgs &a, int64_t c, int *nch, int64_t *kc)
{
    const int64_t k_end = (c - kLag) * kPL;
    int64_t n = a.n_hist / a.ncg;
    if (n < 1) n = 1;
    const int64_t nmax = (k_end + 63) / 64;
    if (n > nmax) n = nmax;
    if (n > a.max_chunks) n = a.max_chunks;
    int64_t q = (k_end + n - 1) / n;
    q = (q + 31) / 32 * 32;
    *kc = q;
    *nch = (int)((k_end + q - 1) / q);
}

__device__ __forceinline__ int64_t blocks_of(const PersistArgs &a, int b)
{
    return (a.bt.N_each[b] + kPL - 1) / kPL;
}

// The recurrence of trajectory b (CTA b: all 16 warps combine, the first four
// step), all of its blocks.
template <class Rhs, int D>
__device__ void recurrence_cta(const PersistArgs &a, int b, double *smem, int *flag)
{
    const DevBatch &bt = a.bt;
    double *sB = smem;                              // [kW] h^a B(d)
    double *sA = sB + kW;                           // [kW] h^a A(d)
    double(*ring)[D] = reinterpret_cast<double(*)[D]>(sA + kW);  // [kRing][D] f rows
    double(*sG)[kPL][D] = reinterpret_cast<double(*)[kPL][D]>(ring + kRing);  // [2][32][D]
    double(*sy)[D] = reinterpret_cast<double(*)[D]>(sG + 2);    // [2][D]
    double *scr = reinterpret_cast<double *>(sy + 2);           // [kThreads][2] combine
    const bool stepper = threadIdx.x < kSubThreads;  // warps 0..3
    const bool act = threadIdx.x / kWarp < D;
    const int i = act ? threadIdx.x / kWarp : 0;
    const int lane = threadIdx.x % kWarp;
    const int64_t Nb = bt.N_each[b];
    const int64_t nb = blocks_of(a, b);
    const double ha = a.kc.h_alpha[0];
    const double ha_ig2 = ha * a.kc.inv_gamma2[0];
    for (int j = threadIdx.x; j < kW; j += kThreads) {
        sB[j] = ha * a.w.B[j];
        sA[j] = ha * a.w.A[j];
    }
    for (int j = threadIdx.x; j < kRing * D; j += kThreads)
        ring[j / D][j % D] = j / D == 0 ? bt.F[(int64_t)b * D + j % D] : 0.0;  // f_0, rows > 0 later
    double p[kMaxParams];
#pragma unroll
    for (int q = 0; q < kMaxParams; ++q) p[q] = bt.params[(int64_t)b * kMaxParams + q];
    const int64_t col = (int64_t)b * D + i;
    const double y0 = bt.y0[col];
    const double y1 = bt.y1 ? bt.y1[col] : 0.0;
    const double f0 = bt.F[col];
    const int cg_lo = (int)((int64_t)b * D / hist::kColsPerCta);
    const int cg_hi = (int)(((int64_t)b * D + D - 1) / hist::kColsPerCta);
    double *Yb = bt.Y + (int64_t)b * (bt.N + 1) * D;
    // combine: R lanes per value (2 kinds x 32 targets x D components)
    constexpr int kVals = 2 * kPL * D;
    constexpr int R = kThreads / kVals >= 8 ? 8 : (kThreads / kVals >= 4 ? 4 : 2);
    all_sync();

    for (int64_t c = 0; c < nb; ++c) {
        const int64_t m0 = c * kPL;
        // far history of the block: wait for its chunks, add them with
        // compensation in a fixed order (lane r: chunks r, r+R, ..; then the
        // R lane sums in order)
        const bool far = c > kLag;
        if (far) {
            int nch;
            int64_t kc;
            plan(a, c, &nch, &kc);
            const int nsg = (nch + kSG - 1) / kSG;
            if (threadIdx.x == 0) {
                bool ok = true;
                for (int g = cg_lo; g <= cg_hi && ok; ++g)
                    ok = wait_geq(a.done + c * a.ncg + g, nsg, a.wait);
                *flag = ok;
            }
            all_sync();
            if (!*flag) break;
            const double *slot = a.spart + (size_t)(c % kSlots) * a.max_sg * 2 * kPL * bt.cols;
            const int v = threadIdx.x / R, r = threadIdx.x % R;
            double s = 0.0, cmp = 0.0;
            if (v < kVals) {
                const int kind = v / (kPL * D), t = (v / D) % kPL, q = v % D;
                const double *src = slot + ((int64_t)kind * kPL + t) * bt.cols + (int64_t)b * D + q;
                const int64_t cs = 2LL * kPL * bt.cols;  // chunk stride
                int ch = r;
                for (; ch + 7 * R < nsg; ch += 8 * R) {
                    double x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = __ldcg(src + (int64_t)(ch + u * R) * cs);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const double t2 = s + x[u];
                        const double bp = t2 - s;
                        cmp += (s - (t2 - bp)) + (x[u] - bp);
                        s = t2;
                    }
                }
                for (; ch < nsg; ch += R) {
                    const double xv = __ldcg(src + (int64_t)ch * cs);
                    const double t2 = s + xv;
                    const double bp = t2 - s;
                    cmp += (s - (t2 - bp)) + (xv - bp);
                    s = t2;
                }
            }
            scr[2 * threadIdx.x] = s;
            scr[2 * threadIdx.x + 1] = cmp;
            all_sync();
            if (v < kVals && r == 0) {
                double ts = scr[2 * threadIdx.x], tc = scr[2 * threadIdx.x + 1];
                for (int u = 1; u < R; ++u) {
                    const double xv = scr[2 * (threadIdx.x + u)];
                    const double t2 = ts + xv;
                    const double bp = t2 - ts;
                    tc += (ts - (t2 - bp)) + (xv - bp) + scr[2 * (threadIdx.x + u) + 1];
                    ts = t2;
                }
                const int kind = v / (kPL * D), t = (v / D) % kPL, q = v % D;
                sG[kind][t][q] = ts + tc;
            }
            all_sync();
        }

        if (stepper) {
            // accumulators of target m = m0+1+lane: y0 + h^a (far + D(m) f_0 +
            // lag blocks), then the block's own points as they appear
            const int64_t m = m0 + 1 + lane;
            const double Tm = bt.y1 ? fma((double)m * a.kc.h, y1, y0) : y0;
            const double aux = Rhs::aux((double)m * a.kc.h, p);
            double accP = fma(ha, far ? sG[0][lane][i] : 0.0, Tm);
            double accC = fma(ha, fma(a.w.D[m], f0, far ? sG[1][lane][i] : 0.0), Tm);
            // points m0 - kLag L .. m0 - 1 (the lag blocks; none before 0):
            // d = m - k = kLag L + 1 + lane - j
            const int lag_rows = (int)(m0 < kLag * kPL ? m0 : kLag * kPL);
            for (int j = kLag * kPL - lag_rows; j < kLag * kPL; ++j) {
                const int64_t k = m0 - kLag * kPL + j;
                const double fk = ring[k % kRing][i];
                const int d = kLag * kPL + 1 + lane - j;
                accP = fma(sB[d], fk, accP);
                accC = fma(sA[d], fk, accC);
            }
            double fk = ring[m0 % kRing][i];
            const int steps = (int)(Nb - m0 < kPL ? Nb - m0 : kPL);
            for (int s = 0; s < steps; ++s) {
                // the newest point k = m0+s; for the owner of target k+1 this
                // completes y^P (accP) and y0 + h^a S^C (accC)
                const int d = lane - s + 1;
                const int dd = d > 0 ? d : 0;  // done targets add B(0) = A(0) = 0
                accP = fma(sB[dd], fk, accP);
                accC = fma(sA[dd], fk, accC);
                const int owner = s;
                double fn = 0.0, yc = 0.0;
                if constexpr (D == 1) {
                    if (lane == owner) {
                        const double fp = Rhs::template one<D>(0, &accP, p, aux);
                        yc = fma(ha_ig2, fp, accC);
                        fn = Rhs::template one<D>(0, &yc, p, aux);
                    }
                } else {
                    if (act && lane == owner) sy[0][i] = accP;
                    sub_sync(kBarStep);
                    if (lane == owner) {
                        double y[D];
#pragma unroll
                        for (int q = 0; q < D; ++q) y[q] = sy[0][q];
                        const double fp = Rhs::template one<D>(i, y, p, aux);
                        yc = fma(ha_ig2, fp, accC);  // corrector
                        if (act) sy[1][i] = yc;
                    }
                    sub_sync(kBarStep);
                    if (lane == owner) {
                        double y[D];
#pragma unroll
                        for (int q = 0; q < D; ++q) y[q] = sy[1][q];
                        fn = Rhs::template one<D>(i, y, p, aux);
                    }
                }
                if (act && lane == owner) {
                    const int64_t mm = m0 + 1 + s;
                    Yb[mm * D + i] = yc;
                    bt.F[mm * bt.ldF + col] = fn;
                    ring[mm % kRing][i] = fn;
                    if (!(finite_bits(yc) && finite_bits(fn))) report_nonfinite(bt.status, mm, b);
                }
                fk = __shfl_sync(0xffffffffu, fn, owner);
            }
        }
        // the block's rows of f are written: publish it
        all_sync();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(a.r_done + b, (int)(c + 1));
        }
    }
    if (threadIdx.x == 0 && !*flag) atomicOr(a.err, 1u);
}

// History CTA w (of n_hist): its chunks of every block's far history, each
// split over kSubs point groups of four warps (group `sub`, thread tid in it,
// tiles at `tiles`); scr: kSubs x 256 doubles for the groups' sums.
__device__ void history_cta(const PersistArgs &a, int w, int sub, int tid, double *tiles,
                            double *scr, int *flag, int *last)
{
    using namespace hist::f64;
    const DevBatch &bt = a.bt;
    double *sF = tiles;
    auto sB = reinterpret_cast<double(*)[kTile + kPL]>(sF + kTile * hist::kColsPerCta);
    auto sA = sB + 1;
    const int bar = 2 + sub;
    for (int64_t c = kLag + 1; c < a.nblk; ++c) {
        int nch;
        int64_t kc;
        plan(a, c, &nch, &kc);
        const int64_t k_end = (c - kLag) * kPL;
        const int tasks = nch * a.ncg;
        double *slot = a.part + (size_t)(c % kSlots) * a.max_chunks * 2 * kPL * bt.cols;
        for (int t = w; t < tasks; t += a.n_hist) {
            const int g = t / nch, ch = t % nch;
            if (threadIdx.x == 0) {
                // the trajectories of columns 4g .. 4g+3 must have finished
                // block c - kLag - 1 (rows up to (c - kLag) L), or all their
                // blocks
                bool ok = true;
                const int b_lo = g * hist::kColsPerCta / bt.dim;
                int b_hi = (g * hist::kColsPerCta + hist::kColsPerCta - 1) / bt.dim;
                if (b_hi > bt.B - 1) b_hi = bt.B - 1;
                for (int b = b_lo; b <= b_hi && ok; ++b) {
                    const int64_t nb = blocks_of(a, b);
                    const int need = (int)(c - kLag < nb ? c - kLag : nb);
                    ok = wait_geq(a.r_done + b, need, a.wait);
                }
                *flag = ok;
            }
            all_sync();
            if (!*flag) {
                if (threadIdx.x == 0) atomicOr(a.err, 1u);
                return;
            }
            // points of the chunk, in kSubs consecutive parts of multiples of 8
            const int64_t k0 = ch * kc, k1 = k0 + kc < k_end ? k0 + kc : k_end;
            const int64_t q = kc / kSubs;
            const int64_t s0 = k0 + sub * q, s1 = sub + 1 < kSubs ? s0 + q : k1;
            hist_fp64_chunk<false, true>(bt.F, bt.ldF, bt.cols, a.w.B, a.w.A, c,
                                         s0 < k1 ? s0 : k1, s1 < k1 ? s1 : k1, scr + sub * 256,
                                         hist::kColsPerCta, g * hist::kColsPerCta, 0, 1, tid, sF,
                                         sB, sA, [bar] { sub_sync(bar); });
            all_sync();
            // the group sums in order, compensated, to the chunk's partial
            const int ncol = min(hist::kColsPerCta, bt.cols - g * hist::kColsPerCta);
            for (int o = threadIdx.x; o < 2 * kPL * hist::kColsPerCta; o += kThreads) {
                const int wc = o % hist::kColsPerCta;
                if (wc >= ncol) continue;
                double s = scr[o], cmp = 0.0;
#pragma unroll
                for (int u = 1; u < kSubs; ++u) {
                    const double xv = scr[u * 256 + o];
                    const double t2 = s + xv;
                    const double bp = t2 - s;
                    cmp += (s - (t2 - bp)) + (xv - bp);
                    s = t2;
                }
                const int kt = o / hist::kColsPerCta;  // kind * 32 + target
                slot[((int64_t)ch * 2 * kPL + kt) * bt.cols + g * hist::kColsPerCta + wc] = s + cmp;
            }
            all_sync();
            // count the chunk in its super-group; the worker that completes
            // the super-group adds its chunk partials (in chunk order,
            // compensated) into the super-group's partial
            const int sg = ch / kSG, sg_lo = sg * kSG;
            const int sg_n = nch - sg_lo < kSG ? nch - sg_lo : kSG;
            if (threadIdx.x == 0) {
                __threadfence();
                const int before = atomicAdd(a.sg_cnt + (c * a.ncg + g) * a.max_sg + sg, 1);
                *last = before == sg_n - 1;
                if (*last) __threadfence();
            }
            all_sync();
            if (*last) {
                double *sslot = a.spart + (size_t)(c % kSlots) * a.max_sg * 2 * kPL * bt.cols;
                const int64_t cs = 2LL * kPL * bt.cols;  // chunk stride
                for (int o = threadIdx.x; o < 2 * kPL * hist::kColsPerCta; o += kThreads) {
                    const int wc = o % hist::kColsPerCta;
                    if (wc >= ncol) continue;
                    const int kt = o / hist::kColsPerCta;
                    const int64_t off = (int64_t)kt * bt.cols + g * hist::kColsPerCta + wc;
                    double s = 0.0, cmp = 0.0;
                    for (int u = 0; u < sg_n; ++u) {
                        const double xv = __ldcg(slot + (int64_t)(sg_lo + u) * cs + off);
                        const double t2 = s + xv;
                        const double bp = t2 - s;
                        cmp += (s - (t2 - bp)) + (xv - bp);
                        s = t2;
                    }
                    sslot[(int64_t)sg * cs + off] = s + cmp;
                }
                all_sync();
                if (threadIdx.x == 0) {
                    __threadfence();
                    atomicAdd(a.done + c * a.ncg + g, 1);
                }
            }
        }
    }
}

template <class Rhs, int D>
__global__ void __launch_bounds__(kThreads, 1) persist_fp64_kernel(const PersistArgs a)
{
    extern __shared__ __align__(16) double psmem[];
    __shared__ int flag, last;
    if (threadIdx.x == 0) flag = 1, last = 0;
    __syncthreads();
    if ((int)blockIdx.x < a.n_rec) {
        recurrence_cta<Rhs, D>(a, blockIdx.x, psmem, &flag);
        return;
    }
    const int sub = threadIdx.x / kSubThreads, tid = threadIdx.x % kSubThreads;
    history_cta(a, (int)blockIdx.x - a.n_rec, sub, tid, psmem + (size_t)sub * kTileDoubles,
                psmem + (size_t)kSubs * kTileDoubles, &flag, &last);
}

template <int D>
constexpr size_t rec_smem_bytes()
{
    return sizeof(double) * (2 * kW + kRing * D + 2 * kPL * D + 2 * D + 2 * kThreads);
}

}  // namespace

int persist_max_ctas(int rhs, int dim)
{
    int n = 0;
    dispatch_rhs(rhs, dim, [&]<class R, int D>() {
        if (cudaFuncSetAttribute(persist_fp64_kernel<R, D>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kPadSmem) != cudaSuccess)
            return;
        int per_sm = 0, sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_fp64_kernel<R, D>,
                                                          kThreads, kPadSmem) != cudaSuccess)
            return;
        n = per_sm * sms;
    });
    cudaGetLastError();
    return n;
}

int persist_workers(int grid, int B) { return grid - B; }

size_t persist_part_elems(int max_chunks, int cols)
{
    return (size_t)kSlots * max_chunks * 2 * kPL * cols;
}

int persist_max_sg(int max_chunks) { return (max_chunks + kSG - 1) / kSG; }

size_t persist_spart_elems(int max_chunks, int cols)
{
    return (size_t)kSlots * persist_max_sg(max_chunks) * 2 * kPL * cols;
}

cudaError_t launch_persist_fp64(int rhs, const DevBatch &bt, const DevWeights &w,
                                const StepConsts &k, int64_t nblk, int grid, int max_chunks,
                                double *part, double *spart, int *sg_cnt, int *done,
                                int *r_done, unsigned *err, long long wait_cycles,
                                cudaStream_t st)
{
    if (w.stride != 0 || grid <= bt.B || max_chunks < 1) return cudaErrorInvalidValue;
    PersistArgs a{};
    a.bt = bt;
    a.w = w;
    a.kc = k;
    a.nblk = nblk;
    a.n_rec = bt.B;
    a.n_hist = grid - bt.B;
    a.ncg = (bt.cols + hist::kColsPerCta - 1) / hist::kColsPerCta;
    a.max_chunks = max_chunks;
    a.max_sg = persist_max_sg(max_chunks);
    a.part = part;
    a.spart = spart;
    a.sg_cnt = sg_cnt;
    a.done = done;
    a.r_done = r_done;
    a.err = err;
    a.wait = wait_cycles > 0 ? wait_cycles : 4000000000LL;
    cudaError_t e = cudaErrorInvalidValue;
    dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        static_assert(rec_smem_bytes<D>() <= kPadSmem, "recurrence CTA shared memory");
        static_assert((kSubs * kTileDoubles + kSubs * 256) * sizeof(double) <= kPadSmem,
                      "history tiles and group sums");
        void *args[] = {&a};
        e = cudaLaunchCooperativeKernel((const void *)persist_fp64_kernel<R, D>, dim3(grid),
                                        dim3(kThreads), args, kPadSmem, st);
    });
    return e;
}

}  // namespace fabm
