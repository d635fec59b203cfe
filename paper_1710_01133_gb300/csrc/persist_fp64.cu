// a2 + a3 + a4 + a5 in double as one persistent launch per solve: the whole
// predictor-corrector of Sec. 2 of arXiv:1710.01133 for a narrow batch (a few
// trajectories), with the recurrence of every trajectory and the far history
// sums running side by side in one cooperative launch instead of ~3 launches
// per 32-step block.
//
// Roles (every CTA on its own SM: the dynamic shared-memory request keeps one
// CTA per SM, and a cooperative launch keeps all of them resident, so the
// CTAs can wait on one another):
//   CTA b < B          the recurrence of trajectory b, block after block
//                      (predictor -> f -> corrector -> f per step, one warp
//                      per component as recurrence.cuh); its h^alpha-scaled
//                      weights and the recent window of f (the two lag
//                      blocks and the block being stepped) stay in shared
//                      memory for the whole solve; after each block it
//                      publishes how many blocks it has finished (r_done[b]).
//   CTA B + w          history worker w: for every block c, the chunks of
//                      the far sums over k < (c-2) L (Sec. 2's k-loop, the
//                      O(N^2) part) assigned to it; it waits until the
//                      trajectories of its four columns have finished block
//                      c-3, whose last rows those chunks read, sums them
//                      (hist_fp64_block, reading f around L1, since other SMs
//                      write it during the launch) and counts the chunk done
//                      (done[c][column group]).
// The recurrence of block c waits for all chunks of its block, adds them in
// chunk order with compensation (FP64), then steps.  Lag 2: block c's far
// history starts once block c-3 is finished, so the recurrences of blocks c-2
// and c-1 hide it.
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
constexpr int kSlots = kLag + 2;                   // blocks whose partials are in flight
constexpr int kThreads = kWarp * hist::kColsPerCta;  // 128
constexpr int kW = (kLag + 1) * kPL + 1;           // weight distances 0 .. (kLag+1) L
constexpr int kRing = (kLag + 1) * kPL + 1;        // rows of f a recurrence CTA keeps
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
    double *part;     // [kSlots][max_chunks][2][32][cols]
    int *done;        // [nblk][ncg] chunks finished, zero at launch
    int *r_done;      // [B] blocks finished per trajectory, zero at launch
    unsigned *err;
    long long wait;   // clock cycles a wait may take
};

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
// one chunk per history CTA, chunks of a multiple of 8 points.
__device__ __forceinline__ void plan(const PersistArgs &a, int64_t c, int *nch, int64_t *kc)
{
    const int64_t k_end = (c - kLag) * kPL;
    int64_t n = a.n_hist / a.ncg;
    if (n < 1) n = 1;
    const int64_t nmax = (k_end + 63) / 64;
    if (n > nmax) n = nmax;
    if (n > a.max_chunks) n = a.max_chunks;
    int64_t q = (k_end + n - 1) / n;
    q = (q + 7) / 8 * 8;
    *kc = q;
    *nch = (int)((k_end + q - 1) / q);
}

__device__ __forceinline__ int64_t blocks_of(const PersistArgs &a, int b)
{
    return (a.bt.N_each[b] + kPL - 1) / kPL;
}

// The recurrence of trajectory b (CTA b), all of its blocks.
template <class Rhs, int D>
__device__ void recurrence_cta(const PersistArgs &a, int b, double *smem, int *flag)
{
    const DevBatch &bt = a.bt;
    double *sB = smem;                              // [kW] h^a B(d)
    double *sA = sB + kW;                           // [kW] h^a A(d)
    double(*ring)[D] = reinterpret_cast<double(*)[D]>(sA + kW);  // [kRing][D] f rows
    double(*sG)[kPL][D] = reinterpret_cast<double(*)[kPL][D]>(ring + kRing);  // [2][32][D]
    double(*sy)[D] = reinterpret_cast<double(*)[D]>(sG + 2);    // [2][D]
    const bool act = threadIdx.x / kWarp < D;
    const int i = act ? threadIdx.x / kWarp : 0;
    const int lane = threadIdx.x % kWarp;
    const int64_t Nb = bt.N_each[b];
    const int64_t nb = blocks_of(a, b);
    const double ha = a.kc.h_alpha[0];
    const double ha_ig2 = ha * a.kc.inv_gamma2[0];
    for (int j = threadIdx.x; j < kW; j += blockDim.x) {
        sB[j] = ha * a.w.B[j];
        sA[j] = ha * a.w.A[j];
    }
    for (int j = threadIdx.x; j < kRing * D; j += blockDim.x)
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
    __syncthreads();

    for (int64_t c = 0; c < nb; ++c) {
        const int64_t m0 = c * kPL;
        // far history of the block: wait for its chunks, add them in order
        // with compensation
        const bool far = c > kLag;
        int nch = 0;
        int64_t kc = 0;
        if (far) {
            plan(a, c, &nch, &kc);
            if (threadIdx.x == 0) {
                bool ok = true;
                for (int g = cg_lo; g <= cg_hi && ok; ++g)
                    ok = wait_geq(a.done + c * a.ncg + g, nch, a.wait);
                *flag = ok;
            }
            __syncthreads();
            if (!*flag) break;
            const double *slot = a.part + (size_t)(c % kSlots) * a.max_chunks * 2 * kPL * bt.cols;
            for (int o = threadIdx.x; o < 2 * kPL * D; o += blockDim.x) {
                const int kind = o / (kPL * D), t = (o / D) % kPL, q = o % D;
                const int64_t off = ((int64_t)kind * kPL + t) * bt.cols + (int64_t)b * D + q;
                double s = 0.0, cmp = 0.0;
                for (int ch = 0; ch < nch; ++ch) {
                    const double v = __ldcg(slot + (int64_t)ch * 2 * kPL * bt.cols + off);
                    const double u = s + v;
                    const double bp = u - s;
                    cmp += (s - (u - bp)) + (v - bp);
                    s = u;
                }
                sG[kind][t][q] = s + cmp;
            }
            __syncthreads();
        }

        // accumulators of target m = m0+1+lane: y0 + h^a (far + D(m) f_0 +
        // lag blocks), then the block's own points as they appear
        const int64_t m = m0 + 1 + lane;
        const double Tm = bt.y1 ? fma((double)m * a.kc.h, y1, y0) : y0;
        const double aux = Rhs::aux((double)m * a.kc.h, p);
        double accP = fma(ha, far ? sG[0][lane][i] : 0.0, Tm);
        double accC = fma(ha, fma(a.w.D[m], f0, far ? sG[1][lane][i] : 0.0), Tm);
        // points m0 - kLag L .. m0 - 1 (the lag blocks; rows < 1 are f_0 or
        // before the start): d = m - k = kLag L + 1 + lane - j
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
                __syncthreads();
                if (lane == owner) {
                    double y[D];
#pragma unroll
                    for (int q = 0; q < D; ++q) y[q] = sy[0][q];
                    const double fp = Rhs::template one<D>(i, y, p, aux);
                    yc = fma(ha_ig2, fp, accC);  // corrector
                    if (act) sy[1][i] = yc;
                }
                __syncthreads();
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
        // the block's rows of f are written: publish it
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(a.r_done + b, (int)(c + 1));
        }
    }
    if (threadIdx.x == 0 && !*flag) atomicOr(a.err, 1u);
}

// History worker w (of n_hist): its chunks of every block's far history.
__device__ void history_cta(const PersistArgs &a, int w, int *flag)
{
    const DevBatch &bt = a.bt;
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
            __syncthreads();
            if (!*flag) {
                if (threadIdx.x == 0) atomicOr(a.err, 1u);
                return;
            }
            hist::f64::hist_fp64_block<false, true>(bt.F, bt.ldF, bt.cols, a.w.B, a.w.A, c, kc,
                                                    k_end, slot, ch, g * hist::kColsPerCta);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(a.done + c * a.ncg + g, 1);
            }
        }
    }
}

template <class Rhs, int D>
__global__ void __launch_bounds__(kThreads, 1) persist_fp64_kernel(const PersistArgs a)
{
    extern __shared__ __align__(16) double psmem[];
    __shared__ int flag;
    if (threadIdx.x == 0) flag = 1;
    __syncthreads();
    if ((int)blockIdx.x < a.n_rec)
        recurrence_cta<Rhs, D>(a, blockIdx.x, psmem, &flag);
    else
        history_cta(a, blockIdx.x - a.n_rec, &flag);
}

template <int D>
constexpr size_t rec_smem_bytes()
{
    return sizeof(double) * (2 * kW + kRing * D + 2 * kPL * D + 2 * D);
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

size_t persist_part_elems(int max_chunks, int cols)
{
    return (size_t)kSlots * max_chunks * 2 * kPL * cols;
}

cudaError_t launch_persist_fp64(int rhs, const DevBatch &bt, const DevWeights &w,
                                const StepConsts &k, int64_t nblk, int grid, int max_chunks,
                                double *part, int *done, int *r_done, unsigned *err,
                                long long wait_cycles, cudaStream_t st)
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
    a.part = part;
    a.done = done;
    a.r_done = r_done;
    a.err = err;
    a.wait = wait_cycles > 0 ? wait_cycles : 4000000000LL;
    cudaError_t e = cudaErrorInvalidValue;
    dispatch_rhs(rhs, bt.dim, [&]<class R, int D>() {
        static_assert(rec_smem_bytes<D>() <= kPadSmem, "recurrence CTA shared memory");
        void *args[] = {&a};
        e = cudaLaunchCooperativeKernel((const void *)persist_fp64_kernel<R, D>, dim3(grid),
                                        dim3(kThreads), args, kPadSmem, st);
    });
    return e;
}

}  // namespace fabm
