// Internal interfaces of the fractional ABM engine (not part of the C ABI).
//
// Index conventions used throughout the CUDA sources.  For the step that
// produces y_m (target m = n+1 in the paper's notation) and a past point k the
// distance is d = m - k >= 1, and the weights of Sec. 2 become
//   B(d) = b_{d-1} = (d^a - (d-1)^a) / Gamma(a+1)                     predictor
//   A(d) = a_{d-1} = ((d+1)^{a+1} - 2 d^{a+1} + (d-1)^{a+1}) / Gamma(a+2)  corrector
//   C(m-1) = c_{m-1}                                        corrector, k = 0 term
// so that  S^P_m = sum_{k<m} B(m-k) f_k  and
//          S^C_m = sum_{k<m} A(m-k) f_k + (C(m-1) - A(m)) f_0.
// The last form lets every history kernel treat k = 0 like any other point;
// the recurrence adds the correction D(m) = C(m-1) - A(m) times f_0.
//
// Time is cut into blocks of L targets: block c holds m = cL+1 .. cL+L.  The
// history kernels sum the "far" part (k < (c-1)L) of every block while the
// recurrence kernel of the previous block runs; the recurrence adds the lag-1
// block and the block's own triangle, step by step.  On the tensor-history
// path (L = 64) a second, one-segment history launch adds the lag-1 block once
// the previous block is done, and the recurrence adds only its own triangle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fabm.h"

// 1/Gamma(a+1), 1/Gamma(a+2) in binary128 as (hi, lo) pairs (weights_x2.c).
extern "C" void fabm_x2_inv_gammas(double alpha, double out[4]);

namespace fabm {

constexpr int kWarp = 32;
constexpr int kRecurL = 32;        // targets per block of the FP64 path
constexpr int kSplitSeg = 64;      // targets per block (= points per segment) of the split path
constexpr int kMaxParams = FABM_MAX_PARAMS;

// Weight vectors on the device, index 0..N.  B[0] = A[0] = D[0] = 0.  With
// one order per component (stride > 0) component i's vectors start at
// B + i*stride (A, D likewise); stride 0: one set for all components.
struct DevWeights {
    const double *B;
    const double *A;
    const double *D;   // D[m] = C(m-1) - A(m)
    int64_t N;
    int64_t stride = 0;
};

// One batch of B trajectories of one solver, as the kernels see it.
struct DevBatch {
    int dim;
    int B;                 // trajectories
    int cols;              // B * dim; column of (b, i) is b*dim + i
    int64_t N;             // steps of the longest trajectory
    const int64_t *N_each; // per-trajectory steps (device)
    const double *y0;      // B x dim
    const double *y1;      // B x dim, y'(0) for 1 < alpha < 2, or NULL (Taylor part y0)
    const double *params;  // B x kMaxParams
    double *F;             // history f_k, (N+1) x ldF, row k = time k; on the
                           // tensor-history path each slot holds a float-float
                           // pair (float2) instead of a double
    int64_t ldF;           // row stride of F (>= cols)
    float *Ff;             // compensated-fp32 history path: f rounded to float, same
                           // layout as F (written by the split recurrence), or NULL
    double *Y;             // output, B x (N+1) x dim (trajectory-major)
    unsigned long long *status;  // [0] = first non-finite (step << 24 | traj), ~0 if none
};

// Step constants; h^alpha and 1/Gamma(alpha+2) per component (all equal for
// a single order).
struct StepConsts {
    double h;
    double h_alpha[FABM_MAX_DIM];     // h^alpha_i
    double inv_gamma2[FABM_MAX_DIM];  // 1/Gamma(alpha_i+2)
};

// a1: weights B(d), A(d), D(m) for d, m = 0..N.
cudaError_t launch_weights(double alpha, int64_t N, double inv_g1, double inv_g2, double *B,
                           double *A, double *D, cudaStream_t st);

// y_0 into Y, f_0 = f(0, y_0) into F row 0 (as a float-float pair when
// f_pairs, the tensor-history path).
cudaError_t launch_init(int rhs, const DevBatch &bt, cudaStream_t st, bool f_pairs = false);

// a2 (FP64): partial far-history sums of target block c from the points
// k in [0, (c-lag)L), split into n_chunks chunks of kc points.
// part: n_chunks x 2 x L x cols (P then C).
cudaError_t launch_hist_fp64(const DevBatch &bt, const DevWeights &w, int64_t c, int L, int lag,
                             int n_chunks, int64_t kc, double *part, cudaStream_t st);

// a3: G[pc][a][col] = sum over chunks of part (fixed order).
cudaError_t launch_hist_reduce(const double *part, int n_chunks, int L, int cols, double *G,
                               cudaStream_t st);

// a4 + a5: steps of block c (L = 32 targets) for every trajectory; G holds the
// far history of block c over the points k < (c - lag) L (2 x L x cols) or is
// NULL when c <= lag; the lag blocks (lag 1 or 2) before block c are summed by
// the recurrence.  split = false: all in double; split = true: FP64 bases and
// corrector update, short-range sums and f in float-float (recur_block_split).
cudaError_t launch_recur(int rhs, const DevBatch &bt, const DevWeights &w, const StepConsts &k,
                         int64_t c, int L, int lag, bool split, const double *G, cudaStream_t st);

// Message returned by fabm_last_error() on the calling thread.
void set_last_error(const char *msg);

// Host-side fault injection (fabm_inject_alloc_failures): true when the
// device allocation about to be made must fail as if the device were out of
// memory (the allocator is then not called).  Consumes one injected failure.
bool take_injected_alloc_failure();

// ---- split path (history on tensor cores) ----

// f of segment seg (64 points) -> bf16 slices Fs and per-column exponents Ef.
cudaError_t launch_slice_f(const DevBatch &bt, int n_ct, int64_t seg, __nv_bfloat16 *Fs, int *Ef,
                           cudaStream_t st);

// Hankel weight tiles and exponents for the lags 1..g_max.
cudaError_t launch_hankel_weights(const double *WB, const double *WA, int64_t g_max,
                                  __nv_bfloat16 *WH, int *Ew, cudaStream_t st);

// Kernel attributes of the tensor kernel (dynamic shared memory); call once
// per device before the first launch (and outside any graph capture).
cudaError_t prepare_hist_split();

// float2 elements of the partial-sum buffer for n_chunks chunks.
size_t split_part_elems(int n_chunks, int cols);

// History of block c over the segments seg0 .. seg0+n_seg-1 (all before block
// c) on tensor cores: n_chunks chunks of segments (1 <= n_chunks <= n_seg) per
// column tile of 128, written to the partial chunks chunk0 .. chunk0+n_chunks-1.
// The far part of block c is seg0 = 0, n_seg = c-1; the newest segment is
// seg0 = c-1, n_seg = 1.
cudaError_t launch_hist_split(const __nv_bfloat16 *Fs, const int *Ef, const __nv_bfloat16 *WH,
                              const int *Ew, int64_t c, int seg0, int n_seg, int chunk0,
                              int n_chunks, int n_ct, int cols, float2 *part, unsigned int *err,
                              long long wait_cycles, cudaStream_t st);

// G[kind][t][col] = sum of the float-float partials over chunks, for blocks
// of L targets: accumulated in double with compensation and rounded once, or
// (_ff, tensor path) accumulated in compensated float-float and kept as pairs.
cudaError_t launch_combine_split(const float2 *part, int n_chunks, int cols, int L, double *G,
                                 cudaStream_t st);
cudaError_t launch_combine_split_ff(const float2 *part, int n_chunks, int cols, int L,
                                    float2 *G, cudaStream_t st);

// out[i] = scale * W[i] as a float-float pair, i < n.
cudaError_t launch_ff_weights(const double *W, double scale, int64_t n, float2 *out,
                              cudaStream_t st);

// ---- tensor path, wide far history (history_far.cu) ----
// Point groups of 128 (two blocks of 64); the far history of a pair of blocks
// (target group C: m = 128C+1 .. 128C+128) over the groups 0 .. C-2 on tensor
// cores with 128 targets per MMA, one weight kind per CTA.

// f of group S -> bf16 slices Fs (far_group_slice_elems() per group and
// column tile) and per-column exponents Ef (128 per group and column tile).
cudaError_t launch_slice_group(const DevBatch &bt, int n_ct, int64_t S, __nv_bfloat16 *Fs, int *Ef,
                               cudaStream_t st);
// Hankel weight tiles (far_group_tile_elems() per group lag) and exponents
// (2 per lag) for the group lags 2 .. G_max.
cudaError_t launch_hankel_group(const double *WB, const double *WA, int64_t G_max,
                                __nv_bfloat16 *WH, int *Ew, cudaStream_t st);
size_t far_group_tile_elems();
size_t far_group_slice_elems();
// Kernel attributes of the wide far kernel; call once per device, outside any
// graph capture.
cudaError_t prepare_hist_far();
// float2 elements of the wide far kernel's partials for n_chunks chunks.
size_t far_part_elems(int n_chunks, int cols);
// Far history of target group C over the point groups 0 .. n_grp-1 (n_grp <=
// C-1), n_chunks chunks of groups per column tile and kind:
// part[chunk][kind][128][cols] float-float pairs.
cudaError_t launch_hist_far(const __nv_bfloat16 *Fs, const int *Ef, const __nv_bfloat16 *WH,
                            const int *Ew, int64_t C, int n_grp, int n_chunks, int n_ct, int cols,
                            float2 *part, unsigned int *err, long long wait_cycles,
                            cudaStream_t st);
// out[kind][t][col] (128 targets) = far[.][kind][t][col] over n_far chunks,
// float-float, fixed order.
cudaError_t launch_sum_far(const float2 *far, int n_far, int cols, float2 *out, cudaStream_t st);

// a4 + a5 on the tensor-history path, one lane per column (recurrence_cols.cu):
// the 64 steps of block c given the history of every point k < 64c as
// float-float pairs: G[kind][g_off + t][col] (rows of g_rows per kind; NULL:
// none) plus near[ch][kind][t][col] (64 rows per kind) over n_near chunks.  WB, WA: h^a B(d), h^a A(d)
// for d = 0..64; WD: h^a D(m), m = 0..N; all float-float pairs, one order.
// warps_per_cta (1..12) warps of 32/dim trajectories per CTA, or 0: one lane
// per target, a CTA of dim warps per trajectory (narrow batches).  X: the table
// of the time-only part of f for block c (launch_aux_table), required when
// rhs_has_forcing(rhs), else ignored.  y's slots receive float-float
// increments; launch_finish_y turns them into y after the last block.
struct HistIn {
    const float2 *G = nullptr;     // [2][g_rows][cols], or NULL
    int g_rows = 64, g_off = 0;
    const float2 *near = nullptr;  // [n_near][2][64][cols]
    int n_near = 0;
};
cudaError_t launch_recur_cols(int rhs, const DevBatch &bt, const float2 *WB, const float2 *WA,
                              const float2 *WD, const StepConsts &k, int64_t c, const HistIn &hin,
                              const float2 *X, int warps_per_cta, cudaStream_t st);
// The right-hand side has a time-dependent part (forcing).
bool rhs_has_forcing(int rhs, int dim);
// X[a][b] = aux(t_{64c+1+a}, params of b) as float-float pairs, a < 64, b < B.
cudaError_t launch_aux_table(int rhs, const DevBatch &bt, double h, int64_t c, float2 *X,
                             cudaStream_t st);
// y = T + increment in double for the rows m_lo .. m_hi (1 <= m_lo, m_hi <= N)
// of every trajectory, rows past its N_each excepted.
cudaError_t launch_finish_y(const DevBatch &bt, double h, int64_t m_lo, int64_t m_hi,
                            cudaStream_t st);
// Kernel attributes (dynamic shared memory) of the column recurrence for one
// right-hand side; call before the first launch, outside any graph capture.
cudaError_t prepare_recur_cols(int rhs, int dim);
// Warps the column recurrence needs for B trajectories of dimension dim.
int recur_cols_warps(int dim, int64_t B);

// ---- FP64, persistent (persist_fp64.cu) ----

// CTAs of the persistent FP64 kernel that can be resident at once on the
// current device (0: cooperative launch unavailable).
int persist_max_ctas(int rhs, int dim);
// History workers of a persistent launch of `grid` CTAs for B trajectories
// (the most chunks per block it uses).
int persist_workers(int grid, int B);
// doubles of the persistent kernel's chunk-partial slots and super-group
// (16 chunks) partial slots; super-groups per (block, column group) at most.
size_t persist_part_elems(int max_chunks, int cols);
size_t persist_spart_elems(int max_chunks, int cols);
int persist_max_sg(int max_chunks);
// The whole FP64 solve of a batch (after launch_init) as one cooperative
// launch of `grid` CTAs: bt.B recurrence CTAs and grid - bt.B history CTAs
// (chunks per block at most max_chunks, e.g. persist_workers(grid, B)).
// sg_cnt: nblk x ceil(cols/4) x persist_max_sg(max_chunks) ints, done: nblk x
// ceil(cols/4) ints, r_done: B ints, all zero; err: set on a wait timeout.
cudaError_t launch_persist_fp64(int rhs, const DevBatch &bt, const DevWeights &w,
                                const StepConsts &k, int64_t nblk, int grid, int max_chunks,
                                double *part, double *spart, int *sg_cnt, int *done,
                                int *r_done, unsigned *err, long long wait_cycles,
                                cudaStream_t st);

// ---- FP64X2 precision (double-double history) ----

// Low parts of the double-double weights; the high parts are the DevWeights
// vectors (same layout and stride).
struct DevWeightsLo {
    const double *B;
    const double *A;
    const double *D;
};

// a1 in double-double on the device: B, A, D for d = 0..n as (hi, lo) pairs,
// given 1/Gamma(a+1) and 1/Gamma(a+2) as pairs (weights_dd.cu).
cudaError_t launch_weights_x2(double alpha, int64_t n, double ig1_hi, double ig1_lo,
                              double ig2_hi, double ig2_lo, double *Bh, double *Bl, double *Ah,
                              double *Al, double *Dh, double *Dl, cudaStream_t st);

// a2 in double-double: partial far-history sums of target block c (32 targets)
// over k < (c-lag)*32 as (hi, lo) pairs, n_chunks x 2 x 32 x cols.
cudaError_t launch_hist_x2(const DevBatch &bt, const DevWeights &w, const DevWeightsLo &wl,
                           int64_t c, int lag, int n_chunks, int64_t kc, double2 *part,
                           cudaStream_t st);
// a3: G = sum over chunks in double-double, rounded once to double.
cudaError_t launch_reduce_x2(const double2 *part, int n_chunks, int cols, double *G, cudaStream_t st);

// ---- split path for narrow batches (compensated fp32 on CUDA cores) ----

// y[i] = (float)x[i], i < n.
cudaError_t launch_to_float(const double *x, int64_t n, float *y, cudaStream_t st);

// Far history of block c (32 targets) over k < (c-lag)*32 in compensated fp32;
// partials as float2 (sum, -compensation), n_chunks x 2 x 32 x cols.
// wstride > 0: one order per component (weights of component i at WBf + i*wstride).
cudaError_t launch_hist_fp32c(const DevBatch &bt, const float *WBf, const float *WAf,
                              int64_t wstride, int64_t c, int lag, int n_chunks, int64_t kc,
                              float2 *part, cudaStream_t st);

}  // namespace fabm
