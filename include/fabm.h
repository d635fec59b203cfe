/*
 * fabm.h -- C ABI of the GB300 fractional Adams-Bashforth-Moulton engine.
 *
 * The engine solves Caputo systems  D^alpha y = f(t, y),  y(0) = y0,  0 < alpha < 2
 * (y'(0) also given for 1 < alpha < 2; one order per component allowed),
 * on the uniform grid t_n = n h, n = 0..N, with the predictor-corrector of
 * Section 2 of Bonchis, Kaslik, Rosu, arXiv:1710.01133 (Eq. abm for the
 * predictor, the corrector and its weights a_n, c_n right after it).  For each
 * step n -> n+1 it forms the two hereditary sums over all previous
 * f_k = f(t_k, y_k),
 *     S^P_{n+1} = sum_{k=0}^{n} b_{n-k} f_k
 *     S^C_{n+1} = c_n f_0 + sum_{k=1}^{n} a_{n-k} f_k,
 * then y^P_{n+1} = y0 + h^alpha S^P_{n+1},
 *      y_{n+1}   = y0 + h^alpha (S^C_{n+1} + f(t_{n+1}, y^P_{n+1}) / Gamma(alpha+2))
 * (for 1 < alpha < 2 the Taylor part y0 + t_{n+1} y'(0) takes the place of y0).
 * b_n is taken with a minus sign, ((n+1)^alpha - n^alpha)/Gamma(alpha+1): the
 * paper prints "+", which does not reproduce constant right-hand sides.
 * A system is solved componentwise (Sec. 2, last paragraph).
 *
 * Conventions for every call:
 *   - All pointers are plain host pointers unless a parameter says otherwise.
 *     Host buffers stay owned by the caller; the library copies what it keeps.
 *   - Device memory (history, weights, work space) is owned by the solver and
 *     released by fabm_destroy.
 *   - No call aborts the process.  Every call returns a fabm_status; on failure
 *     fabm_last_error() gives a message for the calling thread.
 *   - A solver may be used by one host thread at a time (FABM_EBUSY otherwise).
 *   - The library runs on the CUDA device that is current when fabm_create is
 *     called, and keeps using it.
 */
#ifndef FABM_H
#define FABM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fabm_solver fabm_solver;

typedef enum {
    FABM_OK = 0,
    FABM_EINVAL = 1,     /* invalid argument (message names it)                     */
    FABM_ENOMEM = 2,     /* host or device allocation failed                        */
    FABM_ECUDA = 3,      /* a CUDA call failed (message has the CUDA error)         */
    FABM_ENONFINITE = 4, /* a solution value became NaN/Inf; message gives
                            trajectory and step, rows up to that step are valid     */
    FABM_ETIMEOUT = 5,   /* a bounded device-side wait gave up (status word set)    */
    FABM_EBUSY = 6       /* solver in use by another thread                         */
} fabm_status;

/* Arithmetic of the history sums. */
enum {
    FABM_FP64 = 0,  /* every step in IEEE double                                   */
    FABM_SPLIT = 1, /* history sums in compensated reduced precision: three-term bf16
                       split on tensor cores (wide batches) or compensated fp32 on
                       CUDA cores (narrow batches); weights computed in double; the
                       steps of a block in float-float arithmetic (about 48 bits),
                       each y formed in double once.  Within 1e-6 of the solution
                       scale of an FP64 solve on every tested workload */
    FABM_FP64X2 = 2 /* the extended-precision mode the paper runs in long double
                       (Sec. 3.4, "memory saving"): weights in double-double from
                       binary128 (fabm_weights_x2), far-history sums in
                       double-double (exact products, compensated sums, combined
                       across chunks in double-double) and rounded once; the
                       steps of a block in double as in FABM_FP64.  About ten FP64
                       operations per history multiply-add */
};

/* Right-hand sides f(t, y) (params in this order; dim as stated). */
enum {
    FABM_RHS_CONST = 0,        /* f_i = p0                      dim >= 1, 1 param   */
    FABM_RHS_TIME = 1,         /* f_i = t                       dim >= 1, 0 params  */
    FABM_RHS_LINEAR = 2,       /* f_i = -p0 y_i                 dim >= 1, 1 param   */
    FABM_RHS_LORENZ = 3,       /* Lorenz-type: p = (sigma, rho, beta), dim 3
                                  f = (s(y-x), x(r-z)-y, xy-bz)                      */
    FABM_RHS_DUFFING = 4,      /* forced oscillator with cubic capacitor, dim 2,
                                  p = (gamma, omega, F):
                                  f = (y, -gamma y - x - x^3 + F cos(omega t))       */
    FABM_RHS_MANUFACTURED = 5, /* f = p0 t^p1 + t^p2 - y, dim 1 (solution t^p2 when
                                  p0 = Gamma(p2+1)/Gamma(p2+1-alpha), p1 = p2-alpha,
                                  y(0) = 0 and, for alpha > 1, y'(0) = 0)           */
    FABM_RHS_LCR = 6           /* forced series LCR circuit, Sec. 5, Eq. sys.LRC,
                                  dim 2, p = (sigma, omega, a, b, f):
                                  f = (y - g(x), -sigma y - x + f sin(omega t)),
                                  g piecewise linear with slopes a (|x|<1), b       */
};

#define FABM_MAX_DIM 4
#define FABM_MAX_PARAMS 8

/* Create a solver for D^alpha y = f(t, y) on t_n = n h, n = 0..N (Sec. 2).
 *   dim        number of components (must match rhs_id, 1..FABM_MAX_DIM)
 *   alpha      fractional order, 0 < alpha < 2.  The Taylor part of the initial
 *              data (the sum over k < ceil(alpha) of t^k/k! y^(k)(0) in Sec. 2) is
 *              y0 for alpha <= 1 and y0 + t y'(0) for 1 < alpha < 2, y'(0) given
 *              to fabm_solve_batch_ic (zero otherwise)
 *   h          step size, h > 0 (T = N h)
 *   N          number of steps, 1 <= N <= 2^31
 *   rhs_id     one of FABM_RHS_*
 *   params     n_params doubles (copied), the rhs parameters
 *   precision  FABM_FP64, FABM_SPLIT or FABM_FP64X2
 *   out        receives the solver handle
 * Computes the weights b, a, c on the device (FABM_FP64X2: on the host, in
 * binary128, then uploaded as double-double).  Errors: FABM_EINVAL for any
 * argument out of range, FABM_ENOMEM, FABM_ECUDA. */
fabm_status fabm_create(int dim, double alpha, double h, int64_t N, int rhs_id,
                        const double *params, int n_params, int precision, fabm_solver **out);

/* As fabm_create with one fractional order per component, D^alpha_i y_i =
 * f_i(t, y) (the systems of Sec. 5 carry an order per equation, alpha1 and
 * alpha2 for the LCR circuit).  alpha: dim orders, each 0 < alpha_i < 2; each
 * component uses its own weights, h^alpha_i and Gamma(alpha_i+2), and y'(0)
 * (fabm_solve_batch_ic) only where alpha_i > 1.  With orders that differ,
 * split precision sums the history with the compensated-fp32 kernel (a tensor
 * tile shares one weight operand across its columns); fabm_copy_weights
 * returns component 0's weights.  Errors as fabm_create. */
fabm_status fabm_create_multi(int dim, const double *alpha, double h, int64_t N, int rhs_id,
                              const double *params, int n_params, int precision,
                              fabm_solver **out);

/* Solve one trajectory.  y0: dim doubles.  out: (N+1) x dim doubles, row n = y_n,
 * row 0 = y0, caller-allocated host memory.  Synchronous. */
fabm_status fabm_solve(fabm_solver *s, const double *y0, double *out);

/* Solve B independent trajectories that share (dim, alpha, h, rhs).
 *   y0           B x dim doubles (host)
 *   traj_params  B x n_params doubles (host) replacing params per trajectory, or NULL
 *   N_each       B step counts 1 <= N_each[b] <= N (host), or NULL for N
 *   out          B x (N+1) x dim doubles, trajectory-major; rows past N_each[b]
 *                are not written.  Host memory, or device memory (allocated by
 *                the caller on the solver's device) when out_on_device != 0.
 *                Pinned host memory (cudaHostAlloc or registered) of 64 MB or
 *                more, with every trajectory running to N, is filled while the
 *                solve runs, group of blocks by group of blocks; other host
 *                memory is filled once at the end.
 * Synchronous.  B = 0 is allowed and does nothing. */
fabm_status fabm_solve_batch(fabm_solver *s, int64_t B, const double *y0, const double *traj_params,
                             const int64_t *N_each, double *out, int out_on_device);

/* As fabm_solve_batch, with the first derivatives y'(0) of the initial data:
 *   y1           B x dim doubles (host), for 1 < alpha < 2; NULL means zero.
 * FABM_EINVAL if y1 is given for alpha <= 1 or holds a non-finite value. */
fabm_status fabm_solve_batch_ic(fabm_solver *s, int64_t B, const double *y0, const double *y1,
                                const double *traj_params, const int64_t *N_each, double *out,
                                int out_on_device);

/* Release the solver and its device memory.  NULL is allowed. */
fabm_status fabm_destroy(fabm_solver *s);

/* Message of the last failed call on this thread ("" if none). */
const char *fabm_last_error(void);

/* History kernels (fabm_set_history_kernel). */
enum {
    FABM_HIST_AUTO = 0,    /* FP64 precision: FABM_HIST_FP64; split precision: tensor
                              cores for batches of at least 64 columns, else FP32C;
                              FP64X2 precision: FABM_HIST_X2                         */
    FABM_HIST_FP64 = 1,    /* double on CUDA cores (FP64 precision only)             */
    FABM_HIST_TENSOR = 2,  /* three-term bf16 split on tcgen05 tensor cores, exact
                              per 64-point segment, far history of each 64-step block
                              with 64 targets per MMA (split precision)              */
    FABM_HIST_FP32C = 3,   /* compensated fp32 on CUDA cores (split precision)       */
    FABM_HIST_X2 = 4,      /* double-double on CUDA cores (FP64X2 precision only)    */
    FABM_HIST_TENSOR_WIDE = 5, /* as FABM_HIST_TENSOR, but the far history of each pair
                              of blocks with 128 targets per MMA (one weight kind per
                              CTA, exact per 128-point group), the latest two or three
                              64-point segments per block with 64; automatic choice
                              on the tensor path where N^2 x columns >= 2^40 (the
                              measured crossover) and N >= 257                       */
    FABM_HIST_FP64_PERSIST = 6 /* FP64 precision, the whole solve as one persistent
                              cooperative launch: one CTA per trajectory runs its
                              recurrence with weights and the recent window of f in
                              shared memory, the other CTAs sum the far history
                              (as FABM_HIST_FP64) and hand it over through device
                              flags; single-order batches of at most 64 trajectories
                              (others run FABM_HIST_FP64); timed by fabm_autotune,
                              not chosen automatically                               */
};

/* Choose the history kernel (one of FABM_HIST_*; must fit the precision).
 * The block length follows from it: 64 targets for FABM_HIST_TENSOR and
 * FABM_HIST_TENSOR_WIDE, 32 otherwise.  fabm_autotune measures the candidates
 * and sets the fastest. */
fabm_status fabm_set_history_kernel(fabm_solver *s, int kernel);
int fabm_get_history_kernel(const fabm_solver *s);
/* History kernel the last solve ran (FABM_HIST_*, after the automatic choice;
 * FABM_HIST_TENSOR_WIDE where its far history used 128 targets per MMA), or -1
 * before the first solve or for a NULL solver. */
int fabm_last_history_kernel(const fabm_solver *s);

/* Step layouts of the split-precision recurrence on the tensor-history path
 * (fabm_set_recurrence_layout); both compute the same steps in float-float. */
enum {
    FABM_REC_AUTO = 0,     /* COLUMNS when the batch has at least 96 warps of columns
                              (96 * 32/dim trajectories) or N * columns >= 2^28
                              (the history dominates), else TARGETS                 */
    FABM_REC_COLUMNS = 1,  /* one lane per column (trajectory, component), 32/dim
                              trajectories per warp: fewest instructions per step    */
    FABM_REC_TARGETS = 2   /* one lane per target, one CTA of dim warps per
                              trajectory: most parallelism for narrow batches        */
};

/* Choose the recurrence layout (one of FABM_REC_*) for later solves on the
 * tensor-history path; other paths ignore it.  FABM_EINVAL for other values,
 * FABM_EBUSY while another thread uses the solver. */
fabm_status fabm_set_recurrence_layout(fabm_solver *s, int layout);
/* The layout set on the solver (FABM_REC_*), or -1 for NULL. */
int fabm_get_recurrence_layout(const fabm_solver *s);
/* Warps per CTA of the lane-per-column recurrence (FABM_REC_COLUMNS) for later
 * solves: 0 chooses automatically (CTAs sized to fill the SMs the tensor CTAs
 * leave free, at most 4 warps each), 1..12 fixes it; the arithmetic and the
 * results do not depend on it.  FABM_EINVAL outside 0..12, FABM_EBUSY while
 * another thread uses the solver. */
fabm_status fabm_set_recurrence_warps(fabm_solver *s, int warps);
/* The width set on the solver (0: automatic), or -1 for NULL. */
int fabm_get_recurrence_warps(const fabm_solver *s);

/* Autotuner: for each candidate setting, times solves of the caller's batch
 * (B, y0, traj_params as for fabm_solve_batch) truncated to n_probe, 2 n_probe
 * and 4 n_probe steps, fits c + alpha n + beta n^2 (fixed costs, the per-step
 * chain, the O(n^2) history) to the three, and keeps the setting whose
 * prediction for all N steps is smallest (a probe that reaches N is timed
 * as it is).
 * Longer probes predict better where the history only dominates late in a
 * long solve.  Candidates: for FABM_FP64 and FABM_FP64X2
 * (with its double-double kernel), the split-k CTA target of the history kernel
 * (152, 304, 608, 1216 CTAs); for FABM_SPLIT, the two tensor-core far-history
 * tilings (FABM_HIST_TENSOR_WIDE: 128 targets per MMA and per far launch;
 * FABM_HIST_TENSOR: 64) each with 0 or 16 SMs (or an automatic number) kept
 * free for the recurrence running beside it, and the compensated-fp32 kernel
 * at 304 and 608 CTAs.  Up to max_report
 * candidates are reported (predicted milliseconds per full solve, history
 * kernel FABM_HIST_*, CTA target or SM reserve); *n_report receives the number
 * tried.  The warps per recurrence CTA (fabm_set_recurrence_warps) are not
 * tuned: truncated probes run the recurrence-dominated early blocks and favour
 * wider CTAs than a full solve does.
 * Any report pointer may be NULL.  Allocates a device output buffer of
 * B x (N+1) x dim doubles for the duration of the call. */
fabm_status fabm_autotune(fabm_solver *s, int64_t B, const double *y0, const double *traj_params,
                          int64_t n_probe, int max_report, double *ms_report, int *kernel_report,
                          int *ctas_report, int *n_report);

/* Time-block length L of the last solve (or of the current choice before any
 * solve).  fabm_set_block accepts only the length of an allowed history
 * kernel (32 or 64) and selects that kernel; it changes the order of summation
 * only. */
fabm_status fabm_set_block(fabm_solver *s, int L);
int fabm_get_block(const fabm_solver *s);

/* Record each solve's launch sequence (both streams) as a CUDA graph and
 * replay it while the batch size, the longest trajectory and the buffers stay
 * the same (1, the default), or launch kernel by kernel (0).  Inputs (y0,
 * parameters, per-trajectory lengths) are read from device memory by the
 * kernels, so a cached graph serves any inputs of the same shape. */
fabm_status fabm_set_graphs(fabm_solver *s, int enable);

/* Failure handling (Sec. 5 of the design has no counterpart in the paper; these
 * make the library's error paths testable without faulting a GPU).
 *
 * fabm_set_wait_limit: the tensor-core history kernel waits on barriers that
 * other warps of its CTA complete; each such wait gives up after `cycles` SM
 * clock cycles (0: the default, about 2 s at 2 GHz).  A CTA that gives up sets
 * the solver's status word, waits for its own copies and MMAs in flight, frees
 * its tensor memory and returns, and the solve returns FABM_ETIMEOUT; the
 * solver stays usable.  A tiny limit forces that path.  FABM_EINVAL for
 * cycles < 0.
 *
 * fabm_inject_alloc_failures: the next n device allocations the library makes
 * (solver work space, server admissions; process-wide) fail as if the device
 * were out of memory, without calling the allocator: the call that needed the
 * memory returns FABM_ENOMEM (a server marks that request failed with
 * FABM_ENOMEM), and later calls allocate normally.  n = 0 cancels what is left.
 * FABM_EINVAL for n < 0. */
fabm_status fabm_set_wait_limit(fabm_solver *s, int64_t cycles);
fabm_status fabm_inject_alloc_failures(int n);

/* Copy the first n device weights of the solver to host arrays (n <= N+1):
 *   B[d] = b_{d-1}, A[d] = a_{d-1} (d >= 1; index 0 holds 0),
 *   D[m] = c_{m-1} - a_{m-1}       (m >= 1; index 0 holds 0),
 * the predictor weights of Eq. abm and the corrector weights of Sec. 2 in the
 * distance form d = (n+1) - k used by the kernels.  Any of B, A, D may be NULL. */
fabm_status fabm_copy_weights(fabm_solver *s, int64_t n, double *B, double *A, double *D);
/* FABM_FP64X2 solvers: the low parts of the double-double weights whose high
 * parts fabm_copy_weights returns (value = high + low), computed on the device
 * in double-double arithmetic.  FABM_EINVAL for other precisions or n outside
 * 0..N+1. */
fabm_status fabm_copy_weights_lo(fabm_solver *s, int64_t n, double *Bl, double *Al, double *Dl);

/* The weights B(d), A(d), D(m) of fabm_copy_weights for d, m = 0..n in
 * double-double: hi is the double nearest the value, lo the rounded rest
 * (about 1e-27 relative for n <= 2^20).  Evaluated on the host in binary128
 * from cancellation-free rewrites of the printed differences; needs no GPU.
 * Arrays of n+1 doubles each.  FABM_EINVAL unless 0 < alpha < 2, n >= 0 and no
 * pointer is NULL. */
fabm_status fabm_weights_x2(double alpha, int64_t n, double *B_hi, double *B_lo, double *A_hi,
                            double *A_lo, double *D_hi, double *D_lo);

/* Stroboscopic samples of solved trajectories, the sampling behind the
 * bifurcation diagram of Sec. 5 (the attractor of the forced LCR system seen
 * once per forcing period 2 pi / omega, plotted against the amplitude f).
 *   Y        device array B x (N+1) x dim, the layout fabm_solve_batch writes
 *            (out_on_device = 1); row n of trajectory b is t_n = n h;
 *   N_each   device array of B per-trajectory step counts (rows beyond N_each[b]
 *            are not read), or NULL for N;
 *   samples  device array B x n_samples: samples[b][j] = component comp of
 *            trajectory b at t = t0 + j period, linearly interpolated between the
 *            two grid points around it; NaN where t lies outside [0, N_each[b] h]
 *            or N_each[b] is outside 1..N.
 * Caller-owned device memory; runs on the current device and synchronizes it.
 * FABM_EINVAL for NULL pointers, B or n_samples < 0, N < 1, dim outside
 * 1..FABM_MAX_DIM, comp outside 0..dim-1, h or period not positive, t0 not
 * finite; FABM_ECUDA if the launch fails. */
fabm_status fabm_stroboscope(const double *Y, int64_t B, int64_t N, int dim,
                             const int64_t *N_each, double h, double t0, double period,
                             int64_t n_samples, int comp, double *samples);

/* Number of kernel launches made by the last solve call on this solver. */
int64_t fabm_last_launch_count(const fabm_solver *s);

/* Kernel classes for fabm_kernel_stats. */
enum {
    FABM_KERNEL_WEIGHTS = 0,     /* weight generation (fabm_create)                    */
    FABM_KERNEL_INIT = 1,        /* y_0, f_0                                           */
    FABM_KERNEL_HISTORY = 2,     /* history sums (the O(N^2) part): far segments and,  */
                                 /* tensor path, the newest segment                    */
    FABM_KERNEL_COMBINE = 3,     /* fixed-order combination of history partial sums    */
    FABM_KERNEL_RECURRENCE = 4,  /* in-block predictor/corrector steps (tensor path:   */
                                 /* also the table of the time-only part of f)         */
    FABM_KERNEL_SLICE = 5,       /* split path conversions: f of a finished block ->   */
                                 /* bf16 slices; float-float y -> double at the end    */
    FABM_KERNEL_KINDS = 6
};

/* Per-launch timing.  period > 0 enables it: the launches of every period-th
 * time block (and the initial launch) are bracketed by CUDA events recorded on
 * the stream they run on, and the elapsed times are added up when the solve
 * call returns; period = 1 times every launch, a larger period samples the
 * blocks uniformly and keeps the event overhead small.  period = 0 disables
 * it.  Enabling resets the counters. */
fabm_status fabm_set_timing(fabm_solver *s, int period);

/* Counters since timing was enabled, for one kernel class (timed launches only):
 *   launches  number of timed launches
 *   total_ms  sum of their CUDA-event durations
 *   flops     algorithmic floating-point operations they performed (2 per
 *             multiply-add of a history term; 0 for classes with no history
 *             terms).  Any output pointer may be NULL. */
fabm_status fabm_kernel_stats(const fabm_solver *s, int kind, int64_t *launches, double *total_ms,
                              double *flops);
/* Milliseconds during which the timed launches of one kind ran (the union of
 * their intervals, so launches that overlap on different streams count once);
 * equal to fabm_kernel_stats' total_ms when they never overlap. */
fabm_status fabm_kernel_busy(const fabm_solver *s, int kind, double *busy_ms);

/* ------------------------------------------------------------ serving ---
 * A continuous-batching server for independent solves that differ in right-
 * hand side, dim, alpha, h and N.  Requests wait in arrival order and are
 * admitted while the device memory they need (weights, history, output,
 * partial sums: about (5 dim + 3) x 8 x N bytes) fits in the budget.  Each
 * fabm_server_step advances every admitted request by one block of 32 steps
 * with launches shared by all of them (the history of each request's next
 * block beside the recurrence of its current block), frees finished requests
 * and admits waiting ones; a request's weights and initial values are computed
 * during the step that admits it, and it runs its first block at the next.  A request's result does not depend on the other
 * requests in flight.  Precision FABM_FP64 sums the history in double,
 * FABM_SPLIT in compensated fp32 (requests have few columns, so tensor tiles
 * would be mostly padding); per-step updates and accumulators are double in
 * both.  Calls on one server are serialized by a mutex. */
typedef struct fabm_server fabm_server;

typedef struct {
    int dim;               /* 1..FABM_MAX_DIM, matching rhs_id */
    double alpha;          /* 0 < alpha < 2 (y'(0) = 0 for alpha > 1 unless given) */
    double h;              /* step size > 0 */
    int64_t N;             /* steps, 1..2^31 */
    int rhs_id;            /* FABM_RHS_* */
    const double *params;  /* n_params doubles, copied at submission */
    int n_params;
    const double *y0;      /* dim doubles, copied at submission */
} fabm_request;

enum { FABM_REQ_WAITING = 0, FABM_REQ_RUNNING = 1, FABM_REQ_DONE = 2, FABM_REQ_FAILED = 3 };

/* budget_bytes: device memory the admitted requests may hold together;
 * max_slots: most requests in flight at once. */
fabm_status fabm_server_create(size_t budget_bytes, int precision, int max_slots,
                               fabm_server **out);
/* Queue a request (copied); *ticket identifies it.  For 1 < alpha < 2 the
 * Taylor part of the initial data is y0 alone (y'(0) = 0). */
fabm_status fabm_server_submit(fabm_server *s, const fabm_request *req, int64_t *ticket);
/* As fabm_server_submit with y'(0) for 1 < alpha < 2 (Sec. 2: the Taylor part
 * y0 + t y'(0)).  y1: dim doubles (host, copied); NULL means zero.
 * FABM_EINVAL if y1 is given for alpha <= 1 or holds a non-finite value. */
fabm_status fabm_server_submit_ic(fabm_server *s, const fabm_request *req, const double *y1,
                                  int64_t *ticket);
/* One scheduling step (synchronous): admit, advance all requests admitted at
 * earlier steps by one block, retire finished ones.  Reports the requests in
 * flight and waiting. */
fabm_status fabm_server_step(fabm_server *s, int *n_active, int *n_waiting);
/* State of a request: FABM_REQ_*. */
fabm_status fabm_server_poll(fabm_server *s, int64_t ticket, int *state);
/* Copy a finished request's y_0..y_N ((N+1) x dim doubles, host) and forget it.
 * FABM_EBUSY if it has not finished; the request's own error if it failed
 * (FABM_ENONFINITE, or FABM_ENOMEM when it can never fit the budget). */
fabm_status fabm_server_result(fabm_server *s, int64_t ticket, double *out);
/* Step the server (fabm_server_step, advancing every admitted request) until
 * the request has finished, then fabm_server_result into out.  Errors as
 * fabm_server_result, or a step's error; FABM_EINVAL for an unknown ticket. */
fabm_status fabm_server_wait(fabm_server *s, int64_t ticket, double *out);
/* Checkpoint of a waiting or running request at the current block boundary:
 * its problem, the index of the next block, the history f and solution rows
 * computed so far, the far-history sums of the next block and its status,
 * serialized into buf (host memory, cap bytes, in the host's byte order).
 * *size receives the bytes needed; with buf NULL only the size is reported.
 * The request keeps running; fabm_server_cancel after a checkpoint evicts it
 * (its device memory is released).  FABM_EINVAL for an unknown or finished
 * ticket or cap < *size. */
fabm_status fabm_server_checkpoint(fabm_server *s, int64_t ticket, void *buf, size_t cap,
                                   size_t *size);
/* Queue a request from a checkpoint taken on a server of the same precision
 * (this one or another); once admitted it continues from the saved block and
 * gives the same result, bit for bit, as a run that was never interrupted.
 * FABM_EINVAL for a buffer that is not a consistent checkpoint or a precision
 * mismatch. */
fabm_status fabm_server_resume(fabm_server *s, const void *buf, size_t size, int64_t *ticket);
/* Steps N and dimension of a known request (for sizing the result buffer of a
 * resumed one).  FABM_EINVAL for an unknown ticket. */
fabm_status fabm_server_shape(fabm_server *s, int64_t ticket, int64_t *N, int *dim);
/* Drop a request in any state; a running one releases its device memory at
 * once.  The ticket becomes unknown.  FABM_EINVAL for an unknown ticket. */
fabm_status fabm_server_cancel(fabm_server *s, int64_t ticket);
/* Tickets of requests that finished (done or failed) since the last call, in
 * the order they finished: up to max of them into tickets, their number in *n;
 * the rest are kept for the next call.  Saves polling every request. */
fabm_status fabm_server_finished(fabm_server *s, int64_t *tickets, int max, int *n);
/* Steps run, kernel launches made, device bytes held by admitted requests. */
fabm_status fabm_server_stats(const fabm_server *s, int64_t *steps, int64_t *launches,
                              size_t *bytes_in_use);
fabm_status fabm_server_destroy(fabm_server *s);

/* One FP64 trajectory (as fabm_solve with precision FABM_FP64) without any
 * device allocation, for callers that cannot allocate device memory when they
 * solve: a framework's caching allocator may own the whole device-memory
 * budget, cudaMalloc/cudaFree synchronize the device, or the host process may
 * forbid a plug-in allocations of its own.  The paper has no counterpart; it
 * is a deployment variant of the same kernels.
 *   dim, alpha, h, N, rhs_id, params, n_params  as for fabm_create
 *                                                (N <= 65536, dim <= FABM_MAX_DIM)
 *   y0   dim doubles, host;  out  (N+1) x dim doubles, host, row n = y_n
 * All device buffers (weights, history, split-k partials) live in one static
 * device array of about 7 MB that every GPU loading the library holds until
 * the process exits.  Calls share that array and keep the last call's data;
 * calls are serialized by a host mutex, and work overlapping on the GPU with
 * another user of the array would race.  Every call looks up the array's
 * device address in the calling thread's current context (the address changes
 * after cudaDeviceReset or in another context); the first call in a context may
 * load the library's device code there: make it before any stream capture.
 * Runs on the calling thread's per-thread default stream; synchronous.
 * Errors: FABM_EINVAL (incl. N or dim beyond the array's limits, with a
 * message saying so), FABM_ECUDA, FABM_ENONFINITE. */
fabm_status fabm_solve_noalloc(int dim, double alpha, double h, int64_t N, int rhs_id,
                               const double *params, int n_params, const double *y0, double *out);

#ifdef __cplusplus
}
#endif
#endif /* FABM_H */
