/*
 * sbo.h -- C ABI of libsbo, a GB300 (sm_103a) implementation of the batched primal-dual
 * gradient descent-ascent of PDBO ("Smoothing Binary Optimization: A Primal-Dual
 * Perspective", arXiv 2509.21064).
 *
 * Problem (Eq. 1 with the QUBO objective):   min_{x in {0,1}^n}  F(x) = x^T Q x + c^T x.
 * The library works on the multilinear form of F (Prop. 2.4):
 *     f(x) = 1/2 x^T A x + c'^T x,   A_ij = Q_ij + Q_ji (i != j), A_ii = 0,   c' = c + diag(Q),
 * and on the Lagrangian L(x, y) = f(x) + sum_i y_i g(x_i) with g(x) = x^2 - x (section 3.1,
 * section 4.2).  One iteration of Algorithm 1 for every restart r and coordinate i:
 *     d_i = (A x)_i + c'_i + y_i (2 x_i - 1)
 *     if |x_i - 1/2| <= delta and |d_i| <= grad_tol and y_i <= 0:  x_i <- 1/2 -/+ delta
 *     else                                                          x_i <- clip(x_i - alpha d_i, 0, 1)
 *     y_i <- y_i + beta (x_i^2 - x_i)              (old x_i: simultaneous updates, Eq. 5)
 * B restarts run together; every K iterations (and at T) each restart is rounded to
 * b = [x > 1/2], F(b) is evaluated exactly in int64, and the best candidate is retained
 * (section 4.2).  x^0 ~ Uniform([0,1]^n) and y^0 = ybar (App. C.1).
 *
 * Conventions for every call:
 *   - Every call returns an sbo_status and never aborts, throws or exits; the message of the
 *     last failure on the calling thread is available from sbo_last_error().
 *   - Host input arrays are owned by the caller and are copied (or fully consumed) before the
 *     call returns.  Host output arrays are allocated by the caller.  "_dev" arguments are
 *     device pointers owned by the caller.
 *   - A problem handle owns all device memory it allocates, until sbo_destroy.
 *   - Work is enqueued on the stream given at creation (a cudaStream_t passed as void*;
 *     NULL means the legacy default stream).  Calls that return results to the host
 *     synchronise that stream first.
 *   - Integer data: Q, c are int32.  The exactness rules below are checked at creation and
 *     violations return SBO_ERANGE.
 */
#ifndef SBO_H_
#define SBO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sbo_status {
  SBO_OK = 0,
  SBO_EINVAL = 1,     /* invalid argument (null pointer, bad size, malformed CSR, bad parameter) */
  SBO_ENOMEM = 2,     /* device or host allocation failed */
  SBO_ECUDA = 3,      /* a CUDA runtime/driver call failed, or no usable device */
  SBO_ETIMEOUT = 4,   /* a bounded device-side wait gave up; the kernel returned early */
  SBO_ENOTREADY = 5,  /* results requested before any evaluation took place */
  SBO_ERANGE = 6,     /* data not exactly representable at the requested precision */
  SBO_EDEVICE = 7     /* the device reported an inconsistent state (bounds check failed) */
} sbo_status;

typedef enum sbo_precision {
  SBO_FP32 = 0,       /* A stored FP32, x operand FP32, FP32 accumulation (CUDA cores) */
  SBO_BF16 = 1,       /* A stored BF16 (|A_ij| <= 256), x operand BF16 (RN from the FP32
                         master), FP32 accumulation; dense: tcgen05 tensor cores */
  SBO_FP8_E4M3 = 2    /* sparse only: weights stored E4M3 (|A_ij| <= 16), x operand BF16,
                         FP32 accumulation */
} sbo_precision;

typedef struct sbo_problem sbo_problem;  /* opaque, library-owned */

/* Hyper-parameters of one batched run (Algorithm 1; App. C.1). */
typedef struct sbo_gda_params {
  int32_t restarts;    /* B >= 1 */
  int32_t eval_every;  /* K >= 1: rounding + exact objective at t = K, 2K, ... and at t = iters */
  int64_t iters;       /* T >= 0 */
  double alpha;        /* primal step, > 0 */
  double beta;         /* dual step, >= 0 */
  double ybar;         /* y^0 = ybar * 1 */
  double delta;        /* perturbation tolerance, 0 <= delta < 0.5 */
  double grad_tol;     /* gradient threshold of the perturbation rule (Algorithm 1: 2*delta) */
  uint64_t seed;       /* x^0_{r,i} = top 24 bits of SplitMix64 output r*2^32+i, times 2^-24 */
} sbo_gda_params;

/* ---- creation ------------------------------------------------------------------------
 * sbo_create_dense: Q is n*n row-major int32 on the host; c is n int32 on the host or NULL
 * (zero).  precision: SBO_FP32 or SBO_BF16.  Requires 1 <= n <= 65536, every
 * |A_ij| <= 256 (BF16) or <= 2^24 (FP32), every row sum sum_j |A_ij| < 2^24 (exact FP32
 * accumulation of A b for the objective), and |c'_i| < 2^31.  A is canonicalised on the
 * device (Prop. 2.4).  stream: cudaStream_t or NULL.  On success *out receives the handle.
 */
sbo_status sbo_create_dense(int64_t n, const int32_t* Q, const int32_t* c, int32_t precision,
                            void* stream, sbo_problem** out);

/* sbo_create_dense_i8: the same problem from an int8 Q (entries in [-128, 127]; c as above):
 * a quarter of the bytes to copy to the device, the same canonical form and checks. */
sbo_status sbo_create_dense_i8(int64_t n, const int8_t* Q, const int32_t* c, int32_t precision, void* stream,
                               sbo_problem** out);

/* sbo_create_csr (Eq. 1 with the QUBO objective for a sparse Q, put in the multilinear form of
 * Prop. 2.4; Max-Cut enters as Q = W, c = -W 1, the graph form of section 4.2):
 * Q in CSR on the host: rowptr[n+1] (int64, rowptr[0]=0, non-decreasing,
 * rowptr[n]=nnz), col[nnz] (int32 in [0,n)), val[nnz] (int32); duplicates are summed.
 * c as above.  precision: SBO_FP32, SBO_BF16 or SBO_FP8_E4M3 (weight storage).  A = Q + Q^T
 * with zero diagonal is formed on the host.  Requires 1 <= n < 2^31 and the exactness
 * rules above (|A_ij| <= 16 for E4M3). */
sbo_status sbo_create_csr(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                          const int32_t* val, const int32_t* c, int32_t precision,
                          void* stream, sbo_problem** out);

/* sbo_create_maxkcut: Max-k-Cut on a weighted graph (the paper's appendix on Max-k-Cut): edges
 * (ei[e], ej[e]) with integer weight w[e], each listed once (int32 ends in [0, n), no self-loops;
 * duplicates are summed), k parts with 2 <= k <= 8.  Every vertex carries k logits Z_:,i and the
 * point X_:,i = softmax(Z_:,i) of the simplex; sbo_gda runs the simultaneous gradient
 * descent-ascent of section 3.2 on L(X, y) = Tr(X W X^T) + sum_i y_i (|X_:,i|^2 - 1) with
 * Z^0_{r,i,j} = the x^0 generator at index i k + j and y^0 = ybar (x0, y0 must be NULL).
 * Candidates are argmax parts (ties to the smallest index), scored F = -(weight of the cut);
 * sbo_best and sbo_eval use one byte per vertex holding its part, and sbo_state reports X as
 * [restart][vertex][part] (B n k floats) and y as [restart][vertex].  FP32 throughout; weights
 * and row sums of |w| must stay below 2^24.  Not available: grouped runs, sbo_lagrangian,
 * SBO_OPT_DUAL = 1. */
sbo_status sbo_create_maxkcut(int64_t n, int64_t m, const int32_t* ei, const int32_t* ej, const int32_t* w, int32_t k,
                              void* stream, sbo_problem** out);

/* ---- the batched GDA run ----------------------------------------------------------------
 * sbo_gda_start: (re)initialises the run: allocates the state for B = prm->restarts,
 * x^0 from x0 (host, B*n float32 row-major [r][i], values in [0,1]) or, when x0 is NULL,
 * from the SplitMix64 rule of prm->seed; y^0 = ybar; clears every best.  Asynchronous.
 * sbo_gda_run: enqueues `iters` more iterations (the iteration counter continues), with
 * evaluations at t = K, 2K, ... and t = prm->iters.  Asynchronous.  A sparse run replayed from
 * CUDA graphs may leave the evaluation of its latest evaluation point pending (it then runs beside
 * the next block's iterations); sbo_sync, sbo_best, sbo_restart_best and sbo_trace complete it
 * first, so every result they report covers all evaluation points up to the current t.
 * sbo_gda: start (x0 = NULL) + run(prm->iters) + synchronise.  A handle may run again:
 * each start begins afresh. */
sbo_status sbo_gda_start(sbo_problem* p, const sbo_gda_params* prm, const float* x0);
/* sbo_gda_start_xy: as sbo_gda_start, with the initial duals y0 (host, B*n float32 [r][i], finite)
 * given by the caller instead of ybar (y0 NULL: ybar) -- a warm start, or the continuation of a
 * run saved with sbo_state.  The paper starts from y0 = ybar * 1 (App. C.1). */
sbo_status sbo_gda_start_xy(sbo_problem* p, const sbo_gda_params* prm, const float* x0, const float* y0);
sbo_status sbo_gda_run(sbo_problem* p, int64_t iters);
sbo_status sbo_gda(sbo_problem* p, const sbo_gda_params* prm);

/* sbo_sync (no passage: the end of an asynchronous run of Algorithm 1's loop):
 * waits for the problem's stream; returns SBO_ETIMEOUT / SBO_EDEVICE if a kernel
 * raised the device error word since the last sync (the word is then cleared). */
sbo_status sbo_sync(sbo_problem* p);

/* ---- results (all synchronise first) ---------------------------------------------------
 * sbo_eval (Eq. 1: F(b) = b^T Q b + c^T b at binary points): exact F of `count` binary vectors bits[count*n] (host, 0/1 bytes), into F[count]
 * (host int64), computed on the device with the same kernels as the run's evaluations. */
sbo_status sbo_eval(sbo_problem* p, int64_t count, const uint8_t* bits, int64_t* F);

/* sbo_best (section 4.2: the best of the B runs is retained): global best over all evaluations so
 * far: lexicographic minimum of (F, t, r).
 * x_out (host, n bytes, may be NULL), F_out, iter_out (t), restart_out (r) may be NULL.
 * SBO_ENOTREADY before the first evaluation. */
sbo_status sbo_best(sbo_problem* p, uint8_t* x_out, int64_t* F_out, int64_t* iter_out,
                    int32_t* restart_out);

/* sbo_restart_best (section 4.2, per run of the batch; the earliest t is what the time-to-best
 * measure of the same section reads): per-restart best F and the earliest t that reached it (host arrays of
 * B entries; INT64_MAX / -1 for a restart not yet evaluated). */
sbo_status sbo_restart_best(sbo_problem* p, int64_t* F, int64_t* t);

/* sbo_state (Algorithm 1: the primal-dual iterate (x^t, y^t) of every restart): FP32 copies of the
 * current iterates, X and Y (host, B*n each, [r][i]). */
sbo_status sbo_state(sbo_problem* p, float* X, float* Y);

/* sbo_gradient: the gradient d = dL/dx (Algorithm 1 with Eq. 5: (A x)_i + c'_i + y_i g'(x_i)) that
 * the latest iteration took at (x^{t-1}, y^{t-1}), exactly as the update kernel computed it
 * (host, B*n floats, [r][i]).  Needs SBO_OPT_KEEP_GRAD = 1 at sbo_gda_start and t >= 1, else
 * SBO_ENOTREADY.  Not for Max-k-Cut runs. */
sbo_status sbo_gradient(sbo_problem* p, float* G);

/* sbo_trace (section 4.2: best of the B runs at each evaluation point, the data behind that
 * section's earliest time to the best solution): min_r F at every evaluation so far, in order (host int64[cap]); *count gets
 * the number of evaluations (may exceed cap; only the first cap are written). */
sbo_status sbo_trace(sbo_problem* p, int64_t* minF, int64_t cap, int64_t* count);

/* ---- differentiation -----------------------------------------------------------------------
 * sbo_lagrangian: value and gradients of the Lagrangian (section 3.1) at B points:
 *     L[r] = 1/2 x_r^T A x_r + c'^T x_r + sum_i y_ri (x_ri^2 - x_ri)
 *     GX[r,i] = (A x_r)_i + c'_i + y_ri (2 x_ri - 1),   GY[r,i] = x_ri^2 - x_ri
 * X_dev, Y_dev: device float32 [B][n] row-major (caller-owned).  gout_dev (device float32 [B],
 * may be NULL = all ones) scales row r of GX and GY (the adjoint of a per-restart upstream
 * gradient).  L_dev (B), GX_dev, GY_dev (B*n) are device float32 outputs; any may be NULL.  A x is recomputed on every
 * call (nothing is cached between calls), with the contraction of the problem's precision.
 * stream: cudaStream_t or NULL; the call is asynchronous on it.  Scratch for the operand is kept
 * by the handle: B*n*2 bytes (dense BF16), or n*round_up(B,8)*4 (CSR FP32) or *2 (CSR BF16 /
 * E4M3) bytes in the sparse kernels' variable-major layout.  Dense and CSR QUBO problems; not
 * Max-k-Cut. */
sbo_status sbo_lagrangian(sbo_problem* p, int32_t B, const float* X_dev, const float* Y_dev,
                          const float* gout_dev, float* L_dev, float* GX_dev, float* GY_dev,
                          void* stream);

/* sbo_dual_bound: a certified lower bound on min F (the paper's section on the dual certificate).
 * With y = ybar * 1 and ybar large enough that L(., y) is convex on [0,1]^n (for Max-Cut:
 * ybar >= -lambda_min(W); in general A + 2 ybar I positive semidefinite -- the caller's
 * responsibility, the library does not check it), min over the box of L(., y) <= min F, and for
 * any box point x, L(x) + min over the box of <grad L(x), z - x> <= min over the box of L.  This
 * call runs `iters` projected gradient steps of size alpha on L(., ybar) (the GDA of section 3.2
 * with beta = 0 and one restart: it replaces the problem's current run), polishes the point with
 * min(iters, 500) FP64 projected gradient steps, then forms that bound in FP64 from an FP64
 * product A x: *lower_bound gets it, *value (may be NULL) L(x).  For Max-Cut the
 * cut is at most -(*lower_bound).  QUBO problems only (dense or CSR). */
sbo_status sbo_dual_bound(sbo_problem* p, double ybar, double alpha, int64_t iters, double* lower_bound,
                          double* value);

/* sbo_lagrangian_noalloc: the same computation and arguments as sbo_lagrangian, for dense
 * problems, for callers that cannot allocate device memory -- processes whose device memory
 * belongs to a framework's pool or a fixed budget, and loops that cannot absorb cudaMalloc's
 * implicit synchronisation.  The paper has no counterpart: this is a property of the library,
 * not of the method.  CSR problems return SBO_EINVAL.  It calls no
 * cudaMalloc/cudaFree or other allocating routine; for BF16 problems it stages the BF16 copy
 * of X in one fixed 16 MiB device array that every GPU loading the library holds until the
 * process exits, so it requires B * round_up(n, 8) * 2 <= 16 MiB and returns SBO_EINVAL
 * otherwise (FP32 problems need no scratch and have no limit).  The first call on a device,
 * with that device current, looks up the array's address; make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on the GPU race. */
sbo_status sbo_lagrangian_noalloc(sbo_problem* p, int32_t B, const float* X_dev, const float* Y_dev,
                                  const float* gout_dev, float* L_dev, float* GX_dev, float* GY_dev,
                                  void* stream);

/* ---- execution options -------------------------------------------------------------------
 * sbo_set_option: selects execution details; values take effect at the next sbo_gda_start.
 * SBO_OPT_USE_GRAPH also applies to the next sbo_gda_run of the current run, and SBO_OPT_PDL and
 * SBO_OPT_TIMEOUT_US to its directly launched kernels (replayed graphs keep the values they were
 * captured with until the next start); results depend on none of the three.
 *   SBO_OPT_KERNEL:     0 auto, 1 SIMT FP32 (plain form), 2 tcgen05 (BF16 dense),
 *                       3 tiny-n single-CTA loop (n <= 64, FP32)
 *   SBO_OPT_USE_GRAPH:  1 (default) replay blocks of K iterations from a CUDA graph; 0 launch
 *                       every kernel directly
 *   SBO_OPT_TILE_N:     restarts per tensor-core tile: 0 auto, 64, 128 or 256 (one SM per
 *                       128-row tile), 512: CTA pairs (two SMs per 256 x 256 tile), or
 *                       1064, 1128, 1256: width 64, 128, 256 with the K dimension of every tile
 *                       split over a thread-block cluster of 2-8 SMs, reduced in split order
 *                       through L2 (problems with at most half as many tiles as SMs; others
 *                       fall back to the plain width), or 2128, 2256: the same on CTA pairs, tiles
 *                       of 256 rows x 128 or 256 restarts with the K dimension split over 2-4
 *                       pairs (others fall back to plain tiles of 64 or 128)
 *   SBO_OPT_AUTOTUNE:   1 (default): with SBO_OPT_TILE_N = 0, sbo_gda_start times the tcgen05
 *                       update kernel at every tile width on the run's own buffers and keeps
 *                       the fastest; decisions are cached per (device, n, B, SM count) in the
 *                       process and in the file named by the environment variable
 *                       SBO_TUNE_CACHE (default ~/.cache/sbo/tile_tuning.txt; "off" disables
 *                       the file); 0: a fixed rule
 *   SBO_OPT_SPLIT_K:    largest split-K factor for the tensor-core tiles left over after whole
 *                       rounds over the SMs (default 16; 0 or 1 disables splitting).  Split
 *                       tiles are summed in a fixed order, so results do not depend on it.
 *   SBO_OPT_TIMEOUT_US: budget in microseconds of every bounded device-side wait (default
 *                       4,000,000); on expiry the kernel returns early and sbo_sync reports
 *                       SBO_ETIMEOUT
 *   SBO_OPT_PDL:        1 (default): the sparse kernel's iterations are launched as programmatic
 *                       dependents of the previous kernel (the launch of iteration t+1 overlaps
 *                       iteration t; results identical); 0: plain stream order
 *   SBO_OPT_DUAL:       0 (default): one dual y_i per coordinate (PDBO, Algorithm 1); 1: one dual
 *                       mu per restart on the single constraint sum_i g(x_i) = 0 (the PDBO-s
 *                       variant of section 4's discussion and ablation): the same primal step and
 *                       perturbation rule with mu in place of y_i, and mu <- mu + beta sum_i g(x_i)
 *                       on the old x.  Set before sbo_gda_start; y0 then gives mu0_r = y0[r*n];
 *                       sbo_state reports mu_r in every coordinate of restart r.  Not available in
 *                       grouped runs or the tiny kernel (FP32 problems with n <= 64 use SIMT)
 *   SBO_OPT_G:          constraint function g of the Lagrangian (section 3.1): 0 (default) the
 *                       quadratic x^2 - x; 1 the entropy x log x + (1 - x) log(1 - x) (g(0) = g(1)
 *                       = 0), whose derivative log(x / (1 - x)) is taken at x clamped to
 *                       [1e-6, 1 - 1e-6].  Applies to the run (update and dual step) and to
 *                       sbo_lagrangian; QUBO problems only; sbo_dual_bound always uses the quadratic
 *                       g
 *   SBO_OPT_KEEP_GRAD:  0 (default); 1: every update also writes the gradient d it used into a
 *                       run-owned buffer (4 B per element more device memory and store traffic),
 *                       read with sbo_gradient -- for checking the loop's own gradients.  Set
 *                       before sbo_gda_start; QUBO problems only
 *   SBO_OPT_CSR_FORM:   form of the sparse update kernel: 0 (default) chosen by the autotuner at
 *                       sbo_gda_start (with SBO_OPT_AUTOTUNE = 0: a fixed rule on n, B and the L2
 *                       size), 1 one row per warp with 128 restarts, 2 one row per warp with 256
 *                       restarts, 3 rows strided over one resident wave and software-pipelined (256
 *                       restarts per warp), 4 rows staged in shared memory by bulk copies (a
 *                       producer warp and four consumer warps per CTA), 5, 6, 7 the forms 1, 2, 3
 *                       with L2 eviction priorities for state that overflows L2 (each row's own x
 *                       and y evict-first, the operand written for the next iteration evict-last),
 *                       8 resident: one cooperative CTA per SM (seven SMs in eight) keeps its rows'
 *                       x, y and structure in shared memory for all the iterations of a launch
 *                       (grid barrier between them; graphs whose state fits, about n B <= 3e6 on
 *                       152 SMs; the evaluations beside the next block keep to the SMs left free;
 *                       explicit only, not an autotuner candidate).
 *                       Results are identical in
 *                       every form; the single-constraint form (SBO_OPT_DUAL = 1) keeps the rule
 *   SBO_OPT_EVAL_MODE:  scheduling of the evaluations of sparse and Max-k-Cut runs replayed from
 *                       graphs with K >= 2: 0 (default) and 2 on a graph branch beside the next
 *                       block's steps, 1 in line after each block.  Results are identical in both
 *   SBO_OPT_STEPS_PER_LAUNCH: largest number of GDA iterations one launch of the cluster split-K
 *                       kernel (tile codes 1064-2256) or of the resident sparse form (SBO_OPT_CSR_FORM
 *                       8) runs, with per-coordinate duals: 0 (default)
 *                       4,096, 1 one launch per iteration.  The iterations of a launch meet at a
 *                       grid-wide barrier, so such a launch is cooperative (scheduled only when all
 *                       its CTAs can be resident at once); a wait that outlasts SBO_OPT_TIMEOUT_US
 *                       makes the launch return early with SBO_ETIMEOUT.  Results are identical for
 *                       every value */
enum { SBO_OPT_KERNEL = 1, SBO_OPT_USE_GRAPH = 2, SBO_OPT_TILE_N = 3, SBO_OPT_TIMEOUT_US = 4, SBO_OPT_SPLIT_K = 5,
       SBO_OPT_AUTOTUNE = 6, SBO_OPT_PDL = 7, SBO_OPT_DUAL = 8, SBO_OPT_G = 9, SBO_OPT_KEEP_GRAD = 10,
       SBO_OPT_CSR_FORM = 11, SBO_OPT_EVAL_MODE = 12, SBO_OPT_STEPS_PER_LAUNCH = 13 };
sbo_status sbo_set_option(sbo_problem* p, int32_t option, int64_t value);

/* sbo_info: n, restarts of the current run, the kernel chosen (values of SBO_OPT_KERNEL; 4 the
 * sparse QUBO kernel, 5 the Max-k-Cut kernel), the tile width (dense tensor-core runs) or the
 * sparse update's form (values of SBO_OPT_CSR_FORM, 0 the rule) and the iteration counter t; any
 * pointer may be NULL. */
sbo_status sbo_info(const sbo_problem* p, int64_t* n, int32_t* restarts, int32_t* kernel,
                    int32_t* tile_n, int64_t* t);

/* ---- grouped runs (heterogeneous batches) ---------------------------------------------------
 * A group advances several dense BF16 problems of different n together: every iteration is
 * one persistent tcgen05 launch over the tiles of all members (ordered by decreasing n), and
 * every evaluation one grouped launch plus each member's best bookkeeping (section 4.2 per
 * member).  Members stay owned by the caller and keep their own state and results: read them
 * with sbo_best / sbo_state / sbo_trace on each member after sbo_group_sync.
 * sbo_group_create: count >= 1 distinct dense BF16 problems; stream as for sbo_create_dense.
 * sbo_group_start: prms[count]; members share iters and eval_every (else SBO_EINVAL); starts
 *   every member (x^0 from its seed) on the group's tile width.
 * sbo_group_run / sbo_group_sync: as sbo_gda_run / sbo_sync for the whole group.
 * sbo_group_set_option: SBO_OPT_USE_GRAPH, SBO_OPT_TILE_N (64, 128 or 256 restarts per tile; default
 * 0: sbo_group_start times each width on the group's own instance table over a few update launches
 * and keeps the fastest; set before start). */
typedef struct sbo_group sbo_group;
sbo_status sbo_group_create(int32_t count, sbo_problem* const* problems, void* stream, sbo_group** out);
sbo_status sbo_group_start(sbo_group* g, const sbo_gda_params* prms);
sbo_status sbo_group_run(sbo_group* g, int64_t iters);
sbo_status sbo_group_sync(sbo_group* g);
sbo_status sbo_group_set_option(sbo_group* g, int32_t option, int64_t value);
int64_t sbo_group_launch_count(const sbo_group* g);
void sbo_group_destroy(sbo_group* g);  /* NULL-safe; does not destroy the members */

/* Kernel launches enqueued by this handle since creation (every kernel of the library). */
int64_t sbo_launch_count(const sbo_problem* p);

void sbo_destroy(sbo_problem* p);      /* NULL-safe; synchronises the stream first */
const char* sbo_last_error(void);      /* thread-local; "" when the last call succeeded */
const char* sbo_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SBO_H_ */
