/*
 * fastpfp.h -- C ABI of the GB300 FastPFP solver (libfastpfp.so).
 *
 * FastPFP (Lu, Huang & Liu, "A Fast Projected Fixed-Point Algorithm for
 * Large Graph Matching") matches two undirected weighted attributed graphs:
 *
 *   max_X 1/2 tr(X^T A X A') + lambda tr(X^T K),  K = B B'^T       (Eq. 3)
 *   X 1 <= 1, X^T 1 = 1, X in {0,1}^{n x n'}, n >= n'               (Eq. 4)
 *
 * relaxed to partial doubly stochastic X and solved by the projected
 * fixed-point iteration (Eq. fastPFP, Algorithm 1)
 *
 *   Y[:, :n'] = A X A' + lambda K
 *   repeat { Y <- P1(Y) (Eq. P1);  Y <- max(Y, 0) (Eq. P2) } until Y converges
 *   X <- (1 - alpha) X + alpha Y[:, :n'];  X <- X / max(X)
 *
 * until X converges, followed by the greedy discretisation of Section 4.5.
 *
 * Conventions for every entry point
 *   - Matrices are dense, row-major, contiguous, float32.
 *   - "device" pointers are CUDA global memory on the handle's device; the
 *     caller owns them.  "host" pointers are ordinary host memory.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls that return statistics
 *     synchronise that stream before returning.
 *   - Every call returns FASTPFP_OK (0) or a negative FASTPFP_ERR_* code;
 *     fastpfp_error_string() names it.  On an error no output is valid.
 *   - Orientation: outputs are in the caller's orientation.  Internally the
 *     larger graph indexes the rows (Section 3 assumes n >= n'); the swap
 *     and the transposes are done by the library.
 *   - A handle is not thread safe: one host thread per handle at a time.
 */
#ifndef FASTPFP_H
#define FASTPFP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FASTPFP_OK 0
#define FASTPFP_ERR_ARG (-1)         /* null pointer, bad size, alpha outside [0,1] ...  */
#define FASTPFP_ERR_SIZE (-2)        /* a graph larger than the handle's max_n            */
#define FASTPFP_ERR_CUDA (-3)        /* a CUDA runtime call failed                        */
#define FASTPFP_ERR_TIMEOUT (-4)     /* a device-side barrier wait ran out of its budget  */
#define FASTPFP_ERR_NONFINITE (-5)   /* NaN or Inf met in the iterate                     */
#define FASTPFP_ERR_UNSUPPORTED (-6) /* option not available on this device / build       */

#define FASTPFP_MAX_N 16384          /* largest graph a handle can be created for         */
#define FASTPFP_MAX_K 256            /* largest attribute dimension k                     */

/* Precision of the A X A' products (FP32 accumulation throughout).  FP32:
 * the products of FP32 operands on the tensor cores, every operand split
 * into its TF32 part (rounded to 10 mantissa bits) and its FP32 remainder
 * and multiplied as hi*hi + hi*lo + lo*hi (relative error about 2^-21 per
 * product term, below the FP32 accumulation's own).  FP32_SIMT: the same
 * products on the FP32 FMA pipes (exact FP32 arithmetic).  BF16: both
 * operands of both products rounded to BF16.  FP8: both operands E4M3
 * (round to nearest even, saturating) with one power-of-two scale per
 * operand row, chosen so the row's largest magnitude maps to at most 448,
 * and both scales applied to the FP32 accumulator: A and A' are quantised
 * once per solve, X^T (through a BF16 copy) and T = A X (through its BF16
 * result) before each product.  BF16 and FP8 runs end with FP32
 * iterations (the FP32 products above). */
enum { FASTPFP_FP32 = 0, FASTPFP_BF16 = 1, FASTPFP_FP8 = 2, FASTPFP_FP32_SIMT = 3 };
enum { FASTPFP_ALG_FASTPFP = 0, FASTPFP_ALG_PG = 1, FASTPFP_ALG_FASTGA = 2 };

typedef struct fastpfp_s* fastpfp_t;

/* Parameters of one solve.  Defaults (fastpfp_default_params) follow the
 * paper where it fixes a value: alpha = 0.5 (Section 5), the uniform start
 * X = 1 1^T / (n n') and Y = 0 (after Algorithm 1), X <- X / max(X) on
 * (Remarks after Theorem 1). */
typedef struct {
    float lambda;          /* weight of the attribute term, Eq. (3); >= 0                     */
    float alpha;           /* step size of Eq. (fastPFP), in [0, 1]                           */
    double tol_outer;      /* eps_1: stop when max|X(t+1) - X(t)| < eps_1 (Section 5)         */
    double tol_inner;      /* eps_2: stop P_D when max|Y(u+1) - Y(u)| < eps_2 (Section 5)     */
    int max_outer;         /* I_0: at most this many outer iterations, >= 1                   */
    int max_inner;         /* I_1: at most this many P1/P2 rounds per outer iteration, >= 1   */
    int precision;         /* FASTPFP_FP32, FASTPFP_BF16, FASTPFP_FP8 or FASTPFP_FP32_SIMT for the
                              A X A' products                                                */
    int refine_iters;      /* BF16 / FP8: FP32 outer iterations run after the low-precision
                              phase                                                          */
    double switch_tol;     /* BF16 / FP8: the low-precision phase ends once max|dX| <
                              switch_tol, or once max|dX| shrinks by less than half in an
                              iteration (from its fourth iteration on: the products' rounding
                              noise is near)                                                 */
    int normalize_max;     /* 1: X <- X / max(X) after every outer iteration (Algorithm 1)     */
    int slack_policy;      /* 0: slack columns of Y carry over between outer iterations
                              (Algorithm 1 initialises Y once); 1: reset them to 0            */
    int timeout_ms;        /* budget of every device-side barrier wait; <= 0 means 2000 ms     */
    int profile;           /* 1: record CUDA events on `stream` around every phase of the first
                              128 outer iterations and report per-phase times in the stats;
                              implies loop_mode 1                                            */
    int loop_mode;         /* control of the repeat loop of Algorithm 1.  0: one CUDA graph per
                              solve (or wave), a while node around the outer iteration whose
                              condition a device kernel sets from the stop word after every
                              iteration (no host round trip inside a solve); 1: the host
                              enqueues outer iterations in chunks of 4 and polls the stop word
                              one chunk behind                                               */
    int debug_flags;       /* testing only, 0 in production.  Bit 0: CTA 0 of the first
                              projection launch skips its arrival at the first grid barrier, so
                              every wait of that launch runs out after timeout_ms and the call
                              returns FASTPFP_ERR_TIMEOUT (exercises failure detection without
                              faulting or hanging the device)                                 */
    int algorithm;         /* FASTPFP_ALG_FASTPFP (default): Eq. (fastPFP),
                              X <- (1 - alpha) X + alpha P_d(A X A' + lambda K);
                              FASTPFP_ALG_PG: the projected gradient method of Eq. (pg),
                              X <- P_d(X + alpha (A X A' + lambda K)) (normalize_max applies to
                              both);
                              FASTPFP_ALG_FASTGA: graduated assignment with C = A (x) A'
                              (Appendix, Eqs. GAO3/GAO4) at a fixed beta, the comparison method
                              of Section 5: X <- Y[:, :m] of Sinkhorn normalisation (rows, then
                              columns, to eps_2 or I_1) applied to exp(beta Q / max|Q|),
                              Q = A X A' + lambda K over the slacked N x N matrix (slack columns
                              0), to eps_1 or I_0;
                              precision FP32 or FP32_SIMT only; pairs of a batch run one after
                              another; alpha and normalize_max do not apply                   */
    float beta;            /* FASTPFP_ALG_FASTGA: the fixed inverse temperature beta > 0 of the
                              soft-assignment, applied to Q scaled by its largest magnitude (the
                              paper gives no value or schedule; default 100)                  */
} fastpfp_params;

/* Statistics of one solve (in the canonical orientation). */
typedef struct {
    int outer_iters;        /* outer iterations run                                          */
    int inner_iters_total;  /* P1/P2 rounds summed over all outer iterations                 */
    int inner_iters_max;    /* largest P1/P2 round count of one outer iteration              */
    int converged;          /* 1 if max|dX| < tol_outer was reached; 0 if I_0 stopped it     */
    int lowp_iters;         /* outer iterations run with BF16 or FP8 products                */
    int transposed;         /* 1 if the graphs were swapped (n_a < n_b)                      */
    int status;             /* FASTPFP_OK or the error code of this solve                    */
    int launches;           /* CUDA kernels this solve enqueued                              */
    int wave_pairs;         /* pairs that shared this solve's pdb_kernel launches (a wave of a
                               batched call); 0 when it ran alone through pd_kernel           */
    double final_delta;     /* last max|X(t+1) - X(t)|                                       */
    double objective;       /* Eq. (3) at the returned partial permutation                   */
    float ms_gemm;          /* profile = 1: summed time of the gradient products             */
    float ms_proj;          /* profile = 1: summed time of the projection launches           */
    float ms_disc;          /* profile = 1: time of the discretisation                       */
    int host_syncs;         /* host synchronisations the call made (stream or event waits) while
                               its work was in flight; the same for every pair of a batch     */
} fastpfp_stats;

/* One graph pair of a batch; all pointers are device pointers. */
typedef struct {
    const float* A;     /* n_a x n_a symmetric                       */
    const float* A2;    /* n_b x n_b symmetric                       */
    const float* B;     /* n_a x k, or NULL when k == 0              */
    const float* B2;    /* n_b x k, or NULL when k == 0              */
    int n_a, n_b, k;
    const float* X0;    /* nullable n_a x n_b start                  */
    int32_t* perm_out;  /* n_a entries                               */
    float* X_out;       /* nullable n_a x n_b                        */
} fastpfp_pair;

/* Fills *p with the defaults: lambda 0, alpha 0.5, tol_outer = tol_inner =
 * 1e-6, max_outer 100, max_inner 1000, FP32, refine_iters 8, switch_tol
 * 1e-3, normalize_max 1, slack_policy 0, timeout_ms 2000. */
void fastpfp_default_params(fastpfp_params* p);

/* Creates a solver on CUDA device `device` for graphs of up to max_n nodes.
 * All device scratch (the slacked N x N matrix Y of Section 4.3, X, K, the
 * products, the reduction buffers) is allocated here, sized for max_n, one
 * slot of it for each of the max_batch pairs one fastpfp_match_batched call
 * may carry (about 30 max_n^2 bytes per slot).  Nothing is allocated by the
 * solve calls.  Errors: ERR_ARG (max_n < 1, max_batch < 1,
 * out == NULL), ERR_CUDA (bad device, out of memory). */
int fastpfp_create(fastpfp_t* out, int device, int max_n, int max_batch);

/* Releases the handle and all its device memory.  NULL is ignored. */
void fastpfp_destroy(fastpfp_t h);

/* Solves one pair (Algorithm 1 followed by Section 4.5), all arrays on the
 * device.
 *   A   : n_a x n_a symmetric adjacency of graph 1 (Section 3)
 *   A2  : n_b x n_b symmetric adjacency of graph 2
 *   B,B2: n_a x k and n_b x k node attributes; may be NULL when k == 0 or
 *         p->lambda == 0
 *   X0  : nullable n_a x n_b start; NULL gives the uniform start 1/(n n')
 *   perm_out : n_a int32; perm_out[i] = node of graph 2 matched to node i of
 *              graph 1, or -1 when graph 1 is the larger one and i is left
 *              unmatched (every node of the smaller graph is matched, Eq. 4)
 *   X_out    : nullable n_a x n_b; receives the final soft assignment X
 *   st       : nullable host pointer; receives the statistics
 * Synchronises `stream`.  Errors: ERR_ARG, ERR_SIZE (max(n_a, n_b) > max_n),
 * ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE. */
int fastpfp_match(fastpfp_t h, void* stream,
                  const float* A, int n_a, const float* A2, int n_b,
                  const float* B, const float* B2, int k,
                  const fastpfp_params* p, const float* X0,
                  int32_t* perm_out, float* X_out, fastpfp_stats* st);

/* As fastpfp_match, but every array argument is HOST memory: the library
 * stages the inputs into its own device buffers, solves, and copies
 * perm_out (and X_out) back.  Synchronises `stream`. */
int fastpfp_match_host(fastpfp_t h, void* stream,
                       const float* A, int n_a, const float* A2, int n_b,
                       const float* B, const float* B2, int k,
                       const fastpfp_params* p, const float* X0,
                       int32_t* perm_out, float* X_out, fastpfp_stats* st);

/* Solves `count` independent pairs with the same parameters (Algorithm 1
 * per pair).  pairs[] is a host array of device-pointer descriptors; st is
 * a nullable host array of `count` statistics.  Pairs are solved in waves:
 * pairs whose slacked matrices fit on chip together (tensor memory plus
 * shared memory of all SMs; N <= 4096 each, at most 128 per wave) share one
 * projection launch per outer iteration.  A batch larger than one wave is
 * streamed: pairs that stopped leave the wave, waiting pairs join it in
 * batch order.  With loop_mode 0 (and profile 0) the waves are planned on
 * the device and the whole batch runs as one CUDA graph launch with one
 * host synchronisation; otherwise the host plans them between outer
 * iterations (the same plans, so the same results).  With profile = 1 a
 * wave's phase times are split equally between its pairs.  Synchronises
 * `stream`.  Errors as fastpfp_match, plus ERR_ARG when count > max_batch. */
int fastpfp_match_batched(fastpfp_t h, void* stream, int count, const fastpfp_pair* pairs,
                          const fastpfp_params* p, fastpfp_stats* st);

/* As fastpfp_match_batched, but every pointer of every descriptor is HOST
 * memory: each wave's inputs are copied into the handle's device staging,
 * solved, and perm_out (and X_out) copied back.  Synchronises `stream`. */
int fastpfp_match_batched_host(fastpfp_t h, void* stream, int count, const fastpfp_pair* pairs,
                               const fastpfp_params* p, fastpfp_stats* st);

/* Copies the per-outer-iteration trace of a pair of the last call on this
 * handle: inner_counts[t] = P1/P2 rounds of outer iteration t, deltas[t] =
 * max|X(t+1) - X(t)|.  `pair` is 0 after fastpfp_match / _host, and after
 * fastpfp_match_batched (or _host) the index of any pair within that call.
 * Either array may be NULL.  Returns the number of outer iterations (at most
 * cap entries are written), or ERR_ARG for an index outside the last call. */
int fastpfp_last_trace(fastpfp_t h, int pair, int* inner_counts, double* deltas, int cap);

/* ---- single steps of Algorithm 1, for step-by-step checking ------------ */

/* Gradient of Section 4.1 in canonical orientation (N >= m):
 *   Y[i, j] = sum_l (sum_q A[i,q] X[q,l]) A2[l,j] + lambda * K[i,j]
 * for i < N, j < m; Y has leading dimension ldy >= m.  A is N x N, X is
 * N x m, A2 is m x m, K is N x m (nullable when lambda == 0).  precision
 * selects FP32 (split TF32 on the tensor cores), FP32_SIMT, BF16 or FP8
 * products (FP32 accumulation; each quantises as the solve does, FP8's T
 * through a BF16 copy).  Device pointers;
 * asynchronous on `stream`.  Errors: ERR_ARG, ERR_SIZE, ERR_CUDA. */
int fastpfp_gradient(fastpfp_t h, void* stream, const float* A, const float* X, const float* A2,
                     const float* K, float lambda, int N, int m, float* Y, int ldy, int precision);

/* K = B B2^T (below Eq. 4): B is N x k, B2 is m x k, K is N x m, 1 <= k <=
 * 256.  Device pointers; asynchronous.  Errors: ERR_ARG, ERR_SIZE, ERR_CUDA. */
int fastpfp_affinity(fastpfp_t h, void* stream, const float* B, const float* B2, int N, int m,
                     int k, float* K);

/* Successive projection P_D of Section 4.3 in place on the N x N device
 * matrix Y (leading dimension N): rounds of P1 (Eq. P1, total taken over
 * Y) then P2 (Eq. P2) until max|dY| < tol or max_iter rounds.  *iters and
 * *last_delta (host, nullable) receive the rounds run and the last
 * max|dY|.  Synchronises `stream`.  Errors: ERR_ARG, ERR_SIZE, ERR_CUDA,
 * ERR_TIMEOUT. */
int fastpfp_project(fastpfp_t h, void* stream, float* Y, int N, double tol, int max_iter,
                    int* iters, double* last_delta);

/* Greedy discretisation of Section 4.5 of the N x m device matrix X
 * (N >= m): repeatedly takes the largest remaining entry, ties to the
 * lowest row-major index, and removes its row and column.  row_of_col
 * (device, m int32) receives the row matched to each column.  Bit-exact
 * with the sequential definition for finite X.  Asynchronous.  Errors:
 * ERR_ARG, ERR_SIZE, ERR_CUDA. */
int fastpfp_discretize(fastpfp_t h, void* stream, const float* X, int N, int m,
                       int32_t* row_of_col);

/* ---- learned warm start ----------------------------------------------------
 * The paper recommends the uniform start X = 1 1^T / (n n') and notes that
 * the result depends on the initialisation (discussion after Algorithm 1).
 * These calls build a learned start instead (not part of the paper):
 *   features  F_i = [zscore(deg)_i, hist_i[0..15], zscore(B)_i[0..14]] (32 per
 *             node): weighted degree, histogram of the node's nonzero
 *             incident weights in 16 bins of [0, 1] (clamped) divided by their
 *             count, the first 15 attributes; z-scores over the graph's nodes
 *   MLP       H = relu(F W1 + b1) (128), E = H W2 + b2 (64), one set of weights
 *             for both graphs
 *   start     S = E_big E_small^T / 8; X0 = sinkhorn_iters alternations of
 *             row and column normalisation of exp(S - max S)
 * params is a device array of FASTPFP_MLP_NPARAMS floats: W1 (32 x 128,
 * row-major), b1 (128), W2 (128 x 64), b2 (64). */
#define FASTPFP_MLP_NPARAMS (32 * 128 + 128 + 128 * 64 + 64)

/* X0_out (device, n_a x n_b, caller orientation) = the learned start of the
 * pair; use it as fastpfp_match's X0.  B/B2 may be NULL when k == 0.  Device
 * pointers; asynchronous on `stream`.  Errors: ERR_ARG, ERR_SIZE, ERR_CUDA. */
int fastpfp_warmstart(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2, int n_b,
                      const float* B, const float* B2, int k, const float* params, int sinkhorn_iters,
                      float* X0_out);

/* One training step on a pair whose matching `perm` (device, n_a entries,
 * as fastpfp_match returns it; every node of the smaller graph matched) is
 * the target.  Loss, with t(j) the row matched to column j in canonical
 * orientation and m the smaller graph's size:
 *   L = -(1/m) sum_j [S(t(j), j) - logsumexp_i S(i, j)]
 *       -(1/m) sum_j [S(t(j), j) - logsumexp_j' S(t(j), j')]
 * The gradient of L w.r.t. params is computed by hand-written backward
 * kernels; when step >= 1 an Adam update (beta 0.9 / 0.999, eps 1e-8, bias
 * correction for `step`) with learning rate lr is applied to params using
 * the device moments adam_m / adam_v (FASTPFP_MLP_NPARAMS floats each, start
 * at zero).  step == 0 only evaluates.  *loss_out (host, nullable; the call
 * then synchronises) receives L before the update; grad_out (device,
 * nullable) the gradient.  Errors: ERR_ARG, ERR_SIZE, ERR_CUDA. */
int fastpfp_warmstart_train_step(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2,
                                 int n_b, const float* B, const float* B2, int k, const int32_t* perm,
                                 float* params, float* adam_m, float* adam_v, int step, float lr,
                                 double* loss_out, float* grad_out);

/* ---- entry point for callers that cannot allocate -------------------------
 * The paper has no counterpart to this call; it exists for callers that are
 * not allowed to call cudaMalloc -- for example a plugin that a host
 * application hands a fixed device-memory arena (the application accounts
 * for every byte and refuses allocations made behind its back), or a
 * real-time loop that forbids allocation after start-up (cudaMalloc can
 * block and synchronise the device for an unbounded time).  Such callers
 * cannot create a handle, because fastpfp_create allocates.
 *
 * fastpfp_project_noalloc runs the same successive projection as
 * fastpfp_project, in place on the caller's N x N device matrix Y (row-major,
 * leading dimension N), on the CUDA device that is current.  It allocates
 * nothing: the projection's own scratch (column-sum accumulators, FP64
 * totals, round maxima, barrier and control words) is one file-scope device
 * array of about 130 KB that every GPU which loads this library holds until
 * the process exits.
 *   - N must be a multiple of 4 with 4 <= N <= 4096 and Y 16-byte aligned;
 *     larger N returns FASTPFP_ERR_SIZE, other shapes FASTPFP_ERR_ARG.
 *   - The first call on a device resolves the array's device address and sets
 *     the kernel's attributes for that device.
 *   - Every call on a device shares the one array: the call clears what must
 *     start at zero, but two calls whose work overlaps on the GPU (different
 *     streams, or different host threads) race on it and give wrong results.
 *   - Synchronises `stream`; *iters and *last_delta (host, nullable) as in
 *     fastpfp_project.  Errors: ERR_ARG, ERR_SIZE, ERR_CUDA, ERR_TIMEOUT. */
int fastpfp_project_noalloc(void* stream, float* Y, int N, double tol, int max_iter, int* iters,
                            double* last_delta);

/* Measures the bandwidth of a memory level that can hold the slacked
 * matrix Y of the projection rounds (Section 4.3), on CUDA device `device`,
 * with the rounds' access pattern (every float read and written back once
 * per sweep, 16-byte accesses):
 *   level 0  shared memory, every SM sweeping ~225 KB of its own;
 *   level 1  L2, one 64 MB buffer (the size of Y at N = 4000);
 *   level 2  HBM, one 2 GB buffer;
 *   level 3  tensor memory, every SM sweeping all 512 columns x 128 lanes
 *            (256 KB) of its own with 16-column tcgen05.ld / tcgen05.st
 *            accesses, the wave kernel's band storage.
 * sweeps >= 1 timed sweeps after one warm-up sweep.  *gbs receives the
 * measured read + write bandwidth in GB/s.  Allocates and frees a scratch
 * buffer (levels 1, 2, 3); synchronises the device.  Errors: ERR_ARG (bad level
 * or sweeps, gbs == NULL), ERR_CUDA. */
int fastpfp_bandwidth_probe(int device, int level, int sweeps, double* gbs);

/* Throughput of the gradient's product kernels on CUDA device `device`: one
 * n x n x n product C = A B^T (both operands K-major, values pseudo-random
 * in [-1, 1)) with the kernel `precision` selects (FASTPFP_FP32: the
 * tensor-core kernel on split-TF32 operands, three MMAs per product term;
 * FASTPFP_FP32_SIMT: the SIMT kernel; FASTPFP_BF16 / FASTPFP_FP8: the
 * tensor-core kernel, 128 x 256 tiles, E4M3 with per-row scales), timed alone with CUDA events after one
 * warm-up launch; *tflops = 2 n^3 / (best of reps) in TFLOP/s.  n a multiple
 * of 16 in [256, 16384], reps in [1, 1000].  Allocates and frees about
 * 16 n^2 bytes; synchronises the device.  Errors: ERR_ARG, ERR_CUDA. */
int fastpfp_gemm_probe(int device, int precision, int n, int reps, double* tflops);

/* Tile shapes of the gradient products A X A' + lambda K (Section 4.1).
 * Each solve picks, per grouped launch, the CTA tile of its FP32 products
 * (128 or 64 output rows) and of its tensor-core products, BF16 or E4M3
 * (128 x 256 or 128 x 128 outputs; timed in BF16), from a table kept in the
 * handle, indexed by a size
 * class of the group's largest canonical N (class c covers
 * 2^(c+6) < N <= 2^(c+7); class 0 also N <= 128) and a count class of the
 * group's pairs (1; 2-4; 5-16; 17-32).  The table starts at 128 / 256 in
 * every class.  Results do not depend on the choice: every output is
 * accumulated in the same order whatever the tile. */
#define FASTPFP_TUNE_SIZES 8
#define FASTPFP_TUNE_COUNTS 4

/* Fills the table by timing both tiles of both products for every class
 * the handle can meet (N up to max_n, counts up to min(max_batch, 32)), on
 * problems of the class's largest N (square, N = m) in the handle's own
 * scratch, on `stream`: one untimed launch pair, then `reps` (1..100) timed
 * ones; the faster tile (minimum over reps) wins.  A class whose smallest
 * group already holds four times as many large tiles as the device has SMs,
 * in both products, keeps 128 / 256 unmeasured.  Must not overlap a solve
 * on the same handle.  times_ms (host, nullable) receives
 * FASTPFP_TUNE_SIZES x FASTPFP_TUNE_COUNTS x 4 doubles, row-major: the best
 * time of FP32 tile 128, FP32 tile 64, BF16 tile 256 and BF16 tile 128 of
 * each class (0 where the class was not measured).  Synchronises `stream`.
 * Errors: ERR_ARG, ERR_CUDA, ERR_TIMEOUT (a tensor-core launch gave up). */
int fastpfp_autotune(fastpfp_t h, void* stream, int reps, double* times_ms);

/* The table entry of size class n and count class count (the classes that
 * contain these values): *f32_tile_m (128 or 64) and *tc_tile_n (256 or
 * 128), each nullable.  Errors: ERR_ARG (n < 1, count < 1). */
int fastpfp_get_tiles(fastpfp_t h, int n, int count, int* f32_tile_m, int* tc_tile_n);

/* Sets the table entry of the classes that contain n and count; n <= 0
 * means every size class, count <= 0 every count class.  f32_tile_m must be
 * 128 or 64 and tc_tile_n 256 or 128.  Errors: ERR_ARG. */
int fastpfp_set_tiles(fastpfp_t h, int n, int count, int f32_tile_m, int tc_tile_n);

/* Human-readable name of an error code. */
const char* fastpfp_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* FASTPFP_H */
