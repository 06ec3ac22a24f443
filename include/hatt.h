/*
 * libhatt — Hadamard-avoiding tensor-train recompression (HaTT) on one GB300.
 *
 * C ABI. Every pointer argument is either host memory (marked "host") or
 * device memory of the current CUDA device (marked "device"). The caller owns
 * all memory, inputs, outputs and workspace; the library never allocates
 * device memory and never synchronizes the stream, except where a function
 * says so. `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream). Every entry point returns a tt_status; no entry point aborts,
 * exits or traps.
 *
 * Tensor-train layout (Section 2.2, Eq. (2.1)-(2.2)): a TT of order d has cores
 * T_k of shape r_k x n_k x r_{k+1} (0-based k), r_0 = r_d = 1, stored
 * row-major (C order): entry (a, i, b) of core k is cores[k][(a*n_k + i)*r_{k+1} + b].
 * With this layout the horizontal unfolding H(T_k) (r_k x n_k r_{k+1}) and the
 * vertical unfolding V(T_k) (r_k n_k x r_{k+1}) of Section 2.1 are plain
 * row-major views. The Hadamard product Y ⊙ Z is the TT whose cores are the
 * partial Kronecker products Y_k ⊠ Z_k with combined rank index alpha*s + beta
 * (Section 2.2); it is never formed by tt_hadamard_recompress.
 */
#ifndef HATT_H
#define HATT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_ERR_SHAPE = 1,      /* orders/mode sizes disagree, r_0 != 1 or r_d != 1, aliasing */
  TT_ERR_RANK = 2,       /* a rank or size above the supported bound (see TT_MAX_SMALL_RANK) */
  TT_ERR_ARG = 3,        /* null pointer, negative option, unknown precision/variant */
  TT_ERR_WORKSPACE = 4,  /* workspace smaller than the size reported by the *_plan call */
  TT_ERR_CUDA = 5,       /* a CUDA launch or copy failed; cudaGetLastError() has been cleared */
  TT_ERR_NONFINITE = 6,  /* a non-finite input core or intermediate (tt_device_status) */
  TT_ERR_TIMEOUT = 7,    /* a bounded device wait ran out (tt_device_status, tt_batched_status) */
  TT_ERR_BREAKDOWN = 8   /* a shifted Cholesky QR met a non-positive pivot (tt_device_status) */
} tt_status;

/* Largest sketch / output rank the small dense factorizations accept
 * (Gram, Cholesky and symmetric eigen problems of size rank x rank held in
 * shared memory of one thread block). */
#define TT_MAX_SMALL_RANK 128

/* One TT tensor. Every array is caller-owned.
 *   d      order, d >= 1
 *   n      host[d]    mode sizes n_k >= 1
 *   r      host[d+1]  ranks; read for inputs, written for outputs
 *   cores  host[d]    array of device pointers; core k holds r_k*n_k*r_{k+1} doubles */
typedef struct {
  int32_t d;
  const int64_t *n;
  int64_t *r;
  double **cores;
} tt_t;

/* Arithmetic of tt_hadamard_recompress. Only the right-to-left sketches
 * W^{(k)} (HPCRL-1, Algorithm 3 / Eq. (3.6)) may run in low precision: each of
 * their three products per core rounds its operands (W^{(k+1)} with its norm,
 * the sketch core R_k, Z_k, Y_k and the intermediates) to the named type --
 * FP64 -> FP32 round to nearest even, then for TF32 round to nearest with ties
 * away at 10 mantissa bits, for BF16 round to nearest even at 7 -- and
 * accumulates in FP32; the result is kept in FP64. A perturbed W is just
 * another test matrix: range(C_k W) stays inside range(C_k), so the QR, the
 * projection, the core update and the truncation (all FP64) keep the result
 * exact whenever the sketch rank reaches the separation rank, and otherwise
 * add an error of the order of the sketch's relative perturbation to the
 * randomized range-finder error. The paper computes in FP64 throughout; the
 * low-precision modes have no counterpart in it. */
typedef enum {
  TT_FP64 = 0,           /* every step in IEEE binary64 */
  TT_MIXED_FP32 = 1,     /* HPCRL-1 products: FP32 operands, FP32 accumulation */
  TT_MIXED_TF32 = 2,     /* HPCRL-1 products: TF32 operands, FP32 accumulation */
  TT_MIXED_BF16 = 3,     /* HPCRL-1 products: BF16 operands, FP32 accumulation */
  TT_FP64_TC = 4         /* FP64 accuracy throughout; large products (max(M, N) >= 128,
                            K >= 128, >= 2e7 flops) on the BF16 tensor cores: each row /
                            column scaled by a power of two and cut into 9 slices of 6
                            bits, slice products accumulated exactly in FP32 (<= 9 pairs
                            per level, <= 448 terms of K per accumulation), levels
                            combined in FP64; the error is that of an FP64 product
                            (within 2^-54 of each row's and column's largest entry) */
} tt_precision;

/* Options of tt_hadamard_recompress (the problem statement of Algorithm 4:
 * two TT tensors and target ranks; plus the truncation this library adds).
 *   max_rank     cap on the output ranks; 0 = no cap beyond the sketch rank
 *   tol          relative Frobenius tolerance of the final truncation sweep;
 *                0 = no tolerance truncation. The sweep keeps, at each bond, the
 *                smallest rank whose discarded tail sum sigma_i^2 <= delta^2,
 *                delta = tol * ||X||_F / sqrt(d-1)
 *   sketch_rank  l before clamping; 0 = max_rank + oversample if max_rank > 0,
 *                else the PKP rank max_k r_k s_k (exact recompression)
 *   oversample   used when sketch_rank = 0 (>= 0)
 *   seed         Philox4x32-10 key of the Gaussian sketch TT
 *   precision    a tt_precision
 *   variant      1 = HaTT-1 (HPCRL-1 sketches, Eq. (3.6));
 *                2 = HaTT-2 (HPCRL-2, Eq. (3.7)): before each contraction
 *                W^{(k+1)} is replaced by its leading singular terms, the
 *                R_k with sigma > ep * sigma_max (at least one), and the
 *                contraction runs on R_k <= l_{k+1} columns. The singular
 *                values come from the Gram matrix W^T W (FP64), so directions
 *                below ~1e-8 sigma_max are not resolved and ep < 1e-8 keeps
 *                them (the result is then HaTT-1's up to rounding). R_k stays
 *                in device memory (the contractions read it there), so the
 *                call does not synchronize and can be captured; the
 *                workspace is planned for R_k = l_{k+1}. The batched entry
 *                point takes it; the persistent engine does not.
 *   ep           HaTT-2 truncation threshold, 0 <= ep < 1 (ignored by variant 1)
 *   fixed_ranks  0 = the output cores are compacted to the ranks the truncation kept and
 *                X->r is written from the device by an asynchronous copy (valid once the
 *                stream reaches it); 1 = the output keeps the rank bound of the plan call
 *                (min(l_k, max_rank) when truncating with a cap, else l_k): rows and
 *                columns past the kept ranks are zero, X->r is set on the host before the
 *                call returns, and nothing is read back, so a call whose inputs have fixed
 *                shapes can be captured in a CUDA graph and replayed (time stepping)
 *   seed_offset  NULL, or a device uint64 read when the sketch is generated: the
 *                Philox key is seed + *seed_offset. A captured call then draws a
 *                fresh sketch on every replay if the caller advances the word
 *                between replays (the library never writes it). The batched
 *                entry point requires NULL. */
typedef struct {
  int64_t max_rank;
  double tol;
  int64_t sketch_rank;
  int64_t oversample;
  uint64_t seed;
  int32_t precision;
  int32_t variant;
  double ep;
  int32_t fixed_ranks;
  const uint64_t *seed_offset;
} tt_opts;

/* Rank plan and workspace size of tt_hadamard_recompress.
 * Sketch ranks are clamped (l_k = min(l_req, r_k s_k, n_0..n_{k-1}, n_k..n_{d-1}),
 * then l_k <= l_{k-1} n_{k-1} and l_k <= n_k l_{k+1}) so that every economy
 * QR of Algorithm 4 is well posed.
 *   Y, Z              input TTs (only d, n, r are read; cores may be NULL)
 *   out_rank_bound    host[d+1], written: the sketch ranks l_k, which bound the
 *                     output ranks; output core k needs l_k*n_k*l_{k+1} doubles
 *   workspace_bytes   host, written
 * Synchronous, host only; launches nothing. */
int tt_hadamard_recompress_plan(const tt_t *Y, const tt_t *Z, const tt_opts *opts,
                                int64_t *out_rank_bound, size_t *workspace_bytes);

/* Recompress the Hadamard product Y ⊙ Z (Algorithm 4 with HPCRL-1 of
 * Algorithm 3 and Eq. (3.6); core update of Eq. (3.10)) without forming the
 * rank-r_k s_k PKP cores:
 *   1. Gaussian sketch TT R with the planned ranks (Definition 2.1), generated
 *      on the device from a counter-based RNG;
 *   2. right-to-left sketches W^{(k)} = H(A_{k:d}) H(R_{k:d})^T (Eq. (3.1))
 *      computed from the Y, Z and R cores only, each scaled to unit norm;
 *   3. left-to-right pass: QR of C_k W^{(k)} (diag(R) >= 0), M = Q^T C_k,
 *      C_{k+1} = M x (Y_{k+1} ⊠ Z_{k+1}) evaluated core-wise (Eq. (3.8)-(3.10));
 *   4. if tol > 0 or max_rank is below a sketch rank, a right-to-left
 *      truncation sweep of the left-orthogonal result.
 *   Y, Z       inputs (Y.d == Z.d, Y.n[k] == Z.n[k], r_0 = r_d = s_0 = s_d = 1)
 *   X          output: X->d and X->n must match; X->cores[k] must hold at least
 *              b_k*n_k*b_{k+1} doubles, b the plan's bound. On return (stream
 *              ordered) core k holds the r_k x n_k x r_{k+1} result densely in the
 *              prefix of its buffer, and X->r (host[d+1]) receives the ranks
 *              through a stream-ordered device-to-host copy: read X->r after the
 *              stream has been synchronized (pinned host memory keeps the call
 *              asynchronous; pageable memory makes the copy block). With
 *              opts->fixed_ranks = 1, r = b, set on the host (see tt_opts).
 *              Output buffers must not alias input cores (TT_ERR_SHAPE).
 *   workspace  device, at least the plan's workspace_bytes, 256-byte aligned.
 * Without truncation the result is left-orthogonal (cores 0..d-2 have
 * orthonormal vertical unfoldings).
 * Synchronization: with tol > 0 and a stream that is not being captured, the
 * truncation sweep reads one device flag per cluster level (a short
 * synchronization of `stream`) to stop launching levels that would be skipped;
 * a captured stream gets every level instead. */
int tt_hadamard_recompress(const tt_t *Y, const tt_t *Z, const tt_opts *opts, tt_t *X,
                           void *workspace, size_t workspace_bytes, void *stream);

/* Many independent recompressions in one call (pairs of uneven order, mode
 * sizes and ranks; no counterpart in the paper, whose experiments run one
 * pair at a time). A single small pair leaves most of the GPU idle, so the
 * pairs are spread over `lanes` library-owned CUDA streams (pair j on lane
 * j % lanes, in order within a lane): the caller's `stream` forks into the
 * lanes through an event and waits for all of them at the end, so the call
 * stays stream-ordered (and capturable into a CUDA graph, after a first call
 * outside capture has created the library's streams and events on this
 * device). Each lane reuses one region of the workspace for its pairs.
 *   count            number of pairs (>= 0)
 *   Y, Z, opts, X    host arrays of `count` (as for tt_hadamard_recompress;
 *                    X[j] sized from that pair's tt_hadamard_recompress_plan)
 *   lanes            1..32
 *   workspace        device, 256-byte aligned, at least the batch plan's size
 * Every pair is validated before anything is enqueued; the first pair's
 * error code is returned. */
int tt_hadamard_recompress_batch_plan(int32_t count, const tt_t *Y, const tt_t *Z,
                                      const tt_opts *opts, int32_t lanes,
                                      size_t *workspace_bytes);
int tt_hadamard_recompress_batch(int32_t count, const tt_t *Y, const tt_t *Z,
                                 const tt_opts *opts, tt_t *X, int32_t lanes, void *workspace,
                                 size_t workspace_bytes, void *stream);

/* Workspace size of tt_round and its output rank bound b_k = min(r_k, b_{k-1} n_{k-1})
 * (the bound of the left-to-right QR sweep; the ranks kept are also <= max_rank when
 * max_rank > 0), both host outputs. */
int tt_round_plan(const tt_t *A, int64_t max_rank, double tol, int64_t *out_rank_bound,
                  size_t *workspace_bytes);

/* TT rounding of A (Algorithm 1, Oseledets), synchronizing like
 * tt_hadamard_recompress's truncation when tol > 0: orthogonalization sweep with QR
 * of each vertical unfolding (left to right), then a right-to-left truncation
 * sweep with the same rule as tt_hadamard_recompress (max_rank cap, tol with
 * delta = tol * ||A|| / sqrt(d-1)). B is written like X above; all ranks of A
 * must be <= TT_MAX_SMALL_RANK. */
int tt_round(const tt_t *A, int64_t max_rank, double tol, tt_t *B, void *workspace,
             size_t workspace_bytes, void *stream);

/* tt_round_plan / tt_round with the fixed_ranks option of tt_opts: with
 * fixed_ranks = 1 the output bound is min(b_k, max_rank) (max_rank > 0), B keeps it
 * with zeros past the kept ranks, B->r is set on the host and nothing is read back
 * (capturable). fixed_ranks = 0 is tt_round_plan / tt_round. */
int tt_round_ex_plan(const tt_t *A, int64_t max_rank, double tol, int32_t fixed_ranks,
                     int64_t *out_rank_bound, size_t *workspace_bytes);
int tt_round_ex(const tt_t *A, int64_t max_rank, double tol, int32_t fixed_ranks, tt_t *B,
                void *workspace, size_t workspace_bytes, void *stream);

/* Workspace of tt_dot / tt_norm (host output). */
int tt_dot_plan(const tt_t *A, const tt_t *B, size_t *workspace_bytes);

/* Inner product <A, B> = sum over all entries of A * B, by the left-to-right
 * contraction G_k = sum_i A_k(i)^T G_{k-1} B_k(i), G_0 = 1 (the TT inner product
 * behind the relative errors of Section 5). out: device scalar (double). */
int tt_dot(const tt_t *A, const tt_t *B, double *out, void *workspace, size_t workspace_bytes,
           void *stream);

/* <A, B> like tt_dot, for callers that cannot allocate device memory:
 * latency-critical loops whose rules forbid any allocation once running, and
 * plugins whose host framework owns all device memory through its own
 * allocator and gives them no way to reserve a workspace. No counterpart in
 * the paper.
 *   A, B, out  as tt_dot (out: device scalar)
 * Allocates nothing and calls no allocating routine: its scratch is one fixed
 * 8 MiB array in the device memory of every GPU that loads this library
 * (reserved until the process exits). The first call on a device looks up
 * that array's device address (with the device current) and caches it; make
 * this first call before any stream capture. Calls share the array: two calls
 * that overlap on the GPU (other streams, other host threads) race and must be
 * ordered by the caller. Nothing in the array must start at zero; every buffer
 * is written before it is read. Returns TT_ERR_WORKSPACE, before launching
 * anything, when the workspace tt_dot_plan reports for A, B exceeds 8 MiB.
 * The cached address belongs to the device's context at the first call: after
 * a cudaDeviceReset of that device the process must not call tt_dot_noalloc
 * on it again. */
int tt_dot_noalloc(const tt_t *A, const tt_t *B, double *out, void *stream);

/* Frobenius norm ||A||_F = sqrt(<A, A>); out: device scalar. Workspace as tt_dot(A, A). */
int tt_norm(const tt_t *A, double *out, void *workspace, size_t workspace_bytes, void *stream);

/* The Gaussian sketch TT of Definition 2.1 on the device: core k
 * (ell[k] x n[k] x ell[k+1]) gets i.i.d. N(0, 1/(ell_k n_k ell_{k+1})) entries
 * from Philox4x32-10 (key = seed, counter = (flat index, k, pair, 0)) and the
 * Box-Muller transform of two 52-bit uniforms. This is the sketch
 * tt_hadamard_recompress uses internally for the same seed.
 *   n     host[d], ell host[d+1] with ell[0] = ell[d] = 1
 *   cores host[d] array of device pointers (ell[k]*n[k]*ell[k+1] doubles each) */
int tt_sketch_tt(int32_t d, const int64_t *n, const int64_t *ell, uint64_t seed, uint32_t pair,
                 double **cores, void *stream);

/* Raw Philox4x32-10 blocks (Salmon et al., SC'11): out[4j..4j+3] =
 * Philox(counter = ctr[4j..4j+3], key = (key0, key1)) for j < count.
 * ctr, out: device uint32 arrays of 4*count words. */
int tt_philox4x32_10(const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out,
                     int64_t count, void *stream);

/* Number of CUDA kernels this library has enqueued in the calling process
 * since it was loaded (all entry points, all threads). A diagnostic with no
 * counterpart in the paper: the difference around a call is that call's
 * launch count. Host only; never fails. */
int64_t tt_launch_count(void);

/* ---------------------------------------------------------------- batched
 * Many independent recompressions in ONE persistent launch. Each pair runs
 * HaTT-1 (Algorithm 3, then Algorithm 4) exactly as tt_hadamard_recompress
 * does, with the sketch rank as output rank (no truncation sweep). The paper
 * recompresses one product at a time; the task engine has no counterpart in
 * it. Every pair's launch sequence becomes a chain of stages (its GEMMs, the
 * Cholesky QR passes, norms, sketch cores) split into tasks (output tiles,
 * row blocks, element chunks). One queue holds the tasks of all pairs,
 * interleaved so that the pairs with the longest chains (most stages) start
 * first and, within a round of stages, the pairs with the most predicted
 * flops go first. Resident CTAs take tasks in queue order; a task waits, by a
 * bounded poll of its pair's completion counter, for the pair's earlier
 * stages. Since a task only waits on tasks earlier in the queue, which
 * running CTAs already hold, the launch cannot deadlock.
 *
 * create: plans every pair (Y[j], Z[j], opts[j]; the same checks as
 *   tt_hadamard_recompress_plan) and writes the output ranks (the clamped
 *   sketch ranks) into X[j].r (host). Refuses (TT_ERR_ARG) a pair whose
 *   options need the truncation sweep (tol > 0, or max_rank below a sketch
 *   rank), variant 2, or a precision other than TT_FP64 / TT_MIXED_FP32.
 *   X[j].cores must be device buffers of X[j].r[k]*n[k]*X[j].r[k+1] doubles.
 *   The descriptors' host arrays and device buffers must stay valid while the
 *   plan is used. *workspace_bytes: the device workspace to bind. The plan is
 *   host memory owned by the caller (free it with tt_batched_plan_destroy).
 * bind: lays out the workspace (caller-owned, 256-byte aligned, >= the size
 *   reported), and with autotune = 1 times the candidate tile shapes of the
 *   48 GEMM shape buckets with the most flops that are not yet in the
 *   process-wide cache (the others keep an analytic choice); uploads the task
 *   tables. Synchronizes `stream`; not allowed while it is being captured.
 * run: clears the control words and enqueues the persistent launch on
 *   `stream` (no synchronization; capturable once bound). spin_cap bounds each
 *   wait (polls of ~0.25 us; once any wait has run out every later wait gives
 *   up at once and the results are invalid).
 * status: reads the status word of the last run (synchronizes `stream`):
 *   TT_OK, TT_ERR_TIMEOUT if a wait ran out, TT_ERR_NONFINITE if a norm or a
 *   Gram matrix was not finite (NaN or Inf in an input), TT_ERR_BREAKDOWN.
 * info: number of stages and tasks of the bound plan and resident CTAs.
 * profile: sums over the CTAs of the last run's profile words into out (host
 *   int64[24]): [0] cycles from each CTA's start to its end, [1] cycles
 *   polling for prerequisites, [2] cycles taking tickets, [8 + t] cycles
 *   running tasks of kind t, [16 + t] number of those tasks (t: 0 sketch,
 *   1 GEMM tile, 2 norm partial, 3 norm, 4 first core, 5 Cholesky, 6 QR
 *   apply, 7 set). Synchronizes `stream`.
 * tune_cache: save (save = 1) or load (save = 0) the process-wide tile cache
 *   as text lines "prec M N K batch bm bn" at `path` (host string). */
typedef struct tt_batch_plan tt_batch_plan;
int tt_batched_plan_create(int32_t count, const tt_t *Y, const tt_t *Z, const tt_opts *opts,
                           tt_t *X, tt_batch_plan **plan, size_t *workspace_bytes);
int tt_batched_plan_bind(tt_batch_plan *plan, void *workspace, size_t workspace_bytes,
                         int32_t autotune, void *stream);
int tt_batched_run(tt_batch_plan *plan, int64_t spin_cap, void *stream);
int tt_batched_status(tt_batch_plan *plan, void *stream, int32_t *status);
int tt_batched_plan_info(const tt_batch_plan *plan, int64_t *stages, int64_t *tasks,
                         int32_t *blocks);
int tt_batched_profile(tt_batch_plan *plan, void *stream, int64_t *out);
int tt_batched_plan_destroy(tt_batch_plan *plan);
int tt_batched_tune_cache(const char *path, int32_t save);

/* One batched product C_b = alpha A_b B_b, b < batch, through the library's
 * contraction kernels: the FP64 kernels for TT_FP64; for TT_MIXED_FP32 the
 * SIMT kernel with FP32-rounded operands and FP32 accumulation; for
 * TT_MIXED_TF32 / TT_MIXED_BF16 the tcgen05 tensor-core kernel, operands
 * rounded to the format (as tt_precision states) and FP32 accumulation per
 * K slice, slices summed in FP64; for TT_FP64_TC the FP64-accurate BF16
 * tensor-core products where the size qualifies. No counterpart in the
 * paper: it exposes the kernels of Eq. (3.6)'s contractions to
 * product-level checks.
 *   A  device, batch x M x K, row-major (leading dimension K)
 *   B  device, batch x K x N, row-major (leading dimension N)
 *   C  device, batch x M x N, row-major; written, never read; must not
 *      overlap A or B
 *   M, N, batch >= 0, K >= 1; M K, K N, M N < 2^31 (TT_ERR_SHAPE)
 *   workspace  device, 256-byte aligned, tt_gemm_plan's size
 * Enqueued on `stream`; FP64 products may be timed once per new shape
 * (tt_gemm_autotune). */
int tt_gemm_plan(int32_t precision, int64_t M, int64_t N, int64_t K, int64_t batch,
                 size_t *workspace_bytes);
int tt_gemm(int32_t precision, int64_t M, int64_t N, int64_t K, int64_t batch, const double *A,
            const double *B, double *C, double alpha, void *workspace, size_t workspace_bytes,
            void *stream);

/* FP64 GEMM plan tuning, an implementation detail with no counterpart in the
 * paper. The first time a GEMM shape (sizes, batch, operand layout) runs on a
 * stream that is not being captured, the library times its model's best
 * candidate tilings (single and paired-column forms, ~50 launches on the
 * call's own operands and output) and keeps the fastest for every later
 * launch of that shape in the process, including inside captured graphs.
 * This synchronizes the caller's stream once per tuned shape and allocates
 * nothing. A shape first met during a capture keeps the model's choice, and
 * so do products under 1e7 flops, products that accumulate into their output
 * or carry a device skip flag, and shapes beyond the first 256 tuned. Results
 * differ between tilings only by the order of FP64 rounding.
 * tt_gemm_autotune(0) turns the timing off for shapes not yet run (they keep
 * the model's choice), 1 turns it on (the default). Returns TT_OK; the
 * setting is process-wide. */
int tt_gemm_autotune(int32_t enable);

/* Kernel timer, a diagnostic with no counterpart in the paper: between
 * tt_kernel_timer_start and tt_kernel_timer_stop, each launch of the FP64
 * GEMM kernel that is not being captured into a CUDA graph is bracketed by a
 * pair of CUDA events recorded on the stream it is launched on, and its
 * algorithmic flop count 2*M*N*K*batch is kept, for the first `capacity`
 * launches (later ones run untimed). This is how a caller measures the
 * dominant kernel's average duration on its own stream.
 * start: creates 2*capacity events on the current device (the library owns
 *   them); capacity in [1, 1<<20], else TT_ERR_ARG; TT_ERR_CUDA if event
 *   creation fails; a running timer is stopped and discarded first.
 * stop: waits for the recorded events, writes ms[i] and flops[i] (host
 *   arrays of `capacity` doubles, may be NULL when capacity is 0) for the
 *   i < min(recorded, capacity) launches, *count = number recorded (may be
 *   NULL), destroys the events. TT_ERR_ARG if no timer is running.
 * Host only; one timer per process; not for use while another thread
 * launches through this library. */
int tt_kernel_timer_start(int32_t capacity);
int tt_kernel_timer_stop(double *ms, double *flops, int32_t capacity, int64_t *count);
/* As tt_kernel_timer_stop, and role[i] (host, `capacity` int32, may be NULL)
 * tells what launch i computed: TT_ROLE_METHOD for the contractions HaTT
 * itself is made of (the HPCRL products of Algorithm 3 / eq. (3.6) or (3.7),
 * the core sketch C_k W, the projection Q^T C_k and the core update of
 * eq. (3.10)), which always do their work; TT_ROLE_AUX for every other FP64
 * GEMM launch (Gram matrices and triangular steps of the QR, the truncation
 * sweep and its eigen refinement, inner products, TT rounding), some of which
 * a device flag turns into no-ops once a loop has converged. */
#define TT_ROLE_AUX 0
#define TT_ROLE_METHOD 1
int tt_kernel_timer_stop_ex(double *ms, double *flops, int32_t *role, int32_t capacity,
                            int64_t *count);

/* Periodic central-difference Laplacian of a TT (Section 5, Example 4):
 * L = sum_k I x .. x D_k x .. x I applied to A, D the n_k x n_k second
 * difference (u_{i+1} - 2 u_i + u_{i-1}) * inv_h2 with wrap-around. L has
 * ranks {1, 2 r_1, ..., 2 r_{d-1}, 1} and cores [A_1 | D A_1],
 * [[A_k, D A_k], [0, A_k]], [[D A_d], [A_d]] (for d = 1 the single core
 * D A_1). L: caller-allocated cores of those shapes and L->r set to them
 * (TT_ERR_SHAPE otherwise); stream ordered. */
int tt_laplacian(const tt_t *A, double inv_h2, tt_t *L, void *stream);

/* S = sum_j coef[j] T[j] (count >= 1 TTs of equal order and mode sizes,
 * coef host) with block-diagonal cores: ranks r_k(S) = sum_j r_k(T_j) for
 * the inner bonds, the coefficients multiply the first cores (for d = 1 the
 * single core is the plain sum). S: caller-allocated, S->r set to those
 * ranks (TT_ERR_SHAPE otherwise); stream ordered. */
int tt_lincomb(int32_t count, const tt_t *T, const double *coef, tt_t *S, void *stream);

/* x[i] /= *divisor for i < count (x, divisor: device; stream ordered, so the
 * divisor may be a norm that an earlier call on the stream computes, e.g. the
 * normalization X / ||X|| of the power iteration of Section 5, Example 3).
 * TT_ERR_ARG for a negative count or NULL pointers (count > 0). */
int tt_scale(double *x, int64_t count, const double *divisor, void *stream);

/* Device error word, a diagnostic with no counterpart in the paper. Bits:
 *   1  a bounded wait inside a kernel ran out (the tensor-core products wait
 *      on an mbarrier for their own MMAs); that kernel writes NaN to its
 *      outputs, frees its tensor memory and returns, so nothing hangs or traps;
 *   2  a non-finite value reached a norm ||W^{(k)}|| of the right-to-left
 *      sketches (Algorithm 3) or the Gram matrix of a Cholesky QR pass
 *      (Algorithm 4, tt_round): a NaN or Inf in an input core, or an overflow;
 *      the QR stops there and leaves its matrix as it was;
 *   4  a shifted Cholesky factorization still met a non-positive pivot (QR
 *      breakdown; the shift of shifted Cholesky QR makes this unreachable for
 *      finite inputs, the bit guards against it).
 * Writes the word to *value (host) and clears it; synchronizes the current
 * device. TT_ERR_ARG if value is NULL, TT_ERR_CUDA if the device cannot be read. */
int tt_device_error(int32_t *value);
/* As tt_device_error, reporting the word as a status: TT_ERR_TIMEOUT (bit 1),
 * else TT_ERR_NONFINITE (bit 2), else TT_ERR_BREAKDOWN (bit 4), else TT_OK;
 * clears the word, synchronizes the current device. */
int tt_device_status(int32_t *status);

/* Static description of a status code (never NULL). */
const char *tt_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HATT_H */
