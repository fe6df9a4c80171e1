/*
 * ks.h -- C ABI of the GB300 temporally parallel Kalman filter / RTS smoother.
 *
 * The library computes the filtering and smoothing posteriors of a
 * linear/Gaussian state-space model (Section IV)
 *
 *     x_k = F x_{k-1} + u + q_{k-1},   q ~ N(0, Q),
 *     y_k = H x_k + d + r_k,           r ~ N(0, R),   x_0 ~ N(m0, P0),
 *
 * as two all-prefix-sums (Section II-B):
 *   - Lemma 3 builds one filtering element a_k = (A_k, b_k, C_k, eta_k, J_k)
 *     per measurement; Lemma 4's operator combines them; by Theorem 1 the
 *     prefix a_1 (x) ... (x) a_k has b = filtered mean, C = filtered covariance.
 *   - Lemma 5 builds one smoothing element (E_k, g_k, L_k) per step from the
 *     filtered moments; Lemma 6's operator combines them; by Theorem 2 the
 *     suffix a_k (x) ... (x) a_n has g = smoothed mean, L = smoothed covariance.
 * The scans use block-level elements (Section III-C): each thread folds a
 * contiguous block of steps, blocks are scanned within a thread block, and
 * thread blocks are chained by a decoupled look-back.
 *
 * Conventions (all entry points)
 * ------------------------------
 * - Arithmetic: FP32 on the GPU; the k = 1 element (prior m0, P0) in FP64.
 * - Memory: every pointer argument documented "device" must point to memory
 *   the current CUDA device can read/write (cudaMalloc, torch CUDA tensors).
 *   The caller owns every buffer; the library allocates no device memory and
 *   keeps no state between calls, apart from the block-length table of
 *   ks_set_chunk_rules (host memory).  Scratch lives in the caller's
 *   workspace `ws` (opaque, size from ks_workspace_bytes, 256-byte aligned).
 * - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are stream-ordered and asynchronous, make no host
 *   synchronisation, and may be captured into a CUDA graph.
 * - Layouts: matrices row-major; filtered/smoothed means are [T][nx],
 *   covariances [T][nx][nx] (full, symmetric), all FP32.
 * - Sizes: 1 <= T <= 2^31 - 1.  Supported (nx, ny) pairs are listed by
 *   ks_supported(); others return KS_EUNSUPPORTED.
 * - nx = 32: the operators' dense products run on the tensor cores (3xTF32,
 *   FP32 accumulate) and the inverses of Lemmas 4 and 5 get one FP64-residual
 *   refinement step when their estimated condition number exceeds 1e3.  At
 *   every nx the general Lemma 4 operator (cross-block combines) refines its
 *   (I + C_i J_j)^{-1} the same way (ks_refinements counts them).
 *   ks_smooth and ks_smooth_scan then want fmean, fcov, smean and scov
 *   16-byte aligned (KS_EINVAL otherwise).
 * - Errors: every call returns KS_OK (0) or a negative code.  Argument and
 *   launch errors are returned immediately.  Errors found on the device
 *   (non-finite values, a failed factorisation, a look-back wait that timed
 *   out) are recorded in the workspace's status word and reported by
 *   ks_status().  Calls on one workspace must not overlap on the device.
 */
#ifndef KS_H
#define KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KS_OK 0
#define KS_EINVAL (-1)        /* bad argument: size, null or misaligned pointer */
#define KS_ECUDA (-2)         /* a CUDA launch or copy failed */
#define KS_ENUMERIC (-3)      /* device: non-finite value or failed factorisation */
#define KS_ETIMEOUT (-4)      /* device: bounded look-back wait ran out */
#define KS_EUNSUPPORTED (-5)  /* size not compiled in, or a model form the entry point does not take */

/* Workspace purposes for ks_workspace_bytes(). */
#define KS_WS_SMOOTH 0        /* ks_smooth / ks_filter_scan / ks_smooth_scan scratch */
#define KS_WS_ELEMENTS 1      /* additionally the materialised element arrays of ks_build_elements */

/*
 * Linear/Gaussian model of Sections II and IV.
 *
 * time_varying = 0 (time-invariant): F [nx][nx], u [nx], Q [nx][nx],
 * H [ny][nx], d [ny], R [ny][ny] are DEVICE pointers to FP32 row-major
 * arrays; u and d may be NULL (zero).
 *
 * time_varying = 1: every one of them holds one entry per step, step-major:
 * F [T][nx][nx], u [T][nx], Q [T][nx][nx], H [T][ny][nx], d [T][ny],
 * R [T][ny][ny] (u, d may be NULL).  With 0-based steps, step k is predicted
 * from step k-1 with F[k], u[k], Q[k] (F[0], u[0], Q[0] take the prior
 * N(m0, P0) to step 0) and observed as y[k] = H[k] x_k + d[k] + r_k with
 * r_k ~ N(0, R[k]): Section II's model with its indices shifted by one.
 * Each of these arrays must start on a 16-byte boundary (KS_EINVAL otherwise).
 * Time-varying models are accepted by ks_smooth and ks_smooth_traced for
 * nx in {2, 4, 6, 8} (KS_EUNSUPPORTED elsewhere), and need
 * ks_workspace_bytes(m, T, KS_WS_SMOOTH) bytes (the same as KS_WS_ELEMENTS
 * for them: per-step elements or model constants live in the workspace).
 *
 * m0 [nx] and P0 [nx][nx] are DEVICE pointers to FP64 arrays.  Q, R and P0
 * must be symmetric positive definite (R, P0) / semidefinite with
 * F P F^T + Q definite (Q).
 */
typedef struct ks_model {
    int32_t nx;
    int32_t ny;
    int32_t time_varying;
    int32_t reserved;
    const float *F, *u, *Q, *H, *d, *R;
    const double *m0, *P0;
} ks_model;

/*
 * B independent time-invariant models for a batch of sequences laid end to
 * end.  Every array holds one model per sequence, sequence-major: F [B][nx][nx],
 * u [B][nx] (or NULL), Q [B][nx][nx], H [B][ny][nx], d [B][ny] (or NULL),
 * R [B][ny][ny] FP32; m0 [B][nx], P0 [B][nx][nx] FP64.  offsets [B+1] (int64)
 * gives each sequence's first step on the concatenated axis: offsets[0] = 0,
 * strictly increasing (every sequence has at least one step), offsets[B] =
 * the total number of steps.  All pointers are DEVICE pointers.
 */
typedef struct ks_model_batch {
    int32_t nx;
    int32_t ny;
    int32_t B;
    int32_t reserved;
    const float *F, *u, *Q, *H, *d, *R;
    const double *m0, *P0;
    const int64_t *offsets;
} ks_model_batch;

/* Layout of the materialised filtering elements written by ks_build_elements
 * (Lemma 3) into the workspace: structure of arrays, component-major.  The
 * c-th scalar component of element k (0-based step) is the float at
 *     (float*)((char*)ws + offset_X) + c * ld + k
 * with components row-major within A [nx*nx], b [nx], C [nx*nx], eta [nx],
 * J [nx*nx]. */
typedef struct ks_elements_layout {
    int64_t ld;          /* floats between consecutive components (>= T, multiple of 64) */
    int64_t offset_A, offset_b, offset_C, offset_eta, offset_J;  /* bytes from ws */
} ks_elements_layout;

/* Library version, for the binding's load check. */
int ks_version(void);

/* 1 if the (nx, ny) pair is compiled in, else 0. */
int ks_supported(int nx, int ny);

/* Human-readable text of a status code; never NULL. */
const char *ks_strerror(int code);

/*
 * Bytes of workspace needed for sequences of up to T steps of model `m`
 * (only m->nx, m->ny and m->time_varying are read; host pointer).
 * purpose = KS_WS_SMOOTH or KS_WS_ELEMENTS.  Returns 0 for invalid
 * arguments, and for a time-varying model of an (nx, ny) whose smoother
 * does not take one.
 */
size_t ks_workspace_bytes(const ks_model *m, int64_t T, int purpose);

/*
 * Zero the workspace's status word and scan state (stream-ordered).  Call
 * once on a fresh workspace before its first use.
 */
int ks_workspace_init(void *ws, size_t ws_bytes, void *stream);

/*
 * Element offsets of ks_build_elements' output inside a KS_WS_ELEMENTS
 * workspace (host call, no device work).
 */
int ks_elements_layout_get(const ks_model *m, int64_t T, ks_elements_layout *out);

/*
 * Lemma 3 (Section IV-A): build the T filtering elements (A_k, b_k, C_k,
 * eta_k, J_k) from the measurements y [T][ny] (device, FP32) into the
 * workspace, in the layout of ks_elements_layout_get.  k = 1 is built in
 * FP64 from (m0, P0) with A_1 = 0 and eta_1 = 0, J_1 = 0; for k > 1 the model
 * being time-invariant, A, C, J are the same for every k and only b_k, eta_k
 * depend on y_k.  C and J are stored symmetrised.
 * ws must hold ks_workspace_bytes(m, T, KS_WS_ELEMENTS) bytes.
 */
int ks_build_elements(const ks_model *m, const float *y, int64_t T,
                      void *ws, size_t ws_bytes, void *stream);

/*
 * Forward filtering scan over the elements built by ks_build_elements:
 * inclusive all-prefix-sums under Lemma 4's operator (Theorem 1).  Writes the
 * filtered means fmean [T][nx] = b of each prefix and covariances
 * fcov [T][nx][nx] = C of each prefix (device, FP32).
 */
int ks_filter_scan(const ks_model *m, int64_t T, void *ws, size_t ws_bytes,
                   float *fmean, float *fcov, void *stream);

/*
 * Reverse smoothing scan (Lemmas 5 and 6, Theorem 2): builds the smoothing
 * elements from the filtered moments fmean [T][nx], fcov [T][nx][nx]
 * (device) as it loads them, computes the suffix sums
 * a_k (x) a_{k+1} (x) ... (x) a_T (earlier element on the left) and writes
 * smoothed means smean [T][nx] and covariances scov [T][nx][nx] (device).
 */
int ks_smooth_scan(const ks_model *m, int64_t T, const float *fmean, const float *fcov,
                   void *ws, size_t ws_bytes, float *smean, float *scov, void *stream);

/*
 * End to end: filtering elements built from y as the forward scan loads
 * them (no materialised element arrays), forward scan writing
 * fmean/fcov, then the reverse smoothing scan writing smean/scov.
 * y [T][ny], fmean [T][nx], fcov [T][nx][nx], smean, scov: device, FP32.
 * fmean and fcov may be NULL, in which case the filtered moments are kept
 * in the workspace only (which then needs ks_workspace_bytes(m, T,
 * KS_WS_ELEMENTS) bytes).  smean and scov may both be NULL (with fmean and
 * fcov given): then only the forward scan runs (filtering only).
 */
int ks_smooth(const ks_model *m, const float *y, int64_t T, void *ws, size_t ws_bytes,
              float *fmean, float *fcov, float *smean, float *scov, void *stream);

/*
 * Batched end to end: one forward and one reverse scan over the B sequences
 * laid end to end (segmented scans; no combine crosses into a neighbouring
 * sequence's result because each sequence's first filtering element has
 * A_1 = 0 and its last smoothing element has E_n = 0).  y [total_T][ny] and
 * the outputs [total_T][nx], [total_T][nx][nx] are concatenated in sequence
 * order (device, FP32).  ws: ks_workspace_bytes_batch(nx, ny, B, total_T)
 * bytes.  An inconsistent offsets table is reported by ks_status as
 * KS_EINVAL.
 */
size_t ks_workspace_bytes_batch(int nx, int ny, int B, int64_t total_T);
int ks_smooth_batch(const ks_model_batch *mb, const float *y, int64_t total_T, void *ws, size_t ws_bytes,
                    float *fmean, float *fcov, float *smean, float *scov, void *stream);

/*
 * Block length of the fused scans (Section III-C: each thread folds a block
 * of l consecutive steps; a tile is 128 threads) and how a block is folded.
 * The nx <= 6 entry points ks_smooth, ks_smooth_traced, ks_smooth_batch and
 * ks_smooth_batched are compiled for l in {4, 8, 16, 32} and pick one per
 * call from the call's total number of steps T.  For a time-invariant model
 * a full block can also be folded through per-position coefficients built
 * once per call and model (the linear block fold: Lemma 3's A, C, J are the
 * same at every step, so a block's (b, eta) is affine in its measurements)
 * instead of element by element; `fold` = 1 selects it for ks_smooth,
 * ks_smooth_traced and ks_smooth_batched (ks_smooth_batch always folds element
 * by element).  The built-in choice is 4 steps below 96 Ki steps, 8 below
 * 192 Ki, 16 below 640 Ki and 32 above, folding with the coefficients at 32
 * steps for single sequences and never for ks_smooth_batched.
 * ks_set_chunk_rules replaces it for one state size (nx = 2, 4 or 6; nx = 0:
 * ks_smooth_batched) by `count` rules with strictly increasing T_below: a
 * call uses the first rule whose T_below exceeds its T, else the last one.
 * count = 0 restores the built-in choice.  steps must be 4, 8, 16 or 32, fold
 * 0 or 1, and count <= 16 (KS_EINVAL otherwise).  The table is process state
 * of the library (host memory, guarded by a mutex); results agree to FP32
 * rounding whichever entry runs.  The project's tuner measures the table on
 * the device (package module tune.py).  ks_chunk_steps and ks_chunk_fold
 * return the steps per thread and the fold flag a call of T steps would use
 * (0 for an nx without a table).
 */
typedef struct ks_chunk_rule {
    int64_t T_below;
    int32_t steps;
    int32_t fold;
} ks_chunk_rule;
int ks_set_chunk_rules(int nx, int count, const ks_chunk_rule *rules);
int ks_chunk_steps(int nx, int64_t T);
int ks_chunk_fold(int nx, int64_t T);

/*
 * Batched end to end over sequences of different state sizes, in one
 * preparation, one forward-scan and one reverse-scan launch.  The sequences
 * come in G groups (1 <= G <= 3), one per state size, with distinct
 * (nx, ny) among (2, 1), (4, 2) and (6, 3) (others: KS_EUNSUPPORTED).  A
 * group is a segmented batch exactly as for ks_smooth_batch: its models
 * (ks_model_batch: nx, ny, B >= 1 sequences, per-sequence parameters and the
 * offsets table, device), its total_T steps (= offsets[B]) and its own
 * concatenated arrays y [total_T][ny], fmean, smean [total_T][nx], fcov,
 * scov [total_T][nx][nx] (device, FP32, 16-byte aligned; all required).
 * Each scan launch takes (group, tile) work items from one queue, the
 * largest state size first, and runs the code specialised for the item's
 * size; no combine crosses a sequence start (Lemma 3's A_1 = 0, Lemma 5's
 * E_n = 0) or a group.  ws: ks_workspace_bytes_batched(G, groups) bytes
 * (reads nx, ny, B and total_T), 256-byte aligned, initialised once with
 * ks_workspace_init.  Device-side errors (an inconsistent offsets table:
 * KS_EINVAL) are reported by ks_status.
 */
typedef struct ks_batch_group {
    ks_model_batch models;
    int64_t total_T;
    const float *y;
    float *fmean, *fcov, *smean, *scov;
} ks_batch_group;
size_t ks_workspace_bytes_batched(int G, const ks_batch_group *groups);
int ks_smooth_batched(int G, const ks_batch_group *groups, void *ws, size_t ws_bytes, void *stream);

/*
 * ks_smooth with per-kernel timing:/*
 * ks_smooth with per-kernel timing: `events` points to 4 cudaEvent_t handles
 * (passed as void*; any may be NULL) that are recorded on `stream` before the
 * model preparation, before the forward scan kernel, between the two scans
 * and after the reverse scan kernel.  Otherwise identical to ks_smooth.
 */
int ks_smooth_traced(const ks_model *m, const float *y, int64_t T, void *ws, size_t ws_bytes,
                     float *fmean, float *fcov, float *smean, float *scov, void *stream,
                     void *const *events);

/*
 * Synchronise `stream`, read the workspace's device status word, clear it,
 * and return KS_OK, KS_ENUMERIC or KS_ETIMEOUT (or KS_ECUDA if the stream
 * reported an error).  ws: device.
 */
int ks_status(void *ws, void *stream);

/*
 * Testing aid for the bounded look-back waits of the block scans (Section
 * III-C's block-level elements, chained across thread blocks).  Writes two
 * settings into the workspace header (stream-ordered); they persist until
 * changed or until ks_workspace_init:
 *   wait_polls  polls a look-back wait makes before it gives up, records
 *               KS_ETIMEOUT for ks_status and goes on with an empty prefix
 *               (0: the default, about one second);
 *   first_tile  1 makes the forward scan of ks_smooth / ks_smooth_batch at
 *               nx <= 6 number its tiles from 1, so that tile 0 is never
 *               published and tile 1's wait must run out; 0 restores the
 *               normal numbering; other values: KS_EINVAL.
 * Results computed with first_tile = 1 are not meaningful; the call exists so
 * that a test can check, in bounded time, that a wait which runs out is
 * reported and leaves the device usable.  ws: device, >= 256 bytes, 256-byte
 * aligned.
 */
int ks_workspace_set_waits(void *ws, size_t ws_bytes, uint32_t wait_polls, uint32_t first_tile, void *stream);

/*
 * Refinement counter of the workspace (Lemma 4's (I + C_i J_j)^{-1}, and at
 * nx = 32 also Lemma 5's (F P F^T + Q)^{-1}): every inverse whose condition
 * estimate (1-norm, or infinity-norm in the lane-group kernels of nx = 8 and
 * of nx = 32 batches) exceeds 1e3 gets one refinement step with its residual
 * formed in FP64, and each warp or lane group in which that happened adds one
 * to a counter kept beside the status word.  Synchronises `stream`, writes
 * the count accumulated since the workspace was initialised or last read to
 * *count (host) and clears it.  ws: device.  A diagnostic: the results do not
 * depend on reading it.
 */
int ks_refinements(void *ws, void *stream, uint32_t *count);

/*
 * ks_smooth without a workspace, for callers that cannot allocate device/*
 * ks_smooth without a workspace, for callers that cannot allocate device
 * memory: for example a real-time loop that must not take cudaMalloc's
 * implicit device synchronisation or risk its failure once running, or a host
 * application that owns the device memory budget and does not let plug-ins
 * allocate.  The paper has no counterpart; this is an interface convenience.
 *
 * Same computation and arguments as ks_smooth for time-invariant models with
 * nx = 4, ny = 2 (other sizes, or time-varying models: KS_EUNSUPPORTED), with
 * T <= KS_NOALLOC_MAX_T.  KS_EINVAL for a larger T, for NULL fmean or fcov,
 * or for exactly one of smean and scov NULL; both NULL runs the filter only,
 * as in ks_smooth.  The caller still provides every input and output; the
 * scratch lives in a static device array of KS_NOALLOC_SCRATCH_BYTES that
 * every GPU loading this library holds until the process exits.  The
 * function itself allocates nothing.
 *  - Every call looks up that array's device address on the current device
 *    (a host-side query, so the address stays right after a cudaDeviceReset).
 *    The first call on a device also loads the library's device code there;
 *    make that first call before any stream capture.
 *  - All calls on a device share the one array: calls that overlap on the GPU
 *    (different streams or threads without ordering) race and give wrong
 *    results.  Each call clears the state it needs, so sequential calls are
 *    independent.
 *  - Device-side errors: if status_out (device pointer, may be NULL) is given,
 *    the call's device status bits are copied there at the end of the call,
 *    stream-ordered: 0 = ok, bit 0 = non-finite value or failed factorisation,
 *    bit 1 = a look-back wait ran out.
 */
#define KS_NOALLOC_MAX_T 1048576
#define KS_NOALLOC_SCRATCH_BYTES 4194304
int ks_smooth_noalloc(const ks_model *m, const float *y, int64_t T, float *fmean, float *fcov,
                      float *smean, float *scov, int32_t *status_out, void *stream);

/*
 * Marginal log-likelihood (Section III-C: the filtering prefix also carries
 * p(y_1:k)): one parallel pass over the filtered moments gives every
 *   log p(y_k | y_1:k-1) = log N(y_k; H (F xbar_{k-1} + u) + d,
 *                                 H (F P_{k-1} F^T + Q) H^T + R)
 * (k = 1 from (m0, P0), in FP64), and log p(y_1:T) is their sum.
 * y [T][ny], fmean [T][nx], fcov [T][nx][nx]: device, FP32 (the filtered
 * moments of ks_smooth or ks_filter_scan; may be NULL when T = 1).
 * ll [T] (device FP32, may be NULL): the per-step terms.  total (device, one
 * double, may be NULL): their sum, accumulated in FP64.  At least one of ll
 * and total.  status (device uint32): cleared, then set to 1 when a
 * predictive covariance fails its Cholesky factorisation or a term is not
 * finite.  Allocates nothing; no workspace.
 */
int ks_loglik(const ks_model *m, const float *y, int64_t T, const float *fmean, const float *fcov,
              float *ll, double *total, uint32_t *status, void *stream);

/*
 * Time sharding (Section III-C's block-level elements with one block per
 * device): a sequence split into consecutive shards, each on its own device,
 * is smoothed with one exchange of one element per shard and scan:
 *   1. each shard folds its filtering elements into one element
 *      (ks_filter_aggregate); the shards' aggregates are exchanged;
 *   2. shard s combines the aggregates of shards 0..s-1 (ks_filter_combine_batch):
 *      the result has A = 0 and its (b, C) is the filtered posterior at the step
 *      before the shard, so the shard's forward scan is ks_smooth(..., smean =
 *      scov = NULL) with that posterior as the model's (m0, P0) (Lemma 3's
 *      k = 1 element is exactly "posterior (x) measurement element");
 *   3. each shard folds its smoothing elements into one element
 *      (ks_smoother_aggregate); the aggregates are exchanged;
 *   4. shard s combines those of shards s+1..S-1 (ks_smoother_combine_batch):
 *      the result has E = 0 and its (g, L) is the smoothed posterior at the
 *      step after the shard; appended to the shard's filtered moments as one
 *      extra step, Lemma 5's last-step element turns it into the suffix
 *      entering the shard, so the shard's reverse scan is ks_smooth_scan over
 *      T + 1 steps.
 *
 * ks_filter_aggregate: out = a_1 (x) ... (x) a_T over the shard's steps
 * (Lemma 4, packed filter element, device [3nx^2 + 2nx]).  y [T][ny]: the
 * shard's measurements (device).  first != 0: the shard starts the sequence,
 * and its first element is Lemma 3's k = 1 element from (m0, P0); otherwise
 * every element is a measurement element.
 * ks_smoother_aggregate: out = the fold of the shard's Lemma 5 elements built
 * from its filtered moments (packed smoother element, device [2nx^2 + nx]);
 * last != 0: the shard ends the sequence, and its last element is Lemma 5's
 * k = n element (E = 0).
 * Workspace: ks_workspace_bytes_aggregate(m, T) bytes, 256-byte aligned.
 * Offered for nx <= 6 (KS_EUNSUPPORTED otherwise).
 */
size_t ks_workspace_bytes_aggregate(const ks_model *m, int64_t T);
int ks_filter_aggregate(const ks_model *m, const float *y, int64_t T, int first, void *ws,
                        size_t ws_bytes, float *out, void *stream);
int ks_smoother_aggregate(const ks_model *m, int64_t T, const float *fmean, const float *fcov,
                          int last, void *ws, size_t ws_bytes, float *out, void *stream);

/*
 * Batched Lemma 4 / Lemma 6 operators on `count` independent element pairs,
 * for operator-level testing and for callers that run their own scans.
 * Elements are packed per element (no padding) in device memory, FP32:
 *   filter element  = A[nx*nx] b[nx] C[nx*nx] eta[nx] J[nx*nx]
 *   smoother element = E[nx*nx] g[nx] L[nx*nx]
 * out[i] = left[i] (x) right[i].  C, J, L of the results are symmetrised.
 */
int ks_filter_combine_batch(int nx, int64_t count, const float *left, const float *right,
                            float *out, void *ws, size_t ws_bytes, void *stream);
int ks_smoother_combine_batch(int nx, int64_t count, const float *left, const float *right,
                              float *out, void *ws, size_t ws_bytes, void *stream);

/*
 * Discrete-state (hidden Markov model) filter and smoother: Section III's
 * general elements and operators (Definitions 1 and 2, Theorems 1 and 2)
 * with every integral a sum over the K states, the counting-measure case the
 * paper's Section VI points to.
 *
 * Model: x_0 ~ pi [K], p(x_k = j | x_k-1 = i) = Pi[i][j] ([K][K], rows sum
 * to one), and the measurements only through their likelihoods
 * lik [T][K], lik[k][j] = p(y_k | x_k = j) >= 0 (any emission model; a row
 * needs a positive entry).  pi and Pi: device FP32 (ks_hmm holds device
 * pointers; the struct itself is a host object).  Supported K:
 * ks_hmm_supported(K) (2, 4, 8, 16 and 32); others return KS_EUNSUPPORTED.
 * At K = 16 and 32 lik must be 16-byte aligned (KS_EINVAL otherwise).
 *
 * ks_hmm_smooth writes, device FP32:
 *   filt   [T][K]  p(x_k | y_1:k)      (required; the smoother reads it back);
 *   smooth [T][K]  p(x_k | y_1:T)      (NULL: filter only);
 *   loglik [T]     log p(y_1:k)        (NULL: not written).
 * The marginal likelihoods come from the filtering scan itself (Theorem 1's
 * g), carried as logarithms.  ws: ks_hmm_workspace_bytes(K, T) bytes,
 * 256-byte aligned, initialised once with ks_workspace_init; its status word
 * is read with ks_status (bit 0: a likelihood row with no positive finite
 * entry, an impossible observation sequence or a non-finite result; bit 1: a
 * look-back wait ran out).  Stream-ordered, no host synchronisation.
 */
typedef struct ks_hmm {
    int32_t K;
    int32_t reserved;
    const float *pi, *Pi;
} ks_hmm;

int ks_hmm_supported(int K);
size_t ks_hmm_workspace_bytes(int K, int64_t T);
int ks_hmm_smooth(const ks_hmm *h, const float *lik, int64_t T, void *ws, size_t ws_bytes, float *filt,
                  float *smooth, float *loglik, void *stream);
/* The same, recording events[0..3] (cudaEvent_t, entries may be NULL) around
 * the preparation, filter and smoother launches. */
int ks_hmm_smooth_traced(const ks_hmm *h, const float *lik, int64_t T, void *ws, size_t ws_bytes, float *filt,
                         float *smooth, float *loglik, void *stream, void *const *events);

#ifdef __cplusplus
}
#endif

#endif /* KS_H */
