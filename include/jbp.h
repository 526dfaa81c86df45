/*
 * jbp.h -- C ABI of the GB300 joint FFT belief-propagation decoder.
 *
 * The library decodes frames of K users who share one regular GF(q) LDPC code
 * (q = 2^m, m = 1..6) and whose PAM levels add on a real AWGN channel:
 *
 *     y_t = sum_k (2 c_{k, pi_k^{-1}(t)} - (q-1)) + w_t,   w_t ~ N(0, sigma2).
 *
 * Each decoding iteration is sum-product belief propagation on the joint
 * factor graph, run as hand-written sm_103a CUDA kernels:
 *   (a) channel node: each user's extrinsic q-ary message from the other users'
 *       distributions (prefix/suffix convolution over the integer symbol sum,
 *       no division) scored against y_t;
 *   (b) check node (FFT-QSPA): the variable-to-check rule of the paper's
 *       appendix "Q-ary LDPC code", eq. (app_ldpc_v2c), then eq. (app_ldpc_c2v)
 *       evaluated in the Walsh-Hadamard domain (appendix "Complexity
 *       derivation", paragraph FFT-BP): permute by the edge coefficient, WHT,
 *       leave-one-out product, inverse WHT, inverse permutation;
 *   (c) variable node: the marginal of eq. (app_ldpc_marginal);
 *   (d) hard decision, syndrome check (eq. app_ldpc_check_eq) and per-frame
 *       early exit on convergence (Table 1 caption: at most 50 iterations
 *       with early exit).
 *
 * Messages are FP32 probability vectors scaled to a largest entry of 1 (their
 * natural logs are the decoder's max-normalised log-messages).  A c2v message
 * is floored at 1e-12 of its maximum; a channel message is floored at 1e-12.
 * The schedule is flooding: per iteration all channel nodes, then all checks,
 * then the decisions.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a jbp_status.  On failure jbp_last_error() returns a
 *     thread-local message describing the most recent failure of this thread.
 *     No C++ exception crosses this interface.
 *   - Field: GF(2^m) with the primitive polynomials x+1, x^2+x+1, x^3+x+1,
 *     x^4+x+1, x^5+x^2+1, x^6+x+1; symbol index bits are the polynomial
 *     coefficients (bit i = coefficient of x^i).
 *   - Layouts are row-major and frame-major.  Check-major edges: edge
 *     e = j*dc + d is the d-th nonzero of row j of H.
 *   - "device pointer" means memory of the handle's GPU (cudaMalloc or any
 *     allocator of that device); "host pointer" means pageable or pinned host
 *     memory.  The library never frees memory it did not allocate.
 */
#ifndef JBP_H
#define JBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JBP_OK = 0,
    JBP_EINVAL = 1,    /* invalid argument (NULL handle, bad size, unsupported shape)   */
    JBP_ENOMEM = 2,    /* device or host allocation failed, or the memory budget is hit */
    JBP_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error)       */
    JBP_EAGAIN = 4,    /* jbp_poll: the request is not finished yet                     */
    JBP_ETIMEOUT = 5,  /* a bounded device-side wait expired                            */
    JBP_ECLOSED = 6    /* the context is shutting down / ticket unknown or consumed     */
} jbp_status;

/* Check-node transform precision.  FP32: Walsh-Hadamard butterflies in FP32 on
 * the CUDA cores.  The others run the transform as a dense +-1 matrix product on
 * the tensor cores with BF16 operands and FP32 accumulation: BF16X3 splits each
 * FP32 operand into three BF16 terms (about FP32 accuracy), BF16X2 into two
 * (hi/lo), BF16 uses one. */
typedef enum { JBP_PREC_FP32 = 0, JBP_PREC_BF16X2 = 1, JBP_PREC_BF16 = 2, JBP_PREC_BF16X3 = 3 } jbp_precision;

/* Channel-node algorithm (kernel (a)).  TRELLIS: the exact FP32 sum-product
 * over the integer symbol sums (prefix convolutions and scored suffixes; the
 * reference numerics).  DFT: the same extrinsic messages as a correlation in
 * the frequency domain of the sum alphabet (DFT length L >= K(q-1)+1), with the
 * forward and inverse transforms issued as matrix products on the tensor cores
 * (FP16 operand terms, FP32 accumulation).  Its error is absolute, a few 1e-4
 * of each message's maximum at most ((K+2) 2^-9 + K 2^-12 by construction),
 * rather than relative per entry, so entries far below the maximum are not
 * resolved; a channel use whose peak the transform cannot resolve is computed
 * by the trellis in the same call.  It runs in the step form for 2 <= K <= 8
 * and q = 16, 32, 64; other handles of the context keep the trellis
 * (jbp_query_channel tells which).  AUTO: DFT except where the register-
 * resident trellis applies (q <= 16 and K <= 4), which is the faster node there
 * and keeps the fused form where a frame fits it.  Under AUTO, jbp_create also
 * times both nodes on a decoder that has the DFT form (at 1 frame and at the
 * frame count that fills the SMs), and its serving pools run, block by block,
 * the node measured faster for the pool's current frame count (the DFT node
 * has a latency floor per tile of channel uses, so a pool of a few frames runs
 * the trellis); a served frame then matches its decode alone within the DFT
 * node's bound, not bit for bit.  No paper counterpart: the paper prints no
 * channel-node kernel. */
typedef enum { JBP_CHAN_TRELLIS = 0, JBP_CHAN_DFT = 1, JBP_CHAN_AUTO = 2 } jbp_channel_node;

/* Launch form of jbp_decode.  AUTO picks FUSED when one frame's message state
 * fits in one SM's shared memory, else STEP.  FUSED: one persistent kernel runs
 * every iteration of a group of frames with all messages in shared memory.
 * STEP: one kernel per node type per iteration, messages resident in HBM.
 * PLAIN: the STEP kernels launched for one frame at a time (the per-frame
 * reference form used for comparison). */
typedef enum { JBP_FORM_AUTO = 0, JBP_FORM_FUSED = 1, JBP_FORM_STEP = 2, JBP_FORM_PLAIN = 3 } jbp_form;

typedef struct jbp_ctx jbp_ctx;  /* one GPU, its streams, memory budget and serving loop */
typedef struct jbp_h jbp_h;      /* one (code, K, q, channel) decoder bound to a context  */

/* Parity-check matrix H (P x n over GF(q)): every check has dc edges (dc = 3,
 * 4 or 6); dv is the largest variable degree, and a variable may have fewer
 * edges (an irregular variable-degree profile; the paper's construction of H
 * samples a sparse support with no degree regularity).  chk_var [P*dc]: variable
 * index of each edge; chk_coef [P*dc]: nonzero coefficient H_{j,l} in 1..q-1.
 * Host pointers, copied by jbp_create; the caller keeps ownership.  The fused
 * form's fast (position-major) shape and the tensor-core variants need dc = 4,
 * the former also every variable of degree 2; other codes run the step form or
 * the fused form's team shape. */
typedef struct {
    int32_t n, P, q, dv, dc;
    const int32_t *chk_var;
    const uint8_t *chk_coef;
} jbp_code;

/* Channel.  sigma2 > 0: noise variance.  interleave = 1: perm [K*n] gives
 * pi_k(i), the channel use that carries user k's symbol i (each row a
 * permutation of 0..n-1).  interleave = 0: every pi_k is the identity and perm
 * may be NULL.  Host pointer, copied by jbp_create. */
typedef struct {
    double sigma2;
    int32_t interleave;
    const int32_t *perm;
} jbp_channel;

/* Context options.  iters: maximum iterations T (>= 1).  early_stop: 1 stops a
 * frame at the first iteration after which all K syndromes are zero.
 * precision: jbp_precision of the check-node transform (the tensor-core
 * variants run in the step form; AUTO then picks STEP).  mem_budget_bytes:
 * cap on the device memory the context allocates (0 = 90% of free memory at
 * creation).  device: CUDA device ordinal.  block_iters: iterations per
 * serving block (0 = 5).  channel_node: jbp_channel_node (DFT runs in the step
 * form; AUTO then picks STEP for the handles that use it).  reserved: zero. */
typedef struct {
    int32_t iters;
    int32_t early_stop;
    int32_t precision;
    int32_t device;
    int64_t mem_budget_bytes;
    int32_t block_iters;
    int32_t channel_node;
    int32_t reserved[6];
} jbp_options;

/* One decode call.  F >= 0 frames.  y [F*n] FP32 channel outputs.  Outputs:
 * hat [F*K*n] decided symbols; iters [F] iterations run (the stopping
 * iteration, or T); ok [F*K] 1 where user k's syndrome is zero after the last
 * iteration run; logpost [F*K*n*q] optional (may be NULL) max-normalised
 * log-posterior of the last iteration run.
 * on_device = 0: host pointers; the call copies in and out and returns when
 * the outputs are written (a batch of 8,192 frames or more goes in eight parts
 * whose copies overlap the other parts' decodes; the outputs are those of one
 * launch).  on_device = 1: device pointers; the work is
 * enqueued on `stream` (a cudaStream_t, NULL = the handle's own stream) and the
 * call returns without waiting; outputs are valid once that stream reaches
 * this point.  form: jbp_form.  sigma2 [F]: optional (NULL = the handle's
 * channel) per-frame noise variance, host or device like the other buffers.
 * Buffers must not overlap. */
typedef struct {
    int32_t F;
    const float *y;
    uint8_t *hat;
    int32_t *iters;
    uint8_t *ok;
    float *logpost;
    int32_t on_device;
    int32_t form;
    void *stream;
    const float *sigma2;
} jbp_batch;

/* Create a context on opt->device.  Fails with JBP_EINVAL on bad options,
 * JBP_ECUDA if the device cannot be used.  *out owns streams and a serving
 * thread (started on the first jbp_submit). */
int jbp_context_create(const jbp_options *opt, jbp_ctx **out);

/* Stop the serving thread, wait for in-flight work, free everything the
 * context owns.  Handles of this context must be destroyed first. */
int jbp_context_destroy(jbp_ctx *ctx);

/* Bind a decoder for `code`, K >= 1 users (K <= 16) and GF(q) (q = code->q)
 * to the context: step a0 of the decoder, its one-time setup.  Defined by the
 * paper's appendix "Q-ary LDPC code": the code is the null space over GF(Q) of
 * a sparse parity-check matrix H (eq. app_ldpc_check_eq; every row a check
 * sum_l H_{j,l} c_l = 0 over GF(Q)), H built as in its paragraph "Construction
 * of H" (a sparse support with nonzero coefficients on GF(Q)*), and symbols
 * map to field elements by a fixed bijection (the index bits are the
 * polynomial coefficients of the field listed at the top of this file).  The
 * call deep-copies chk_var, chk_coef and the interleavers pi_k to the device;
 * builds the GF(q) multiply and divide tables (jbp_gf_tables), the per-user
 * slot tables of the fused form and the check order of its shared-memory
 * layout; the caller keeps ownership of every host array.  Supported shapes:
 * q in {2,4,8,16,32,64}, dc in {3, 4, 6}, variable degrees 0..dv with
 * 1 <= dv <= 8, n >= 1; the tensor-core check variants (precision other than
 * FP32) need dc = 4.  Errors: JBP_EINVAL (NULL pointers, unsupported shape, a
 * variable with more than dv edges or a coefficient outside 1..q-1),
 * JBP_ENOMEM (over the context's budget), JBP_ECUDA. */
int jbp_create(jbp_ctx *ctx, const jbp_code *code, int32_t K, int32_t q,
               const jbp_channel *chan, jbp_h **out);

/* Free the handle's device memory.  Its pending submitted requests are
 * cancelled (their tickets poll JBP_ECLOSED). */
int jbp_destroy(jbp_h *h);

/* Decode one batch (see jbp_batch): up to T iterations of joint
 * sum-product BP per frame, flooding schedule.  Each iteration is the
 * channel-node update (kernel (a) above: the K-user PAM-sum factor), the
 * variable-to-check rule eq. (app_ldpc_v2c), the check-to-variable rule
 * eq. (app_ldpc_c2v) in the Walsh-Hadamard domain (appendix "Complexity
 * derivation", paragraph FFT-BP), the marginal eq. (app_ldpc_marginal) and
 * its hard decision (ties -> lowest symbol), then the parity checks
 * eq. (app_ldpc_check_eq): with early_stop a frame ends at the first iteration
 * after which all K users' syndromes are zero (Table 1 caption: at most 50
 * iterations with early exit on convergence), and its outputs are those of that
 * iteration.  Frames are independent; the result of a frame does not depend on
 * the batch it is in.  Errors: JBP_EINVAL (NULL buffers, F < 0, a form the
 * handle cannot run), JBP_ENOMEM, JBP_ECUDA, JBP_ETIMEOUT (a bounded device wait
 * of a tensor-core or staged kernel expired; outputs are then not valid). */
int jbp_decode(jbp_h *h, jbp_batch *batch);

/* Decode several device batches of possibly different decoders (codes, K, q)
 * of one context in one call: the parts run concurrently on the context's
 * stream pool (parts of one handle run in order on one stream; at most 32
 * distinct handles).  Every batch must have on_device = 1.  Work is ordered
 * after prior work on `stream` (NULL = the context's stream; any stream,
 * cudaStreamLegacy included) and completion is ordered before later work on
 * it, through events: the decode itself runs on a stream of the context.  The
 * call returns without waiting.  The first call with a given argument set
 * autotunes each fused part's launch shape (jbp_tune) and runs eagerly; the
 * second captures the whole multi-part decode as one CUDA graph, which later
 * calls with identical arguments (handles, sizes, pointers) replay with one
 * launch, whatever the caller's stream. */
int jbp_decode_many(jbp_ctx *ctx, int32_t nparts, jbp_h *const *handles, const jbp_batch *batches, void *stream);

/* Autotune the fused-form launch shape of a handle on a device batch (runs a
 * few short timed launches that write the first frames' outputs: each distinct
 * shape the planner resolves is timed 5 times and scored by the median; a shape
 * whose launch fails is skipped) and keep the fastest; *threads and
 * *frames_per_cta receive the resolved shape (both >= 1 for a handle with a
 * fused form; 0 when the handle has none).  Returns JBP_ECUDA if no candidate
 * ran.  Synchronous.  With batch == NULL the shape is set from *threads and
 * *frames_per_cta instead (0 = default; threads > 256 selects, for K = 4, the
 * variant that splits each channel use over two lanes).  The per-frame
 * arithmetic does not depend on the shape. */
int jbp_tune(jbp_h *h, const jbp_batch *batch, int32_t *threads, int32_t *frames_per_cta);

/* Serving: queue one frame (y_frame [n] host pointer, copied before return)
 * for continuous batching on the context's device; sigma2 > 0 is this
 * frame's noise variance (<= 0: the handle's channel).  *ticket identifies it.
 * The frame is decoded by the same iteration as jbp_decode (eqs.
 * app_ldpc_v2c, app_ldpc_c2v, app_ldpc_marginal, app_ldpc_check_eq with early
 * exit); the paper has no serving counterpart: requests of any decoder of the
 * context are admitted into resident device pools as slots and memory free
 * up and re-batched every block of iterations.  A decoder that the fused
 * position-major kernel serves (q <= 16, K <= 4, every variable of degree 2,
 * FP32 check, trellis channel node) keeps its pool in that kernel's layout and
 * runs each block as one launch of it (a slot's state goes to shared memory and
 * back to HBM once per block): its served frames equal jbp_decode's fused form
 * bit for bit.  Other decoders' pools run the step form and equal its results
 * (under AUTO with the DFT node, see jbp_channel_node).  Thread-safe.  Errors:
 * JBP_EINVAL (NULL pointer, sigma2 not finite), JBP_ECLOSED (the context is
 * shutting down).  The queue is unbounded: a request waits on the host until a
 * pool slot frees up. */
int jbp_submit(jbp_h *h, const float *y_frame, double sigma2, uint64_t *ticket);

/* Serving: JBP_EAGAIN while the request runs; JBP_OK once finished, with
 * hat [K*n], iters [1] and ok [K] written (host pointers; any may be NULL):
 * the decisions of eq. (app_ldpc_marginal), the iterations run and the
 * syndrome flags of eq. (app_ldpc_check_eq), as jbp_decode gives them for the
 * same frame.  A finished ticket is consumed by the successful poll; polling it
 * again gives JBP_ECLOSED.  Thread-safe; no paper counterpart (serving). */
int jbp_poll(jbp_ctx *ctx, uint64_t ticket, uint8_t *hat, int32_t *iters, uint8_t *ok);

/* Serving statistics since context creation: completed requests, and the
 * p50 / p99 submit-to-finish latency in microseconds (0 when nothing ran). */
int jbp_serving_stats(jbp_ctx *ctx, uint64_t *completed, double *p50_us, double *p99_us);

/* Thread-local message of the last failure on this thread ("" if none). */
const char *jbp_last_error(void);

/* ---- single steps on device buffers (one kernel launch each, enqueued on
 * `stream`, NULL = the handle's stream).  They expose the per-iteration kernels
 * for testing and for callers that schedule iterations themselves.
 * Layouts: msg [F*K*E*q] holds, per edge, the check-to-variable message
 * (before jbp_step_channel, after jbp_step_check) or the variable-to-check
 * message (after jbp_step_channel), as probabilities scaled to max 1 (the
 * uniform start is all ones), 16-byte aligned; ch2v [F*K*n*q] likewise; post [F*K*n*q]
 * max-normalised log-posterior; hat [F*K*n]; ok [F*K]; E = P*dc. ---- */

/* (a) channel node for every channel use of F frames: reads the c2v messages in
 * msg and y [F*n]; writes ch2v and replaces each c2v in msg by the v2c message
 * of the same edge (eq. app_ldpc_v2c with the channel message as local belief). */
int jbp_step_channel(jbp_h *h, int32_t F, const float *y, float *msg, float *ch2v, void *stream);

/* (b) check node for every check: replaces the v2c messages in msg by the new
 * c2v messages (eq. app_ldpc_c2v in the WHT domain); precision: jbp_precision.
 * msg must be 16-byte aligned (JBP_EINVAL otherwise): the kernel moves tiles of
 * it with bulk copies. */
int jbp_step_check(jbp_h *h, int32_t F, float *msg, int32_t precision, void *stream);

/* (c) variable node: post = ch2v + sum of the variable's c2v (max-normalised;
 * post may be NULL) and the hard decision hat (ties -> lowest symbol). */
int jbp_step_var(jbp_h *h, int32_t F, const float *ch2v, const float *msg, float *post,
                 uint8_t *hat, void *stream);

/* (d) syndrome: ok[f*K+k] = 1 iff every check of user k is satisfied by hat. */
int jbp_step_syndrome(jbp_h *h, int32_t F, const uint8_t *hat, uint8_t *ok, void *stream);

/* Decode without allocating memory.  For callers that may not allocate device
 * memory themselves (code running inside another framework's memory pool or
 * under a hard memory cap, or a process that may not call cudaMalloc): the
 * paper has no counterpart; this is a deployment variant of the step-form
 * decode (the same kernels as jbp_decode with JBP_FORM_STEP).  Its working
 * memory -- code tables and message state -- lives in one fixed 16 MiB device
 * array inside the library, which every GPU that loads the library holds until
 * the process exits; no call allocates (no cudaMalloc/cudaFree, no allocating
 * library routine).  code/chan: host pointers as for jbp_create (dc = 4,
 * regular dv, q in 2..64, K in 1..16).  T >= 1 iterations, early_stop as in
 * jbp_options.  y [F*n], hat [F*K*n], iters [F], ok [F*K]: device pointers of the
 * current device.  The work is enqueued on `stream` (a cudaStream_t, NULL = the
 * default stream) and the call returns without waiting.  Errors: JBP_EINVAL for
 * bad arguments, and when F frames of this shape do not fit the fixed array (the
 * message gives the maximum F); JBP_ECUDA for CUDA failures.  The first call on
 * each device looks up the array's device address (set-up); make that first
 * call before any stream capture.  All calls share the array and it keeps the
 * previous call's contents (each call clears what must start at zero); calls
 * whose work overlaps on the GPU race on it, so serialise them.  If a bounded
 * device wait of the check kernel expires during a call (JBP_ETIMEOUT in
 * jbp_decode), that call's outputs are marked instead, since it returns before
 * the work runs: every frame gets iters = -1 and ok = 0. */
int jbp_decode_noalloc(const jbp_code *code, int32_t K, const jbp_channel *chan, int32_t T,
                       int32_t early_stop, int32_t F, const float *y, uint8_t *hat, int32_t *iters,
                       uint8_t *ok, void *stream);

/* Counters of a handle since creation (host pointers, may be NULL):
 * log_fallbacks = channel messages whose linear-domain computation underflowed
 * and were recomputed in log space; tc_timeouts = 1 if a bounded device wait
 * (a tensor-core completion or a staged check tile) ever expired.
 * Synchronises the device. */
int jbp_stats(jbp_h *h, uint64_t *log_fallbacks, int32_t *tc_timeouts);

/* Shape information of a handle (host pointers, any may be NULL): edges E,
 * per-frame device state bytes, and whether one frame fits the fused form. */
int jbp_query(jbp_h *h, int32_t *E, int64_t *state_bytes_per_frame, int32_t *fused_ok);

/* The channel node this handle runs (jbp_channel_node): DFT where the context
 * asked for it and the handle's (K, q) supports it, else TRELLIS.  No paper
 * counterpart: an implementation query. */
int jbp_query_channel(jbp_h *h, int32_t *channel_node);

/* Host only (no GPU, no context): the GF(q) tables jbp_create uploads for the
 * check node's coefficient permutations (step a0 of the decoder's setup), for
 * inspection and tests.  q = 2, 4, ..., 64 with the field polynomials listed at
 * the top of this file.  mul and div (host pointers owned by the caller, q*q
 * bytes each) receive mul[h*q + x] = h x and div[h*q + x] = h^{-1} x (row h = 0
 * of div is zero).  Returns JBP_EINVAL for another q or a NULL table.  The
 * field arithmetic is that of the parity checks, appendix "Q-ary LDPC code",
 * eq. app_ldpc_check_eq: sums over GF(q) of symbols times nonzero entries of H. */
int jbp_gf_tables(int32_t q, uint8_t *mul, uint8_t *div);

/* Host only (no GPU, no context): the constant operand tables the DFT channel
 * node of (K, q) loads, as jbp_create builds them, for inspection and tests.
 * shape (may be NULL) receives {L, W, KB, Nc, chunks}: DFT length L = the first
 * multiple of 16 >= K(q-1)+1; Gaussian-score window W = min(L, 128); forward
 * inner width KB = max(q, W); Nc spectral rows per chunk; chunks = L / Nc.
 * *bytes (required) receives the table size; out (may be NULL) receives the
 * tables, host memory owned by the caller, at least *bytes long:
 *   per chunk c = 0..chunks-1, four tiles of FP16 values:
 *     forward hi, forward lo  [Nc x KB], element (r, x) = F(c*Nc + r, x)
 *     inverse hi, inverse lo  [q x Nc],  element (a, r) = B(a, c*Nc + r)
 *   then L float pairs (cos, sin)(2 pi m / L), m = 0..L-1.
 * F(n, x): spectral row n of the length-L real DFT folded onto frequencies
 * 0..L/2 (pair p = n/2; n = 0: 1, n = 1: (-1)^x (the Nyquist term); else n
 * even: cos, n odd: -sin of 2 pi p x / L).  B(a, n): the inverse over that
 * folded spectrum (n = 0: 1; n = 1: (-1)^a; else n even: 2 cos, n odd: -2 sin
 * of 2 pi p a / L), so that sum_n B(a, n) F(n, x) = L [a == x].  hi = the FP16
 * rounding of the value, lo = the FP16 rounding of the remainder.  A (rows x D)
 * tile stores element (m, k) at byte (m/8)(D/8)128 + (k/8)128 + (m%8)16 + (k%8)2
 * (8x8 core matrices of 128 bytes, consecutive along k, then along m).
 * Returns JBP_EINVAL if (K, q) has no DFT form (q not 16, 32 or 64, K not
 * 2..8) or bytes is NULL.  No paper counterpart: the paper prints no
 * channel-node kernel; the node computed is kernel (a) above. */
int jbp_dft_tables(int32_t K, int32_t q, int32_t *shape, void *out, int64_t *bytes);

/* Measured FP32 multiply-add throughput of `device` (TFLOP/s, 2 flops per
 * multiply-add), the denominator of the ALU roofline the channel-node and
 * fused kernels are reported against.  Runs independent FMA chains on every
 * SM for about `seconds` (0 < seconds <= 60) as three back-to-back launches and
 * returns the median rate in *tflops.  packed = 0: one multiply-add per lane
 * and instruction (FFMA); packed = 1: two-lane FP32 instructions (two
 * multiply-adds per lane and instruction).  Synchronous; allocates a small
 * device buffer; changes no device setting.  Errors: JBP_EINVAL (NULL tflops,
 * seconds out of range), JBP_ECUDA.  No paper counterpart: a measurement
 * utility. */
int jbp_fp32_peak(int32_t device, double seconds, int32_t packed, double *tflops);

/* ---- the paper's own classical path on the evidence interface S ----
 *
 * The paper's baseline decoders (appendix "Complexity derivation", paragraphs
 * SIC-BP and FFT-BP; Table 1) decode K rows from a slot-wise evidence matrix
 * S [n x q] (appendix "Q-ary LDPC code", eq. app_ldpc_local_belief_from_S),
 * produced by a fixed AMP-MMSE slot detector (appendix "Slot-wise AMP--MMSE
 * detector").  A jbp_ura handle holds one code and one detector configuration:
 *
 *   jbp_amp_evidence  y -> S     AMP per slot, eqs. amp_iter_r / amp_iter_u /
 *                                amp_iter_res, Bernoulli-Gaussian denoiser
 *                                eqs. bg_activity_prob / bg_mmse_mean, and
 *                                S[l][a] = log p^(R_a; nu) (paragraph
 *                                "Evidence interface")
 *   jbp_sic_decode    S -> rows  SIC: row k is single-row FFT-BP from local
 *                                beliefs exp(S^(k)) (max-normalised, floored at
 *                                1e-12 of the max), flooding, WHT check
 *                                node, early exit on a zero syndrome; then
 *                                S^(k+1) = S^(k) + cancel_log at each slot's
 *                                decided symbol (the paper leaves the SIC rule
 *                                open; this is the rule built here)
 *   jbp_ura_decode    y -> rows  both, with S kept on the device
 *
 * Slot model (appendix "Unsourced random access"): slot l of a frame carries
 * y_l = A_l u_l + noise in C^ns with A_l = F_{rows_l,:} / sqrt(ns), F_{k,a} =
 * exp(-2 pi i k a / q) (partial DFT, appendix "Sensing-matrix construction"). */
typedef struct jbp_ura jbp_ura;

/* Detector and decoder parameters.  ns: complex channel uses per slot, 1..32
 * (and <= q).  K: rows decoded by SIC, 1..8.  amp_iters >= 0 (I_AMP).
 * bp_iters >= 1 per row; early_stop = 1 ends a row at the first zero
 * syndrome.  rho_bg in (0, 1) and sigma_u2 > 0: the Bernoulli-Gaussian prior of
 * every coordinate.  cancel_log <= 0.  rows [n*ns]: slot l's partial-DFT rows at
 * rows + l*ns, distinct values in 0..q-1; host pointer, copied. */
typedef struct {
    int32_t ns, K, amp_iters, bp_iters, early_stop, reserved;
    double rho_bg, sigma_u2, cancel_log;
    const int32_t *rows;
} jbp_ura_params;

/* Create a handle for a code (regular, (dv, dc) = (2, 3), (2, 4) or (3, 6); q = 16, 32 or 64
 * for the decoder, q = 32 or 64 for the detector) on ctx's device.  The code
 * arrays and rows are copied.  Errors: JBP_EINVAL (bad code or parameters,
 * or one frame's decoder state does not fit shared memory), JBP_ENOMEM,
 * JBP_ECUDA. */
int jbp_ura_create(jbp_ctx *ctx, const jbp_code *code, const jbp_ura_params *p, jbp_ura **out);
int jbp_ura_destroy(jbp_ura *u);

/* Evidence of F frames.  y [F*n*ns*2] (complex, real then imaginary per channel
 * use, slot-major), S [F*n*q] out.  on_device = 1: device pointers, work
 * enqueued on `stream` (NULL = the context's stream), no wait.  on_device = 0:
 * host pointers, the call copies, runs and waits. */
int jbp_amp_evidence(jbp_ura *u, int32_t F, const float *y, float *S, int32_t on_device, void *stream);

/* SIC decode of F frames from evidence S [F*n*q]: hat [F*K*n] (row k of frame
 * f at (f*K + k)*n), iters [F*K] (BP iterations of each row), ok [F*K] (row's
 * syndrome zero).  Pointers and on_device as jbp_amp_evidence. */
int jbp_sic_decode(jbp_ura *u, int32_t F, const float *S, uint8_t *hat, int32_t *iters, uint8_t *ok,
                   int32_t on_device, void *stream);

/* jbp_amp_evidence then jbp_sic_decode; S stays in the handle's device
 * workspace (grown as needed, within the context's memory budget). */
int jbp_ura_decode(jbp_ura *u, int32_t F, const float *y, uint8_t *hat, int32_t *iters, uint8_t *ok,
                   int32_t on_device, void *stream);

/* Symbol and codeword errors after row alignment (eq. app_ura_hungarian): for
 * each of F frames, the assignment of decoded rows to true rows (a permutation
 * of K <= 8 rows) with the fewest symbol mismatches; among equally good ones
 * the first in lexicographic order.  hat, truth [F*K*n] symbols (row k of frame
 * f at (f*K + k)*n); sym_err [F] mismatched symbols and cw_err [F] mismatched
 * rows under that assignment.  on_device = 1: device pointers, work enqueued on
 * `stream` (NULL = the context's stream), no wait; 0: host pointers, the call
 * copies, runs and waits.  An evaluation helper; it does not change a decode. */
int jbp_match_rows(jbp_ctx *ctx, int32_t F, int32_t K, int32_t n, const uint8_t *hat, const uint8_t *truth,
                   int32_t *sym_err, int32_t *cw_err, int32_t on_device, void *stream);

#ifdef __cplusplus
}
#endif
#endif
