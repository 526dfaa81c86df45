/*
 * jbp_oracle.h -- FP64 CPU oracle for joint sum-product belief propagation over
 * K users that share one GF(2^m) LDPC code and are coupled by a PAM-sum channel.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle is the plain, slow, obviously correct
 * statement of what the decoder computes.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no source,
 * header, table or helper with the CUDA library, and the library never calls it.
 *
 * Notation follows the paper's appendix "Q-ary LDPC code": variable nodes
 * l in [L] (here L = n), check nodes j in [P], field F_Q with Q = 2^m, edge
 * coefficients H_{j,l} in F_Q^x, messages m_{l->j}(a) and m_{j->l}(a).
 *
 * Message convention: every message is a log-probability vector over the Q
 * symbols, shifted so that its maximum is 0 ("max-normalised log-message").
 */
#ifndef JBP_ORACLE_H
#define JBP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Parity-check matrix in check-major edge order: edge e = j*dc + d is the d-th
 * nonzero of row j; it joins check j to variable chk_var[e] with coefficient
 * chk_coef[e] (an integer 1..Q-1 read as a polynomial over GF(2)).  Variable
 * degrees may be anything (0 included); every check has exactly dc edges. */
typedef struct {
    int n;               /* L: number of variable nodes per user            */
    int P;               /* number of check nodes                           */
    int dc;              /* check degree                                    */
    int m;               /* Q = 2^m, 1 <= m <= 8                            */
    const int *chk_var;  /* [P*dc]                                          */
    const int *chk_coef; /* [P*dc]                                          */
} or_code;

/* Joint channel: y_t = sum_k level(c_{k, pi_k^{-1}(t)}) + w_t, w_t ~ N(0, sigma2),
 * level(a) = 2a - (Q-1).  perm[k*n + i] = pi_k(i) = channel use that carries
 * user k's symbol i; perm == NULL means pi_k = identity for every user. */
typedef struct {
    int K;
    double sigma2;
    const int *perm;     /* [K*n] or NULL                                   */
} or_chan;

enum { OR_CHECK_WHT = 0, OR_CHECK_DIRECT = 1, OR_CHECK_LITERAL = 2 };

/* ---- field (appendix "Q-ary LDPC code": fixed bijection [Q] -> F_Q) ---- */
int or_gf_poly(int m);                      /* primitive polynomial used for GF(2^m) */
int or_gf_mul(int m, int a, int b);         /* product in GF(2^m)                    */

/* ---- single node updates (one frame, one node) ---- */

/* Channel-node extrinsic for one channel use.  logmu [K*Q]: max-normalised
 * log-messages from the K users' variable nodes; out [K*Q]: max-normalised,
 * clipped at log_floor.  Trellis form (prefix sums forward, scored suffixes
 * backward, log-sum-exp in FP64). */
void or_channel_node(int K, int m, double sigma2, double y, const double *logmu,
                     double log_floor, double *out);
/* Same quantity by enumerating all Q^(K-1) assignments of the other users. */
void or_channel_node_brute(int K, int m, double sigma2, double y, const double *logmu,
                           double log_floor, double *out);

/* Check-node update for one check of degree dc.  coef [dc]; logv2c [dc*Q]
 * (max-normalised); out [dc*Q] max-normalised c2v log-messages.  method:
 * OR_CHECK_WHT (Walsh-Hadamard domain, the FFT-BP form), OR_CHECK_DIRECT
 * (XOR convolutions of the permuted messages) or OR_CHECK_LITERAL (the sum over
 * parity-satisfying assignments written out).  rel_floor: r <- max(r, rel_floor*max r). */
void or_check_node(int m, int dc, const int *coef, const double *logv2c, int method,
                   double rel_floor, double *out);

/* ---- whole-frame steps, batched over F frames (OpenMP over frames) ----
 * Layouts (frame-major): y [F*n]; c2v [F*K*E*Q] with E = P*dc in check-major
 * edge order; ch2v and post [F*K*n*Q]; hat [F*K*n]; ok [F*K]. */
void or_step_channel(const or_code *code, const or_chan *ch, int F, const float *y,
                     const double *c2v, double log_floor, double *ch2v);
void or_step_check(const or_code *code, int K, int F, const double *ch2v,
                   const double *c2v_old, int method, double rel_floor, double *c2v_new);
void or_step_var(const or_code *code, int K, int F, const double *ch2v, const double *c2v,
                 double *post, uint8_t *hat);
/* v2c [F*K*E*Q] of every edge (eq. app_ldpc_v2c), and the check update applied
 * to given v2c messages (the two halves of or_step_check). */
void or_step_v2c(const or_code *code, int K, int F, const double *ch2v, const double *c2v,
                 double *v2c);
void or_step_check_v2c(const or_code *code, int K, int F, const double *v2c, int method,
                       double rel_floor, double *c2v_new);
void or_syndrome(const or_code *code, int K, int F, const uint8_t *hat, uint8_t *ok);

/* ---- full decode ---- */
typedef struct {
    int iters;           /* T: maximum number of iterations                 */
    int early_stop;      /* 1: stop a frame once all K syndromes are zero    */
    int check_method;    /* OR_CHECK_*                                      */
    double rel_floor;    /* c2v floor relative to the max (1e-12), 0 = none  */
    double log_floor;    /* ch2v clip (log(1e-12)), -INFINITY = none         */
    int threads;         /* OpenMP threads, <= 0: library default            */
} or_opts;

/* Decode F frames.  Outputs (NULL = not wanted): hat [F*K*n], iters [F],
 * ok [F*K], post [F*K*n*Q] (final max-normalised log-posterior), margin [F*K*n]
 * (p(1) - p(2) of the sum-normalised posterior), ch2v_out [F*K*n*Q] and
 * c2v_out [F*K*E*Q] (messages of the last iteration run). */
void or_decode(const or_code *code, const or_chan *ch, int F, const float *y,
               const or_opts *o, uint8_t *hat, int32_t *iters, uint8_t *ok,
               double *post, double *margin, double *ch2v_out, double *c2v_out);

/* Exact posterior marginals p(c_{k,i} = a | y) by enumerating the codebook
 * {c : Hc = 0} (all Q^n words tested) and all K-tuples of codewords.  Tiny
 * cases only (Q^n <= 2^20 and |C|^K <= 2^24).  out [K*n*Q] max-normalised logs.
 * Returns |C|, or -1 if the case is too large. */
long or_brute_marginals(const or_code *code, const or_chan *ch, const float *y, double *out);

/* ---- evidence interface: slot-wise AMP detector and SIC FFT-BP ----
 * The paper's own classical baseline decodes K rows from a slot-wise evidence
 * matrix S (L x Q) produced by a fixed AMP-MMSE detector (appendix "Slot-wise
 * AMP--MMSE detector"; appendix "Q-ary LDPC code", eq. app_ldpc_local_belief_from_S;
 * appendix "Complexity derivation", paragraphs SIC-BP and FFT-BP). */

/* Scalar Bernoulli-Gaussian channel R = U + W, W ~ CN(0, nu),
 * U ~ (1-rho) delta_0 + rho CN(0, su2); s = |r|^2.
 * or_bg_log_activity: log of the activity posterior, eq. (bg_activity_prob).
 * or_bg_gain: eta(r)/r, so that eq. (bg_mmse_mean) is eta(r) = gain * r.
 * or_bg_deriv: the complex sensitivity d eta / d r (half the divergence
 * d Re(eta)/d Re(r) + d Im(eta)/d Im(r)), which scales the Onsager term. */
double or_bg_log_activity(double s, double nu, double rho, double su2);
double or_bg_gain(double s, double nu, double rho, double su2);
double or_bg_deriv(double s, double nu, double rho, double su2);

/* AMP-MMSE on one slot, eqs. (amp_iter_r), (amp_iter_u), (amp_iter_res):
 * A = F_{rows,:} / sqrt(ns) with F_{k,a} = exp(-2 pi i k a / Q) (partial DFT,
 * appendix "Sensing-matrix construction"), nu^(i) = |Ytilde^(i)|^2 / ns.
 * y [2*ns] interleaved complex observation; after `iters` iterations the
 * evidence S[a] = log p^(R^(iters)_a; nu^(iters)) (paragraph "Evidence
 * interface").  R_out [2*Q] (final pseudo-observation) and nu_out may be NULL.
 * Q here is any size >= 1 (not only a field size). */
void or_amp_slot(int Q, int ns, const int *rows, const float *y, int iters, double rho,
                 double su2, double *S, double *R_out, double *nu_out);
/* The same iteration for any dictionary A [ns*Q] given by its real and
 * imaginary parts (row-major, A[i*Q + a]). */
void or_amp_dict(int Q, int ns, const double *Ar, const double *Ai, const float *y, int iters,
                 double rho, double su2, double *S, double *R_out, double *nu_out);
/* Batched over F frames of L slots: y [F*L*ns*2], rows [L*ns] (slot l uses
 * rows + l*ns), S [F*L*Q]. */
void or_amp_evidence(int Q, int ns, int L, const int *rows, int F, const float *y, int iters,
                     double rho, double su2, double *S, int threads);

/* Single-row FFT-BP with local beliefs lambda_l(a) proportional to exp(S_{l,a})
 * (eq. app_ldpc_local_belief_from_S), max-normalised and clipped at
 * o->log_floor; flooding: v2c (eq. app_ldpc_v2c), check (the WHT form),
 * marginal and decision (eq. app_ldpc_marginal), early exit when the syndrome
 * is zero.  S [F*n*Q]; outputs as or_decode with K = 1. */
void or_bp_prior(const or_code *code, int F, const double *S, const or_opts *o, uint8_t *hat,
                 int32_t *iters, uint8_t *ok, double *post, double *margin);

/* SIC over K rows: row k is decoded by or_bp_prior from S^(k); then
 * S^(k+1)_{l,a} = S^(k)_{l,a} + cancel_log at a = hat_k[l] (every other entry
 * unchanged), S^(0) = S.  hat [F*K*n], iters [F*K], ok [F*K], margin
 * [F*K*n] (NULL = not wanted). */
void or_sic_decode(const or_code *code, int K, double cancel_log, int F, const double *S,
                   const or_opts *o, uint8_t *hat, int32_t *iters, uint8_t *ok, double *margin);

#ifdef __cplusplus
}
#endif
#endif
