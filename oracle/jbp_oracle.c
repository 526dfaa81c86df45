/*
 * jbp_oracle.c -- FP64 CPU oracle for joint FFT-BP decoding (test infrastructure).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the CUDA library.  It shares no
 * code with the CUDA path.  Every function below is the plain statement of the
 * quantity it computes, in double precision, with no blocking or fusion.
 *
 * Sources:
 *  - GF(Q) symbols and parity checks: appendix "Q-ary LDPC code", paragraphs
 *    on the bijection phi : [Q] -> F_Q and eqs. (app_ldpc_code_def),
 *    (app_ldpc_check_eq).  The bijection is "index bits = polynomial
 *    coefficients" over a fixed primitive polynomial (or_gf_poly).
 *  - Variable-to-check rule: eq. (app_ldpc_v2c).
 *  - Check-to-variable rule: eq. (app_ldpc_c2v) (OR_CHECK_LITERAL), the same
 *    sum as XOR convolutions of the coefficient-permuted messages
 *    (OR_CHECK_DIRECT, appendix "Complexity derivation", paragraph SIC-BP),
 *    and in the Walsh-Hadamard domain (OR_CHECK_WHT, paragraph FFT-BP).
 *  - Marginal and hard decision: eq. (app_ldpc_marginal).
 *  - Early exit on convergence and the 50-iteration cap: Table 1 caption.
 *  - Channel factor: the paper's local belief lambda_l(a) (eq.
 *    app_ldpc_local_belief_from_S) is replaced by the extrinsic message of a
 *    K-user PAM-sum channel node, y_t = sum_k (2 a_k - (Q-1)) + N(0, sigma2).
 *    This factor is this library's channel model, not the paper's; its
 *    extrinsic is the plain marginalisation of the Gaussian likelihood over
 *    the other users' symbols, computed here by a sum trellis in log space and
 *    checked against direct enumeration (or_channel_node_brute).
 *
 * Parity pins (tests/test_oracle_*.py): field axioms and known products;
 * trellis == enumeration; WHT == direct == literal check node; BP marginals ==
 * brute-force marginals on cycle-free joint graphs; K = 1 reduces to
 * single-user Q-ary sum-product; noiseless frames decode; user-permutation
 * equivariance; every early-stopped frame has a zero syndrome.
 */
#include "jbp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* GF(2^m)                                                                  */
/* ------------------------------------------------------------------------ */

int or_gf_poly(int m)
{
    /* primitive polynomials, bit i = coefficient of x^i */
    static const int poly[9] = {0, 0x3, 0x7, 0xB, 0x13, 0x25, 0x43, 0x89, 0x11D};
    return (m >= 1 && m <= 8) ? poly[m] : 0;
}

/* Product of two polynomials over GF(2), reduced modulo the primitive
 * polynomial (shift-and-add, the definition of multiplication in GF(2^m)). */
int or_gf_mul(int m, int a, int b)
{
    int poly = or_gf_poly(m), r = 0;
    while (b) {
        if (b & 1) r ^= a;
        b >>= 1;
        a <<= 1;
        if (a & (1 << m)) a ^= poly;
    }
    return r;
}

typedef struct {
    int m, Q;
    int *mul;  /* [Q*Q] */
    int *inv;  /* [Q]   */
} gf_t;

static void gf_make(gf_t *g, int m)
{
    g->m = m;
    g->Q = 1 << m;
    g->mul = (int *)malloc(sizeof(int) * g->Q * g->Q);
    g->inv = (int *)calloc(g->Q, sizeof(int));
    for (int a = 0; a < g->Q; ++a)
        for (int b = 0; b < g->Q; ++b) {
            g->mul[a * g->Q + b] = or_gf_mul(m, a, b);
            if (g->mul[a * g->Q + b] == 1) g->inv[a] = b;
        }
}

static void gf_free(gf_t *g)
{
    free(g->mul);
    free(g->inv);
}

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */

/* log(exp(a) + exp(b)) */
static double lse2(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double hi = a > b ? a : b, lo = a > b ? b : a;
    return hi + log1p(exp(lo - hi));
}

/* shift a log vector so that its maximum is 0, then clip at log_floor */
static void normalise_log(double *v, int Q, double log_floor)
{
    double mx = -INFINITY;
    for (int a = 0; a < Q; ++a) mx = v[a] > mx ? v[a] : mx;
    for (int a = 0; a < Q; ++a) {
        double x = v[a] - mx;
        v[a] = x < log_floor ? log_floor : x;
    }
}

static int parity_sign(int x, int w)
{
    return (__builtin_popcount((unsigned)(x & w)) & 1) ? -1 : 1;
}

/* ------------------------------------------------------------------------ */
/* Channel node                                                             */
/* ------------------------------------------------------------------------ */

/* log N(y; sum of levels, sigma2) up to a constant, as a function of the
 * integer symbol sum v = sum_k a_k: the levels sum to 2v - K(Q-1). */
static double log_gauss(double y, int v, int K, int Q, double sigma2)
{
    double d = y - (double)(2 * v - K * (Q - 1));
    return -d * d / (2.0 * sigma2);
}

void or_channel_node(int K, int m, double sigma2, double y, const double *logmu,
                     double log_floor, double *out)
{
    const int Q = 1 << m, D = Q - 1, S = K * D, W = S + 1;
    /* Fk[k*W + s]: log-distribution of the symbol sum of users 0..k-1 (s <= kD).
     * Bk[k*W + v]: log of sum over users k..K-1 of the Gaussian likelihood
     * times their messages, given that users 0..k-1 sum to v (v <= kD). */
    double *Fk = (double *)malloc(sizeof(double) * K * W);
    double *Bk = (double *)malloc(sizeof(double) * (K + 1) * W);
    for (int i = 0; i < K * W; ++i) Fk[i] = -INFINITY;
    for (int i = 0; i < (K + 1) * W; ++i) Bk[i] = -INFINITY;

    Fk[0] = 0.0; /* F_0 = delta at sum 0 */
    for (int k = 0; k + 1 < K; ++k)
        for (int s = 0; s <= (k + 1) * D; ++s) {
            double acc = -INFINITY;
            for (int b = 0; b < Q; ++b) {
                int s0 = s - b;
                if (s0 < 0 || s0 > k * D) continue;
                acc = lse2(acc, Fk[k * W + s0] + logmu[k * Q + b]);
            }
            Fk[(k + 1) * W + s] = acc;
        }

    for (int v = 0; v <= S; ++v) Bk[K * W + v] = log_gauss(y, v, K, Q, sigma2);
    for (int k = K - 1; k >= 0; --k)
        for (int v = 0; v <= k * D; ++v) {
            double acc = -INFINITY;
            for (int b = 0; b < Q; ++b) acc = lse2(acc, logmu[k * Q + b] + Bk[(k + 1) * W + v + b]);
            Bk[k * W + v] = acc;
        }

    /* extrinsic for user k: combine the others below (F_k) and above (B_{k+1}) */
    for (int k = 0; k < K; ++k) {
        for (int a = 0; a < Q; ++a) {
            double acc = -INFINITY;
            for (int s = 0; s <= k * D; ++s) acc = lse2(acc, Fk[k * W + s] + Bk[(k + 1) * W + s + a]);
            out[k * Q + a] = acc;
        }
        normalise_log(out + k * Q, Q, log_floor);
    }
    free(Fk);
    free(Bk);
}

void or_channel_node_brute(int K, int m, double sigma2, double y, const double *logmu,
                           double log_floor, double *out)
{
    const int Q = 1 << m;
    long combos = 1;
    for (int k = 1; k < K; ++k) combos *= Q;
    int *a = (int *)malloc(sizeof(int) * K);
    for (int k = 0; k < K; ++k) {
        for (int ak = 0; ak < Q; ++ak) {
            double acc = -INFINITY;
            for (long c = 0; c < combos; ++c) {
                long r = c;
                for (int j = 0; j < K; ++j) {
                    if (j == k) { a[j] = ak; continue; }
                    a[j] = (int)(r % Q);
                    r /= Q;
                }
                int v = 0;
                double lp = 0.0;
                for (int j = 0; j < K; ++j) {
                    v += a[j];
                    if (j != k) lp += logmu[j * Q + a[j]];
                }
                acc = lse2(acc, lp + log_gauss(y, v, K, Q, sigma2));
            }
            out[k * Q + ak] = acc;
        }
        normalise_log(out + k * Q, Q, log_floor);
    }
    free(a);
}

/* ------------------------------------------------------------------------ */
/* Check node                                                               */
/* ------------------------------------------------------------------------ */

static void check_node_g(const gf_t *g, int dc, const int *coef, const double *logv2c,
                         int method, double rel_floor, double *out)
{
    const int Q = g->Q;
    double *p = (double *)malloc(sizeof(double) * dc * Q);   /* linear v2c          */
    double *pt = (double *)malloc(sizeof(double) * dc * Q);  /* permuted: x = h*b   */
    double *Wp = (double *)malloc(sizeof(double) * dc * Q);  /* WHT of pt           */
    double *conv = (double *)malloc(sizeof(double) * Q);
    double *tmp = (double *)malloc(sizeof(double) * Q);
    double *r = (double *)malloc(sizeof(double) * Q);
    int *asg = (int *)malloc(sizeof(int) * dc);

    for (int d = 0; d < dc; ++d)
        for (int b = 0; b < Q; ++b) {
            p[d * Q + b] = exp(logv2c[d * Q + b]);
            /* the edge carries x = H_{j,l} * a; its distribution is p(a) at x */
            pt[d * Q + g->mul[coef[d] * Q + b]] = p[d * Q + b];
        }

    if (method == OR_CHECK_WHT)
        for (int d = 0; d < dc; ++d)
            for (int w = 0; w < Q; ++w) {
                double acc = 0.0;
                for (int x = 0; x < Q; ++x) acc += pt[d * Q + x] * parity_sign(x, w);
                Wp[d * Q + w] = acc;
            }

    for (int d = 0; d < dc; ++d) {
        const int h = coef[d];
        if (method == OR_CHECK_WHT) {
            /* pointwise product of the other edges' transforms, inverse transform */
            for (int w = 0; w < Q; ++w) {
                double prod = 1.0;
                for (int e = 0; e < dc; ++e)
                    if (e != d) prod *= Wp[e * Q + w];
                tmp[w] = prod;
            }
            for (int x = 0; x < Q; ++x) {
                double acc = 0.0;
                for (int w = 0; w < Q; ++w) acc += tmp[w] * parity_sign(x, w);
                conv[x] = acc / Q;
            }
            for (int a = 0; a < Q; ++a) r[a] = conv[g->mul[h * Q + a]];
        } else if (method == OR_CHECK_DIRECT) {
            /* XOR convolution of the other edges' permuted distributions */
            for (int x = 0; x < Q; ++x) conv[x] = (x == 0) ? 1.0 : 0.0;
            for (int e = 0; e < dc; ++e) {
                if (e == d) continue;
                for (int x = 0; x < Q; ++x) {
                    double acc = 0.0;
                    for (int x1 = 0; x1 < Q; ++x1) acc += conv[x1] * pt[e * Q + (x ^ x1)];
                    tmp[x] = acc;
                }
                memcpy(conv, tmp, sizeof(double) * Q);
            }
            for (int a = 0; a < Q; ++a) r[a] = conv[g->mul[h * Q + a]];
        } else {
            /* eq. (app_ldpc_c2v): sum over assignments of the other neighbours that
             * satisfy H_{j,l} a + sum H_{j,l'} a_{l'} = 0 */
            for (int a = 0; a < Q; ++a) r[a] = 0.0;
            long combos = 1;
            for (int e = 1; e < dc; ++e) combos *= Q;
            for (long c = 0; c < combos; ++c) {
                long rem = c;
                int s = 0;
                double prod = 1.0;
                for (int e = 0; e < dc; ++e) {
                    if (e == d) continue;
                    asg[e] = (int)(rem % Q);
                    rem /= Q;
                    s ^= g->mul[coef[e] * Q + asg[e]];
                    prod *= p[e * Q + asg[e]];
                }
                /* characteristic 2: H a = s  <=>  a = H^{-1} s */
                int a = g->mul[g->inv[h] * Q + s];
                r[a] += prod;
            }
        }
        double mx = 0.0;
        for (int a = 0; a < Q; ++a) mx = r[a] > mx ? r[a] : mx;
        for (int a = 0; a < Q; ++a) {
            double v = r[a] < rel_floor * mx ? rel_floor * mx : r[a];
            out[d * Q + a] = (v > 0.0) ? log(v) - log(mx) : -INFINITY;
        }
    }
    free(p); free(pt); free(Wp); free(conv); free(tmp); free(r); free(asg);
}

void or_check_node(int m, int dc, const int *coef, const double *logv2c, int method,
                   double rel_floor, double *out)
{
    gf_t g;
    gf_make(&g, m);
    check_node_g(&g, dc, coef, logv2c, method, rel_floor, out);
    gf_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Whole-frame steps                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n, P, dc, E, Q, m;
    const int *chk_var, *chk_coef;
    int *var_ptr;   /* [n+1] CSR of the edges of each variable */
    int *var_edge;  /* [E]                                      */
} graph_t;

static void graph_make(graph_t *G, const or_code *c)
{
    G->n = c->n; G->P = c->P; G->dc = c->dc; G->E = c->P * c->dc;
    G->m = c->m; G->Q = 1 << c->m;
    G->chk_var = c->chk_var; G->chk_coef = c->chk_coef;
    G->var_ptr = (int *)calloc(G->n + 1, sizeof(int));
    G->var_edge = (int *)malloc(sizeof(int) * (G->E > 0 ? G->E : 1));
    for (int e = 0; e < G->E; ++e) G->var_ptr[c->chk_var[e] + 1]++;
    for (int i = 0; i < G->n; ++i) G->var_ptr[i + 1] += G->var_ptr[i];
    int *fill = (int *)calloc(G->n, sizeof(int));
    for (int e = 0; e < G->E; ++e) {
        int i = c->chk_var[e];
        G->var_edge[G->var_ptr[i] + fill[i]++] = e;
    }
    free(fill);
}

static void graph_free(graph_t *G)
{
    free(G->var_ptr);
    free(G->var_edge);
}

/* inverse interleavers: use_to_pos[k*n + t] = i with pi_k(i) = t */
static int *invert_perm(const or_chan *ch, int n)
{
    int *inv = (int *)malloc(sizeof(int) * ch->K * n);
    for (int k = 0; k < ch->K; ++k)
        for (int i = 0; i < n; ++i) {
            int t = ch->perm ? ch->perm[k * n + i] : i;
            inv[k * n + t] = i;
        }
    return inv;
}

/* channel step for one frame.  The message from variable l of user k into its
 * channel factor is eq. (app_ldpc_v2c) with the channel factor in place of
 * check j: the product of all incoming check messages. */
static void frame_channel(const graph_t *G, const or_chan *ch, const int *use_to_pos,
                          const float *y, const double *c2v, double log_floor, double *ch2v)
{
    const int K = ch->K, Q = G->Q, n = G->n, E = G->E;
    double *logmu = (double *)malloc(sizeof(double) * K * Q);
    double *out = (double *)malloc(sizeof(double) * K * Q);
    for (int t = 0; t < n; ++t) {
        for (int k = 0; k < K; ++k) {
            int i = use_to_pos[k * n + t];
            for (int a = 0; a < Q; ++a) {
                double s = 0.0;
                for (int q = G->var_ptr[i]; q < G->var_ptr[i + 1]; ++q)
                    s += c2v[((size_t)k * E + G->var_edge[q]) * Q + a];
                logmu[k * Q + a] = s;
            }
            normalise_log(logmu + k * Q, Q, -INFINITY);
        }
        or_channel_node(K, G->m, ch->sigma2, (double)y[t], logmu, log_floor, out);
        for (int k = 0; k < K; ++k) {
            int i = use_to_pos[k * n + t];
            memcpy(ch2v + ((size_t)k * n + i) * Q, out + k * Q, sizeof(double) * Q);
        }
    }
    free(logmu);
    free(out);
}

/* variable-to-check messages of one frame, eq. (app_ldpc_v2c) with the
 * channel message as the local belief: v2c_e = ch2v_l + sum of the c2v of the
 * other edges of variable l (max-normalised, not clipped) */
static void frame_v2c(const graph_t *G, int K, const double *ch2v, const double *c2v,
                      double *v2c)
{
    const int Q = G->Q, n = G->n, E = G->E;
    for (int k = 0; k < K; ++k)
        for (int e = 0; e < E; ++e) {
            int i = G->chk_var[e];
            double *o = v2c + ((size_t)k * E + e) * Q;
            for (int a = 0; a < Q; ++a) {
                double s = ch2v[((size_t)k * n + i) * Q + a];
                for (int q = G->var_ptr[i]; q < G->var_ptr[i + 1]; ++q)
                    if (G->var_edge[q] != e) s += c2v[((size_t)k * E + G->var_edge[q]) * Q + a];
                o[a] = s;
            }
            normalise_log(o, Q, -INFINITY);
        }
}

/* check-node update of every check of one frame from given v2c messages */
static void frame_check_v2c(const graph_t *G, const gf_t *g, int K, const double *v2c,
                            int method, double rel_floor, double *c2v_new)
{
    const int Q = G->Q, E = G->E, dc = G->dc;
    for (int k = 0; k < K; ++k)
        for (int j = 0; j < G->P; ++j)
            check_node_g(g, dc, G->chk_coef + j * dc, v2c + ((size_t)k * E + j * dc) * Q, method,
                         rel_floor, c2v_new + ((size_t)k * E + j * dc) * Q);
}

/* check step for one frame: v2c, then the check update */
static void frame_check(const graph_t *G, const gf_t *g, int K, const double *ch2v,
                        const double *c2v_old, int method, double rel_floor, double *c2v_new)
{
    const size_t sc = (size_t)K * G->E * G->Q;
    double *v2c = (double *)malloc(sizeof(double) * (sc ? sc : 1));
    frame_v2c(G, K, ch2v, c2v_old, v2c);
    frame_check_v2c(G, g, K, v2c, method, rel_floor, c2v_new);
    free(v2c);
}

/* marginal eq. (app_ldpc_marginal) and hard decision (ties -> lowest index) */
static void frame_var(const graph_t *G, int K, const double *ch2v, const double *c2v,
                      double *post, uint8_t *hat, double *margin)
{
    const int Q = G->Q, n = G->n, E = G->E;
    double *b = (double *)malloc(sizeof(double) * Q);
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < n; ++i) {
            for (int a = 0; a < Q; ++a) {
                double s = ch2v[((size_t)k * n + i) * Q + a];
                for (int q = G->var_ptr[i]; q < G->var_ptr[i + 1]; ++q)
                    s += c2v[((size_t)k * E + G->var_edge[q]) * Q + a];
                b[a] = s;
            }
            int best = 0;
            for (int a = 1; a < Q; ++a)
                if (b[a] > b[best]) best = a;
            normalise_log(b, Q, -INFINITY);
            if (hat) hat[(size_t)k * n + i] = (uint8_t)best;
            if (post) memcpy(post + ((size_t)k * n + i) * Q, b, sizeof(double) * Q);
            if (margin) {
                double z = 0.0, p1 = 0.0, p2 = 0.0;
                for (int a = 0; a < Q; ++a) z += exp(b[a]);
                for (int a = 0; a < Q; ++a) {
                    double pa = exp(b[a]) / z;
                    if (pa > p1) { p2 = p1; p1 = pa; }
                    else if (pa > p2) p2 = pa;
                }
                margin[(size_t)k * n + i] = p1 - p2;
            }
        }
    free(b);
}

/* eq. (app_ldpc_check_eq): ok[k] = 1 iff every check of user k is satisfied */
static void frame_syndrome(const graph_t *G, const gf_t *g, int K, const uint8_t *hat, uint8_t *ok)
{
    const int Q = G->Q, n = G->n, dc = G->dc;
    for (int k = 0; k < K; ++k) {
        int good = 1;
        for (int j = 0; j < G->P && good; ++j) {
            int s = 0;
            for (int d = 0; d < dc; ++d) {
                int e = j * dc + d;
                s ^= g->mul[G->chk_coef[e] * Q + hat[(size_t)k * n + G->chk_var[e]]];
            }
            good = (s == 0);
        }
        ok[k] = (uint8_t)good;
    }
}

static void set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

void or_step_channel(const or_code *code, const or_chan *ch, int F, const float *y,
                     const double *c2v, double log_floor, double *ch2v)
{
    graph_t G;
    graph_make(&G, code);
    int *inv = invert_perm(ch, code->n);
    const size_t sc = (size_t)ch->K * G.E * G.Q, sv = (size_t)ch->K * G.n * G.Q;
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f)
        frame_channel(&G, ch, inv, y + (size_t)f * G.n, c2v + f * sc, log_floor, ch2v + f * sv);
    free(inv);
    graph_free(&G);
}

void or_step_check(const or_code *code, int K, int F, const double *ch2v,
                   const double *c2v_old, int method, double rel_floor, double *c2v_new)
{
    graph_t G;
    gf_t g;
    graph_make(&G, code);
    gf_make(&g, code->m);
    const size_t sc = (size_t)K * G.E * G.Q, sv = (size_t)K * G.n * G.Q;
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f)
        frame_check(&G, &g, K, ch2v + f * sv, c2v_old + f * sc, method, rel_floor, c2v_new + f * sc);
    gf_free(&g);
    graph_free(&G);
}

void or_step_v2c(const or_code *code, int K, int F, const double *ch2v, const double *c2v,
                 double *v2c)
{
    graph_t G;
    graph_make(&G, code);
    const size_t sc = (size_t)K * G.E * G.Q, sv = (size_t)K * G.n * G.Q;
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f) frame_v2c(&G, K, ch2v + f * sv, c2v + f * sc, v2c + f * sc);
    graph_free(&G);
}

void or_step_check_v2c(const or_code *code, int K, int F, const double *v2c, int method,
                       double rel_floor, double *c2v_new)
{
    graph_t G;
    gf_t g;
    graph_make(&G, code);
    gf_make(&g, code->m);
    const size_t sc = (size_t)K * G.E * G.Q;
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f)
        frame_check_v2c(&G, &g, K, v2c + f * sc, method, rel_floor, c2v_new + f * sc);
    gf_free(&g);
    graph_free(&G);
}

void or_step_var(const or_code *code, int K, int F, const double *ch2v, const double *c2v,
                 double *post, uint8_t *hat)
{
    graph_t G;
    graph_make(&G, code);
    const size_t sc = (size_t)K * G.E * G.Q, sv = (size_t)K * G.n * G.Q;
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f)
        frame_var(&G, K, ch2v + f * sv, c2v + f * sc, post ? post + f * sv : NULL,
                  hat ? hat + (size_t)f * K * G.n : NULL, NULL);
    graph_free(&G);
}

void or_syndrome(const or_code *code, int K, int F, const uint8_t *hat, uint8_t *ok)
{
    graph_t G;
    gf_t g;
    graph_make(&G, code);
    gf_make(&g, code->m);
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f)
        frame_syndrome(&G, &g, K, hat + (size_t)f * K * G.n, ok + (size_t)f * K);
    gf_free(&g);
    graph_free(&G);
}

/* ------------------------------------------------------------------------ */
/* Full decode: flooding schedule, per iteration channel -> check -> var    */
/* ------------------------------------------------------------------------ */

void or_decode(const or_code *code, const or_chan *ch, int F, const float *y,
               const or_opts *o, uint8_t *hat, int32_t *iters, uint8_t *ok,
               double *post, double *margin, double *ch2v_out, double *c2v_out)
{
    graph_t G;
    gf_t g;
    graph_make(&G, code);
    gf_make(&g, code->m);
    int *inv = invert_perm(ch, code->n);
    const int K = ch->K;
    const size_t sc = (size_t)K * G.E * G.Q, sv = (size_t)K * G.n * G.Q, sh = (size_t)K * G.n;
    set_threads(o->threads);

#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f) {
        double *c2v_old = (double *)calloc(sc ? sc : 1, sizeof(double)); /* uniform: log 1 */
        double *c2v_new = (double *)calloc(sc ? sc : 1, sizeof(double));
        double *ch2v = (double *)malloc(sizeof(double) * (sv ? sv : 1));
        double *pst = (double *)malloc(sizeof(double) * (sv ? sv : 1));
        double *mrg = (double *)malloc(sizeof(double) * (sh ? sh : 1));
        uint8_t *h = (uint8_t *)malloc(sh ? sh : 1);
        uint8_t *okf = (uint8_t *)malloc(K);
        int t_run = 0;
        for (int t = 1; t <= o->iters; ++t) {
            frame_channel(&G, ch, inv, y + (size_t)f * G.n, c2v_old, o->log_floor, ch2v);
            frame_check(&G, &g, K, ch2v, c2v_old, o->check_method, o->rel_floor, c2v_new);
            double *sw = c2v_old; c2v_old = c2v_new; c2v_new = sw;
            frame_var(&G, K, ch2v, c2v_old, pst, h, mrg);
            frame_syndrome(&G, &g, K, h, okf);
            t_run = t;
            int all = 1;
            for (int k = 0; k < K; ++k) all &= okf[k];
            if (o->early_stop && all) break;
        }
        if (o->iters <= 0) { /* no iteration: decisions from nothing are undefined */
            memset(h, 0, sh); memset(okf, 0, K);
            for (size_t i = 0; i < sv; ++i) pst[i] = 0.0;
            for (size_t i = 0; i < sh; ++i) mrg[i] = 0.0;
        }
        if (hat) memcpy(hat + f * sh, h, sh);
        if (iters) iters[f] = t_run;
        if (ok) memcpy(ok + (size_t)f * K, okf, K);
        if (post) memcpy(post + f * sv, pst, sizeof(double) * sv);
        if (margin) memcpy(margin + f * sh, mrg, sizeof(double) * sh);
        if (ch2v_out && o->iters > 0) memcpy(ch2v_out + f * sv, ch2v, sizeof(double) * sv);
        if (c2v_out) memcpy(c2v_out + f * sc, c2v_old, sizeof(double) * sc);
        free(c2v_old); free(c2v_new); free(ch2v); free(pst); free(mrg); free(h); free(okf);
    }
    free(inv);
    gf_free(&g);
    graph_free(&G);
}

/* ------------------------------------------------------------------------ */
/* Exact marginals by enumeration (eq. app_ldpc_code_def for the codebook)  */
/* ------------------------------------------------------------------------ */

long or_brute_marginals(const or_code *code, const or_chan *ch, const float *y, double *out)
{
    const int n = code->n, Q = 1 << code->m, K = ch->K, dc = code->dc;
    double words = pow((double)Q, (double)n);
    if (words > (double)(1 << 20)) return -1;
    gf_t g;
    gf_make(&g, code->m);
    long W = (long)words, C = 0;
    int *cw = (int *)malloc(sizeof(int) * n * (W > 0 ? W : 1));
    int *word = (int *)malloc(sizeof(int) * (n ? n : 1));
    for (long w = 0; w < W; ++w) {
        long r = w;
        for (int i = 0; i < n; ++i) { word[i] = (int)(r % Q); r /= Q; }
        int good = 1;
        for (int j = 0; j < code->P && good; ++j) {
            int s = 0;
            for (int d = 0; d < dc; ++d) {
                int e = j * dc + d;
                s ^= g.mul[code->chk_coef[e] * Q + word[code->chk_var[e]]];
            }
            good = (s == 0);
        }
        if (good) memcpy(cw + (size_t)C++ * n, word, sizeof(int) * n);
    }
    double tuples = pow((double)C, (double)K);
    if (tuples > (double)(1 << 24)) { free(cw); free(word); gf_free(&g); return -1; }
    int *use_to_pos = invert_perm(ch, n);
    for (int i = 0; i < K * n * Q; ++i) out[i] = -INFINITY;
    int *pick = (int *)calloc(K, sizeof(int));
    for (long tix = 0; tix < (long)tuples; ++tix) {
        long r = tix;
        for (int k = 0; k < K; ++k) { pick[k] = (int)(r % C); r /= C; }
        double ll = 0.0;
        for (int t = 0; t < n; ++t) {
            int v = 0;
            for (int k = 0; k < K; ++k) v += cw[(size_t)pick[k] * n + use_to_pos[k * n + t]];
            ll += log_gauss((double)y[t], v, K, Q, ch->sigma2);
        }
        for (int k = 0; k < K; ++k)
            for (int i = 0; i < n; ++i) {
                double *slot = out + ((size_t)k * n + i) * Q + cw[(size_t)pick[k] * n + i];
                *slot = lse2(*slot, ll);
            }
    }
    for (int ki = 0; ki < K * n; ++ki) normalise_log(out + (size_t)ki * Q, Q, -INFINITY);
    free(pick); free(use_to_pos); free(cw); free(word);
    gf_free(&g);
    return C;
}

/* ------------------------------------------------------------------------ */
/* Evidence interface: Bernoulli-Gaussian denoiser, slot AMP, SIC FFT-BP    */
/* ------------------------------------------------------------------------ */

static const double OR_PI = 3.14159265358979323846;

/* log of the circular complex Gaussian density phi(r; 0, v) at |r|^2 = s */
static double log_cn(double s, double v)
{
    return -s / v - log(OR_PI * v);
}

/* eq. (bg_activity_prob): rho phi1 / ((1-rho) phi0 + rho phi1), in logs */
double or_bg_log_activity(double s, double nu, double rho, double su2)
{
    double a1 = log(rho) + log_cn(s, nu + su2);
    double a0 = log(1.0 - rho) + log_cn(s, nu);
    double mx = a0 > a1 ? a0 : a1;
    return a1 - (mx + log(exp(a0 - mx) + exp(a1 - mx)));
}

/* eq. (bg_mmse_mean): eta = p^ * su2 / (nu + su2) * r */
double or_bg_gain(double s, double nu, double rho, double su2)
{
    return exp(or_bg_log_activity(s, nu, rho, su2)) * su2 / (nu + su2);
}

/* eta(r) = g(s) r with s = r conj(r): d eta / d r = g(s) + s g'(s); with
 * log p^ = a1 - log(exp(a0) + exp(a1)), d p^/ds = p^ (1 - p^) (1/nu - 1/(nu+su2)) */
double or_bg_deriv(double s, double nu, double rho, double su2)
{
    double p = exp(or_bg_log_activity(s, nu, rho, su2));
    double c = su2 / (nu + su2);
    double dp = p * (1.0 - p) * (1.0 / nu - 1.0 / (nu + su2));
    return c * (p + s * dp);
}

void or_amp_dict(int Q, int ns, const double *Ar, const double *Ai, const float *y, int iters,
                 double rho, double su2, double *S, double *R_out, double *nu_out)
{
    double *Ur = (double *)calloc(Q, sizeof(double)), *Ui = (double *)calloc(Q, sizeof(double));
    double *Rr = (double *)malloc(sizeof(double) * Q), *Ri = (double *)malloc(sizeof(double) * Q);
    double *Tr = (double *)malloc(sizeof(double) * ns), *Ti = (double *)malloc(sizeof(double) * ns);
    double *Nr = (double *)malloc(sizeof(double) * ns), *Ni = (double *)malloc(sizeof(double) * ns);
    for (int i = 0; i < ns; ++i) { Tr[i] = y[2 * i]; Ti[i] = y[2 * i + 1]; }
    double nu = 0.0;
    for (int it = 0; it <= iters; ++it) {
        /* nu^(i) = |Ytilde^(i)|^2 / ns */
        nu = 0.0;
        for (int i = 0; i < ns; ++i) nu += Tr[i] * Tr[i] + Ti[i] * Ti[i];
        nu /= ns;
        /* eq. (amp_iter_r): R = U + A^H Ytilde */
        for (int a = 0; a < Q; ++a) {
            double sr = Ur[a], si = Ui[a];
            for (int i = 0; i < ns; ++i) {
                /* conj(A) * T */
                sr += Ar[i * Q + a] * Tr[i] + Ai[i * Q + a] * Ti[i];
                si += Ar[i * Q + a] * Ti[i] - Ai[i * Q + a] * Tr[i];
            }
            Rr[a] = sr;
            Ri[a] = si;
        }
        if (it == iters) break;
        /* eq. (amp_iter_u): U = eta(R; nu), and the Onsager sum of eta' */
        double dsum = 0.0;
        for (int a = 0; a < Q; ++a) {
            double s = Rr[a] * Rr[a] + Ri[a] * Ri[a];
            double gn = or_bg_gain(s, nu, rho, su2);
            Ur[a] = gn * Rr[a];
            Ui[a] = gn * Ri[a];
            dsum += or_bg_deriv(s, nu, rho, su2);
        }
        /* eq. (amp_iter_res): Ytilde' = Y - A U + Ytilde / ns * sum eta' */
        for (int i = 0; i < ns; ++i) {
            double sr = y[2 * i], si = y[2 * i + 1];
            for (int a = 0; a < Q; ++a) {
                sr -= Ar[i * Q + a] * Ur[a] - Ai[i * Q + a] * Ui[a];
                si -= Ar[i * Q + a] * Ui[a] + Ai[i * Q + a] * Ur[a];
            }
            Nr[i] = sr + Tr[i] * dsum / ns;
            Ni[i] = si + Ti[i] * dsum / ns;
        }
        memcpy(Tr, Nr, sizeof(double) * ns);
        memcpy(Ti, Ni, sizeof(double) * ns);
    }
    /* evidence interface: S = log p^(R^(I); nu^(I)) */
    for (int a = 0; a < Q; ++a) S[a] = or_bg_log_activity(Rr[a] * Rr[a] + Ri[a] * Ri[a], nu, rho, su2);
    if (R_out)
        for (int a = 0; a < Q; ++a) { R_out[2 * a] = Rr[a]; R_out[2 * a + 1] = Ri[a]; }
    if (nu_out) *nu_out = nu;
    free(Ur); free(Ui); free(Rr); free(Ri);
    free(Tr); free(Ti); free(Nr); free(Ni);
}

void or_amp_slot(int Q, int ns, const int *rows, const float *y, int iters, double rho,
                 double su2, double *S, double *R_out, double *nu_out)
{
    /* A[i][a] = exp(-2 pi i rows[i] a / Q) / sqrt(ns), real and imaginary parts */
    double *Ar = (double *)malloc(sizeof(double) * ns * Q);
    double *Ai = (double *)malloc(sizeof(double) * ns * Q);
    const double scale = 1.0 / sqrt((double)ns);
    for (int i = 0; i < ns; ++i)
        for (int a = 0; a < Q; ++a) {
            long ka = ((long)rows[i] * a) % Q;
            double ang = -2.0 * OR_PI * (double)ka / (double)Q;
            Ar[i * Q + a] = cos(ang) * scale;
            Ai[i * Q + a] = sin(ang) * scale;
        }
    or_amp_dict(Q, ns, Ar, Ai, y, iters, rho, su2, S, R_out, nu_out);
    free(Ar); free(Ai);
}

void or_amp_evidence(int Q, int ns, int L, const int *rows, int F, const float *y, int iters,
                     double rho, double su2, double *S, int threads)
{
    set_threads(threads);
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f)
        for (int l = 0; l < L; ++l)
            or_amp_slot(Q, ns, rows + (size_t)l * ns, y + ((size_t)f * L + l) * ns * 2, iters, rho, su2,
                        S + ((size_t)f * L + l) * Q, NULL, NULL);
}

/* One row: the local beliefs are the channel messages of a K = 1 decode, held
 * fixed; each iteration is check (v2c then the WHT check update), marginal,
 * decision, syndrome. */
static void frame_bp_prior(const graph_t *G, const gf_t *g, const double *S, const or_opts *o,
                           uint8_t *hat, int32_t *iters, uint8_t *ok, double *post, double *margin)
{
    const int Q = G->Q, n = G->n;
    const size_t sc = (size_t)G->E * Q, sv = (size_t)n * Q;
    double *lam = (double *)malloc(sizeof(double) * (sv ? sv : 1));
    double *c2v_old = (double *)calloc(sc ? sc : 1, sizeof(double));
    double *c2v_new = (double *)calloc(sc ? sc : 1, sizeof(double));
    double *pst = (double *)calloc(sv ? sv : 1, sizeof(double));
    double *mrg = (double *)calloc(n ? n : 1, sizeof(double));
    uint8_t *h = (uint8_t *)calloc(n ? n : 1, 1);
    uint8_t okf = 0;
    memcpy(lam, S, sizeof(double) * sv);
    for (int i = 0; i < n; ++i) normalise_log(lam + (size_t)i * Q, Q, o->log_floor);
    int t_run = 0;
    for (int t = 1; t <= o->iters; ++t) {
        frame_check(G, g, 1, lam, c2v_old, o->check_method, o->rel_floor, c2v_new);
        double *sw = c2v_old; c2v_old = c2v_new; c2v_new = sw;
        frame_var(G, 1, lam, c2v_old, pst, h, mrg);
        frame_syndrome(G, g, 1, h, &okf);
        t_run = t;
        if (o->early_stop && okf) break;
    }
    if (hat) memcpy(hat, h, n);
    if (iters) *iters = t_run;
    if (ok) *ok = okf;
    if (post) memcpy(post, pst, sizeof(double) * sv);
    if (margin) memcpy(margin, mrg, sizeof(double) * n);
    free(lam); free(c2v_old); free(c2v_new); free(pst); free(mrg); free(h);
}

void or_bp_prior(const or_code *code, int F, const double *S, const or_opts *o, uint8_t *hat,
                 int32_t *iters, uint8_t *ok, double *post, double *margin)
{
    graph_t G;
    gf_t g;
    graph_make(&G, code);
    gf_make(&g, code->m);
    const size_t sv = (size_t)G.n * G.Q;
    set_threads(o->threads);
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f)
        frame_bp_prior(&G, &g, S + f * sv, o, hat ? hat + (size_t)f * G.n : NULL, iters ? iters + f : NULL,
                       ok ? ok + f : NULL, post ? post + f * sv : NULL, margin ? margin + (size_t)f * G.n : NULL);
    gf_free(&g);
    graph_free(&G);
}

void or_sic_decode(const or_code *code, int K, double cancel_log, int F, const double *S,
                   const or_opts *o, uint8_t *hat, int32_t *iters, uint8_t *ok, double *margin)
{
    graph_t G;
    gf_t g;
    graph_make(&G, code);
    gf_make(&g, code->m);
    const int n = G.n, Q = G.Q;
    const size_t sv = (size_t)n * Q;
    set_threads(o->threads);
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f) {
        double *Sk = (double *)malloc(sizeof(double) * (sv ? sv : 1));
        uint8_t *h = (uint8_t *)calloc(n ? n : 1, 1);
        memcpy(Sk, S + f * sv, sizeof(double) * sv);
        for (int k = 0; k < K; ++k) {
            const size_t r = (size_t)f * K + k;
            int32_t it = 0;
            uint8_t okk = 0;
            frame_bp_prior(&G, &g, Sk, o, h, &it, &okk, NULL, margin ? margin + r * n : NULL);
            if (hat) memcpy(hat + r * n, h, n);
            if (iters) iters[r] = it;
            if (ok) ok[r] = okk;
            /* cancel the decoded row's evidence before the next row */
            for (int i = 0; i < n; ++i) Sk[(size_t)i * Q + h[i]] += cancel_log;
        }
        free(Sk);
        free(h);
    }
    gf_free(&g);
    graph_free(&G);
}
