// jbp_device.cuh -- per-node device routines of joint FFT belief propagation.
//
// Message format: every stored message is an FP32 probability vector over the q
// symbols scaled so that its largest entry is 1 (the log-message of the decoder
// is its natural log).  A c2v message is floored at kRelFloor of its maximum
// (after the inverse transform); a channel message is floored at kRelFloor.
// Storing probabilities rather than logs keeps the hot loops free of exp/log;
// the relative precision of a stored entry is 2^-24 at every magnitude.
//
// Message block of one (frame, user): the check-major edges e = 4j + d, edge e
// at blk + j*cbs + d*q (cbs = 4q in HBM, 4q + 4 in shared memory to spread
// banks).  Channel messages: ch2v[(k*n + i)*q + a], dense.
//
// Two execution shapes per node type:
//   thread: one thread owns a unit (channel use, check of one user, variable of
//           one user) with all its q-vectors in registers (q <= 16);
//   team:   T = min(q, 32) lanes of one warp own a unit, lane tl holding
//           symbols a = v*T + tl (q = 32, 64, and the channel for K > 4).
// Teams synchronise only their own lanes (team masks), so teams may diverge.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jbp {

constexpr float kRelFloor = 1e-12f;
// linear channel output whose maximum is below this: redo in log space.  At
// 1e-24 every entry down to the 1e-12 floor (relative to the maximum) is still a
// normal FP32 number, so no entry the floor keeps is lost to underflow.
constexpr float kFallbackMax = 1e-24f;
constexpr int kMaxDv = 8;
constexpr int kMaxK = 16;
constexpr int kDC = 4;                   // check degree of the kernels
constexpr float kNegInf = -__builtin_inff();

// Device view of one decoder: code, interleavers, channel and GF tables.
struct Graph {
    int n, P, E, dc, dv, K, Q;
    float inv_sigma2;         // 1 / noise variance of every frame, unless sigma2_f is set
    const int32_t* chk_var;   // [E]     variable of check-major edge e
    const uint8_t* chk_coef;  // [E]     H_{j,l} of edge e
    const int32_t* var_edge;  // [n*dv]  edges of variable i, ascending
    const int32_t* use_pos;   // [K*n]   use_pos[k*n+t] = pi_k^{-1}(t)
    const uint8_t* gf_mul;    // [Q*Q]   gf_mul[h*Q+x] = h*x
    const uint8_t* gf_div;    // [Q*Q]   gf_div[h*Q+x] = h^{-1}*x
    unsigned long long* log_fallbacks;   // counts channel messages redone in log space (may be null)
    const int32_t* pos_of;    // [K*n]   pos_of[k*n+i] = pi_k(i)                 (fused layout)
    const uint16_t* slot;     // [K*E]   pi_k(var of e)*2 + (e's rank in its var) (fused layout)
    int* tc_error;            // set to 1 if a tensor-core wait expired (may be null: FP32 only)
    const float* sigma2_f;    // [F]     per-frame noise variance of this batch (may be null)
    const uint16_t* chk_order;  // [K*P] order of the check units in the fused check phase (may be null)
    const unsigned char* dft_tab = nullptr;   // DFT tables of the tensor-core channel node (null: trellis)
    int var_reg = 1;          // 1: every variable has exactly dv edges; 0: var_edge rows end early with -1
};

// Edges of variable i: g.dv when the code is variable-regular, else the entries
// of its var_edge row before the first -1 (rows are padded to the largest degree).
__device__ __forceinline__ int var_degree(const Graph& g, int i)
{
    if (g.var_reg) return g.dv;
    int d = 0;
    while (d < g.dv && g.var_edge[i * g.dv + d] >= 0) ++d;
    return d;
}

// 1 / sigma2 of frame f
__device__ __forceinline__ float frame_inv_s2(const Graph& g, long f)
{
    return g.sigma2_f ? __frcp_rn(g.sigma2_f[f]) : g.inv_sigma2;
}

__device__ __forceinline__ float* edge_ptr(float* blk, int e, int cbs, int Q)
{
    return blk + (e >> 2) * cbs + (e & 3) * Q;
}
__device__ __forceinline__ const float* edge_ptr(const float* blk, int e, int cbs, int Q)
{
    return blk + (e >> 2) * cbs + (e & 3) * Q;
}

template <int Q>
struct Shape {
    static_assert(Q >= 2 && Q <= 64 && (Q & (Q - 1)) == 0, "q must be 2..64, a power of two");
    static constexpr int T = Q < 32 ? Q : 32;
    static constexpr int V = Q / T;
    static constexpr int LOGT = T == 2 ? 1 : T == 4 ? 2 : T == 8 ? 3 : T == 16 ? 4 : 5;
};

struct TeamLane {
    int tl;          // lane within the team
    unsigned mask;   // the team's lanes within the warp
};

template <int T>
__device__ __forceinline__ TeamLane team_lane()
{
    const int lane = threadIdx.x & 31;
    TeamLane L;
    L.tl = lane & (T - 1);
    L.mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(T - 1)));
    return L;
}

template <int T>
__device__ __forceinline__ float team_max(float v, unsigned mask)
{
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, T));
    return v;
}

// ---------------------------------------------------------------------------
// register vector helpers (thread shape)
// ---------------------------------------------------------------------------

template <int Q>
__device__ __forceinline__ void vload(const float* p, float (&v)[Q])
{
    if constexpr (Q % 4 == 0) {
#pragma unroll
        for (int i = 0; i < Q / 4; ++i) {
            const float4 t = reinterpret_cast<const float4*>(p)[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q / 2; ++i) {
            const float2 t = reinterpret_cast<const float2*>(p)[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    }
}

template <int Q>
__device__ __forceinline__ void vstore(float* p, const float (&v)[Q])
{
    if constexpr (Q % 4 == 0) {
#pragma unroll
        for (int i = 0; i < Q / 4; ++i)
            reinterpret_cast<float4*>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < Q / 2; ++i) reinterpret_cast<float2*>(p)[i] = make_float2(v[2 * i], v[2 * i + 1]);
    }
}

// max of three floats in one instruction (the maximum is one of the inputs, so
// the result equals fmaxf(fmaxf(a, b), c) bit for bit on non-NaN inputs)
__device__ __forceinline__ float fmax3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Largest entry, as a tree of three-input maxima (depth log3 N, not N - 1).
template <int N>
__device__ __forceinline__ float vmax(const float (&v)[N])
{
    if constexpr (N == 1) {
        return v[0];
    } else if constexpr (N == 2) {
        return fmaxf(v[0], v[1]);
    } else {
        constexpr int M = (N + 2) / 3;
        float t[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int a = 3 * i;
            if (a + 2 < N) t[i] = fmax3f(v[a], v[a + 1], v[a + 2]);
            else if (a + 1 < N) t[i] = fmaxf(v[a], v[a + 1]);
            else t[i] = v[a];
        }
        return vmax<M>(t);
    }
}

// Index of the largest entry, the lowest index among equal maxima (the rule of a
// scan that replaces its best only on a strictly larger value), as a tree: a
// node keeps its left (lower-index) child unless the right one is larger.
template <int LO, int HI, int N>
__device__ __forceinline__ void vargmax_rng(const float (&v)[N], float& bv, int& bi)
{
    if constexpr (HI - LO == 1) {
        bv = v[LO];
        bi = LO;
    } else {
        constexpr int MID = LO + (HI - LO + 1) / 2;
        float lv, rv;
        int li, ri;
        vargmax_rng<LO, MID, N>(v, lv, li);
        vargmax_rng<MID, HI, N>(v, rv, ri);
        const bool r = rv > lv;
        bv = r ? rv : lv;
        bi = r ? ri : li;
    }
}

template <int N>
__device__ __forceinline__ int vargmax(const float (&v)[N])
{
    float bv;
    int bi;
    vargmax_rng<0, N, N>(v, bv, bi);
    return bi;
}

// ---------------------------------------------------------------------------
// Channel node
// ---------------------------------------------------------------------------
//
// With a_k the symbol of user k and s = sum_k a_k, the likelihood of y is
// G(s) = exp(-(y - (2s - K(q-1)))^2 / (2 sigma2)), and the message to user k is
//   ch2v_k(a) ~ sum over the other users' symbols of G(a + sum_{j!=k} a_j) prod mu_j(a_j),
// a leave-one-out combination of the K incoming messages mu_j.  The exponent is
// taken relative to the nearest symbol sum s*: with r = y - (2s* - K(q-1)) and
// d = s* - s, -(y - L_s)^2/(2 sigma2) + (y - L_s*)^2/(2 sigma2) = -2 d (r + d)/sigma2,
// which keeps its relative accuracy for every entry that matters.

// 2^x by the special-function unit's approximation (PTX ex2.approx.ftz.f32;
// relative error about 2^-22, results below 2^-126 flushed to zero)
__device__ __forceinline__ float exp2_approx(float x)
{
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x));
    return e;
}

struct GaussTerm {
    int ss;          // nearest symbol sum s*
    float ssf;       // s* as a float (exact: a small integer)
    float r;         // y - (2 s* - K(q-1))
    float inv_s2;    // 1 / sigma2
    float k2;        // -2 log2(e) / sigma2
    float k2r;       // k2 r
    // the exponent (natural log) of the score of sum value s
    __device__ __forceinline__ float expo(int s) const
    {
        // d = s* - s is exact in FP32 (small integers), so subtracting floats
        // gives the value an integer subtraction and conversion would
        const float d = ssf - (float)s;
        return -2.0f * d * (r + d) * inv_s2;
    }
    // the score itself, exp(expo(s)) = 2^(d (k2 d + k2 r)): one addition, one
    // multiply-add, one product and one base-2 exponential
    __device__ __forceinline__ float score(int s) const
    {
        const float d = ssf - (float)s;
        return exp2_approx(d * fmaf(k2, d, k2r));
    }
};

__device__ __forceinline__ GaussTerm gauss_term(float y, int K, int Q, float inv_s2)
{
    const int KD = K * (Q - 1);
    float sf = rintf((y + (float)KD) * 0.5f);
    sf = fminf(fmaxf(sf, 0.0f), (float)KD);
    GaussTerm t;
    t.ss = (int)sf;
    t.ssf = sf;
    t.r = y - (float)(2 * t.ss - KD);
    t.inv_s2 = inv_s2;
    t.k2 = -2.0f * 1.4426950408889634f * inv_s2;
    t.k2r = t.k2 * t.r;
    return t;
}

// -- thread shape: K <= 4, q <= 16, every array in registers -----------------
//
// Leave-one-out without division by a balanced split of the users (for K = 4:
// {0,1} | {2,3}): with P23 = mu_2 (*) mu_3 (integer convolution) and the scored
// suffix H23(v) = sum_s P23(s) G(v + s), the messages to users 0 and 1 are
// sum_b mu_1(b) H23(a + b) and sum_b mu_0(b) H23(a + b); users 2 and 3 use the
// mirror quantities.  K = 3 uses the prefix F_2 = mu_0 (*) mu_1 and the suffix
// B_2(v) = sum_b mu_2(b) G(v + b).  G is streamed (one exp per sum value per pass).

template <int NA, int NB>
__device__ __forceinline__ void rconv(const float (&A)[NA], const float (&B)[NB], float (&C)[NA + NB - 1])
{
#pragma unroll
    for (int i = 0; i < NA + NB - 1; ++i) C[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int j = 0; j < NB; ++j) C[i + j] = fmaf(A[i], B[j], C[i + j]);
}

// H(v) = sum_s P(s) X(v + s), v in [0, NX - NP]
template <int NP, int NX>
__device__ __forceinline__ void rcorr(const float (&P)[NP], const float (&X)[NX], float (&H)[NX - NP + 1])
{
#pragma unroll
    for (int v = 0; v < NX - NP + 1; ++v) {
        float acc = 0.0f;
#pragma unroll
        for (int s = 0; s < NP; ++s) acc = fmaf(P[s], X[v + s], acc);
        H[v] = acc;
    }
}

// H1(v) = sum_s P1(s) G(v + s), H2 likewise, one pass over G(w), w in [0, W)
template <int NP1, int NH1, int NP2, int NH2>
__device__ __forceinline__ void rcorr_g2(const float (&P1)[NP1], float (&H1)[NH1], const float (&P2)[NP2],
                                        float (&H2)[NH2], const GaussTerm& gt)
{
    constexpr int W1 = NH1 + NP1 - 1, W2 = NH2 + NP2 - 1, W = W1 > W2 ? W1 : W2;
#pragma unroll
    for (int v = 0; v < NH1; ++v) H1[v] = 0.0f;
#pragma unroll
    for (int v = 0; v < NH2; ++v) H2[v] = 0.0f;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const float g = gt.score(w);
#pragma unroll
        for (int v = 0; v < NH1; ++v)
            if (w - v >= 0 && w - v < NP1) H1[v] = fmaf(P1[w - v], g, H1[v]);
#pragma unroll
        for (int v = 0; v < NH2; ++v)
            if (w - v >= 0 && w - v < NP2) H2[v] = fmaf(P2[w - v], g, H2[v]);
    }
}

template <int NP, int NH>
__device__ __forceinline__ void rcorr_g(const float (&P)[NP], float (&H)[NH], const GaussTerm& gt)
{
#pragma unroll
    for (int v = 0; v < NH; ++v) H[v] = 0.0f;
#pragma unroll
    for (int w = 0; w < NH + NP - 1; ++w) {
        const float g = gt.score(w);
#pragma unroll
        for (int v = 0; v < NH; ++v)
            if (w - v >= 0 && w - v < NP) H[v] = fmaf(P[w - v], g, H[v]);
    }
}

// Log-space recomputation of user k's message (rare: taken when the linear pass
// of that user underflows).  mu: the linear incoming messages (> 0 or 0).
template <int K, int Q>
__device__ __noinline__ void chan_user_log(const float (&mu)[K][Q], int k, const GaussTerm& gt, float (&out)[Q])
{
    constexpr int D = Q - 1, S = (K - 1) * D + 1;
    float F[S], Fn[S];
#pragma unroll 1
    for (int s = 0; s < S; ++s) F[s] = kNegInf;
    F[0] = 0.0f;
    int len = 1;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        if (j == k) continue;
#pragma unroll 1
        for (int s = 0; s < len + D; ++s) {
            float acc = kNegInf;
#pragma unroll 1
            for (int b = 0; b <= D; ++b) {
                if (s - b < 0 || s - b >= len) continue;
                const float t = F[s - b] + __logf(mu[j][b]);
                const float hi = fmaxf(acc, t), lo = fminf(acc, t);
                acc = (lo == kNegInf) ? hi : hi + log1pf(__expf(lo - hi));
            }
            Fn[s] = acc;
        }
        len += D;
#pragma unroll 1
        for (int s = 0; s < len; ++s) F[s] = Fn[s];
    }
    float mx = kNegInf;
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        float acc = kNegInf;
#pragma unroll 1
        for (int s = 0; s < len; ++s) {
            const float t = F[s] + gt.expo(s + a);
            const float hi = fmaxf(acc, t), lo = fminf(acc, t);
            acc = (lo == kNegInf) ? hi : hi + log1pf(__expf(lo - hi));
        }
        out[a] = acc;
        mx = fmaxf(mx, acc);
    }
#pragma unroll 1
    for (int a = 0; a < Q; ++a) out[a] = fmaxf(__expf(out[a] - mx), kRelFloor);
}

// Normalise a linear channel output to max 1 and floor it; rerun in log space
// if it underflowed.
template <int K, int Q>
__device__ __forceinline__ void chan_finish(const float (&mu)[K][Q], int k, const GaussTerm& gt, float (&o)[Q],
                                            unsigned long long* fallbacks)
{
    const float mx = vmax(o);
    if (!(mx >= kFallbackMax)) {
        if (fallbacks) atomicAdd(fallbacks, 1ull);
        chan_user_log<K, Q>(mu, k, gt, o);
        return;
    }
    const float inv = __frcp_rn(mx);
#pragma unroll
    for (int a = 0; a < Q; ++a) o[a] = fmaxf(o[a] * inv, kRelFloor);
}

// Extrinsic messages of one channel use; calls emit(k, out_k) per user as soon
// as its message is final (max 1, floored).
template <int K, int Q, class Emit>
__device__ __forceinline__ void chan_reg(const float (&mu)[K][Q], const GaussTerm& gt, unsigned long long* fb,
                                         Emit emit)
{
    constexpr int D = Q - 1;
    if constexpr (K == 1) {
        float o[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) o[a] = gt.score(a);
        chan_finish<K, Q>(mu, 0, gt, o, fb);
        emit(0, o);
    } else if constexpr (K == 2) {
        float o0[Q], o1[Q];
        rcorr_g2<Q, Q, Q, Q>(mu[1], o0, mu[0], o1, gt);
        chan_finish<K, Q>(mu, 0, gt, o0, fb);
        emit(0, o0);
        chan_finish<K, Q>(mu, 1, gt, o1, fb);
        emit(1, o1);
    } else if constexpr (K == 3) {
        float F2[2 * D + 1];
        rconv(mu[0], mu[1], F2);
        float o2[Q], B2[2 * D + 1];
        rcorr_g2<2 * D + 1, Q, Q, 2 * D + 1>(F2, o2, mu[2], B2, gt);
        chan_finish<K, Q>(mu, 2, gt, o2, fb);
        emit(2, o2);
        float o[Q];
        rcorr(mu[0], B2, o);
        chan_finish<K, Q>(mu, 1, gt, o, fb);
        emit(1, o);
        rcorr(mu[1], B2, o);
        chan_finish<K, Q>(mu, 0, gt, o, fb);
        emit(0, o);
    } else {
        static_assert(K == 4, "thread-shape channel node is built for K <= 4");
        float o[Q];
        {
            float P23[2 * D + 1], H23[2 * D + 1];
            rconv(mu[2], mu[3], P23);
            rcorr_g<2 * D + 1, 2 * D + 1>(P23, H23, gt);
            rcorr(mu[1], H23, o);
            chan_finish<K, Q>(mu, 0, gt, o, fb);
            emit(0, o);
            rcorr(mu[0], H23, o);
            chan_finish<K, Q>(mu, 1, gt, o, fb);
            emit(1, o);
        }
        {
            float P01[2 * D + 1], H01[2 * D + 1];
            rconv(mu[0], mu[1], P01);
            rcorr_g<2 * D + 1, 2 * D + 1>(P01, H01, gt);
            rcorr(mu[3], H01, o);
            chan_finish<K, Q>(mu, 2, gt, o, fb);
            emit(2, o);
            rcorr(mu[2], H01, o);
            chan_finish<K, Q>(mu, 3, gt, o, fb);
            emit(3, o);
        }
    }
}

// Outputs of the channel node for user k's variable i (variable degree 2): its
// channel message o (max 1, floored) into ch2v_f, and each of its two c2v
// messages in the user's message blocks blk replaced by the v2c message of the
// same edge (eq. app_ldpc_v2c with the channel message as the local belief:
// v2c_0 = ch2v * c2v_1, v2c_1 = ch2v * c2v_0, each rescaled to max 1).
template <int Q>
__device__ __forceinline__ void chan_store_user(const Graph& g, float* blk, int cbs, float* ch2v_f, int k, int i,
                                                const float (&o)[Q])
{
    vstore<Q>(ch2v_f + ((size_t)k * g.n + i) * Q, o);
    float* p0 = edge_ptr(blk, g.var_edge[2 * i], cbs, Q);
    float* p1 = edge_ptr(blk, g.var_edge[2 * i + 1], cbs, Q);
    float c0[Q], c1[Q];
    vload<Q>(p0, c0);
    vload<Q>(p1, c1);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const float t = c0[a];
        c0[a] = o[a] * c1[a];
        c1[a] = o[a] * t;
    }
    const float i0 = __frcp_rn(vmax(c0)), i1 = __frcp_rn(vmax(c1));
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        c0[a] *= i0;
        c1[a] *= i1;
    }
    vstore<Q>(p0, c0);
    vstore<Q>(p1, c1);
}

// One channel use u of one frame, thread shape (variable degree 2).  msg_f:
// the frame's message blocks (user k at msg_f + k*ustride); ch2v_f: the frame's
// channel messages.  Reads the c2v of the K variables on this use, writes their
// channel messages and replaces each of their two c2v by the v2c message of the
// same edge (chan_store_user).
template <int K, int Q>
__device__ __forceinline__ void chan_thread(const Graph& g, float* msg_f, size_t ustride, int cbs, float* ch2v_f,
                                            float y, float inv_s2, int u)
{
    float mu[K][Q];
    int var[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        var[k] = g.use_pos[k * g.n + u];
        const float* blk = msg_f + k * ustride;
        float a0[Q], a1[Q];
        vload<Q>(edge_ptr(blk, g.var_edge[2 * var[k]], cbs, Q), a0);
        vload<Q>(edge_ptr(blk, g.var_edge[2 * var[k] + 1], cbs, Q), a1);
#pragma unroll
        for (int a = 0; a < Q; ++a) a0[a] *= a1[a];
        const float inv = __frcp_rn(vmax(a0));
#pragma unroll
        for (int a = 0; a < Q; ++a) mu[k][a] = a0[a] * inv;
    }
    const GaussTerm gt = gauss_term(y, K, Q, inv_s2);
    chan_reg<K, Q>(mu, gt, g.log_fallbacks, [&](int k, const float (&o)[Q]) {
        chan_store_user<Q>(g, msg_f + k * ustride, cbs, ch2v_f, k, var[k], o);
    });
}

// -- team shape: any K <= 16, q <= 64 (linear trellis, log-space on underflow)

struct LinSR {
    static constexpr bool kLog = false;
    __device__ static __forceinline__ float zero() { return 0.0f; }
    __device__ static __forceinline__ float mac(float acc, float a, float b) { return fmaf(a, b, acc); }
    __device__ static __forceinline__ float rescale(float x, float mx) { return mx > 0.0f ? x * (__frcp_rn(mx)) : x; }
};

struct LogSR {
    static constexpr bool kLog = true;
    __device__ static __forceinline__ float zero() { return kNegInf; }
    __device__ static __forceinline__ float mac(float acc, float a, float b)
    {
        const float t = a + b;
        const float hi = fmaxf(acc, t), lo = fminf(acc, t);
        return (lo == kNegInf) ? hi : hi + log1pf(__expf(lo - hi));
    }
    __device__ static __forceinline__ float rescale(float x, float mx) { return x - mx; }
};

// Offset of the prefix array F_k (k >= 2) inside the prefix buffer; F_1 is mu_0.
__host__ __device__ __forceinline__ int prefix_offset(int k, int D)
{
    return k < 2 ? 0 : D * ((k - 1) * k / 2 - 1) + (k - 2);
}

// Floats of team scratch for one channel use: mu[K*Q] | prefixes | B0 | B1 | res[K*Q].
__host__ __device__ __forceinline__ int chan_scratch_floats(int K, int Q)
{
    const int D = Q - 1, S = K * D;
    return 2 * K * Q + prefix_offset(K, D) + 2 * (S + 1);
}

// Team-shape channel messages of use u: prefixes F_0 = delta_0, F_{j+1} = F_j (*) mu_j,
// scored suffixes B_K = G, B_j(v) = sum_b mu_j(b) B_{j+1}(v + b), messages
// ch2v_k(a) ~ sum_s F_k(s) B_{k+1}(s + a); every prefix and suffix rescaled to max 1.
// res [K*Q] receives the final messages (max 1, floored).  Returns true
// (team-uniform) if the linear pass underflowed; the caller reruns in LogSR.
template <int Q, class SR>
__device__ bool chan_trellis(const Graph& g, const float* msg_f, size_t ustride, int cbs, float y, float inv_s2,
                             int u, float* sc, float* res, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V, D = Q - 1;
    const int K = g.K, S = K * D;
    float* mu = sc;
    float* Fb = mu + K * Q;
    float* B = Fb + prefix_offset(K, D);
    float* Bn = B + S + 1;
    bool bad = false;

    for (int k = 0; k < K; ++k) {
        const int i = g.use_pos[k * g.n + u];
        const float* blk = msg_f + k * ustride;
        float l[V];
#pragma unroll
        for (int v = 0; v < V; ++v) l[v] = SR::kLog ? 0.0f : 1.0f;
        const int deg = var_degree(g, i);
        for (int d = 0; d < deg; ++d) {
            const float* m = edge_ptr(blk, g.var_edge[i * g.dv + d], cbs, Q);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float x = m[v * T + L.tl];
                l[v] = SR::kLog ? l[v] + __logf(x) : l[v] * x;
            }
        }
        float mx = l[0];
#pragma unroll
        for (int v = 1; v < V; ++v) mx = fmaxf(mx, l[v]);
        mx = team_max<T>(mx, L.mask);
#pragma unroll
        for (int v = 0; v < V; ++v) mu[k * Q + v * T + L.tl] = SR::rescale(l[v], mx);
    }

    const GaussTerm gt = gauss_term(y, K, Q, inv_s2);
    for (int s = L.tl; s <= S; s += T) B[s] = SR::kLog ? gt.expo(s) : gt.score(s);

    for (int j = 1; j + 1 < K; ++j) {
        __syncwarp(L.mask);
        const float* Fj = (j == 1) ? mu : Fb + prefix_offset(j, D);
        float* Fn = Fb + prefix_offset(j + 1, D);
        const int len = (j + 1) * D + 1, jD = j * D;
        float lmx = kNegInf;
        for (int s = L.tl; s < len; s += T) {
            const int b0 = s - jD > 0 ? s - jD : 0, b1 = s < D ? s : D;
            float acc = SR::zero();
            for (int b = b0; b <= b1; ++b) acc = SR::mac(acc, mu[j * Q + b], Fj[s - b]);
            Fn[s] = acc;
            lmx = fmaxf(lmx, acc);
        }
        const float mx = team_max<T>(lmx, L.mask);
        if (!SR::kLog && !(mx > 0.0f)) bad = true;
        for (int s = L.tl; s < len; s += T) Fn[s] = SR::rescale(Fn[s], mx);
    }

    for (int k = K - 1; k >= 0; --k) {
        __syncwarp(L.mask);
        const float* Fk = (k == 1) ? mu : Fb + prefix_offset(k, D);
        float o[V];
        float lmx = kNegInf;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int a = v * T + L.tl;
            if (k == 0) {
                o[v] = B[a];
            } else {
                float acc = SR::zero();
                const int kD = k * D;
                for (int s = 0; s <= kD; ++s) acc = SR::mac(acc, Fk[s], B[s + a]);
                o[v] = acc;
            }
            lmx = fmaxf(lmx, o[v]);
        }
        const float mx = team_max<T>(lmx, L.mask);
        if (!SR::kLog && !(mx >= kFallbackMax)) bad = true;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float r = SR::kLog ? __expf(o[v] - mx) : o[v] * (__frcp_rn(mx));
            res[k * Q + v * T + L.tl] = fmaxf(r, kRelFloor);
        }
        if (k > 0) {
            const int len = k * D + 1;
            float lm2 = kNegInf;
            for (int s = L.tl; s < len; s += T) {
                float acc = SR::zero();
#pragma unroll 4
                for (int b = 0; b <= D; ++b) acc = SR::mac(acc, mu[k * Q + b], B[s + b]);
                Bn[s] = acc;
                lm2 = fmaxf(lm2, acc);
            }
            const float m2 = team_max<T>(lm2, L.mask);
            if (!SR::kLog && !(m2 > 0.0f)) bad = true;
            for (int s = L.tl; s < len; s += T) Bn[s] = SR::rescale(Bn[s], m2);
            float* t = B;
            B = Bn;
            Bn = t;
        }
    }
    __syncwarp(L.mask);
    return bad;
}

// -- team shape, register-blocked linear trellis -----------------------------
//
// The three trellis operations are correlations Y(o) = sum_t A(t) X(o + t + xoff)
// (a prefix convolution is the correlation with the reversed message and
// xoff = -(q-1)).  A team computes one with each lane owning kBR consecutive
// outputs and, when there are fewer output blocks than lanes, a contiguous
// chunk of the taps; the chunks' partial sums are combined with shuffles.  A
// sliding window keeps the X values in registers, so a lane loads one X and
// one A per tap for kBR multiply-adds.  kBR is odd: lanes start kBR words
// apart, which maps the 32 lanes of a warp onto 32 distinct banks, and the tap
// chunk length is odd for the same reason.  X arrays carry zero pads (BlkPad)
// so that no load needs a bounds check.

constexpr int kBR = 9;

// outputs per lane for a field size: 9 at q = 64, 7 below (measured faster
// there); both odd, and both within the 48-float right pad (overrun <= 2 BR + 1)
template <int Q>
struct CorrBlock {
    static constexpr int BR = Q >= 64 ? 9 : 7;
};

template <int Q>
struct BlkPad {
    static constexpr int L = Q;            // left zero pad (prefix convolutions read X(s - (q-1)))
    static constexpr int R = Q + 48;       // right pad: convolution tails (zeros), block and window overrun
};

__host__ __device__ __forceinline__ int blk_pad(int Q) { return Q + Q + 48; }

// Y(o) for o < L at Y[o]; A(t) at A[t] (t < NT; AREV: A(NT-1-t)); X(i) at X[i]
// (i may run BR + q beyond the data, into zero pads; BR outputs per lane).  mode 0: rescale Y to
// max 1; mode 1: normalise to max 1 and floor at kRelFloor.  Returns the team
// max before scaling.
template <int T, bool AREV, int BR = kBR>
__device__ __forceinline__ float team_corr(float* Y, int L, const float* A, int NT, const float* X, int xoff, int mode,
                                        TeamLane Lr)
{
    const int nb = (L + BR - 1) / BR;
    int C = 1;
    while (C * 2 * nb <= T) C *= 2;
    const int passes = (nb + T - 1) / T;  // only when C == 1 and nb > T
    int tc = (NT + C - 1) / C;
    if (C > 1) tc |= 1;
    float mx_all = kNegInf;
    for (int ps = 0; ps < passes; ++ps) {
        const int ob = (C == 1) ? (Lr.tl + ps * T) : (Lr.tl / C);
        const int c = (C == 1) ? 0 : (Lr.tl % C);
        const bool active = ob < nb;
        const int o0 = ob * BR;
        const int tb = min(NT, c * tc), te = min(NT, tb + tc);
        float acc[BR];
#pragma unroll
        for (int r = 0; r < BR; ++r) acc[r] = 0.0f;
        if (active && tb < te) {
            float xw[2 * BR];
            const float* xp = X + o0 + tb + xoff;
#pragma unroll
            for (int i = 0; i < 2 * BR - 1; ++i) xw[i] = xp[i];
            const float* ap = AREV ? A + (NT - 1 - tb) : A + tb;
            int t0 = tb;
            // full groups of BR taps
            for (; t0 + BR <= te; t0 += BR) {
#pragma unroll
                for (int j = 0; j < BR; ++j) {
                    const float a = AREV ? ap[-(t0 - tb) - j] : ap[(t0 - tb) + j];
#pragma unroll
                    for (int r = 0; r < BR; ++r) acc[r] = fmaf(a, xw[r + j], acc[r]);
                }
                if (t0 + BR < te) {
#pragma unroll
                    for (int i = 0; i < BR - 1; ++i) xw[i] = xw[i + BR];
                    const float* xn = xp + (t0 - tb) + 2 * BR - 1;
#pragma unroll
                    for (int i = 0; i < BR; ++i) xw[BR - 1 + i] = xn[i];
                }
            }
            // tail
            if (t0 < te) {
#pragma unroll
                for (int j = 0; j < BR; ++j) {
                    if (t0 + j < te) {
                        const float a = AREV ? ap[-(t0 - tb) - j] : ap[(t0 - tb) + j];
#pragma unroll
                        for (int r = 0; r < BR; ++r) acc[r] = fmaf(a, xw[r + j], acc[r]);
                    }
                }
            }
        }
        for (int off = 1; off < C; off <<= 1)
#pragma unroll
            for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(Lr.mask, acc[r], off, T);
        float lmx = kNegInf;
        if (active && c == 0) {
#pragma unroll
            for (int r = 0; r < BR; ++r)
                if (o0 + r < L) {
                    lmx = fmaxf(lmx, acc[r]);
                    Y[o0 + r] = acc[r];
                }
        }
        mx_all = fmaxf(mx_all, lmx);
    }
    const float mx = team_max<T>(mx_all, Lr.mask);
    __syncwarp(Lr.mask);
    const float inv = mx > 0.0f ? __frcp_rn(mx) : 0.0f;
    for (int o = Lr.tl; o < L; o += T) Y[o] = mode ? fmaxf(Y[o] * inv, kRelFloor) : Y[o] * inv;
    __syncwarp(Lr.mask);
    return mx;
}

// Scratch of the blocked trellis (floats): mu[K*Q] | F_1..F_{K-1} (each with
// zero pads) | B0, B1 (likewise) | res[K*Q].
__host__ __device__ __forceinline__ int blk_arr_floats(int len, int Q) { return len + blk_pad(Q); }

__host__ __device__ __forceinline__ int blk_prefix_offset(int j, int Q)
{
    const int D = Q - 1;
    int f = 0;
    for (int i = 1; i < j; ++i) f += blk_arr_floats(i * D + 1, Q);
    return f;
}

__host__ __device__ __forceinline__ int blk_scratch_floats(int K, int Q)
{
    const int D = Q - 1, S = K * D;
    return K * Q + blk_prefix_offset(K, Q) + 2 * blk_arr_floats(S + 1, Q) + K * Q;
}

// Zero a team's blocked-trellis scratch (the pads must read as zero).
template <int T>
__device__ __forceinline__ void blk_clear(float* sc, int floats, TeamLane Lr)
{
    for (int i = Lr.tl; i < floats; i += T) sc[i] = 0.0f;
    __syncwarp(Lr.mask);
}

// Team-shape channel messages of use u, linear domain, register-blocked.
// Same quantity as chan_trellis<Q, LinSR>; res [K*Q] gets the final messages.
// Returns true if the pass underflowed (the caller reruns in log space and then
// clears the scratch again).
template <int Q>
__device__ bool chan_blocked(const Graph& g, const float* msg_f, size_t ustride, int cbs, float y, float inv_s2, int u,
                             float* sc, float* res, TeamLane Lr)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V, D = Q - 1, PL = BlkPad<Q>::L;
    const int K = g.K, S = K * D;
    float* mu = sc;
    float* Fb = mu + K * Q;                               // F_j data at Fb + blk_prefix_offset(j) + PL
    float* B = Fb + blk_prefix_offset(K, Q) + PL;         // data pointers (pads before and after)
    float* Bn = B + blk_arr_floats(S + 1, Q);
    bool bad = false;
    for (int k = 0; k < K; ++k) {
        const int i = g.use_pos[k * g.n + u];
        const float* blk = msg_f + k * ustride;
        float l[V];
#pragma unroll
        for (int v = 0; v < V; ++v) l[v] = 1.0f;
        const int deg = var_degree(g, i);
        for (int d = 0; d < deg; ++d) {
            const float* m = edge_ptr(blk, g.var_edge[i * g.dv + d], cbs, Q);
#pragma unroll
            for (int v = 0; v < V; ++v) l[v] *= m[v * T + Lr.tl];
        }
        float mx = l[0];
#pragma unroll
        for (int v = 1; v < V; ++v) mx = fmaxf(mx, l[v]);
        mx = team_max<T>(mx, Lr.mask);
        const float inv = __frcp_rn(mx);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int a = v * T + Lr.tl;
            mu[k * Q + a] = l[v] * inv;
            if (k == 0) Fb[PL + a] = l[v] * inv;   // F_1 = mu_0, padded copy
        }
    }
    const GaussTerm gt = gauss_term(y, K, Q, inv_s2);
    for (int s = Lr.tl; s <= S; s += T) B[s] = gt.score(s);
    __syncwarp(Lr.mask);
    for (int j = 1; j + 1 < K; ++j) {
        const float m = team_corr<T, true, CorrBlock<Q>::BR>(Fb + blk_prefix_offset(j + 1, Q) + PL, (j + 1) * D + 1, mu + j * Q, Q,
                                           Fb + blk_prefix_offset(j, Q) + PL, -(Q - 1), 0, Lr);
        if (!(m > 0.0f)) bad = true;
    }
    for (int k = K - 1; k >= 0; --k) {
        if (k == 0) {
            float mx = kNegInf;
            for (int a = Lr.tl; a < Q; a += T) mx = fmaxf(mx, B[a]);
            mx = team_max<T>(mx, Lr.mask);
            if (!(mx >= kFallbackMax)) bad = true;
            const float inv = mx > 0.0f ? __frcp_rn(mx) : 0.0f;
            for (int a = Lr.tl; a < Q; a += T) res[a] = fmaxf(B[a] * inv, kRelFloor);
            __syncwarp(Lr.mask);
        } else {
            const float* Fk = Fb + blk_prefix_offset(k, Q) + PL;
            const float m = team_corr<T, false, CorrBlock<Q>::BR>(res + k * Q, Q, Fk, k * D + 1, B, 0, 1, Lr);
            if (!(m >= kFallbackMax)) bad = true;
            const float m2 = team_corr<T, false, CorrBlock<Q>::BR>(Bn, k * D + 1, mu + k * Q, Q, B, 0, 0, Lr);
            if (!(m2 > 0.0f)) bad = true;
            float* t = B;
            B = Bn;
            Bn = t;
        }
    }
    return bad;
}

// Team shape: store the channel messages res of use u and turn the c2v of the
// K variables on this use into v2c in place.
template <int Q>
__device__ void chan_write_team(const Graph& g, float* msg_f, size_t ustride, int cbs, float* ch2v_f,
                                const float* res, int u, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
    for (int k = 0; k < g.K; ++k) {
        const int i = g.use_pos[k * g.n + u];
        float* blk = msg_f + k * ustride;
        float ch[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            ch[v] = res[k * Q + v * T + L.tl];
            ch2v_f[((size_t)k * g.n + i) * Q + v * T + L.tl] = ch[v];
        }
        float cv[kMaxDv][V];
        const int deg = var_degree(g, i);
#pragma unroll
        for (int d = 0; d < kMaxDv; ++d)
            if (d < deg) {
                const float* m = edge_ptr(blk, g.var_edge[i * g.dv + d], cbs, Q);
#pragma unroll
                for (int v = 0; v < V; ++v) cv[d][v] = m[v * T + L.tl];
            }
#pragma unroll
        for (int d = 0; d < kMaxDv; ++d)
            if (d < deg) {
                float l[V];
                float lmx = kNegInf;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    float s = ch[v];
#pragma unroll
                    for (int d2 = 0; d2 < kMaxDv; ++d2)
                        if (d2 < deg && d2 != d) s *= cv[d2][v];
                    l[v] = s;
                    lmx = fmaxf(lmx, s);
                }
                const float inv = __frcp_rn(team_max<T>(lmx, L.mask));
                float* m = edge_ptr(blk, g.var_edge[i * g.dv + d], cbs, Q);
#pragma unroll
                for (int v = 0; v < V; ++v) m[v * T + L.tl] = l[v] * inv;
            }
    }
}

// ---------------------------------------------------------------------------
// Check node (FFT-QSPA, FP32 Walsh-Hadamard butterflies)
// ---------------------------------------------------------------------------
//
// For check j of one user, in place (v2c in, c2v out), edges d = 0..3 with
// coefficient h_d: the edge carries x = h_d a, so p~_d(x) = v2c_d(h_d^{-1} x);
// P_d = WHT(p~_d) with P(w) = sum_x p(x) (-1)^{popcount(x & w)}; Q_d = prod of the
// other three P (prefix/suffix, no division); r_d = WHT(Q_d) (the 1/q factor
// cancels in the normalisation); c2v_d(a) = max(r_d(h_d a), kRelFloor max r_d) / max r_d.

template <int Q>
__device__ __forceinline__ void wht_reg(float (&p)[Q])
{
#pragma unroll
    for (int s = 1; s < Q; s <<= 1)
#pragma unroll
        for (int x = 0; x < Q; ++x)
            if (!(x & s)) {
                const float a = p[x], b = p[x | s];
                p[x] = a + b;
                p[x | s] = a - b;
            }
}

// Thread shape (q <= 16).  blk: check j's four edge vectors (blk + d*Q).
template <int Q>
__device__ __forceinline__ void check_thread(float* blk, const uint8_t* coef, const uint8_t* gdiv)
{
    float P[kDC][Q];
    int h[kDC];
#pragma unroll
    for (int d = 0; d < kDC; ++d) {
        h[d] = coef[d];
        const uint8_t* dv = gdiv + h[d] * Q;
#pragma unroll
        for (int x = 0; x < Q; ++x) P[d][x] = blk[d * Q + dv[x]];
    }
#pragma unroll
    for (int d = 0; d < kDC; ++d) wht_reg<Q>(P[d]);
    float R[kDC][Q];
#pragma unroll
    for (int x = 0; x < Q; ++x) {
        const float l01 = P[0][x] * P[1][x], r23 = P[2][x] * P[3][x];
        R[0][x] = P[1][x] * r23;
        R[1][x] = P[0][x] * r23;
        R[2][x] = l01 * P[3][x];
        R[3][x] = l01 * P[2][x];
    }
#pragma unroll
    for (int d = 0; d < kDC; ++d) {
        wht_reg<Q>(R[d]);
        const float mx = vmax(R[d]);
        const float fl = kRelFloor * mx, inv = __frcp_rn(mx);
        const uint8_t* dv = gdiv + h[d] * Q;
#pragma unroll
        for (int x = 0; x < Q; ++x) blk[d * Q + dv[x]] = fmaxf(R[d][x], fl) * inv;
    }
}

// In-team Walsh-Hadamard transform over the index x = v*T + tl.
template <int Q>
__device__ __forceinline__ void wht_team(float (&p)[Shape<Q>::V], TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
#pragma unroll
    for (int s = 1; s < T; s <<= 1) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float o = __shfl_xor_sync(L.mask, p[v], s, T);
            p[v] = (L.tl & s) ? (o - p[v]) : (p[v] + o);
        }
    }
#pragma unroll
    for (int s = 1; s < V; s <<= 1) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (!(v & s)) {
                const float a = p[v], b = p[v | s];
                p[v] = a + b;
                p[v | s] = a - b;
            }
        }
    }
}

// Value of the team-distributed vector r at index x (x may differ per lane).
template <int Q>
__device__ __forceinline__ float team_gather(const float (&r)[Shape<Q>::V], int x, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V, LOGT = Shape<Q>::LOGT;
    const int src = x & (T - 1);
    float out = 0.0f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float t = __shfl_sync(L.mask, r[v], src, T);
        if ((x >> LOGT) == v) out = t;
    }
    return out;
}

// Team shape (any q), split into the loads of one check and the rest, so that
// a team can issue the loads of several checks before computing any of them.
template <int Q>
struct CheckRegs {
    float P[kDC][Shape<Q>::V];
    int h[kDC];
};

template <int Q>
__device__ __forceinline__ void check_team_load(const float* blk, const uint8_t* coef, const uint8_t* gdiv,
                                                TeamLane L, CheckRegs<Q>& c)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
#pragma unroll
    for (int d = 0; d < kDC; ++d) {
        c.h[d] = coef[d];
#pragma unroll
        for (int v = 0; v < V; ++v) c.P[d][v] = blk[d * Q + gdiv[c.h[d] * Q + v * T + L.tl]];
    }
}

template <int Q>
__device__ __forceinline__ void check_team_finish(float* blk, CheckRegs<Q>& c, const uint8_t* gmul, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
#pragma unroll
    for (int d = 0; d < kDC; ++d) wht_team<Q>(c.P[d], L);
    float R[kDC][V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float l01 = c.P[0][v] * c.P[1][v], r23 = c.P[2][v] * c.P[3][v];
        R[0][v] = c.P[1][v] * r23;
        R[1][v] = c.P[0][v] * r23;
        R[2][v] = l01 * c.P[3][v];
        R[3][v] = l01 * c.P[2][v];
    }
    __syncwarp(L.mask);
#pragma unroll
    for (int d = 0; d < kDC; ++d) {
        wht_team<Q>(R[d], L);
        float lmx = R[d][0];
#pragma unroll
        for (int v = 1; v < V; ++v) lmx = fmaxf(lmx, R[d][v]);
        const float mx = team_max<T>(lmx, L.mask);
        const float fl = kRelFloor * mx, inv = __frcp_rn(mx);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int a = v * T + L.tl;
            const float r = team_gather<Q>(R[d], gmul[c.h[d] * Q + a], L);
            blk[d * Q + a] = fmaxf(r, fl) * inv;
        }
    }
}

// Team shape (any q).  blk: check j's four edge vectors.
template <int Q>
__device__ void check_team(float* blk, const uint8_t* coef, const uint8_t* gmul, const uint8_t* gdiv, TeamLane L)
{
    CheckRegs<Q> c;
    check_team_load<Q>(blk, coef, gdiv, L, c);
    check_team_finish<Q>(blk, c, gmul, L);
}

// ---------------------------------------------------------------------------
// Variable node, decision, syndrome
// ---------------------------------------------------------------------------

// Marginal eq. (app_ldpc_marginal) of variable i of one user, its hard decision
// (ties -> lowest symbol) and optionally the max-normalised log-posterior.
template <int Q>
__device__ __forceinline__ void var_thread(const Graph& g, const float* ch2v_fk, const float* blk, int cbs, int i,
                                           float* logpost_fk, uint8_t* hat_fk)
{
    float b[Q];
    vload<Q>(ch2v_fk + (size_t)i * Q, b);
    const int deg = var_degree(g, i);
    for (int d = 0; d < deg; ++d) {
        float t[Q];
        vload<Q>(edge_ptr(blk, g.var_edge[i * g.dv + d], cbs, Q), t);
#pragma unroll
        for (int a = 0; a < Q; ++a) b[a] *= t[a];
    }
    float bv = b[0];
    int bi = 0;
#pragma unroll
    for (int a = 1; a < Q; ++a)
        if (b[a] > bv) {
            bv = b[a];
            bi = a;
        }
    hat_fk[i] = (uint8_t)bi;
    if (logpost_fk) {
        const float l = __logf(bv);
        float o[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) o[a] = __logf(b[a]) - l;
        vstore<Q>(logpost_fk + (size_t)i * Q, o);
    }
}

template <int Q>
__device__ void var_team(const Graph& g, const float* ch2v_fk, const float* blk, int cbs, int i, float* logpost_fk,
                         uint8_t* hat_fk, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
    float b[V];
#pragma unroll
    for (int v = 0; v < V; ++v) b[v] = ch2v_fk[(size_t)i * Q + v * T + L.tl];
    const int deg = var_degree(g, i);
    for (int d = 0; d < deg; ++d) {
        const float* m = edge_ptr(blk, g.var_edge[i * g.dv + d], cbs, Q);
#pragma unroll
        for (int v = 0; v < V; ++v) b[v] *= m[v * T + L.tl];
    }
    float bv = b[0];
    int bi = L.tl;
#pragma unroll
    for (int v = 1; v < V; ++v)
        if (b[v] > bv) {
            bv = b[v];
            bi = v * T + L.tl;
        }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(L.mask, bv, o, T);
        const int oi = __shfl_xor_sync(L.mask, bi, o, T);
        if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if (L.tl == 0) hat_fk[i] = (uint8_t)bi;
    if (logpost_fk) {
        const float l = __logf(bv);
#pragma unroll
        for (int v = 0; v < V; ++v) logpost_fk[(size_t)i * Q + v * T + L.tl] = __logf(b[v]) - l;
    }
}

// ---------------------------------------------------------------------------
// Position-major transposed layout (fused kernel, thread shape, dv = 2)
// ---------------------------------------------------------------------------
//
// User k's variable i is stored at its channel-use position p = pi_k(i), so the
// channel node of use p finds every user's variable at the same position.  32
// consecutive positions are interleaved in chunks of W symbols (W = 1: chunks of
// 4 halve the load instructions of the channel and variable phases but cost the
// check phase's permuted gathers more address arithmetic and bank conflicts;
// measured 5% slower on K=4, q=16):
// symbol a of the q-vector at position p of row r lives at
//   ((r * q/W + a/W) * 32 + p % 32) * W + a % W,
// so a thread reads its vector as q/W aligned W-float loads and the 32 threads
// of a warp on consecutive positions cover consecutive banks.  Rows: ch2v row =
// k*NB + p/32; msg row = (k*NB + p/32)*2 + d for the variable's d-th edge
// (ascending edge id).

constexpr int kLanes = 32;

template <int Q>
struct PosW {
    static constexpr int W = 1;
};

// Users 2 and 3 rotate their rows' 32 positions by 16: the lane-pair shape has
// lanes 2m and 2m+1 read users {0, 1} and {2, 3} at the same position, which
// would otherwise fall on one bank.  Consecutive positions of a row still cover
// all 32 banks.
__host__ __device__ __forceinline__ int pos_rot(int k) { return (k & 2) << 3; }

template <int Q>
__device__ __forceinline__ int pos_vec(int row, int p, int k)
{
    return row * Q * kLanes + ((p + pos_rot(k)) & (kLanes - 1)) * PosW<Q>::W;
}

// offset of symbol a inside a position vector
template <int Q>
__device__ __forceinline__ int pos_sym(int a)
{
    constexpr int W = PosW<Q>::W;
    return (a / W) * (kLanes * W) + (a % W);
}

template <int Q>
__device__ __forceinline__ void sload(const float* base, float (&v)[Q])
{
    constexpr int W = PosW<Q>::W;
#pragma unroll
    for (int c = 0; c < Q / W; ++c) {
        if constexpr (W == 4) {
            const float4 t = *reinterpret_cast<const float4*>(base + c * kLanes * W);
            v[4 * c] = t.x; v[4 * c + 1] = t.y; v[4 * c + 2] = t.z; v[4 * c + 3] = t.w;
        } else if constexpr (W == 1) {
            v[c] = base[c * kLanes];
        } else {
            const float2 t = *reinterpret_cast<const float2*>(base + c * kLanes * W);
            v[2 * c] = t.x; v[2 * c + 1] = t.y;
        }
    }
}

template <int Q>
__device__ __forceinline__ void sstore(float* base, const float (&v)[Q])
{
    constexpr int W = PosW<Q>::W;
#pragma unroll
    for (int c = 0; c < Q / W; ++c) {
        if constexpr (W == 4)
            *reinterpret_cast<float4*>(base + c * kLanes * W) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        else if constexpr (W == 1)
            base[c * kLanes] = v[c];
        else
            *reinterpret_cast<float2*>(base + c * kLanes * W) = make_float2(v[2 * c], v[2 * c + 1]);
    }
}

// Channel node of use p, thread shape, position-major layout.  msg_f / ch2v_f:
// the frame's blocks; NB = ceil(n / 32).  hat_f (may be null): before the
// channel messages are replaced, the previous iteration's posterior
// ch2v * c2v_0 * c2v_1 of each variable on this use (eq. app_ldpc_marginal) is
// formed from the messages already loaded here and its decision (ties -> lowest
// symbol) stored at hat_f[k*NB*32 + p]: the decision phase of the previous
// iteration, folded into this one.
template <int K, int Q>
__device__ __forceinline__ void chan_thread_pos(const Graph& g, float* msg_f, float* ch2v_f, int NB, float y,
                                                float inv_s2, int p, uint8_t* hat_f = nullptr)
{
    float mu[K][Q];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int row = (k * NB + (p >> 5)) * 2;
        float a0[Q], a1[Q];
        sload<Q>(msg_f + pos_vec<Q>(row, p, k), a0);
        sload<Q>(msg_f + pos_vec<Q>(row + 1, p, k), a1);
#pragma unroll
        for (int a = 0; a < Q; ++a) a0[a] *= a1[a];
        if (hat_f) {
            float b[Q];
            sload<Q>(ch2v_f + pos_vec<Q>(k * NB + (p >> 5), p, k), b);
#pragma unroll
            for (int a = 0; a < Q; ++a) b[a] *= a0[a];
            hat_f[k * NB * 32 + p] = (uint8_t)vargmax<Q>(b);
        }
        const float inv = __frcp_rn(vmax(a0));
#pragma unroll
        for (int a = 0; a < Q; ++a) mu[k][a] = a0[a] * inv;
    }
    const GaussTerm gt = gauss_term(y, K, Q, inv_s2);
    chan_reg<K, Q>(mu, gt, g.log_fallbacks, [&](int k, const float (&o)[Q]) {
        const int row = (k * NB + (p >> 5)) * 2;
        sstore<Q>(ch2v_f + pos_vec<Q>(k * NB + (p >> 5), p, k), o);
        float* p0 = msg_f + pos_vec<Q>(row, p, k);
        float* p1 = msg_f + pos_vec<Q>(row + 1, p, k);
        float c0[Q], c1[Q];
        sload<Q>(p0, c0);
        sload<Q>(p1, c1);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float t = c0[a];
            c0[a] = o[a] * c1[a];
            c1[a] = o[a] * t;
        }
        const float i0 = __frcp_rn(vmax(c0)), i1 = __frcp_rn(vmax(c1));
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            c0[a] *= i0;
            c1[a] *= i1;
        }
        sstore<Q>(p0, c0);
        sstore<Q>(p1, c1);
    });
}

// Channel node of use p for K = 4 split over a pair of lanes (lanes 2m, 2m+1 of
// a warp; `half` = lane & 1, `mask` = the pair's lanes).  Lane h owns users
// 2h and 2h+1: it forms their pair convolution P_own = mu_{2h} (*) mu_{2h+1},
// receives the other half's by shuffles, scores it
// against G (the suffix H), and emits its users' messages
// sum_b mu_{2h+1}(b) H(a+b) and sum_b mu_{2h}(b) H(a+b).  Each lane does half
// of the single-thread work with about half the registers, with the same sums
// in the same order (bit-identical to chan_thread_pos).  hat_f (may be null):
// the folded decision of the previous iteration for the lane's two users, as
// in chan_thread_pos.
template <int Q>
__device__ __forceinline__ void chan_pair_pos(const Graph& g, float* msg_f, float* ch2v_f, int NB, float y,
                                              float inv_s2, int p, int half, unsigned mask, uint8_t* hat_f)
{
    constexpr int D = Q - 1, K = 4, NP = 2 * D + 1;
    float mu[2][Q];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int k = 2 * half + j;
        const int row = (k * NB + (p >> 5)) * 2;
        float a0[Q], a1[Q];
        sload<Q>(msg_f + pos_vec<Q>(row, p, k), a0);
        sload<Q>(msg_f + pos_vec<Q>(row + 1, p, k), a1);
#pragma unroll
        for (int a = 0; a < Q; ++a) a0[a] *= a1[a];
        if (hat_f) {
            float b[Q];
            sload<Q>(ch2v_f + pos_vec<Q>(k * NB + (p >> 5), p, k), b);
#pragma unroll
            for (int a = 0; a < Q; ++a) b[a] *= a0[a];
            hat_f[k * NB * 32 + p] = (uint8_t)vargmax<Q>(b);
        }
        const float inv = __frcp_rn(vmax(a0));
#pragma unroll
        for (int a = 0; a < Q; ++a) mu[j][a] = a0[a] * inv;
    }
    // own pair convolution, then the other half's by shuffles
    float Po[NP];
    {
        float Pown[NP];
        rconv(mu[0], mu[1], Pown);
#pragma unroll
        for (int i = 0; i < NP; ++i) Po[i] = __shfl_xor_sync(mask, Pown[i], 1);
    }
    const GaussTerm gt = gauss_term(y, K, Q, inv_s2);
    float H[NP];
    rcorr_g<NP, NP>(Po, H, gt);
    // one user at a time (16 registers of output live, not 32): user 2h gets
    // sum_b mu_{2h+1}(b) H(a+b), user 2h+1 gets sum_b mu_{2h}(b) H(a+b)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        float o[Q];
        rcorr(mu[1 - j], H, o);
        float mx = vmax(o);
        const bool bad = !(mx >= kFallbackMax);
        // the log-space recomputation needs all four incoming messages: pair-uniform
        if (__shfl_xor_sync(mask, bad ? 1 : 0, 1) || bad) {
            float mu4[K][Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const float x0 = __shfl_xor_sync(mask, mu[0][a], 1), x1 = __shfl_xor_sync(mask, mu[1][a], 1);
                mu4[2 * half][a] = mu[0][a];
                mu4[2 * half + 1][a] = mu[1][a];
                mu4[2 * (1 - half)][a] = x0;
                mu4[2 * (1 - half) + 1][a] = x1;
            }
            if (bad) {
                if (g.log_fallbacks) atomicAdd(g.log_fallbacks, 1ull);
                chan_user_log<K, Q>(mu4, 2 * half + j, gt, o);
                mx = 1.0f;
            }
        }
        const float inv = __frcp_rn(mx);
#pragma unroll
        for (int a = 0; a < Q; ++a) o[a] = fmaxf(o[a] * inv, kRelFloor);
        const int k = 2 * half + j;
        const int row = (k * NB + (p >> 5)) * 2;
        sstore<Q>(ch2v_f + pos_vec<Q>(k * NB + (p >> 5), p, k), o);
        float* p0 = msg_f + pos_vec<Q>(row, p, k);
        float* p1 = msg_f + pos_vec<Q>(row + 1, p, k);
        float c0[Q], c1[Q];
        sload<Q>(p0, c0);
        sload<Q>(p1, c1);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float t = c0[a];
            c0[a] = o[a] * c1[a];
            c1[a] = o[a] * t;
        }
        const float i0 = __frcp_rn(vmax(c0)), i1 = __frcp_rn(vmax(c1));
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            c0[a] *= i0;
            c1[a] *= i1;
        }
        sstore<Q>(p0, c0);
        sstore<Q>(p1, c1);
    }
}

// Index h^{-1} x for every x from the images of the basis vectors: multiplying
// by a fixed field element is GF(2)-linear, so h^{-1} x is the XOR of
// h^{-1} 2^b over the set bits b of x.
template <int Q>
__device__ __forceinline__ int gf_lin(const int (&basis)[6], int x)
{
    int r = 0;
#pragma unroll
    for (int b = 0; (1 << b) < Q; ++b)
        if (x & (1 << b)) r ^= basis[b];
    return r;
}

// Record of one check unit (check j of user k) for the position-major check
// phase, built once per CTA: for each edge d, off.{x,y,z,w}[d] = the offset of
// the edge's message vector in the frame's message block (bits 0..23; symbol a
// at + a*32) with the edge coefficient h in bits 24..31; basis.{x,y}: 16 bits
// per edge, the images h^{-1} 2^b (b < log2 q, 4 bits each) from which the
// permuted symbol h^{-1} x of any x is an XOR (division by h is GF(2)-linear).
struct CheckRec {
    uint4 off;
    uint2 basis;
};

template <int Q>
__device__ __forceinline__ CheckRec check_rec(const Graph& g, int NB, int k, int j)
{
    unsigned o[kDC], b[kDC];
#pragma unroll
    for (int d = 0; d < kDC; ++d) {
        const int e = 4 * j + d, sl = g.slot[k * g.E + e], pp = sl >> 1, h = g.chk_coef[e];
        o[d] = (unsigned)(pos_vec<Q>((k * NB + (pp >> 5)) * 2 + (sl & 1), pp, k)) | ((unsigned)h << 24);
        unsigned bb = 0;
        for (int t = 0; (1 << t) < Q; ++t) bb |= (unsigned)g.gf_div[h * Q + (1 << t)] << (4 * t);
        b[d] = bb;
    }
    CheckRec r;
    r.off = make_uint4(o[0], o[1], o[2], o[3]);
    r.basis = make_uint2(b[0] | (b[1] << 16), b[2] | (b[3] << 16));
    return r;
}

__device__ __forceinline__ int rec_coef(unsigned o) { return (int)(o >> 24); }

// position-order index of the edge's variable in the frame's decisions
// (k*NB*32 + position): its message row is (k*NB + position/32)*2 + slot, and
// its position within the row is rotated by pos_rot(k)
template <int Q>
__device__ __forceinline__ int rec_hat(unsigned o, int NB)
{
    // rk = k NB + position / 32; users k >= 2 (rk >= 2 NB, K <= 4) rotate by pos_rot = 16
    const unsigned v = o & 0xFFFFFFu, rk = (v / (Q * kLanes)) >> 1;
    const unsigned rot = rk >= 2u * (unsigned)NB ? (unsigned)pos_rot(2) : 0u;
    return (int)((rk << 5) | ((v - rot) & (kLanes - 1)));
}

// user k of the record's unit, from rk = k NB + position / 32 (K <= 4: three comparisons)
template <int Q>
__device__ __forceinline__ int rec_user(unsigned o, int NB)
{
    const unsigned rk = ((o & 0xFFFFFFu) / (Q * kLanes)) >> 1, nb = (unsigned)NB;
    return (int)(rk >= nb) + (int)(rk >= 2u * nb) + (int)(rk >= 3u * nb);
}

// Check node of one unit (check j of user k), thread shape, position-major
// layout, from its record: the edge coefficient permutation p_e(b) = v2c_e(h^-1 b)
// gathered through XORs of the basis images, the WHT of each edge (eq.
// app_ldpc_c2v in the transform domain), the leave-one-out products, the inverse
// WHT, the 1e-12 floor relative to the maximum and the scaling to max 1, and the
// scatter back through the same permutation.
template <int Q>
__device__ __forceinline__ void check_thread_rec(float* msg_f, const uint4& r, const uint2& rb)
{
    static_assert(PosW<Q>::W == 1, "offset XOR trick needs one symbol per chunk");
    const unsigned o[kDC] = {r.x, r.y, r.z, r.w};
    const unsigned bw[kDC] = {rb.x & 0xFFFFu, rb.x >> 16, rb.y & 0xFFFFu, rb.y >> 16};
    float P[kDC][Q];
    float* base[kDC];
    int basis[kDC][6];
#pragma unroll
    for (int d = 0; d < kDC; ++d) {
        base[d] = msg_f + (o[d] & 0xFFFFFFu);
#pragma unroll
        for (int b = 0; b < 6; ++b) basis[d][b] = ((1 << b) < Q) ? (int)((bw[d] >> (4 * b)) & 15u) * kLanes : 0;
#pragma unroll
        for (int x = 0; x < Q; ++x) P[d][x] = base[d][gf_lin<Q>(basis[d], x)];
    }
#pragma unroll
    for (int d = 0; d < kDC; ++d) wht_reg<Q>(P[d]);
#pragma unroll
    for (int x = 0; x < Q; ++x) {
        const float p0 = P[0][x], p1 = P[1][x], p2 = P[2][x], p3 = P[3][x];
        const float l01 = p0 * p1, r23 = p2 * p3;
        P[0][x] = p1 * r23;
        P[1][x] = p0 * r23;
        P[2][x] = l01 * p3;
        P[3][x] = l01 * p2;
    }
#pragma unroll
    for (int d = 0; d < kDC; ++d) {
        wht_reg<Q>(P[d]);
        const float mx = vmax(P[d]);
        const float fl = kRelFloor * mx, inv = __frcp_rn(mx);
#pragma unroll
        for (int x = 0; x < Q; ++x) base[d][gf_lin<Q>(basis[d], x)] = fmaxf(P[d][x], fl) * inv;
    }
}

// Posterior and decision of the variable at position p of user k.
template <int Q>
__device__ __forceinline__ int var_thread_pos(const float* msg_f, const float* ch2v_f, int NB, int k, int p,
                                              float* logpost_ki)
{
    float b[Q], c0[Q], c1[Q];
    const int row = k * NB + (p >> 5);
    sload<Q>(ch2v_f + pos_vec<Q>(row, p, k), b);
    sload<Q>(msg_f + pos_vec<Q>(2 * row, p, k), c0);
    sload<Q>(msg_f + pos_vec<Q>(2 * row + 1, p, k), c1);
#pragma unroll
    for (int a = 0; a < Q; ++a) b[a] *= c0[a] * c1[a];
    const int bi = vargmax<Q>(b);
    if (logpost_ki) {
        const float bv = vmax<Q>(b);
        const float l = __logf(bv);
        float o[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) o[a] = __logf(b[a]) - l;
        vstore<Q>(logpost_ki, o);
    }
    return bi;
}

// eq. (app_ldpc_check_eq) for check j of one user's decisions.
__device__ __forceinline__ bool check_satisfied(const Graph& g, const uint8_t* hat_fk, int j, const uint8_t* gmul)
{
    int s = 0;
    for (int d = 0; d < g.dc; ++d) {
        const int e = j * g.dc + d;
        s ^= gmul[g.chk_coef[e] * g.Q + hat_fk[g.chk_var[e]]];
    }
    return s == 0;
}

}  // namespace jbp
