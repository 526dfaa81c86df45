// jbp_device.cuh -- per-node device routines of joint FFT belief propagation.
//
// Every routine works on one "unit" (a channel use, a check of one user, a
// variable of one user) with a team of T = min(q, 32) lanes of one warp; lane
// tl owns the symbols a = v*T + tl, v < V = q/T.  Teams synchronise only with
// their own lanes (team masks), so teams of one warp may diverge.  Pointers are
// generic: the same routines run on HBM-resident state (step kernels) and on
// shared-memory state (fused kernel).
//
// Message convention: FP32 log-probabilities with maximum 0.  A stored c2v
// message is floored at kRelFloor of its maximum (in the linear domain after
// the inverse transform); a channel message is clipped at kLogFloor.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jbp {

constexpr float kRelFloor = 1e-12f;
constexpr float kLogFloor = -27.631021115928547f;  // ln(1e-12)
constexpr float kFallbackMax = 1e-30f;             // linear trellis underflow guard
constexpr int kMaxDv = 8;
constexpr int kMaxK = 16;
constexpr float kNegInf = -__builtin_inff();

// Device view of one decoder: code, interleavers, channel and GF tables.
struct Graph {
    int n, P, E, dc, dv, K, Q;
    float inv_sigma2;
    const int32_t* chk_var;   // [E]     variable of check-major edge e
    const uint8_t* chk_coef;  // [E]     H_{j,l} of edge e
    const int32_t* var_edge;  // [n*dv]  edges of variable i, ascending
    const int32_t* use_pos;   // [K*n]   use_pos[k*n+t] = pi_k^{-1}(t)
    const uint8_t* gf_mul;    // [Q*Q]   gf_mul[h*Q+x] = h*x
    const uint8_t* gf_div;    // [Q*Q]   gf_div[h*Q+x] = h^{-1}*x
};

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

template <int T>
__device__ __forceinline__ bool team_any(bool p, unsigned mask)
{
    int v = p ? 1 : 0;
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(mask, v, o, T);
    return v != 0;
}

// ---------------------------------------------------------------------------
// Channel node
// ---------------------------------------------------------------------------

// Sum-product arithmetic of the trellis: linear domain (fast path) or log
// domain (taken when the linear pass underflows).
struct LinSR {
    static constexpr bool kLog = false;
    __device__ static __forceinline__ float zero() { return 0.0f; }
    __device__ static __forceinline__ float mac(float acc, float a, float b) { return fmaf(a, b, acc); }
    __device__ static __forceinline__ float from_log(float l) { return __expf(l); }
    __device__ static __forceinline__ float rescale(float x, float mx) { return mx > 0.0f ? x * (1.0f / mx) : x; }
    __device__ static __forceinline__ float to_log(float x, float mx) { return __logf(x) - __logf(mx); }
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
    __device__ static __forceinline__ float from_log(float l) { return l; }
    __device__ static __forceinline__ float rescale(float x, float mx) { return x - mx; }
    __device__ static __forceinline__ float to_log(float x, float mx) { return x - mx; }
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

// Extrinsic channel messages of channel use u of one frame.
//
// With a_k the symbol of user k and s = sum_k a_k, the likelihood of y_u is
// G(s) = exp(-(y_u - (2s - K(q-1)))^2 / (2 sigma2)).  The message to user k is
//   ch2v_k(a) ~ sum_s F_k(s) B_{k+1}(s + a),
// with prefixes F_0 = delta_0, F_{j+1} = F_j (*) mu_j (integer convolution) and
// scored suffixes B_K = G, B_j(v) = sum_b mu_j(b) B_{j+1}(v + b).  Nothing is
// divided out.  Every prefix and suffix is rescaled to a maximum of 1.  The
// exponent uses the nearest symbol sum s*: with r = y - (2s* - K(q-1)) and
// d = s* - s, -(y - L_s)^2/(2 sigma2) + (y - L_s*)^2/(2 sigma2) = -2 d (r + d)/sigma2.
//
// msg_f: the frame's message block [K][E][Q] (c2v).  res [K*Q] receives the
// max-normalised, clipped log messages.  Returns true (team-uniform) if the
// linear pass lost a message to underflow; the caller then reruns in LogSR.
template <int Q, class SR>
__device__ bool chan_trellis(const Graph& g, const float* msg_f, float y, int u, float* sc,
                             float* res, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V, D = Q - 1;
    const int K = g.K, S = K * D;
    float* mu = sc;
    float* Fb = mu + K * Q;
    float* B = Fb + prefix_offset(K, D);
    float* Bn = B + S + 1;
    bool bad = false;

    // messages of the K variables into this channel node: product of all c2v
    for (int k = 0; k < K; ++k) {
        const int i = g.use_pos[k * g.n + u];
        const float* mk = msg_f + (size_t)k * g.E * Q;
        float l[V];
#pragma unroll
        for (int v = 0; v < V; ++v) l[v] = 0.0f;
        for (int d = 0; d < g.dv; ++d) {
            const float* m = mk + (size_t)g.var_edge[i * g.dv + d] * Q;
#pragma unroll
            for (int v = 0; v < V; ++v) l[v] += m[v * T + L.tl];
        }
        float mx = l[0];
#pragma unroll
        for (int v = 1; v < V; ++v) mx = fmaxf(mx, l[v]);
        mx = team_max<T>(mx, L.mask);
#pragma unroll
        for (int v = 0; v < V; ++v) mu[k * Q + v * T + L.tl] = SR::from_log(l[v] - mx);
    }

    // likelihood over the symbol sum
    {
        const int KD = K * D;
        float sf = rintf((y + (float)KD) * 0.5f);
        sf = fminf(fmaxf(sf, 0.0f), (float)KD);
        const int ss = (int)sf;
        const float r = y - (float)(2 * ss - KD);
        for (int s = L.tl; s <= S; s += T) {
            const float dl = (float)(ss - s);
            const float e = -2.0f * dl * (r + dl) * g.inv_sigma2;
            B[s] = SR::kLog ? e : __expf(e);
        }
    }

    // prefixes F_2 .. F_{K-1}
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

    // scored suffixes and the extrinsic outputs, last user first
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
        for (int v = 0; v < V; ++v) res[k * Q + v * T + L.tl] = fmaxf(SR::to_log(o[v], mx), kLogFloor);
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

// Store the channel messages of use u and turn the c2v messages of the K
// variables on this use into v2c messages in place (eq. app_ldpc_v2c with the
// channel message as the local belief): v2c_e = ch2v + sum of the other edges'
// c2v, max-normalised.  Only this team touches these edges in this step.
template <int Q>
__device__ void chan_write(const Graph& g, float* msg_f, float* ch2v_f, const float* res, int u,
                           TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
    for (int k = 0; k < g.K; ++k) {
        const int i = g.use_pos[k * g.n + u];
        float* mk = msg_f + (size_t)k * g.E * Q;
        float ch[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            ch[v] = res[k * Q + v * T + L.tl];
            ch2v_f[((size_t)k * g.n + i) * Q + v * T + L.tl] = ch[v];
        }
        float cv[kMaxDv][V];
        int eidx[kMaxDv];
#pragma unroll
        for (int d = 0; d < kMaxDv; ++d) {
            if (d < g.dv) {
                eidx[d] = g.var_edge[i * g.dv + d];
#pragma unroll
                for (int v = 0; v < V; ++v) cv[d][v] = mk[(size_t)eidx[d] * Q + v * T + L.tl];
            }
        }
#pragma unroll
        for (int d = 0; d < kMaxDv; ++d) {
            if (d < g.dv) {
                float l[V];
                float lmx = kNegInf;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    float s = ch[v];
#pragma unroll
                    for (int d2 = 0; d2 < kMaxDv; ++d2)
                        if (d2 < g.dv && d2 != d) s += cv[d2][v];
                    l[v] = s;
                    lmx = fmaxf(lmx, s);
                }
                const float mx = team_max<T>(lmx, L.mask);
#pragma unroll
                for (int v = 0; v < V; ++v) mk[(size_t)eidx[d] * Q + v * T + L.tl] = l[v] - mx;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Check node (FFT-QSPA, FP32 butterflies)
// ---------------------------------------------------------------------------

// In-team Walsh-Hadamard transform in natural (Sylvester) order over the index
// x = v*T + tl: P(w) = sum_x p(x) (-1)^{popcount(x & w)}.
template <int Q>
__device__ __forceinline__ void wht(float (&p)[Shape<Q>::V], TeamLane L)
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

// Check-node update of check j of one user (msg_fk: that user's [E][Q] block),
// in place: v2c of the DC edges in, c2v out.
//   x_e = h_e a_e carries the edge; p~_e(x) = v2c_e(h_e^{-1} x);
//   P_e = WHT(p~_e); Q_e = prod_{e' != e} P_e' (prefix/suffix, no division);
//   r_e = WHT(Q_e) (the 1/q factor cancels in the normalisation);
//   c2v_e(a) = log max(r_e(h_e a), kRelFloor * max r_e) - log max r_e.
template <int Q, int DC>
__device__ void check_unit_fp32(const Graph& g, float* msg_fk, int j, const uint8_t* gmul,
                                const uint8_t* gdiv, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
    float P[DC][V];
    int h[DC];
#pragma unroll
    for (int d = 0; d < DC; ++d) {
        const int e = j * DC + d;
        h[d] = g.chk_coef[e];
        const float* m = msg_fk + (size_t)e * Q;
#pragma unroll
        for (int v = 0; v < V; ++v) P[d][v] = __expf(m[gdiv[h[d] * Q + v * T + L.tl]]);
    }
#pragma unroll
    for (int d = 0; d < DC; ++d) wht<Q>(P[d], L);

    float R[DC][V];
    {
        float pre[V];
#pragma unroll
        for (int v = 0; v < V; ++v) pre[v] = 1.0f;
#pragma unroll
        for (int d = 0; d < DC; ++d) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                R[d][v] = pre[v];
                pre[v] *= P[d][v];
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) pre[v] = 1.0f;
#pragma unroll
        for (int d = DC - 1; d >= 0; --d) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                R[d][v] *= pre[v];
                pre[v] *= P[d][v];
            }
        }
    }
    __syncwarp(L.mask);
#pragma unroll
    for (int d = 0; d < DC; ++d) {
        wht<Q>(R[d], L);
        float lmx = R[d][0];
#pragma unroll
        for (int v = 1; v < V; ++v) lmx = fmaxf(lmx, R[d][v]);
        const float mx = team_max<T>(lmx, L.mask);
        const float lgmx = __logf(mx);
        float* m = msg_fk + (size_t)(j * DC + d) * Q;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int a = v * T + L.tl;
            const float r = team_gather<Q>(R[d], gmul[h[d] * Q + a], L);
            m[a] = __logf(fmaxf(r, kRelFloor * mx)) - lgmx;
        }
    }
}

// ---------------------------------------------------------------------------
// Variable node, decision, syndrome
// ---------------------------------------------------------------------------

// Marginal eq. (app_ldpc_marginal) of variable i of one user and its hard
// decision (ties -> lowest symbol).  post_fk may be null.
template <int Q>
__device__ void var_unit(const Graph& g, const float* ch2v_fk, const float* msg_fk, int i,
                         float* post_fk, uint8_t* hat_fk, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
    float b[V];
#pragma unroll
    for (int v = 0; v < V; ++v) b[v] = ch2v_fk[(size_t)i * Q + v * T + L.tl];
    for (int d = 0; d < g.dv; ++d) {
        const float* m = msg_fk + (size_t)g.var_edge[i * g.dv + d] * Q;
#pragma unroll
        for (int v = 0; v < V; ++v) b[v] += m[v * T + L.tl];
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
    if (post_fk) {
#pragma unroll
        for (int v = 0; v < V; ++v) post_fk[(size_t)i * Q + v * T + L.tl] = b[v] - bv;
    }
}

// eq. (app_ldpc_check_eq) for check j of one user's decisions.
__device__ __forceinline__ bool check_satisfied(const Graph& g, const uint8_t* hat_fk, int j,
                                                const uint8_t* gmul)
{
    int s = 0;
    for (int d = 0; d < g.dc; ++d) {
        const int e = j * g.dc + d;
        s ^= gmul[g.chk_coef[e] * g.Q + hat_fk[g.chk_var[e]]];
    }
    return s == 0;
}

}  // namespace jbp
