// jbp_ura.cu -- the paper's own classical path on the evidence interface S:
//
//  * k_amp: the slot-wise AMP-MMSE detector (appendix "Slot-wise AMP--MMSE
//    detector": eqs. amp_iter_r, amp_iter_u, amp_iter_res with the
//    Bernoulli-Gaussian denoiser of eqs. bg_activity_prob, bg_mmse_mean, and
//    the evidence S_{l,a} = log p^(R_a; nu) of paragraph "Evidence
//    interface").  One warp per slot.  The dictionary is a partial DFT
//    (appendix "Sensing-matrix construction"), so A^H r and A u are radix-2
//    transforms of length q held two points per lane and exchanged by warp
//    shuffles: A^H r scatters r onto the slot's rows and runs a
//    decimation-in-frequency transform with positive exponent (output in
//    bit-reversed order); the denoiser is elementwise, so it works in that
//    order, and A u runs a decimation-in-time transform with negative exponent
//    (bit-reversed input, natural output) and gathers the slot's rows.
//
//  * k_sic: SIC over K rows (appendix "Complexity derivation", paragraphs
//    SIC-BP and FFT-BP; appendix "Q-ary LDPC code", eqs.
//    app_ldpc_local_belief_from_S, app_ldpc_v2c, app_ldpc_c2v,
//    app_ldpc_marginal), codes with (dv, dc) = (2, 3), (2, 4) or (3, 6).
//    One warp per frame keeps one row's BP state in
//    shared memory: local beliefs lambda (max 1, floored at kRelFloor) and one
//    message per edge (v2c before a check update, c2v after it), as
//    probabilities scaled to max 1.  Each iteration: the check update in the
//    Walsh-Hadamard domain (leave-one-out by prefix/suffix products), then per
//    variable the marginal, the decision and the next v2c, then the syndrome;
//    the row stops when it is zero.  Before row k the evidence of every
//    earlier row's decided symbol is lowered by cancel_log.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "jbp_internal.h"

namespace jbp {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ float2 shfl2(float2 v, int src)
{
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int Q>
struct AmpShape {
    static_assert(Q == 32 || Q == 64, "the slot detector is built for q = 32 and q = 64");
    static constexpr int V = Q / 32;              // points per lane: position e = lane + 32 v
    static constexpr int LOGQ = Q == 64 ? 6 : 5;  // stages
};

// Twiddle of stage s (half-size h = Q/2 >> s) for this lane: w_{2h}^{lane mod h}
// with w_m = exp(-2 pi i / m), read from tw[k] = exp(-2 pi i k / Q).
template <int Q>
__device__ __forceinline__ void stage_twiddles(const float2* tw, int lane, float2 (&w)[AmpShape<Q>::LOGQ])
{
#pragma unroll
    for (int s = 0; s < AmpShape<Q>::LOGQ; ++s) {
        const int h = (Q / 2) >> s;
        w[s] = tw[(lane & (h - 1)) * (Q / (2 * h))];
    }
}

// Decimation in frequency, natural input, bit-reversed output:
// X_k = sum_e x_e exp(+2 pi i e k / Q) (conjugate twiddles).
template <int Q>
__device__ __forceinline__ void dif_inverse(float2 (&x)[AmpShape<Q>::V], const float2 (&w)[AmpShape<Q>::LOGQ],
                                            int lane)
{
    constexpr int V = AmpShape<Q>::V;
#pragma unroll
    for (int s = 0; s < AmpShape<Q>::LOGQ; ++s) {
        const int h = (Q / 2) >> s;
        const float2 ws = conj2(w[s]);
        if (h == 32) {   // pair (lane, lane + 32) held by one lane
            const float2 a = x[0], b = x[V - 1];
            x[0] = make_float2(a.x + b.x, a.y + b.y);
            x[V - 1] = cmul(make_float2(a.x - b.x, a.y - b.y), ws);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 p = shfl_xor2(x[v], h);
                x[v] = (lane & h) ? cmul(make_float2(p.x - x[v].x, p.y - x[v].y), ws)
                                  : make_float2(x[v].x + p.x, x[v].y + p.y);
            }
        }
    }
}

// Decimation in time, bit-reversed input, natural output:
// X_k = sum_a u_a exp(-2 pi i a k / Q) where position e holds u at bitrev(e).
template <int Q>
__device__ __forceinline__ void dit_forward(float2 (&x)[AmpShape<Q>::V], const float2 (&w)[AmpShape<Q>::LOGQ],
                                            int lane)
{
    constexpr int V = AmpShape<Q>::V;
#pragma unroll
    for (int s = AmpShape<Q>::LOGQ - 1; s >= 0; --s) {
        const int h = (Q / 2) >> s;
        if (h == 32) {
            const float2 bw = cmul(x[V - 1], w[s]);
            const float2 a = x[0];
            x[0] = make_float2(a.x + bw.x, a.y + bw.y);
            x[V - 1] = make_float2(a.x - bw.x, a.y - bw.y);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 t = (lane & h) ? cmul(x[v], w[s]) : x[v];
                const float2 p = shfl_xor2(t, h);
                x[v] = (lane & h) ? make_float2(p.x - t.x, p.y - t.y) : make_float2(t.x + p.x, t.y + p.y);
            }
        }
    }
}

// Scalar Bernoulli-Gaussian channel at s = |r|^2 and noise variance nu:
// x = log((1-rho) phi(r;0,nu) / (rho phi(r;0,nu+su2))), so that
// log p^ = -softplus(x) and log(1 - p^) = x - softplus(x).
struct BgOut {
    float logp, gain, deriv;
};

__device__ __forceinline__ BgOut bg_eval(float s, float nu, float log_odds, float su2)
{
    const float k1 = su2 / (nu * (nu + su2));
    const float x = log_odds + log1pf(su2 / nu) - s * k1;
    const float sp = fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x)));
    const float p = expf(-sp), omp = expf(x - sp);
    const float c = su2 / (nu + su2);
    BgOut o;
    o.logp = -sp;
    o.gain = p * c;
    o.deriv = c * (p + s * p * omp * k1);
    return o;
}

template <int Q>
__global__ void __launch_bounds__(256) k_amp(UraDev u, int F, const float* __restrict__ y, float* __restrict__ S)
{
    constexpr int V = AmpShape<Q>::V, LOGQ = AmpShape<Q>::LOGQ;
    __shared__ float2 tw_s[Q];
    for (int i = threadIdx.x; i < Q; i += blockDim.x) tw_s[i] = make_float2(u.tw[2 * i], u.tw[2 * i + 1]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float2 w[LOGQ];
    stage_twiddles<Q>(tw_s, lane, w);
    const int ns = u.ns;
    const float inv_ns = 1.0f / (float)ns;
    const long tasks = (long)F * u.n;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const bool act = lane < ns;
    for (long task = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < tasks; task += nwarps) {
        const int l = (int)(task % u.n);
        const int r = act ? u.rows[l * ns + lane] : 0;
        const float2 yv = act ? reinterpret_cast<const float2*>(y)[task * ns + lane] : make_float2(0.f, 0.f);
        // lane holding the row that lands on position e = lane + 32 v (-1: none)
        int src[V];
#pragma unroll
        for (int v = 0; v < V; ++v) src[v] = -1;
        for (int i = 0; i < ns; ++i) {
            const int ri = __shfl_sync(0xffffffffu, r, i);
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (ri == lane + 32 * v) src[v] = i;
        }
        float2 T = yv;
        float2 U[V], R[V];
#pragma unroll
        for (int v = 0; v < V; ++v) U[v] = make_float2(0.f, 0.f);
        float nu = 0.f;
        for (int it = 0;; ++it) {
            nu = warp_sum(T.x * T.x + T.y * T.y) * inv_ns;
            // R = U + A^H T
            float2 z[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 t = shfl2(T, src[v] < 0 ? 0 : src[v]);
                z[v] = src[v] < 0 ? make_float2(0.f, 0.f) : t;
            }
            dif_inverse<Q>(z, w, lane);
#pragma unroll
            for (int v = 0; v < V; ++v)
                R[v] = make_float2(U[v].x + z[v].x * u.inv_sqrt_ns, U[v].y + z[v].y * u.inv_sqrt_ns);
            if (it == u.amp_iters) break;
            // U = eta(R; nu) and the Onsager sum of eta'
            float dsum = 0.f;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const BgOut o = bg_eval(R[v].x * R[v].x + R[v].y * R[v].y, nu, u.log_odds, u.su2);
                U[v] = make_float2(o.gain * R[v].x, o.gain * R[v].y);
                dsum += o.deriv;
            }
            dsum = warp_sum(dsum);
            // T = y - A U + T / ns * sum eta'
            float2 X[V];
#pragma unroll
            for (int v = 0; v < V; ++v) X[v] = U[v];
            dit_forward<Q>(X, w, lane);
            float2 au = shfl2(X[0], r & 31);
            if (V == 2) {
                const float2 hi = shfl2(X[V - 1], r & 31);
                if (r >> 5) au = hi;
            }
            const float on = dsum * inv_ns;
            T = act ? make_float2(yv.x - au.x * u.inv_sqrt_ns + T.x * on, yv.y - au.y * u.inv_sqrt_ns + T.y * on)
                    : make_float2(0.f, 0.f);
        }
        // evidence at symbol bitrev(e)
        float* Sl = S + task * Q;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int a = (int)(__brev((unsigned)(lane + 32 * v)) >> (32 - LOGQ));
            Sl[a] = bg_eval(R[v].x * R[v].x + R[v].y * R[v].y, nu, u.log_odds, u.su2).logp;
        }
    }
}

// ---------------------------------------------------------------------------
// SIC row decoder
// ---------------------------------------------------------------------------

// Check update of one check of degree DC, in place (v2c in, c2v out), team
// shape: the edge carries x = h a; P_d = WHT of p~_d(x) = v2c_d(h_d^{-1} x);
// Q_d = product of the other P (prefix/suffix, no division); r_d = WHT(Q_d);
// c2v_d(a) = max(r_d(h_d a), kRelFloor max r_d) / max r_d.
template <int Q, int DC>
__device__ __forceinline__ void check_team_dc(float* blk, const uint8_t* coef, const uint8_t* gmul,
                                              const uint8_t* gdiv, TeamLane L)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V;
    float Pv[DC][V];
    int h[DC];
#pragma unroll
    for (int d = 0; d < DC; ++d) {
        h[d] = coef[d];
#pragma unroll
        for (int v = 0; v < V; ++v) Pv[d][v] = blk[d * Q + gdiv[h[d] * Q + v * T + L.tl]];
    }
#pragma unroll
    for (int d = 0; d < DC; ++d) wht_team<Q>(Pv[d], L);
    float R[DC][V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        float pre[DC + 1], suf[DC + 1];
        pre[0] = 1.0f;
        suf[DC] = 1.0f;
#pragma unroll
        for (int d = 0; d < DC; ++d) pre[d + 1] = pre[d] * Pv[d][v];
#pragma unroll
        for (int d = DC - 1; d >= 0; --d) suf[d] = suf[d + 1] * Pv[d][v];
#pragma unroll
        for (int d = 0; d < DC; ++d) R[d][v] = pre[d] * suf[d + 1];
    }
    __syncwarp(L.mask);
#pragma unroll
    for (int d = 0; d < DC; ++d) {
        wht_team<Q>(R[d], L);
        float lmx = R[d][0];
#pragma unroll
        for (int v = 1; v < V; ++v) lmx = fmaxf(lmx, R[d][v]);
        const float mx = team_max<T>(lmx, L.mask);
        const float fl = kRelFloor * mx, inv = 1.0f / mx;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int a = v * T + L.tl;
            const float r = team_gather<Q>(R[d], gmul[h[d] * Q + a], L);
            blk[d * Q + a] = fmaxf(r, fl) * inv;
        }
    }
}

// Team argmax with ties to the lowest symbol: (value, symbol) of this lane's
// best is merged across the team.
template <int T>
__device__ __forceinline__ int team_argmax(float val, int idx, unsigned mask)
{
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(mask, val, o, T);
        const int oi = __shfl_xor_sync(mask, idx, o, T);
        if (ov > val || (ov == val && oi < idx)) {
            val = ov;
            idx = oi;
        }
    }
    return idx;
}

}  // namespace

constexpr int kSicMaxWarps = 16;   // frames (warps) per CTA of the SIC kernel

// Shared memory of the SIC kernel: CTA tables, then one region per warp.
struct SicLayout {
    int tables;     // bytes: gf_mul, gf_div [Q*Q], coef [E], chk_var [E], var_edge [dv*n] (int16)
    int per_warp;   // bytes: msg [E*Q] + lambda [n*Q] floats, decisions [K*n]
};

static SicLayout sic_layout(const UraDev& u)
{
    const int E = u.P * u.dc;
    SicLayout s;
    int t = 2 * u.Q * u.Q + E;
    t = (t + 3) & ~3;
    t += 2 * E + 2 * u.dv * u.n;
    s.tables = (t + 15) & ~15;
    s.per_warp = 4 * (E + u.n) * u.Q + ((u.K * u.n + 15) & ~15);
    return s;
}

namespace {

template <int Q, int DC, int DV>
__global__ void __launch_bounds__(32 * kSicMaxWarps, 1) k_sic(UraDev u, SicLayout lay, int F, const float* __restrict__ S,
                                             uint8_t* __restrict__ hat, int32_t* __restrict__ iters,
                                             uint8_t* __restrict__ ok)
{
    constexpr int T = Shape<Q>::T, V = Shape<Q>::V, TPW = 32 / T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = u.n, P = u.P, E = P * DC, K = u.K;
    uint8_t* s_mul = smem;
    uint8_t* s_div = s_mul + Q * Q;
    uint8_t* s_coef = s_div + Q * Q;
    int16_t* s_cv = reinterpret_cast<int16_t*>(smem + ((2 * Q * Q + E + 3) & ~3));
    int16_t* s_ve = s_cv + E;
    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) {
        s_mul[i] = u.gf_mul[i];
        s_div[i] = u.gf_div[i];
    }
    for (int i = threadIdx.x; i < E; i += blockDim.x) {
        s_coef[i] = u.chk_coef[i];
        s_cv[i] = (int16_t)u.chk_var[i];
    }
    for (int i = threadIdx.x; i < DV * n; i += blockDim.x) s_ve[i] = (int16_t)u.var_edge[i];
    __syncthreads();

    const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* msg = reinterpret_cast<float*>(smem + lay.tables + warp * lay.per_warp);
    float* lam = msg + (size_t)E * Q;
    uint8_t* hs = reinterpret_cast<uint8_t*>(lam + (size_t)n * Q);
    const TeamLane L = team_lane<T>();
    const int team = lane / T;

    for (int f = blockIdx.x * W + warp; f < F; f += gridDim.x * W) {
        const float* Sf = S + (size_t)f * n * Q;
        for (int k = 0; k < K; ++k) {
            // local beliefs of row k: exp(S^(k) - max), floored; every edge starts as v2c = lambda
            for (int i = team; i < n; i += TPW) {
                float x[V];
                float mx = -__builtin_inff();
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int a = v * T + L.tl;
                    int cnt = 0;
                    for (int k2 = 0; k2 < k; ++k2) cnt += hs[k2 * n + i] == a;
                    x[v] = Sf[(size_t)i * Q + a] + u.cancel_log * (float)cnt;
                    mx = fmaxf(mx, x[v]);
                }
                mx = team_max<T>(mx, L.mask);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int a = v * T + L.tl;
                    const float lv = fmaxf(expf(x[v] - mx), kRelFloor);
                    lam[(size_t)i * Q + a] = lv;
#pragma unroll
                    for (int d = 0; d < DV; ++d) msg[(size_t)s_ve[DV * i + d] * Q + a] = lv;
                }
            }
            __syncwarp();
            int t_run = 0;
            bool sat = false;
            for (int t = 1; t <= u.bp_iters; ++t) {
                for (int j = team; j < P; j += TPW)
                    check_team_dc<Q, DC>(msg + (size_t)j * DC * Q, s_coef + j * DC, s_mul, s_div, L);
                __syncwarp();
                for (int i = team; i < n; i += TPW) {
                    // marginal lambda * prod_d c_d and, per edge d, v2c_d = lambda * prod_{d' != d} c_d'
                    int e[DV];
#pragma unroll
                    for (int d = 0; d < DV; ++d) e[d] = s_ve[DV * i + d];
                    float vo[DV][V], mo[DV];
#pragma unroll
                    for (int d = 0; d < DV; ++d) mo[d] = 0.0f;
                    float best = -1.0f;
                    int bi = 0;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int a = v * T + L.tl;
                        const float l = lam[(size_t)i * Q + a];
                        float c[DV];
#pragma unroll
                        for (int d = 0; d < DV; ++d) c[d] = msg[(size_t)e[d] * Q + a];
                        float b = l;
#pragma unroll
                        for (int d = 0; d < DV; ++d) b *= c[d];
                        if (b > best) {
                            best = b;
                            bi = a;
                        }
#pragma unroll
                        for (int d = 0; d < DV; ++d) {
                            float w = l;
#pragma unroll
                            for (int d2 = 0; d2 < DV; ++d2)
                                if (d2 != d) w *= c[d2];
                            vo[d][v] = w;
                            mo[d] = fmaxf(mo[d], w);
                        }
                    }
                    const int dec = team_argmax<T>(best, bi, L.mask);
#pragma unroll
                    for (int d = 0; d < DV; ++d) {
                        const float inv = 1.0f / team_max<T>(mo[d], L.mask);
#pragma unroll
                        for (int v = 0; v < V; ++v) msg[(size_t)e[d] * Q + v * T + L.tl] = vo[d][v] * inv;
                    }
                    if (L.tl == 0) hs[k * n + i] = (uint8_t)dec;
                }
                __syncwarp();
                bool unsat = false;
                for (int j = lane; j < P; j += 32) {
                    int s = 0;
#pragma unroll
                    for (int d = 0; d < DC; ++d) {
                        const int e = j * DC + d;
                        s ^= s_mul[s_coef[e] * Q + hs[k * n + s_cv[e]]];
                    }
                    unsat |= s != 0;
                }
                unsat = __any_sync(0xffffffffu, unsat);
                t_run = t;
                if (!unsat) {
                    sat = true;
                    if (u.early_stop) break;
                } else {
                    sat = false;
                }
            }
            uint8_t* hk = hat + ((size_t)f * K + k) * n;
            for (int i = lane; i < n; i += 32) hk[i] = hs[k * n + i];
            if (lane == 0) {
                iters[(size_t)f * K + k] = t_run;
                ok[(size_t)f * K + k] = sat ? 1 : 0;
            }
            __syncwarp();
        }
    }
}

template <int Q, int DC, int DV>
cudaError_t launch_sic_t(const UraDev& u, const DeviceInfo& di, int F, const float* S, uint8_t* hat,
                         int32_t* iters, uint8_t* ok, cudaStream_t s)
{
    const SicLayout lay = sic_layout(u);
    // per launch: the attribute belongs to the current device
    cudaError_t e = cudaFuncSetAttribute(k_sic<Q, DC, DV>, cudaFuncAttributeMaxDynamicSharedMemorySize, di.smem_optin);
    if (e != cudaSuccess) return e;
    // warps (frames) per CTA: the most resident warps per SM, no wider than the
    // batch needs to cover every SM once
    const int w_cap = (int)std::min<long>(kSicMaxWarps, std::max<long>(1, ((long)F + di.sm_count - 1) / di.sm_count));
    int W = 0, best = 0, per_sm_best = 0;
    for (int w = 1; w <= w_cap; ++w) {
        const int smem = lay.tables + w * lay.per_warp;
        if (smem > di.smem_optin) break;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sic<Q, DC, DV>, 32 * w, smem);
        if (e != cudaSuccess) return e;
        if (per_sm * w > best) {
            best = per_sm * w;
            W = w;
            per_sm_best = per_sm;
        }
    }
    if (W < 1 || per_sm_best < 1) return cudaErrorInvalidConfiguration;
    const int smem = lay.tables + W * lay.per_warp;
    const long need = ((long)F + W - 1) / W;
    const int grid = (int)std::min<long>(need, (long)per_sm_best * di.sm_count);
    k_sic<Q, DC, DV><<<grid, 32 * W, smem, s>>>(u, lay, F, S, hat, iters, ok);
    return cudaGetLastError();
}

template <int Q>
cudaError_t launch_amp_t(const UraDev& u, const DeviceInfo& di, int F, const float* y, float* S, cudaStream_t s)
{
    const long tasks = (long)F * u.n;
    const long need = (tasks + 7) / 8;   // 8 warps per CTA, one slot per warp
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_amp<Q>, 256, 0);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long>(need, (long)std::max(per_sm, 1) * di.sm_count);
    k_amp<Q><<<grid, 256, 0, s>>>(u, F, y, S);
    return cudaGetLastError();
}

// Row alignment of eq. (app_ura_hungarian): one warp per frame builds the K x K
// matrix of symbol mismatches between decoded row k and true row j, then scans
// all K! assignments in lexicographic order (Lehmer codes split across the
// lanes) and keeps the first one with the fewest mismatches; it reports that
// assignment's symbol errors and codeword (row) errors.  K <= 8.
constexpr int kMatchMaxK = 8;

__global__ void __launch_bounds__(256) k_match_rows(int F, int K, int n, const uint8_t* __restrict__ hat,
                                                    const uint8_t* __restrict__ truth, int32_t* sym_err,
                                                    int32_t* cw_err)
{
    __shared__ int cost_s[8][kMatchMaxK * kMatchMaxK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* cost = cost_s[warp];
    int fact = 1;
    for (int i = 2; i <= K; ++i) fact *= i;
    for (long f = (long)blockIdx.x * (blockDim.x >> 5) + warp; f < F; f += (long)gridDim.x * (blockDim.x >> 5)) {
        const uint8_t* h = hat + (size_t)f * K * n;
        const uint8_t* x = truth + (size_t)f * K * n;
        for (int pr = 0; pr < K * K; ++pr) {
            const int k = pr / K, j = pr % K;
            int c = 0;
            for (int i = lane; i < n; i += 32) c += h[(size_t)k * n + i] != x[(size_t)j * n + i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0) cost[pr] = c;
        }
        __syncwarp();
        int best = 0x7fffffff, best_r = 0x7fffffff;
        for (int r = lane; r < fact; r += 32) {
            // r-th permutation in lexicographic order (factorial number system)
            int avail = (1 << K) - 1, rem = r, sum = 0, div = fact;
            for (int k = 0; k < K; ++k) {
                div /= (K - k);
                int idx = rem / div;
                rem %= div;
                int j = 0;
                for (;; ++j)
                    if ((avail >> j) & 1) {
                        if (idx == 0) break;
                        --idx;
                    }
                avail &= ~(1 << j);
                sum += cost[k * K + j];
            }
            if (sum < best) {
                best = sum;
                best_r = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ob = __shfl_xor_sync(0xffffffffu, best, o), orr = __shfl_xor_sync(0xffffffffu, best_r, o);
            if (ob < best || (ob == best && orr < best_r)) {
                best = ob;
                best_r = orr;
            }
        }
        if (lane == 0) {
            int avail = (1 << K) - 1, rem = best_r, div = fact, cw = 0;
            for (int k = 0; k < K; ++k) {
                div /= (K - k);
                int idx = rem / div;
                rem %= div;
                int j = 0;
                for (;; ++j)
                    if ((avail >> j) & 1) {
                        if (idx == 0) break;
                        --idx;
                    }
                avail &= ~(1 << j);
                cw += cost[k * K + j] > 0;
            }
            sym_err[f] = best;
            cw_err[f] = cw;
        }
        __syncwarp();
    }
}

}  // namespace

int sic_warps_per_cta(const UraDev& u, const DeviceInfo& di)
{
    const SicLayout lay = sic_layout(u);
    const int room = di.smem_optin - lay.tables;
    if (room < lay.per_warp) return 0;
    return std::min(kSicMaxWarps, room / lay.per_warp);
}

cudaError_t launch_match_rows(const DeviceInfo& di, int F, int K, int n, const uint8_t* hat, const uint8_t* truth,
                              int32_t* sym_err, int32_t* cw_err, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    if (K < 1 || K > kMatchMaxK || n < 1) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long>(((long)F + 7) / 8, (long)di.sm_count * 8);
    k_match_rows<<<grid, 256, 0, s>>>(F, K, n, hat, truth, sym_err, cw_err);
    return cudaGetLastError();
}

cudaError_t launch_amp(const UraDev& u, const DeviceInfo& di, int F, const float* y, float* S, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    switch (u.Q) {
        case 32: return launch_amp_t<32>(u, di, F, y, S, s);
        case 64: return launch_amp_t<64>(u, di, F, y, S, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sic(const UraDev& u, const DeviceInfo& di, int F, const float* S, uint8_t* hat, int32_t* iters,
                       uint8_t* ok, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
#define JBP_SIC_CASE(QQ, DD, VV) \
    if (u.Q == QQ && u.dc == DD && u.dv == VV) return launch_sic_t<QQ, DD, VV>(u, di, F, S, hat, iters, ok, s);
    JBP_SIC_CASE(16, 3, 2) JBP_SIC_CASE(16, 4, 2) JBP_SIC_CASE(16, 6, 3)
    JBP_SIC_CASE(32, 3, 2) JBP_SIC_CASE(32, 4, 2) JBP_SIC_CASE(32, 6, 3)
    JBP_SIC_CASE(64, 3, 2) JBP_SIC_CASE(64, 4, 2) JBP_SIC_CASE(64, 6, 3)
#undef JBP_SIC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace jbp
