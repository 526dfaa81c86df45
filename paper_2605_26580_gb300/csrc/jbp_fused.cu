// jbp_fused.cu -- fused form: one persistent kernel runs all iterations of a
// group of frames with the whole message state in shared memory.
//
// A CTA owns G frames at a time.  Shared memory (per CTA):
//   msg  [G][K][P][cbs] f32   c2v / v2c (max 1) per check block, cbs = 4q + 4
//                             (the 16-byte pad spreads thread-shape accesses
//                             over the banks); updated in place
//   ch2v [G][K][n][q]   f32   channel messages
//   y    [G][n]         f32
//   scratch [teams][chan_scratch_floats] f32   (team-shape channel only)
//   hat  [G][K][n] u8, unsat [G][K] u8, active [G] u8, gf mul/div [q*q] u8
// Per iteration: (A) channel nodes + in-place v2c, (B) check nodes,
// (C) decisions, (D) syndromes, (E) per-frame stop; __syncthreads between.
// Global memory sees only y in and hat/iters/ok (and the optional log-posterior) out.
//
// Thread shape (q <= 16; channel also K <= 4 and variable degree 2): one thread
// per unit, vectors in registers.  Team shape otherwise.
#include <algorithm>

#include "jbp_internal.h"

namespace jbp {
namespace {

constexpr int kFusedMaxThreads = 256;
constexpr size_t kStaticSmemMargin = 256;   // static __shared__ words of k_fused

struct FusedLayout {
    size_t msg, ch2v, y, scratch, hat, unsat, active, gmul, gdiv, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline int fused_cbs(int Q) { return 4 * Q + 4; }

__host__ __device__ inline FusedLayout fused_layout(const Graph& g, int G, int teams, int scf)
{
    FusedLayout L;
    size_t o = 0;
    L.msg = o;     o = align16(o + sizeof(float) * (size_t)G * g.K * g.P * fused_cbs(g.Q));
    L.ch2v = o;    o = align16(o + sizeof(float) * (size_t)G * g.K * g.n * g.Q);
    L.y = o;       o = align16(o + sizeof(float) * (size_t)G * g.n);
    L.scratch = o; o = align16(o + sizeof(float) * (size_t)teams * scf);
    L.hat = o;     o = align16(o + (size_t)G * g.K * g.n);
    L.unsat = o;   o = align16(o + (size_t)G * g.K);
    L.active = o;  o = align16(o + (size_t)G);
    L.gmul = o;    o = align16(o + (size_t)g.Q * g.Q);
    L.gdiv = o;    o = align16(o + (size_t)g.Q * g.Q);
    L.total = o;
    return L;
}

// KC > 0: thread-shape channel with KC users; KC == 0: team-shape channel.
template <int Q, int KC>
__global__ void __launch_bounds__(kFusedMaxThreads) k_fused(Graph g, int F, int G, const float* __restrict__ y,
                                                            int T_it, int early_stop, uint8_t* hat,
                                                            int32_t* iters, uint8_t* ok, float* logpost, int scf)
{
    constexpr int T = Shape<Q>::T;
    constexpr bool kThreadCheck = Q <= 16;
    extern __shared__ __align__(16) unsigned char sm[];
    const int teams = blockDim.x / T, team = threadIdx.x / T;
    const FusedLayout lay = fused_layout(g, G, KC > 0 ? 0 : teams, scf);
    const int cbs = fused_cbs(Q);
    float* s_msg = reinterpret_cast<float*>(sm + lay.msg);
    float* s_ch2v = reinterpret_cast<float*>(sm + lay.ch2v);
    float* s_y = reinterpret_cast<float*>(sm + lay.y);
    float* sc = reinterpret_cast<float*>(sm + lay.scratch) + (size_t)team * scf;
    float* res = sc + scf - g.K * Q;
    uint8_t* s_hat = sm + lay.hat;
    uint8_t* s_unsat = sm + lay.unsat;
    uint8_t* s_active = sm + lay.active;
    uint8_t* s_mul = sm + lay.gmul;
    uint8_t* s_div = sm + lay.gdiv;
    __shared__ int s_nactive;

    const TeamLane L = team_lane<T>();
    const int K = g.K, n = g.n, P = g.P;
    const size_t us = (size_t)P * cbs, fs = (size_t)K * us, vs = (size_t)K * n * Q;

    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) {
        s_mul[i] = g.gf_mul[i];
        s_div[i] = g.gf_div[i];
    }
    if constexpr (KC == 0) blk_clear<T>(sc, scf, L);

    const int groups = (F + G - 1) / G;
    for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
        const int f0 = grp * G, gc = min(G, F - f0);
        // uniform c2v messages (all ones), y, control words
        for (size_t i = threadIdx.x; i < (size_t)gc * fs; i += blockDim.x) s_msg[i] = 1.0f;
        for (int i = threadIdx.x; i < gc * n; i += blockDim.x) s_y[i] = y[(size_t)f0 * n + i];
        for (int i = threadIdx.x; i < gc * K; i += blockDim.x) s_unsat[i] = 0;
        for (int i = threadIdx.x; i < G; i += blockDim.x) s_active[i] = i < gc ? 1 : 0;
        __syncthreads();

        for (int t = 1; t <= T_it; ++t) {
            // (A) channel nodes, v2c in place
            if constexpr (KC > 0) {
                for (int unit = threadIdx.x; unit < gc * n; unit += blockDim.x) {
                    const int gi = unit / n, u = unit % n;
                    if (!s_active[gi]) continue;
                    chan_thread<KC, Q>(g, s_msg + gi * fs, us, cbs, s_ch2v + gi * vs, s_y[gi * n + u],
                                       frame_inv_s2(g, f0 + gi), u);
                }
            } else {
                for (int unit = team; unit < gc * n; unit += teams) {
                    const int gi = unit / n, u = unit % n;
                    if (!s_active[gi]) continue;
                    float* msg_f = s_msg + gi * fs;
                    const float yv = s_y[gi * n + u], is2 = frame_inv_s2(g, f0 + gi);
                    if (chan_blocked<Q>(g, msg_f, us, cbs, yv, is2, u, sc, res, L)) {
                        if (g.log_fallbacks && L.tl == 0) atomicAdd(g.log_fallbacks, 1ull);
                        chan_trellis<Q, LogSR>(g, msg_f, us, cbs, yv, is2, u, sc, res, L);
                        blk_clear<T>(sc, scf - K * Q, L);
                    }
                    chan_write_team<Q>(g, msg_f, us, cbs, s_ch2v + gi * vs, res, u, L);
                }
            }
            __syncthreads();
            // (B) check nodes
            if constexpr (kThreadCheck) {
                for (int unit = threadIdx.x; unit < gc * K * P; unit += blockDim.x) {
                    const int gi = unit / (K * P), j = unit % P;
                    if (!s_active[gi]) continue;
                    check_thread<Q>(s_msg + (size_t)unit * cbs, g.chk_coef + 4 * j, s_div);
                }
            } else {
                for (int unit = team; unit < gc * K * P; unit += teams) {
                    const int gi = unit / (K * P), j = unit % P;
                    if (!s_active[gi]) continue;
                    check_team<Q>(s_msg + (size_t)unit * cbs, g.chk_coef + 4 * j, s_mul, s_div, L);
                }
            }
            __syncthreads();
            // (C) posterior and decisions
            if constexpr (kThreadCheck) {
                for (int unit = threadIdx.x; unit < gc * K * n; unit += blockDim.x) {
                    const int gi = unit / (K * n), rem = unit % (K * n), k = rem / n, i = rem % n;
                    if (!s_active[gi]) continue;
                    const size_t fk = (size_t)gi * K + k;
                    float* lp = logpost ? logpost + ((size_t)(f0 + gi) * K + k) * n * Q : nullptr;
                    var_thread<Q>(g, s_ch2v + fk * n * Q, s_msg + fk * us, cbs, i, lp, s_hat + fk * n);
                }
            } else {
                for (int unit = team; unit < gc * K * n; unit += teams) {
                    const int gi = unit / (K * n), rem = unit % (K * n), k = rem / n, i = rem % n;
                    if (!s_active[gi]) continue;
                    const size_t fk = (size_t)gi * K + k;
                    float* lp = logpost ? logpost + ((size_t)(f0 + gi) * K + k) * n * Q : nullptr;
                    var_team<Q>(g, s_ch2v + fk * n * Q, s_msg + fk * us, cbs, i, lp, s_hat + fk * n, L);
                }
            }
            __syncthreads();
            // (D) syndromes
            for (int w = threadIdx.x; w < gc * K * P; w += blockDim.x) {
                const int gi = w / (K * P), rem = w % (K * P), k = rem / P, j = rem % P;
                if (!s_active[gi]) continue;
                if (!check_satisfied(g, s_hat + ((size_t)gi * K + k) * n, j, s_mul)) s_unsat[gi * K + k] = 1;
            }
            if (threadIdx.x == 0) s_nactive = 0;
            __syncthreads();
            // (E) per-frame stop
            for (int gi = threadIdx.x; gi < gc; gi += blockDim.x) {
                if (!s_active[gi]) continue;
                bool all = true;
                for (int k = 0; k < K; ++k) {
                    const bool okk = s_unsat[gi * K + k] == 0;
                    ok[(size_t)(f0 + gi) * K + k] = okk ? 1 : 0;
                    s_unsat[gi * K + k] = 0;
                    all = all && okk;
                }
                iters[f0 + gi] = t;
                if (early_stop && all) s_active[gi] = 0;
                else atomicAdd(&s_nactive, 1);
            }
            __syncthreads();
            if (s_nactive == 0) break;
        }
        for (int i = threadIdx.x; i < gc * K * n; i += blockDim.x) hat[(size_t)f0 * K * n + i] = s_hat[i];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Position-major fused kernel (thread shape: q <= 16, K <= 4, dv = 2)
// ---------------------------------------------------------------------------
//
// Shared memory per CTA (NB = ceil(n/32), every q-vector interleaved over 32
// positions, see jbp_device.cuh):
//   msg  [G][K*NB*2][q][32] f32   c2v / v2c of each variable's two edges, in place
//   ch2v [G][K*NB][q][32]   f32
//   y    [G][NB*32] f32, hat [G][K][NB*32] u8 (position order), unsat [G][K], active [G]
//   rec  [K*P] uint4, recb [K*P] uint2: one record per check unit in the order
//        the check phase runs them (CheckRec), gf mul [q*q] u8 (shared by the G frames)
// Phase A reads and writes consecutive banks; phase B gathers each check's
// four edges through its record (the only irregular access of an iteration).

struct PosLayout {
    size_t msg, ch2v, y, hat, unsat, active, rec, recb, gmul, total;
};

__host__ __device__ inline PosLayout pos_layout(const Graph& g, int G)
{
    const size_t NB = (size_t)(g.n + 31) / 32;
    PosLayout L;
    size_t o = 0;
    L.msg = o;    o = align16(o + sizeof(float) * (size_t)G * g.K * NB * 2 * g.Q * 32);
    L.ch2v = o;   o = align16(o + sizeof(float) * (size_t)G * g.K * NB * g.Q * 32);
    L.y = o;      o = align16(o + sizeof(float) * (size_t)G * NB * 32);
    L.hat = o;    o = align16(o + (size_t)G * g.K * NB * 32);
    L.unsat = o;  o = align16(o + (size_t)G * g.K);
    L.active = o; o = align16(o + (size_t)G);
    L.rec = o;    o = align16(o + sizeof(uint4) * (size_t)g.K * g.P);
    L.recb = o;   o = align16(o + sizeof(uint2) * (size_t)g.K * g.P);
    L.gmul = o;   o = align16(o + (size_t)g.Q * g.Q);
    L.total = o;
    return L;
}

// PAIR (K = 4 only): each channel use split over a lane pair, up to 512 threads
// (128 registers); otherwise one thread per channel use, up to 256 threads.
template <int Q, int KC, bool PAIR>
constexpr int pos_max_threads() { return PAIR ? 512 : kFusedMaxThreads; }

// POOL: serving-pool mode (FusedPool): G = 1, frame f0 is pool
// slot f0, iterations t0 + 1 .. min(t0 + pool.block, T_it) with t0 = iters[f0],
// state loaded from and stored to the pool, the unfolded phase order.
template <int Q, int KC, bool PAIR = false, bool POOL = false>
__global__ void __launch_bounds__(pos_max_threads<Q, KC, PAIR>()) k_fused_pos(Graph g, int F, int G, const float* __restrict__ y,
                                                                int T_it, int early_stop, uint8_t* hat,
                                                                int32_t* iters, uint8_t* ok, float* logpost,
                                                                FusedPool pool)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const PosLayout lay = pos_layout(g, G);
    const int n = g.n, P = g.P, E = g.E, NB = (n + 31) / 32;
    constexpr int K = KC;
    float* s_msg = reinterpret_cast<float*>(sm + lay.msg);
    float* s_ch2v = reinterpret_cast<float*>(sm + lay.ch2v);
    float* s_y = reinterpret_cast<float*>(sm + lay.y);
    uint8_t* s_hat = sm + lay.hat;
    uint8_t* s_unsat = sm + lay.unsat;
    uint8_t* s_active = sm + lay.active;
    uint4* s_rec = reinterpret_cast<uint4*>(sm + lay.rec);
    uint2* s_recb = reinterpret_cast<uint2*>(sm + lay.recb);
    uint8_t* s_mul = sm + lay.gmul;
    __shared__ int s_nactive;

    const size_t fs = (size_t)K * NB * 2 * Q * 32, vs = (size_t)K * NB * Q * 32, hs = (size_t)K * NB * 32;
    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) s_mul[i] = g.gf_mul[i];
    for (int i = threadIdx.x; i < K * P; i += blockDim.x) {
        const int u = g.chk_order ? g.chk_order[i] : i;
        const CheckRec r = check_rec<Q>(g, NB, u / P, u % P);
        s_rec[i] = r.off;
        s_recb[i] = r.basis;
    }

    constexpr bool in_pool = POOL;
    // a pool slot's state between shared memory and HBM (16-byte words)
    auto pool_state = [&](int f, bool load) {
        float4* gm = reinterpret_cast<float4*>(pool.msg + (size_t)f * fs);
        float4* gv = reinterpret_cast<float4*>(pool.ch2v + (size_t)f * vs);
        float4* sm4 = reinterpret_cast<float4*>(s_msg);
        float4* sv4 = reinterpret_cast<float4*>(s_ch2v);
        for (size_t i = threadIdx.x; i < fs / 4; i += blockDim.x) {
            if (load) sm4[i] = gm[i];
            else gm[i] = sm4[i];
        }
        for (size_t i = threadIdx.x; i < vs / 4; i += blockDim.x) {
            if (load) sv4[i] = gv[i];
            else gv[i] = sv4[i];
        }
    };

    const int groups = (F + G - 1) / G;
    for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
        const int f0 = grp * G, gc = min(G, F - f0);
        int t0 = 0, t_end = T_it;
        if constexpr (POOL) {
            if (!pool.active[f0]) continue;   // uniform across the CTA
            t0 = iters[f0];
            t_end = min(T_it, t0 + pool.block);
        }
        if (POOL && t0 > 0) pool_state(f0, true);
        else
            for (size_t i = threadIdx.x; i < (size_t)gc * fs; i += blockDim.x) s_msg[i] = 1.0f;
        for (int i = threadIdx.x; i < gc * n; i += blockDim.x) s_y[(i / n) * NB * 32 + i % n] = y[(size_t)f0 * n + i];
        for (int i = threadIdx.x; i < gc * K; i += blockDim.x) s_unsat[i] = 0;
        for (int i = threadIdx.x; i < G; i += blockDim.x) s_active[i] = i < gc ? 1 : 0;
        __syncthreads();

        // Without a log-posterior output the decision phase of iteration t is
        // folded into the channel phase of iteration t + 1 (which loads the same
        // messages), and its syndromes and stop test run between that channel
        // phase and the next check phase; a final pass decides after the last
        // iteration.
        const bool fold = logpost == nullptr && !in_pool;
        auto phase_decide = [&]() {
            for (int unit = threadIdx.x; unit < gc * K * n; unit += blockDim.x) {
                const int gi = unit / (K * n), rem = unit % (K * n), k = rem / n, p = rem % n;
                if (!s_active[gi]) continue;
                float* lp = nullptr;
                if (logpost) lp = logpost + (((size_t)(f0 + gi) * K + k) * n + g.use_pos[k * n + p]) * Q;
                s_hat[gi * hs + k * NB * 32 + p] = (uint8_t)var_thread_pos<Q>(s_msg + gi * fs, s_ch2v + gi * vs,
                                                                              NB, k, p, lp);
            }
        };
        // syndrome of the check unit with record r in frame gi (eq. app_ldpc_check_eq)
        auto unit_syndrome = [&](int gi, const uint4& r) {
            const uint8_t* hf = s_hat + gi * hs;
            const unsigned o[kDC] = {r.x, r.y, r.z, r.w};
            int sy = 0;
#pragma unroll
            for (int d = 0; d < kDC; ++d) sy ^= s_mul[rec_coef(o[d]) * Q + hf[rec_hat<Q>(o[d], NB)]];
            if (sy) s_unsat[gi * K + rec_user<Q>(o[0], NB)] = 1;
        };
        // per-frame stop after iteration t (syndromes already recorded); returns the frames still active
        auto phase_finish = [&](int t) {
            if (threadIdx.x == 0) s_nactive = 0;
            __syncthreads();
            for (int gi = threadIdx.x; gi < gc; gi += blockDim.x) {
                if (!s_active[gi]) continue;
                bool all = true;
                for (int k = 0; k < K; ++k) {
                    const bool okk = s_unsat[gi * K + k] == 0;
                    ok[(size_t)(f0 + gi) * K + k] = okk ? 1 : 0;
                    s_unsat[gi * K + k] = 0;
                    all = all && okk;
                }
                iters[f0 + gi] = t;
                if (early_stop && all) s_active[gi] = 0;
                else atomicAdd(&s_nactive, 1);
            }
            __syncthreads();
            return s_nactive;
        };
        // A thread's units are u, u + step, ... over gc frames of `per` units each:
        // (frame, index) pairs formed and advanced by subtraction (a thread's first
        // unit lies in the first frame or close to it), not by a division per unit.
        auto advance = [](int step, int per, int& gi, int& i) {
            i += step;
            while (i >= per) {
                i -= per;
                ++gi;
            }
        };
        const int KP = K * P;
        auto phase_stop = [&](int t) {
            int gi0 = 0, i0 = 0;
            advance(threadIdx.x, KP, gi0, i0);
            for (int gi = gi0, i = i0; gi < gc; advance(blockDim.x, KP, gi, i)) {
                if (!s_active[gi]) continue;
                unit_syndrome(gi, s_rec[i]);
            }
            return phase_finish(t);
        };
        bool all_stopped = false;
        for (int t = t0 + 1; t <= t_end; ++t) {
            // (A) channel nodes, v2c in place (and, folded, the decisions of iteration t - 1)
            const bool dec = fold && t > 1;
            if constexpr (PAIR && K == 4) {
                const int half = threadIdx.x & 1;
                const unsigned pmask = 3u << (threadIdx.x & 30);
                int gi0 = 0, p0 = 0;
                advance(threadIdx.x >> 1, n, gi0, p0);
                for (int gi = gi0, p = p0; gi < gc; advance(blockDim.x >> 1, n, gi, p)) {
                    if (!s_active[gi]) continue;
                    chan_pair_pos<Q>(g, s_msg + gi * fs, s_ch2v + gi * vs, NB, s_y[gi * NB * 32 + p],
                                     frame_inv_s2(g, f0 + gi), p, half, pmask, dec ? s_hat + gi * hs : nullptr);
                }
            } else {
                int gi0 = 0, p0 = 0;
                advance(threadIdx.x, n, gi0, p0);
                for (int gi = gi0, p = p0; gi < gc; advance(blockDim.x, n, gi, p)) {
                    if (!s_active[gi]) continue;
                    chan_thread_pos<K, Q>(g, s_msg + gi * fs, s_ch2v + gi * vs, NB, s_y[gi * NB * 32 + p],
                                          frame_inv_s2(g, f0 + gi), p, dec ? s_hat + gi * hs : nullptr);
                }
            }
            __syncthreads();
            // (B) check nodes, in the bank-spreading order of chk_order; folded, each
            // unit also tests its check against the decisions of iteration t - 1
            const bool syn = fold && t > 1;
            int cg0 = 0, ci0 = 0;
            advance(threadIdx.x, KP, cg0, ci0);
            for (int gi = cg0, i = ci0; gi < gc; advance(blockDim.x, KP, gi, i)) {
                if (!s_active[gi]) continue;
                const uint4 r = s_rec[i];
                if (syn) unit_syndrome(gi, r);
                check_thread_rec<Q>(s_msg + gi * fs, r, s_recb[i]);
            }
            __syncthreads();
            if (syn && phase_finish(t - 1) == 0) {
                all_stopped = true;
                break;
            }
            if (!fold) {
                // (C) posterior and decisions (position order), (D) syndromes, (E) per-frame stop
                phase_decide();
                __syncthreads();
                if (phase_stop(t) == 0) {
                    all_stopped = true;
                    break;
                }
            }
        }
        if (fold && !all_stopped) {
            // decisions, syndromes and stop of the last iteration
            phase_decide();
            __syncthreads();
            phase_stop(T_it);
        }
        if (POOL && !all_stopped && t_end < T_it) {
            // the slot goes on in a later block: keep its state
            pool_state(f0, false);
            __syncthreads();
            continue;
        }
        if (POOL && threadIdx.x == 0) {
            pool.active[f0] = 0;
            pool.fin[f0] = 1;
        }
        // decisions back to variable order
        for (int w = threadIdx.x; w < gc * K * n; w += blockDim.x) {
            const int gi = w / (K * n), rem = w % (K * n), k = rem / n, i = rem % n;
            hat[(size_t)f0 * K * n + w] = s_hat[gi * hs + k * NB * 32 + g.pos_of[k * n + i]];
        }
        __syncthreads();
    }
}

template <int Q, int KC, bool PAIR>
bool plan_pos_v(const Graph& g, const DeviceInfo& di, int F, int threads, int fpc_hint, FusedPlan* plan)
{
    int Gmax = 0;
    for (int G = 1; G <= 4096; ++G) {
        if (pos_layout(g, G).total + kStaticSmemMargin > (size_t)di.smem_optin) break;
        Gmax = G;
    }
    if (Gmax == 0) return false;
    int G = fpc_hint > 0 ? std::min(fpc_hint, Gmax) : Gmax;
    G = std::max(1, std::min(G, (F + di.sm_count - 1) / di.sm_count));
    plan->frames_per_cta = G;
    plan->threads = threads;
    plan->smem_bytes = (int)pos_layout(g, G).total;
    plan->variant = PAIR ? 1 : 0;
    int occ = 0;
    if (cudaFuncSetAttribute(k_fused_pos<Q, KC, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             plan->smem_bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_pos<Q, KC, PAIR>, threads, plan->smem_bytes) !=
            cudaSuccess ||
        occ < 1)
        return false;
    plan->grid = std::max(1, std::min((F + G - 1) / G, di.sm_count * occ));
    return true;
}

// Launch shape: threads_hint > 256 selects the lane-pair channel (K = 4); the
// default is one thread per channel use at 256 threads.
template <int Q, int KC>
bool plan_pos(const Graph& g, const DeviceInfo& di, int F, int threads_hint, int fpc_hint, FusedPlan* plan)
{
    int threads = threads_hint > 0 ? threads_hint : kFusedMaxThreads;
    threads = std::max(64, std::min(512, threads / 64 * 64));
    if constexpr (KC == 4) {
        if (threads > kFusedMaxThreads) return plan_pos_v<Q, KC, true>(g, di, F, threads, fpc_hint, plan);
    }
    return plan_pos_v<Q, KC, false>(g, di, F, std::min(threads, kFusedMaxThreads), fpc_hint, plan);
}

template <int Q, int KC, bool PAIR>
cudaError_t fused_pos_v(const Graph& g, const FusedPlan& p, int F, const float* y, int T_it, int early_stop,
                        uint8_t* hat, int32_t* iters, uint8_t* ok, float* post, cudaStream_t s,
                        const FusedPool& pool = FusedPool())
{
    if (pool.msg) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_pos<Q, KC, PAIR, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes);
        if (e != cudaSuccess) return e;
        k_fused_pos<Q, KC, PAIR, true><<<p.grid, p.threads, p.smem_bytes, s>>>(g, F, 1, y, T_it, early_stop, hat,
                                                                                iters, ok, nullptr, pool);
        return cudaGetLastError();
    }
    cudaError_t e =
        cudaFuncSetAttribute(k_fused_pos<Q, KC, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes);
    if (e != cudaSuccess) return e;
    k_fused_pos<Q, KC, PAIR><<<p.grid, p.threads, p.smem_bytes, s>>>(g, F, p.frames_per_cta, y, T_it, early_stop,
                                                                      hat, iters, ok, post, pool);
    return cudaGetLastError();
}

template <int Q, int KC>
cudaError_t fused_pos(const Graph& g, const FusedPlan& p, int F, const float* y, int T_it, int early_stop,
                      uint8_t* hat, int32_t* iters, uint8_t* ok, float* post, cudaStream_t s,
                      const FusedPool& pool = FusedPool())
{
    if constexpr (KC == 4) {
        if (p.variant == 1)
            return fused_pos_v<Q, KC, true>(g, p, F, y, T_it, early_stop, hat, iters, ok, post, s, pool);
    }
    return fused_pos_v<Q, KC, false>(g, p, F, y, T_it, early_stop, hat, iters, ok, post, s, pool);
}

template <int Q, int KC>
bool plan_qk(const Graph& g, const DeviceInfo& di, int F, int threads_hint, int fpc_hint, FusedPlan* plan)
{
    constexpr int T = Shape<Q>::T;
    const int scf = blk_scratch_floats(g.K, Q);
    int threads = threads_hint > 0 ? threads_hint : 256;
    threads = std::max(32, std::min(kFusedMaxThreads, threads / 32 * 32));
    for (; threads >= 32; threads -= 32) {
        const int teams = KC > 0 ? 0 : threads / T;
        int Gmax = 0;
        for (int G = 1; G <= 4096; ++G) {
            if (fused_layout(g, G, teams, scf).total + kStaticSmemMargin > (size_t)di.smem_optin) break;
            Gmax = G;
        }
        if (Gmax == 0) continue;
        int G = fpc_hint > 0 ? std::min(fpc_hint, Gmax) : Gmax;
        // keep every SM busy: no more frames per CTA than F / SMs (at least 1)
        G = std::max(1, std::min(G, (F + di.sm_count - 1) / di.sm_count));
        plan->frames_per_cta = G;
        plan->threads = threads;
        plan->smem_bytes = (int)fused_layout(g, G, teams, scf).total;
        const int groups = (F + G - 1) / G;
        int occ = 0;
        if (cudaFuncSetAttribute(k_fused<Q, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem_bytes) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused<Q, KC>, threads, plan->smem_bytes) !=
                cudaSuccess ||
            occ < 1)
            return false;
        plan->grid = std::max(1, std::min(groups, di.sm_count * occ));
        return true;
    }
    return false;
}

template <int Q, int KC>
cudaError_t fused_qk(const Graph& g, const FusedPlan& p, int F, const float* y, int T_it, int early_stop, uint8_t* hat,
                     int32_t* iters, uint8_t* ok, float* post, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_fused<Q, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes);
    if (e != cudaSuccess) return e;
    k_fused<Q, KC><<<p.grid, p.threads, p.smem_bytes, s>>>(g, F, p.frames_per_cta, y, T_it, early_stop, hat, iters,
                                                            ok, post, blk_scratch_floats(g.K, Q));
    return cudaGetLastError();
}

// Which k_fused<Q, KC> instance serves this graph.
inline int fused_kc(const Graph& g)
{
    return (g.Q <= 16 && g.dv == 2 && g.K <= 4 && g.n <= 32767 && g.slot && g.pos_of) ? g.K : 0;
}

}  // namespace

#define JBP_FUSED_DISPATCH(FN_POS, FN_TEAM, ...)                                     \
    do {                                                                             \
        const int kc = fused_kc(g);                                                  \
        switch (g.Q * 8 + kc) {                                                      \
            case 2 * 8 + 0: return FN_TEAM<2, 0>(__VA_ARGS__);                       \
            case 2 * 8 + 1: return FN_POS<2, 1>(__VA_ARGS__);                        \
            case 2 * 8 + 2: return FN_POS<2, 2>(__VA_ARGS__);                        \
            case 2 * 8 + 3: return FN_POS<2, 3>(__VA_ARGS__);                        \
            case 2 * 8 + 4: return FN_POS<2, 4>(__VA_ARGS__);                        \
            case 4 * 8 + 0: return FN_TEAM<4, 0>(__VA_ARGS__);                       \
            case 4 * 8 + 1: return FN_POS<4, 1>(__VA_ARGS__);                        \
            case 4 * 8 + 2: return FN_POS<4, 2>(__VA_ARGS__);                        \
            case 4 * 8 + 3: return FN_POS<4, 3>(__VA_ARGS__);                        \
            case 4 * 8 + 4: return FN_POS<4, 4>(__VA_ARGS__);                        \
            case 8 * 8 + 0: return FN_TEAM<8, 0>(__VA_ARGS__);                       \
            case 8 * 8 + 1: return FN_POS<8, 1>(__VA_ARGS__);                        \
            case 8 * 8 + 2: return FN_POS<8, 2>(__VA_ARGS__);                        \
            case 8 * 8 + 3: return FN_POS<8, 3>(__VA_ARGS__);                        \
            case 8 * 8 + 4: return FN_POS<8, 4>(__VA_ARGS__);                        \
            case 16 * 8 + 0: return FN_TEAM<16, 0>(__VA_ARGS__);                     \
            case 16 * 8 + 1: return FN_POS<16, 1>(__VA_ARGS__);                      \
            case 16 * 8 + 2: return FN_POS<16, 2>(__VA_ARGS__);                      \
            case 16 * 8 + 3: return FN_POS<16, 3>(__VA_ARGS__);                      \
            case 16 * 8 + 4: return FN_POS<16, 4>(__VA_ARGS__);                      \
            case 32 * 8 + 0: return FN_TEAM<32, 0>(__VA_ARGS__);                     \
            case 64 * 8 + 0: return FN_TEAM<64, 0>(__VA_ARGS__);                     \
            default: break;                                                          \
        }                                                                            \
    } while (0)

bool fused_plan(const Graph& g, const DeviceInfo& di, int F, int threads_hint, int fpc_hint, FusedPlan* plan)
{
    if (g.dc != kDC || F <= 0) return false;
    JBP_FUSED_DISPATCH(plan_pos, plan_qk, g, di, F, threads_hint, fpc_hint, plan);
    return false;
}

cudaError_t launch_fused(const Graph& g, const FusedPlan& plan, int F, const float* y, int T_it, int early_stop,
                         uint8_t* hat, int32_t* iters, uint8_t* ok, float* post, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    JBP_FUSED_DISPATCH(fused_pos, fused_qk, g, plan, F, y, T_it, early_stop, hat, iters, ok, post, s);
    return cudaErrorInvalidValue;
}

#define JBP_POS_DISPATCH(FN, ...)                                                    \
    switch (g.Q * 8 + fused_kc(g)) {                                                 \
        case 2 * 8 + 1: return FN<2, 1>(__VA_ARGS__);                                \
        case 2 * 8 + 2: return FN<2, 2>(__VA_ARGS__);                                \
        case 2 * 8 + 3: return FN<2, 3>(__VA_ARGS__);                                \
        case 2 * 8 + 4: return FN<2, 4>(__VA_ARGS__);                                \
        case 4 * 8 + 1: return FN<4, 1>(__VA_ARGS__);                                \
        case 4 * 8 + 2: return FN<4, 2>(__VA_ARGS__);                                \
        case 4 * 8 + 3: return FN<4, 3>(__VA_ARGS__);                                \
        case 4 * 8 + 4: return FN<4, 4>(__VA_ARGS__);                                \
        case 8 * 8 + 1: return FN<8, 1>(__VA_ARGS__);                                \
        case 8 * 8 + 2: return FN<8, 2>(__VA_ARGS__);                                \
        case 8 * 8 + 3: return FN<8, 3>(__VA_ARGS__);                                \
        case 8 * 8 + 4: return FN<8, 4>(__VA_ARGS__);                                \
        case 16 * 8 + 1: return FN<16, 1>(__VA_ARGS__);                              \
        case 16 * 8 + 2: return FN<16, 2>(__VA_ARGS__);                              \
        case 16 * 8 + 3: return FN<16, 3>(__VA_ARGS__);                              \
        case 16 * 8 + 4: return FN<16, 4>(__VA_ARGS__);                              \
        default: break;                                                              \
    }

bool fused_pool_plan(const Graph& g, const DeviceInfo& di, int cap, int threads_hint, FusedPlan* plan,
                     size_t* msg_floats, size_t* ch2v_floats)
{
    if (g.dc != kDC || cap <= 0 || fused_kc(g) == 0) return false;
    const size_t NB = (size_t)(g.n + 31) / 32;
    *msg_floats = (size_t)g.K * NB * 2 * g.Q * 32;
    *ch2v_floats = (size_t)g.K * NB * g.Q * 32;
    JBP_POS_DISPATCH(plan_pos, g, di, cap, threads_hint, 1, plan);
    return false;
}

cudaError_t launch_fused_pool(const Graph& g, const FusedPlan& plan, int F, const float* y, int T, int early_stop,
                              uint8_t* hat, int32_t* t, uint8_t* ok, const FusedPool& pool, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    if (plan.frames_per_cta != 1 || !pool.msg || pool.block < 1) return cudaErrorInvalidValue;
    FusedPlan p = plan;
    p.grid = std::min(plan.grid, F);
    JBP_POS_DISPATCH(fused_pos, g, p, F, y, T, early_stop, hat, t, ok, nullptr, s, pool);
    return cudaErrorInvalidValue;
}

}  // namespace jbp
