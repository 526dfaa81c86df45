// jbp_step.cu -- step form: one kernel per node type per iteration, message
// state resident in HBM.
//
// HBM layout per frame f (frame-major, q contiguous, cbs = 4q):
//   msg  [K][E][q]  FP32 messages (max 1) on check-major edges: c2v, or v2c
//                   between the channel and check steps (updated in place)
//   ch2v [K][n][q]  FP32 channel messages (max 1)
// Each kernel is a persistent grid-stride loop over units with a grid sized to
// fill every SM at the occupancy the block shape allows.
#include <algorithm>

#include "jbp_internal.h"

namespace jbp {
namespace {

constexpr int kStepThreads = 256;

template <class Kern>
int persistent_grid(Kern kern, int threads, size_t smem, const DeviceInfo& di, long units_per_block, long units)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess || occ < 1) occ = 1;
    long need = (units + units_per_block - 1) / units_per_block;
    long cap = (long)di.sm_count * occ;
    return (int)std::max(1L, std::min(need, cap));
}

template <int Q>
__device__ __forceinline__ void load_gf(const Graph& g, uint8_t* smul, uint8_t* sdiv)
{
    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) {
        smul[i] = g.gf_mul[i];
        sdiv[i] = g.gf_div[i];
    }
    __syncthreads();
}

// (a) channel node + in-place v2c, thread shape: one thread per (frame, channel use).
template <int Q, int KC>
__global__ void __launch_bounds__(kStepThreads) k_channel_thread(Graph g, int F, const float* __restrict__ y,
                                                                 float* msg, float* ch2v,
                                                                 const uint8_t* __restrict__ active)
{
    const long total = (long)F * g.n;
    const size_t us = (size_t)g.E * Q, fs = (size_t)KC * us, vs = (size_t)KC * g.n * Q;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int f = (int)(t / g.n), u = (int)(t % g.n);
        if (active && !active[f]) continue;
        chan_thread<KC, Q>(g, msg + f * fs, us, 4 * Q, ch2v + f * vs, y[(size_t)f * g.n + u], frame_inv_s2(g, f), u);
    }
}

// (a) team shape: T lanes per (frame, channel use), trellis in shared scratch.
// FIX: only the channel uses that the tensor-core channel node left to the
// trellis (a NaN in the first entry of user 0's channel message).
template <int Q, bool FIX = false>
__global__ void __launch_bounds__(kStepThreads) k_channel_team(Graph g, int F, const float* __restrict__ y,
                                                               float* msg, float* ch2v,
                                                               const uint8_t* __restrict__ active, int sc_floats)
{
    constexpr int T = Shape<Q>::T;
    extern __shared__ float smem[];
    const int teams = blockDim.x / T, team = threadIdx.x / T;
    float* sc = smem + (size_t)team * sc_floats;
    float* res = sc + sc_floats - g.K * Q;
    const TeamLane L = team_lane<T>();
    const long total = (long)F * g.n;
    const size_t us = (size_t)g.E * Q, fs = (size_t)g.K * us, vs = (size_t)g.K * g.n * Q;
    blk_clear<T>(sc, sc_floats, L);
    auto one_use = [&](long unit) {   // the channel node of one (frame, channel use), team-uniform
        const int f = (int)(unit / g.n), u = (int)(unit % g.n);
        float* msg_f = msg + f * fs;
        const float yv = y[(size_t)f * g.n + u], is2 = frame_inv_s2(g, f);
        if (chan_blocked<Q>(g, msg_f, us, 4 * Q, yv, is2, u, sc, res, L)) {
            if (g.log_fallbacks && L.tl == 0) atomicAdd(g.log_fallbacks, 1ull);
            chan_trellis<Q, LogSR>(g, msg_f, us, 4 * Q, yv, is2, u, sc, res, L);
            blk_clear<T>(sc, sc_floats - g.K * Q, L);
        }
        chan_write_team<Q>(g, msg_f, us, 4 * Q, ch2v + f * vs, res, u, L);
    };
    if constexpr (FIX) {
        // each lane tests one channel use; the team then runs the flagged ones
        for (long base = ((long)blockIdx.x * teams + team) * T; base < total; base += (long)gridDim.x * teams * T) {
            const long unit = base + L.tl;
            bool flag = false;
            if (unit < total) {
                const int f = (int)(unit / g.n), u = (int)(unit % g.n);
                flag = (!active || active[f]) && isnan(ch2v[f * vs + (size_t)g.use_pos[u] * Q]);
            }
            unsigned bits = __ballot_sync(L.mask, flag) >> ((threadIdx.x & 31) & ~(T - 1));
            if constexpr (T < 32) bits &= (1u << T) - 1u;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                one_use(base + b);
            }
        }
    } else {
        for (long unit = (long)blockIdx.x * teams + team; unit < total; unit += (long)gridDim.x * teams) {
            if (active && !active[unit / g.n]) continue;
            one_use(unit);
        }
    }
}

// (b) check node (FP32 Walsh-Hadamard butterflies), shared-memory staged: a CTA
// takes tiles of consecutive check blocks (contiguous in HBM), brought in by one
// TMA bulk copy each (double-buffered, completion on an mbarrier) and written
// back by a TMA bulk store; max(1, q/16) lanes per check run the transforms,
// 16 symbols per lane in registers.  Every wait is bounded: on expiry the CTA records the error in
// g.tc_error, waits (bounded) for its copies in flight and returns.
constexpr int kStageThreads = 128;   // threads per CTA; a tile holds kStageThreads / LPC checks
constexpr long long kStageSpin = 1ll << 24;

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ bool mbar_done(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity)
{
    long long spins = 0;
    bool done;
    while (!(done = mbar_done(mbar, parity)) && ++spins < kStageSpin) {
    }
    return done;
}

// Check j on a block in shared memory, LPC = max(1, q/16) lanes per check,
// lane l holding the 16 symbols x = 16 l + j (j < 16): the coefficient
// permutation x -> h^{-1} x is GF(2)-linear, so each permuted offset is an XOR
// of the images of the basis vectors; the transform's stages over the low four
// bits of x run in registers and the rest across the check's lanes; the
// leave-one-out products are formed one edge at a time (same association as
// check_thread).
template <int Q>
struct StageShape {
    static constexpr int LPC = Q > 16 ? Q / 16 : 1;   // lanes per check
    static constexpr int W = Q / LPC;                  // symbols per lane
};

template <int Q>
__device__ __forceinline__ void wht_lanes(float (&p)[StageShape<Q>::W], int l, unsigned mask)
{
    constexpr int LPC = StageShape<Q>::LPC, W = StageShape<Q>::W;
    wht_reg<W>(p);
#pragma unroll
    for (int o = 1; o < LPC; o <<= 1) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const float t = __shfl_xor_sync(mask, p[j], o, LPC);
            p[j] = (l & o) ? (t - p[j]) : (p[j] + t);
        }
    }
}

template <int Q, int DC>
__device__ __forceinline__ void check_lanes_lin(float* blk, const uint8_t* coef, const uint8_t* gdiv, int l,
                                                unsigned mask)
{
    constexpr int LPC = StageShape<Q>::LPC, W = StageShape<Q>::W;
    float P[DC][W];
    int basis[DC][4];   // images of the low four basis vectors
    int lane_off[DC];   // image of 16 l
#pragma unroll
    for (int d = 0; d < DC; ++d) {
        const uint8_t* dv = gdiv + coef[d] * Q;
#pragma unroll
        for (int b = 0; b < 4; ++b) basis[d][b] = ((1 << b) < W) ? dv[1 << b] : 0;
        lane_off[d] = LPC > 1 ? dv[W * l] : 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            int o = lane_off[d];
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (j & (1 << b)) o ^= basis[d][b];
            P[d][j] = blk[d * Q + o];
        }
    }
#pragma unroll
    for (int d = 0; d < DC; ++d) wht_lanes<Q>(P[d], l, mask);
#pragma unroll
    for (int d = 0; d < DC; ++d) {
        // leave-one-out product of the other DC - 1 transforms: for DC = 4 the
        // pairing (P0 P1)(P2 P3) of check_thread, otherwise prefix times suffix
        float R[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if constexpr (DC == 4) {
                const float l01 = P[0][j] * P[1][j], r23 = P[2][j] * P[3][j];
                R[j] = d == 0 ? P[1][j] * r23 : d == 1 ? P[0][j] * r23 : d == 2 ? l01 * P[3][j] : l01 * P[2][j];
            } else {
                float pre = 1.0f, suf = 1.0f;
#pragma unroll
                for (int e = 0; e < d; ++e) pre *= P[e][j];
#pragma unroll
                for (int e = DC - 1; e > d; --e) suf *= P[e][j];
                R[j] = pre * suf;
            }
        }
        wht_lanes<Q>(R, l, mask);
        float mx = vmax(R);
#pragma unroll
        for (int o = 1; o < LPC; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(mask, mx, o, LPC));
        const float fl = kRelFloor * mx, inv = __frcp_rn(mx);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            int o = lane_off[d];
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (j & (1 << b)) o ^= basis[d][b];
            blk[d * Q + o] = fmaxf(R[j], fl) * inv;
        }
    }
}

template <int Q, int DC>
__global__ void __launch_bounds__(kStageThreads, 3) k_check_staged(Graph g, long total, float* msg,
                                                                  const uint8_t* __restrict__ active)
{
    constexpr int CB = DC * Q;   // floats per check block
    constexpr int LPC = StageShape<Q>::LPC, kStageChecks = kStageThreads / LPC;
    extern __shared__ __align__(128) float tiles[];   // [2][kStageChecks * CB]
    __shared__ __align__(8) uint64_t mbar_s[2];
    __shared__ uint8_t sdiv[Q * Q];
    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) sdiv[i] = g.gf_div[i];
    const uint32_t mb0 = s_addr(&mbar_s[0]), mb1 = s_addr(&mbar_s[1]);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long ntiles = (total + kStageChecks - 1) / kStageChecks;
    const long per_frame = (long)g.K * g.P;
    auto tile_bytes = [&](long t) -> uint32_t {
        const long c = total - t * kStageChecks;
        return (uint32_t)((c < kStageChecks ? c : kStageChecks) * CB * sizeof(float));
    };
    auto tile_ptr = [&](long t) { return msg + (size_t)t * kStageChecks * CB; };
    // parity of each buffer's mbarrier, and whether a load into it is in flight
    // (or landed and not yet consumed)
    uint32_t par0 = 0, par1 = 0;
    bool pend0 = false, pend1 = false;
    long tile = blockIdx.x;
    if (tile < ntiles) {
        if (threadIdx.x == 0) bulk_load(s_addr(tiles), tile_ptr(tile), tile_bytes(tile), mb0);
        pend0 = true;
    }
    bool failed = false;
    for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
        const bool odd = it & 1;
        float* buf = tiles + (odd ? (size_t)kStageChecks * CB : 0);
        float* other = tiles + (odd ? 0 : (size_t)kStageChecks * CB);
        const long next = tile + gridDim.x;
        if (next < ntiles) {
            if (threadIdx.x == 0) {
                // the bulk store that last read the other buffer must be done reading it
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                bulk_load(s_addr(other), tile_ptr(next), tile_bytes(next), odd ? mb0 : mb1);
            }
            if (odd) pend0 = true;
            else pend1 = true;
        }
        const bool done = mbar_wait_bounded(odd ? mb1 : mb0, odd ? par1 : par0);
        if (__syncthreads_or(done ? 0 : 1)) {
            failed = true;
            break;
        }
        if (odd) {
            par1 ^= 1;
            pend1 = false;
        } else {
            par0 ^= 1;
            pend0 = false;
        }
        const int slot = threadIdx.x / LPC, l = threadIdx.x % LPC;
        const unsigned mask = LPC == 1 ? 0xffffffffu : (((1u << LPC) - 1u) << ((threadIdx.x & 31) & ~(LPC - 1)));
        const long c = tile * kStageChecks + slot;
        if (c < total && (!active || active[c / per_frame]))
            check_lanes_lin<Q, DC>(buf + slot * CB, g.chk_coef + DC * (int)(c % g.P), sdiv, l, mask);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) bulk_store(tile_ptr(tile), s_addr(buf), tile_bytes(tile));
    }
    if (threadIdx.x == 0) {
        if (failed) {
            if (g.tc_error) atomicExch(g.tc_error, 1);
            // loads still in flight land in this CTA's shared memory: wait for them (bounded)
            if (pend0) mbar_wait_bounded(mb0, par0);
            if (pend1) mbar_wait_bounded(mb1, par1);
        }
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

// (c) posterior and decision, thread shape for q <= 16 and dv = 2: one thread
// per (frame, user, variable) with 16-byte loads of the channel message and
// of both edge messages.
template <int Q>
__global__ void __launch_bounds__(kStepThreads) k_var_thread(Graph g, int F, const float* __restrict__ ch2v,
                                                             const float* __restrict__ msg, float* logpost,
                                                             uint8_t* hat, const uint8_t* __restrict__ active)
{
    const long per_frame = (long)g.K * g.n, total = (long)F * per_frame;
    const int cbs = 4 * Q;
    for (long unit = (long)blockIdx.x * blockDim.x + threadIdx.x; unit < total; unit += (long)gridDim.x * blockDim.x) {
        const int f = (int)(unit / per_frame);
        if (active && !active[f]) continue;
        const int rem = (int)(unit % per_frame), k = rem / g.n, i = rem % g.n;
        const size_t fk = (size_t)f * g.K + k;
        const float* blk = msg + fk * g.E * Q;
        const float* c0 = ch2v + (fk * g.n + i) * Q;
        const float* p0 = edge_ptr(blk, g.var_edge[2 * i], cbs, Q);
        const float* p1 = edge_ptr(blk, g.var_edge[2 * i + 1], cbs, Q);
        float b[Q], m0[Q], m1[Q];
        if constexpr (Q >= 4) {
#pragma unroll
            for (int x = 0; x < Q; x += 4) {
                const float4 u = *reinterpret_cast<const float4*>(c0 + x);
                const float4 v = *reinterpret_cast<const float4*>(p0 + x);
                const float4 w = *reinterpret_cast<const float4*>(p1 + x);
                b[x] = u.x; b[x + 1] = u.y; b[x + 2] = u.z; b[x + 3] = u.w;
                m0[x] = v.x; m0[x + 1] = v.y; m0[x + 2] = v.z; m0[x + 3] = v.w;
                m1[x] = w.x; m1[x + 1] = w.y; m1[x + 2] = w.z; m1[x + 3] = w.w;
            }
        } else {
#pragma unroll
            for (int x = 0; x < Q; ++x) {
                b[x] = c0[x];
                m0[x] = p0[x];
                m1[x] = p1[x];
            }
        }
        float bv = -1.0f;
        int bi = 0;
#pragma unroll
        for (int x = 0; x < Q; ++x) {
            b[x] *= m0[x];
            b[x] *= m1[x];
            if (b[x] > bv) {
                bv = b[x];
                bi = x;
            }
        }
        hat[fk * g.n + i] = (uint8_t)bi;
        if (logpost) {
            const float l = __logf(bv);
#pragma unroll
            for (int x = 0; x < Q; ++x) logpost[(fk * g.n + i) * Q + x] = __logf(b[x]) - l;
        }
    }
}

// (c) posterior and decision.  Team per (frame, user, variable).
template <int Q>
__global__ void __launch_bounds__(kStepThreads) k_var(Graph g, int F, const float* __restrict__ ch2v,
                                                      const float* __restrict__ msg, float* logpost, uint8_t* hat,
                                                      const uint8_t* __restrict__ active)
{
    constexpr int T = Shape<Q>::T;
    const int teams = blockDim.x / T, team = threadIdx.x / T;
    const TeamLane L = team_lane<T>();
    const long per_frame = (long)g.K * g.n, total = (long)F * per_frame;
    for (long unit = (long)blockIdx.x * teams + team; unit < total; unit += (long)gridDim.x * teams) {
        const int f = (int)(unit / per_frame);
        if (active && !active[f]) continue;
        const int rem = (int)(unit % per_frame), k = rem / g.n, i = rem % g.n;
        const size_t fk = (size_t)f * g.K + k;
        var_team<Q>(g, ch2v + fk * g.n * Q, msg + fk * g.E * Q, 4 * Q, i, logpost ? logpost + fk * g.n * Q : nullptr,
                    hat + fk * g.n, L);
    }
}

// (c) posterior and decision for q >= 32 and dv = 2: four lanes per (frame,
// user, variable), q/4 symbols per lane read with 16-byte loads.
template <int Q>
__global__ void __launch_bounds__(kStepThreads) k_var_quad(Graph g, int F, const float* __restrict__ ch2v,
                                                           const float* __restrict__ msg, float* logpost,
                                                           uint8_t* hat, const uint8_t* __restrict__ active)
{
    static_assert(Q >= 16, "four lanes of at least four symbols");
    constexpr int W = Q / 4;
    const int sub = threadIdx.x & 3;
    const unsigned mask = 0xfu << ((threadIdx.x & 31) & ~3);
    const long per_frame = (long)g.K * g.n, total = (long)F * per_frame;
    const int cbs = 4 * Q;
    const long first = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 2, stride = ((long)gridDim.x * blockDim.x) >> 2;
    for (long unit = first; unit < total; unit += stride) {
        const int f = (int)(unit / per_frame);
        if (active && !active[f]) continue;
        const int rem = (int)(unit % per_frame), k = rem / g.n, i = rem % g.n;
        const size_t fk = (size_t)f * g.K + k;
        const float* blk = msg + fk * g.E * Q;
        const float* c0 = ch2v + (fk * g.n + i) * Q + sub * W;
        const float* p0 = edge_ptr(blk, g.var_edge[2 * i], cbs, Q) + sub * W;
        const float* p1 = edge_ptr(blk, g.var_edge[2 * i + 1], cbs, Q) + sub * W;
        float b[W], m0[W], m1[W];
#pragma unroll
        for (int x = 0; x < W; x += 4) {
            const float4 u = *reinterpret_cast<const float4*>(c0 + x);
            const float4 v = *reinterpret_cast<const float4*>(p0 + x);
            const float4 w = *reinterpret_cast<const float4*>(p1 + x);
            b[x] = u.x; b[x + 1] = u.y; b[x + 2] = u.z; b[x + 3] = u.w;
            m0[x] = v.x; m0[x + 1] = v.y; m0[x + 2] = v.z; m0[x + 3] = v.w;
            m1[x] = w.x; m1[x + 1] = w.y; m1[x + 2] = w.z; m1[x + 3] = w.w;
        }
        float bv = -1.0f;
        int bi = 0;
#pragma unroll
        for (int x = 0; x < W; ++x) {
            b[x] *= m0[x];
            b[x] *= m1[x];
            if (b[x] > bv) {
                bv = b[x];
                bi = sub * W + x;
            }
        }
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            const float ov = __shfl_xor_sync(mask, bv, o, 4);
            const int oi = __shfl_xor_sync(mask, bi, o, 4);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (sub == 0) hat[fk * g.n + i] = (uint8_t)bi;
        if (logpost) {
            const float l = __logf(bv);
            float* lp = logpost + (fk * g.n + i) * Q + sub * W;
#pragma unroll
            for (int x = 0; x < W; ++x) lp[x] = __logf(b[x]) - l;
        }
    }
}

// (d) syndrome: unsat[f*K+k] = 1 if a check of user k is unsatisfied.
template <int Q>
__global__ void __launch_bounds__(kStepThreads) k_syndrome(Graph g, int F, const uint8_t* __restrict__ hat,
                                                           uint8_t* unsat, const uint8_t* __restrict__ active)
{
    __shared__ uint8_t smul[Q * Q], sdiv[Q * Q];
    load_gf<Q>(g, smul, sdiv);
    const long per_frame = (long)g.K * g.P, total = (long)F * per_frame;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int f = (int)(t / per_frame);
        if (active && !active[f]) continue;
        const int rem = (int)(t % per_frame), k = rem / g.P, j = rem % g.P;
        const size_t fk = (size_t)f * g.K + k;
        if (!check_satisfied(g, hat + fk * g.n, j, smul)) unsat[fk] = 1;
    }
}

// After iteration t: record iterations and ok flags, stop converged frames.
__global__ void k_finalize(int F, int K, int t, int early_stop, StepCtl c)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
        if (!c.active[f]) continue;
        bool all = true;
        for (int k = 0; k < K; ++k) {
            const bool okk = c.unsat[(size_t)f * K + k] == 0;
            c.ok[(size_t)f * K + k] = okk ? 1 : 0;
            c.unsat[(size_t)f * K + k] = 0;
            all = all && okk;
        }
        c.iters[f] = t;
        if (early_stop && all) c.active[f] = 0;
    }
}

__global__ void k_fill(float* p, size_t count, float value)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        p[i] = value;
}

__global__ void k_ok_from_unsat(int n, const uint8_t* unsat, uint8_t* ok)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) ok[i] = unsat[i] ? 0 : 1;
}

template <int Q, int KC>
cudaError_t channel_thread_q(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                             const uint8_t* active, cudaStream_t s)
{
    const long units = (long)F * g.n;
    const int grid = persistent_grid(k_channel_thread<Q, KC>, kStepThreads, 0, di, kStepThreads, units);
    k_channel_thread<Q, KC><<<grid, kStepThreads, 0, s>>>(g, F, y, msg, ch2v, active);
    return cudaGetLastError();
}

template <int Q, bool FIX = false>
cudaError_t channel_team_q(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                           const uint8_t* active, cudaStream_t s)
{
    constexpr int T = Shape<Q>::T;
    const int scf = blk_scratch_floats(g.K, Q);
    const size_t per_team = (size_t)scf * sizeof(float);
    int threads = kStepThreads;
    while (threads > 32 && (size_t)(threads / T) * per_team > (size_t)di.smem_optin) threads -= 32;
    const size_t smem = (size_t)(threads / T) * per_team;
    if (smem > (size_t)di.smem_optin) return cudaErrorInvalidConfiguration;
    cudaError_t e =
        cudaFuncSetAttribute(k_channel_team<Q, FIX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long units = (long)F * g.n;
    // the hand-off pass gives each team T channel uses to test per step
    const int grid = persistent_grid(k_channel_team<Q, FIX>, threads, smem, di, (threads / T) * (FIX ? T : 1), units);
    k_channel_team<Q, FIX><<<grid, threads, smem, s>>>(g, F, y, msg, ch2v, active, scf);
    return cudaGetLastError();
}

template <int Q>
cudaError_t channel_q(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                      const uint8_t* active, cudaStream_t s)
{
    if constexpr (Q <= 16) {
        if (g.dv == 2 && g.var_reg) {
            switch (g.K) {
                case 1: return channel_thread_q<Q, 1>(g, di, F, y, msg, ch2v, active, s);
                case 2: return channel_thread_q<Q, 2>(g, di, F, y, msg, ch2v, active, s);
                case 3: return channel_thread_q<Q, 3>(g, di, F, y, msg, ch2v, active, s);
                case 4: return channel_thread_q<Q, 4>(g, di, F, y, msg, ch2v, active, s);
                default: break;
            }
        }
    }
    return channel_team_q<Q>(g, di, F, y, msg, ch2v, active, s);
}

template <int Q, int DC>
cudaError_t check_qd(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active, cudaStream_t s)
{
    const long units = (long)F * g.K * g.P;
    constexpr int checks_per_tile = kStageThreads / StageShape<Q>::LPC;
    const size_t smem = 2ull * checks_per_tile * DC * Q * sizeof(float);
    cudaError_t e =
        cudaFuncSetAttribute(k_check_staged<Q, DC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = persistent_grid(k_check_staged<Q, DC>, kStageThreads, smem, di, checks_per_tile, units);
    k_check_staged<Q, DC><<<grid, kStageThreads, smem, s>>>(g, units, msg, active);
    return cudaGetLastError();
}

// check degrees built: 3, 4 and 6 (codes of rate 1/3 with dv = 2, rate 1/2 with
// (2, 4) and (3, 6), and any variable-degree profile with these check degrees)
template <int Q>
cudaError_t check_q(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active, cudaStream_t s)
{
    switch (g.dc) {
        case 3: return check_qd<Q, 3>(g, di, F, msg, active, s);
        case 4: return check_qd<Q, 4>(g, di, F, msg, active, s);
        case 6: return check_qd<Q, 6>(g, di, F, msg, active, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int Q>
cudaError_t var_q(const Graph& g, const DeviceInfo& di, int F, const float* ch2v, const float* msg, float* post,
                  uint8_t* hat, const uint8_t* active, cudaStream_t s)
{
    constexpr int T = Shape<Q>::T;
    const long units = (long)F * g.K * g.n;
    if (g.dv == 2 && g.var_reg) {
        if constexpr (Q <= 16) {
            const int grid = persistent_grid(k_var_thread<Q>, kStepThreads, 0, di, kStepThreads, units);
            k_var_thread<Q><<<grid, kStepThreads, 0, s>>>(g, F, ch2v, msg, post, hat, active);
        } else {
            const int grid = persistent_grid(k_var_quad<Q>, kStepThreads, 0, di, kStepThreads / 4, units);
            k_var_quad<Q><<<grid, kStepThreads, 0, s>>>(g, F, ch2v, msg, post, hat, active);
        }
        return cudaGetLastError();
    }
    const int grid = persistent_grid(k_var<Q>, kStepThreads, 0, di, kStepThreads / T, units);
    k_var<Q><<<grid, kStepThreads, 0, s>>>(g, F, ch2v, msg, post, hat, active);
    return cudaGetLastError();
}

template <int Q>
cudaError_t syndrome_q(const Graph& g, const DeviceInfo& di, int F, const uint8_t* hat, uint8_t* unsat,
                       const uint8_t* active, cudaStream_t s)
{
    const long units = (long)F * g.K * g.P;
    const int grid = persistent_grid(k_syndrome<Q>, kStepThreads, 0, di, kStepThreads, units);
    k_syndrome<Q><<<grid, kStepThreads, 0, s>>>(g, F, hat, unsat, active);
    return cudaGetLastError();
}

}  // namespace

#define JBP_DISPATCH_Q(QV, CALL)                         \
    switch (QV) {                                        \
        case 2: { constexpr int Qc = 2; return CALL; }   \
        case 4: { constexpr int Qc = 4; return CALL; }   \
        case 8: { constexpr int Qc = 8; return CALL; }   \
        case 16: { constexpr int Qc = 16; return CALL; } \
        case 32: { constexpr int Qc = 32; return CALL; } \
        case 64: { constexpr int Qc = 64; return CALL; } \
        default: return cudaErrorInvalidValue;           \
    }

cudaError_t launch_channel(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                           const uint8_t* active, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    if (g.dft_tab) return launch_channel_dft(g, di, F, y, msg, ch2v, active, s);
    JBP_DISPATCH_Q(g.Q, (channel_q<Qc>(g, di, F, y, msg, ch2v, active, s)));
}

cudaError_t launch_channel_fix(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                               const uint8_t* active, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    switch (g.Q) {
        case 16: return channel_team_q<16, true>(g, di, F, y, msg, ch2v, active, s);
        case 32: return channel_team_q<32, true>(g, di, F, y, msg, ch2v, active, s);
        case 64: return channel_team_q<64, true>(g, di, F, y, msg, ch2v, active, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_check(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active, int precision,
                         cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    // tensor-core transforms for q >= 16; smaller fields use the FP32 butterflies
    if (precision != 0 && g.Q >= 16) return launch_check_tc(g, di, F, msg, active, precision, s);
    JBP_DISPATCH_Q(g.Q, (check_q<Qc>(g, di, F, msg, active, s)));
}

cudaError_t launch_var(const Graph& g, const DeviceInfo& di, int F, const float* ch2v, const float* msg, float* post,
                       uint8_t* hat, const uint8_t* active, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    JBP_DISPATCH_Q(g.Q, (var_q<Qc>(g, di, F, ch2v, msg, post, hat, active, s)));
}

cudaError_t launch_syndrome(const Graph& g, const DeviceInfo& di, int F, const uint8_t* hat, uint8_t* unsat,
                            const uint8_t* active, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    JBP_DISPATCH_Q(g.Q, (syndrome_q<Qc>(g, di, F, hat, unsat, active, s)));
}

cudaError_t launch_finalize(int F, int K, int t, int early_stop, StepCtl ctl, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    const int threads = 256, grid = std::min((F + threads - 1) / threads, 4096);
    k_finalize<<<grid, threads, 0, s>>>(F, K, t, early_stop, ctl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// resident pools (serving): admission, per-frame finalisation, harvest
// ---------------------------------------------------------------------------

// Frame i of an admission goes to pool slot slot[i]: its channel output and
// noise variance are copied in, every message starts uniform (all ones), its
// iteration count and syndrome flags are cleared and it becomes active.
__global__ void k_pool_admit(int m, const int32_t* __restrict__ slot, const float* __restrict__ adm_y,
                             const float* __restrict__ adm_sig, PoolState p)
{
    const size_t per = (size_t)p.msg_floats;
    for (int i = blockIdx.y; i < m; i += gridDim.y) {
        const int f = slot[i];
        float* msg = p.msg + (size_t)f * per;
        for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < per; j += (size_t)gridDim.x * blockDim.x)
            msg[j] = 1.0f;
        if (blockIdx.x == 0) {
            for (int j = threadIdx.x; j < p.n; j += blockDim.x) p.y[(size_t)f * p.n + j] = adm_y[(size_t)i * p.n + j];
            for (int k = threadIdx.x; k < p.K; k += blockDim.x) p.unsat[(size_t)f * p.K + k] = 0;
            if (threadIdx.x == 0) {
                p.sig[f] = adm_sig[i];
                p.t[f] = 0;
                p.fin[f] = 0;
                p.active[f] = 1;
            }
        }
    }
}

// After one iteration of the pool: every active frame counts it, records its
// syndrome flags and stops (fin = 1) at a zero syndrome (early stop) or at T.
__global__ void k_pool_finalize(int F, int T, int early_stop, PoolState p)
{
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
        if (!p.active[f]) continue;
        bool all = true;
        for (int k = 0; k < p.K; ++k) {
            const bool okk = p.unsat[(size_t)f * p.K + k] == 0;
            p.ok[(size_t)f * p.K + k] = okk ? 1 : 0;
            p.unsat[(size_t)f * p.K + k] = 0;
            all = all && okk;
        }
        const int t = ++p.t[f];
        if ((early_stop && all) || t >= T) {
            p.active[f] = 0;
            p.fin[f] = 1;
        }
    }
}

// Frames that finished during the block are packed, in any order, into the
// harvest area (host-mapped memory): slot, iterations, K syndrome flags and K*n
// decisions each.  count is a device counter cleared before the launch.
__global__ void k_pool_harvest(int F, PoolState p, int32_t* count, int32_t* out_slot, int32_t* out_iters,
                               uint8_t* out_ok, uint8_t* out_hat)
{
    __shared__ int idx;
    const int KN = p.K * p.n;
    for (int f = blockIdx.x; f < F; f += gridDim.x) {
        if (!p.fin[f]) continue;   // uniform across the block
        __syncthreads();
        if (threadIdx.x == 0) {
            idx = atomicAdd(count, 1);
            out_slot[idx] = f;
            out_iters[idx] = p.t[f];
            p.fin[f] = 0;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < p.K; k += blockDim.x) out_ok[(size_t)idx * p.K + k] = p.ok[(size_t)f * p.K + k];
        for (int j = threadIdx.x; j < KN; j += blockDim.x) out_hat[(size_t)idx * KN + j] = p.hat[(size_t)f * KN + j];
    }
}

cudaError_t launch_pool_admit(int m, const int32_t* slot, const float* adm_y, const float* adm_sig,
                              const PoolState& p, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    const int gx = (int)std::min<size_t>(((size_t)p.msg_floats + 255) / 256, 64);
    const dim3 grid(gx, std::min(m, 4096));
    k_pool_admit<<<grid, 256, 0, s>>>(m, slot, adm_y, adm_sig, p);
    return cudaGetLastError();
}

cudaError_t launch_pool_finalize(int F, int T, int early_stop, const PoolState& p, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    const int threads = 256, grid = std::min((F + threads - 1) / threads, 4096);
    k_pool_finalize<<<grid, threads, 0, s>>>(F, T, early_stop, p);
    return cudaGetLastError();
}

cudaError_t launch_pool_harvest(int F, const PoolState& p, int32_t* count, int32_t* out_slot, int32_t* out_iters,
                                uint8_t* out_ok, uint8_t* out_hat, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    k_pool_harvest<<<std::min(F, 4096), 128, 0, s>>>(F, p, count, out_slot, out_iters, out_ok, out_hat);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* p, size_t count, float value, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const int threads = 256;
    const size_t grid = std::min<size_t>((count + threads - 1) / threads, 8192);
    k_fill<<<(int)grid, threads, 0, s>>>(p, count, value);
    return cudaGetLastError();
}

cudaError_t launch_ok_from_unsat(int F, int K, const uint8_t* unsat, uint8_t* ok, cudaStream_t s)
{
    const int n = F * K;
    if (n <= 0) return cudaSuccess;
    const int threads = 256, grid = std::min((n + threads - 1) / threads, 4096);
    k_ok_from_unsat<<<grid, threads, 0, s>>>(n, unsat, ok);
    return cudaGetLastError();
}

}  // namespace jbp
