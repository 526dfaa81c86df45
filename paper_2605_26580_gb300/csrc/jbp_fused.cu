// jbp_fused.cu -- fused form: one persistent kernel runs all iterations of a
// group of frames with the whole message state in shared memory.
//
// A CTA owns G frames at a time.  Shared memory (per CTA):
//   msg  [G][K][E][q] f32   c2v / v2c on check-major edges (updated in place)
//   ch2v [G][K][n][q] f32   channel messages
//   y    [G][n]       f32
//   scratch [teams][chan_scratch_floats] f32   channel trellis per team
//   hat  [G][K][n] u8, unsat [G][K] u8, active [G] u8, gf mul/div [q*q] u8
// Per iteration: (A) channel nodes + in-place v2c, (B) check nodes,
// (C) decisions, (D) syndromes, (E) per-frame stop; __syncthreads between.
// Global memory sees only y in and hat/iters/ok (and the optional posterior) out.
#include <algorithm>

#include "jbp_internal.h"

namespace jbp {
namespace {

constexpr int kFusedMaxThreads = 512;
constexpr size_t kStaticSmemMargin = 256;   // static __shared__ words of k_fused

struct FusedLayout {
    size_t msg, ch2v, y, scratch, hat, unsat, active, gmul, gdiv, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline FusedLayout fused_layout(const Graph& g, int G, int teams, int scf)
{
    FusedLayout L;
    size_t o = 0;
    L.msg = o;     o = align16(o + sizeof(float) * (size_t)G * g.K * g.E * g.Q);
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

template <int Q, int DC>
__global__ void __launch_bounds__(kFusedMaxThreads) k_fused(Graph g, int F, int G, const float* __restrict__ y,
                                                            int T_it, int early_stop, uint8_t* hat,
                                                            int32_t* iters, uint8_t* ok, float* post, int scf)
{
    constexpr int T = Shape<Q>::T;
    extern __shared__ __align__(16) unsigned char sm[];
    const int teams = blockDim.x / T, team = threadIdx.x / T;
    const FusedLayout lay = fused_layout(g, G, teams, scf);
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
    const int K = g.K, n = g.n, E = g.E, P = g.P;
    const size_t fs = (size_t)K * E * Q, vs = (size_t)K * n * Q;

    for (int i = threadIdx.x; i < Q * Q; i += blockDim.x) {
        s_mul[i] = g.gf_mul[i];
        s_div[i] = g.gf_div[i];
    }

    const int groups = (F + G - 1) / G;
    for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
        const int f0 = grp * G, gc = min(G, F - f0);
        // uniform c2v (log 1 = 0), y, control words
        for (size_t i = threadIdx.x; i < (size_t)gc * fs; i += blockDim.x) s_msg[i] = 0.0f;
        for (int i = threadIdx.x; i < gc * n; i += blockDim.x) s_y[i] = y[(size_t)f0 * n + i];
        for (int i = threadIdx.x; i < gc * K; i += blockDim.x) s_unsat[i] = 0;
        for (int i = threadIdx.x; i < G; i += blockDim.x) s_active[i] = i < gc ? 1 : 0;
        __syncthreads();

        for (int t = 1; t <= T_it; ++t) {
            // (A) channel nodes, v2c in place
            for (int unit = team; unit < gc * n; unit += teams) {
                const int gi = unit / n, u = unit % n;
                if (!s_active[gi]) continue;
                float* msg_f = s_msg + gi * fs;
                const float yv = s_y[gi * n + u];
                if (chan_trellis<Q, LinSR>(g, msg_f, yv, u, sc, res, L))
                    chan_trellis<Q, LogSR>(g, msg_f, yv, u, sc, res, L);
                chan_write<Q>(g, msg_f, s_ch2v + gi * vs, res, u, L);
            }
            __syncthreads();
            // (B) check nodes
            for (int unit = team; unit < gc * K * P; unit += teams) {
                const int gi = unit / (K * P), rem = unit % (K * P), k = rem / P, j = rem % P;
                if (!s_active[gi]) continue;
                check_unit_fp32<Q, DC>(g, s_msg + gi * fs + (size_t)k * E * Q, j, s_mul, s_div, L);
            }
            __syncthreads();
            // (C) posterior and decisions
            for (int unit = team; unit < gc * K * n; unit += teams) {
                const int gi = unit / (K * n), rem = unit % (K * n), k = rem / n, i = rem % n;
                if (!s_active[gi]) continue;
                const size_t fk = (size_t)gi * K + k;
                float* pst = post ? post + ((size_t)(f0 + gi) * K + k) * n * Q : nullptr;
                var_unit<Q>(g, s_ch2v + fk * n * Q, s_msg + fk * E * Q, i, pst, s_hat + fk * n, L);
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

template <int Q>
bool plan_q(const Graph& g, const DeviceInfo& di, int F, int threads_hint, int fpc_hint, FusedPlan* plan)
{
    constexpr int T = Shape<Q>::T;
    if (g.dc != 4 || F <= 0) return false;
    const int scf = chan_scratch_floats(g.K, Q);
    int threads = threads_hint > 0 ? threads_hint : 256;
    threads = std::max(32, std::min(kFusedMaxThreads, threads / 32 * 32));
    for (; threads >= 32; threads -= 32) {
        const int teams = threads / T;
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
        if (cudaFuncSetAttribute(k_fused<Q, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem_bytes) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused<Q, 4>, threads, plan->smem_bytes) !=
                cudaSuccess ||
            occ < 1)
            return false;
        plan->grid = std::max(1, std::min(groups, di.sm_count * occ));
        return true;
    }
    return false;
}

template <int Q>
cudaError_t fused_q(const Graph& g, const FusedPlan& p, int F, const float* y, int T_it, int early_stop,
                    uint8_t* hat, int32_t* iters, uint8_t* ok, float* post, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_fused<Q, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem_bytes);
    if (e != cudaSuccess) return e;
    k_fused<Q, 4><<<p.grid, p.threads, p.smem_bytes, s>>>(g, F, p.frames_per_cta, y, T_it, early_stop, hat, iters,
                                                           ok, post, chan_scratch_floats(g.K, Q));
    return cudaGetLastError();
}

}  // namespace

bool fused_plan(const Graph& g, const DeviceInfo& di, int F, int threads_hint, int fpc_hint, FusedPlan* plan)
{
    switch (g.Q) {
        case 2: return plan_q<2>(g, di, F, threads_hint, fpc_hint, plan);
        case 4: return plan_q<4>(g, di, F, threads_hint, fpc_hint, plan);
        case 8: return plan_q<8>(g, di, F, threads_hint, fpc_hint, plan);
        case 16: return plan_q<16>(g, di, F, threads_hint, fpc_hint, plan);
        case 32: return plan_q<32>(g, di, F, threads_hint, fpc_hint, plan);
        case 64: return plan_q<64>(g, di, F, threads_hint, fpc_hint, plan);
        default: return false;
    }
}

cudaError_t launch_fused(const Graph& g, const FusedPlan& plan, int F, const float* y, int T_it, int early_stop,
                         uint8_t* hat, int32_t* iters, uint8_t* ok, float* post, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    switch (g.Q) {
        case 2: return fused_q<2>(g, plan, F, y, T_it, early_stop, hat, iters, ok, post, s);
        case 4: return fused_q<4>(g, plan, F, y, T_it, early_stop, hat, iters, ok, post, s);
        case 8: return fused_q<8>(g, plan, F, y, T_it, early_stop, hat, iters, ok, post, s);
        case 16: return fused_q<16>(g, plan, F, y, T_it, early_stop, hat, iters, ok, post, s);
        case 32: return fused_q<32>(g, plan, F, y, T_it, early_stop, hat, iters, ok, post, s);
        case 64: return fused_q<64>(g, plan, F, y, T_it, early_stop, hat, iters, ok, post, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace jbp
