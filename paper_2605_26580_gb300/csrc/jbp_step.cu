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
template <int Q>
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
    for (long unit = (long)blockIdx.x * teams + team; unit < total; unit += (long)gridDim.x * teams) {
        const int f = (int)(unit / g.n), u = (int)(unit % g.n);
        if (active && !active[f]) continue;
        float* msg_f = msg + f * fs;
        const float yv = y[(size_t)f * g.n + u], is2 = frame_inv_s2(g, f);
        if (chan_blocked<Q>(g, msg_f, us, 4 * Q, yv, is2, u, sc, res, L)) {
            if (g.log_fallbacks && L.tl == 0) atomicAdd(g.log_fallbacks, 1ull);
            chan_trellis<Q, LogSR>(g, msg_f, us, 4 * Q, yv, is2, u, sc, res, L);
            blk_clear<T>(sc, sc_floats - g.K * Q, L);
        }
        chan_write_team<Q>(g, msg_f, us, 4 * Q, ch2v + f * vs, res, u, L);
    }
}

// (b) check node (FP32 Walsh-Hadamard butterflies).  Team per (frame, user, check).
template <int Q>
__global__ void __launch_bounds__(kStepThreads) k_check(Graph g, int F, float* msg, const uint8_t* __restrict__ active)
{
    constexpr int T = Shape<Q>::T;
    __shared__ uint8_t smul[Q * Q], sdiv[Q * Q];
    load_gf<Q>(g, smul, sdiv);
    const int teams = blockDim.x / T, team = threadIdx.x / T;
    const TeamLane L = team_lane<T>();
    const long per_frame = (long)g.K * g.P, total = (long)F * per_frame;
    for (long unit = (long)blockIdx.x * teams + team; unit < total; unit += (long)gridDim.x * teams) {
        const int f = (int)(unit / per_frame);
        if (active && !active[f]) continue;
        const long fk_j = unit;   // ((f*K + k)*P + j): blocks are contiguous in this order
        const int j = (int)(unit % g.P);
        check_team<Q>(msg + (size_t)fk_j * 4 * Q, g.chk_coef + 4 * j, smul, sdiv, L);
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

template <int Q>
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
    cudaError_t e = cudaFuncSetAttribute(k_channel_team<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long units = (long)F * g.n;
    const int grid = persistent_grid(k_channel_team<Q>, threads, smem, di, threads / T, units);
    k_channel_team<Q><<<grid, threads, smem, s>>>(g, F, y, msg, ch2v, active, scf);
    return cudaGetLastError();
}

template <int Q>
cudaError_t channel_q(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                      const uint8_t* active, cudaStream_t s)
{
    if constexpr (Q <= 16) {
        if (g.dv == 2) {
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

template <int Q>
cudaError_t check_q(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active, cudaStream_t s)
{
    constexpr int T = Shape<Q>::T;
    if (g.dc != kDC) return cudaErrorInvalidValue;
    const long units = (long)F * g.K * g.P;
    const int grid = persistent_grid(k_check<Q>, kStepThreads, 0, di, kStepThreads / T, units);
    k_check<Q><<<grid, kStepThreads, 0, s>>>(g, F, msg, active);
    return cudaGetLastError();
}

template <int Q>
cudaError_t var_q(const Graph& g, const DeviceInfo& di, int F, const float* ch2v, const float* msg, float* post,
                  uint8_t* hat, const uint8_t* active, cudaStream_t s)
{
    constexpr int T = Shape<Q>::T;
    const long units = (long)F * g.K * g.n;
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
    JBP_DISPATCH_Q(g.Q, (channel_q<Qc>(g, di, F, y, msg, ch2v, active, s)));
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
