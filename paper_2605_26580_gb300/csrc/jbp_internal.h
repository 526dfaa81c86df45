// jbp_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "jbp_device.cuh"

namespace jbp {

// Per-frame control words of the step form (device memory, F entries each).
struct StepCtl {
    uint8_t* active;   // 1 while the frame iterates
    uint8_t* unsat;    // [F*K] 1 if some check of user k is unsatisfied
    int32_t* iters;    // iterations run
    uint8_t* ok;       // [F*K]
};

struct DeviceInfo {
    int sm_count;
    int smem_optin;   // max dynamic shared memory per block (bytes)
};

// Step kernels (jbp_step.cu).  active may be null (all frames active).
cudaError_t launch_channel(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg,
                           float* ch2v, const uint8_t* active, cudaStream_t s);
cudaError_t launch_check(const Graph& g, const DeviceInfo& di, int F, float* msg,
                         const uint8_t* active, int precision, cudaStream_t s);
cudaError_t launch_var(const Graph& g, const DeviceInfo& di, int F, const float* ch2v,
                       const float* msg, float* post, uint8_t* hat, const uint8_t* active,
                       cudaStream_t s);
cudaError_t launch_syndrome(const Graph& g, const DeviceInfo& di, int F, const uint8_t* hat,
                            uint8_t* unsat, const uint8_t* active, cudaStream_t s);
cudaError_t launch_finalize(int F, int K, int t, int early_stop, StepCtl ctl, cudaStream_t s);
cudaError_t launch_fill(float* p, size_t count, float value, cudaStream_t s);

// Check node on the tensor cores (jbp_check_tc.cu): the Walsh-Hadamard
// transforms as +-1 matrix products with BF16 operands split into `precision`
// terms (JBP_PREC_BF16X2 / BF16 / BF16X3) and FP32 accumulation.
cudaError_t launch_check_tc(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active,
                            int precision, cudaStream_t s);
// Channel node as DFTs over the symbol-sum alphabet on the tensor cores
// (jbp_channel_dft.cu).  Tile: 128 channel uses (rows).  U = K(q-1)+1 sum
// values; L >= U the DFT length (a multiple of 16); W the width of the window of
// the Gaussian score G that is transformed (the rest is below the message floor
// for W = L, and below exp(-2 (W/2 - 1)^2 / sigma2) of the maximum otherwise);
// KB = max(q, W) the inner dimension of the forward DFT matrix; Nc the real
// spectral columns per chunk.  The inverse-DFT accumulators of KG = min(K, 256/q)
// users stay in tensor memory; with K > KG the users go in NP passes, each
// recomputing the forward spectra.  Built for 2 <= K <= 8 and q = 16, 32, 64.
constexpr int kDftRows = 128;
constexpr int kDftThreads = 256;
constexpr int kDftSmemMax = 226 * 1024;   // dynamic part; the kernel's static part is under 1 KB
struct DftShape {
    int U, L, W, KB, Nc, chunks, tmem_cols, smem, KG, NP;
    bool ok;
};
__host__ __device__ constexpr DftShape dft_shape(int K, int Q)
{
    DftShape s{};
    s.U = K * (Q - 1) + 1;
    s.L = (s.U + 15) / 16 * 16;
    s.W = s.L < 128 ? s.L : 128;
    s.KB = Q > s.W ? Q : s.W;
    s.ok = false;
    if (Q < 16 || Q > 64 || (Q & (Q - 1)) || K < 2 || K > 8) return s;
    s.KG = K < 256 / Q ? K : 256 / Q;
    s.NP = (K + s.KG - 1) / s.KG;
    // mu tiles + G window (one FP16 term each) + twiddles + message offsets + alignment slack
    const int fixed = K * kDftRows * Q * 2 + kDftRows * s.W * 2 + s.L * 8 + kDftRows * K * 12 + 1024;
    for (int nc = 128; nc >= 16; nc /= 2) {
        // tensor-memory columns; a thread holds (K + 1) nc / 2 spectral values in registers
        if (s.L % nc || s.KG * Q + (K + 1) * nc > 512 || (K + 1) * nc > 192) continue;
        // forward chunk (hi, lo) + inverse chunk (hi, lo) + X tiles of one pass (hi, lo)
        const int sm = fixed + nc * s.KB * 4 + Q * nc * 4 + s.KG * kDftRows * nc * 4;
        if (sm > kDftSmemMax) continue;
        s.Nc = nc;
        s.smem = sm;
        s.ok = true;
        break;
    }
    if (!s.ok) return s;
    s.chunks = s.L / s.Nc;
    const int need = s.KG * Q + (K + 1) * s.Nc;
    s.tmem_cols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
    return s;
}
// Bytes of the device tables of one (K, q) and their contents (host memory):
// per chunk the forward DFT rows (FP16 hi, lo) and the inverse DFT rows (hi,
// lo) in tensor-core tile order, then L twiddles (cos, sin)(2 pi m / L).
size_t dft_table_bytes(int K, int Q);
void dft_build_table(int K, int Q, unsigned char* out);
// Per-handle part that follows those tables: for every channel use u and user k
// (index u*K + k) three int32 offsets, in floats: the variable's two c2v messages
// within a frame's msg block and its channel message within the frame's ch2v.
size_t dft_offsets_bytes(int K, int n);
void dft_build_offsets(int K, int Q, int n, int E, const int32_t* use_pos, const int32_t* var_edge, int32_t* out);
// Launches the tensor-core kernel, then the FP32 trellis on the channel uses it
// could not resolve (launch_channel_fix).
cudaError_t launch_channel_dft(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                               const uint8_t* active, cudaStream_t s);
// Team-shape trellis on the channel uses whose user-0 channel message starts
// with a NaN (left by the tensor-core channel node); q = 16, 32, 64 (jbp_step.cu).
cudaError_t launch_channel_fix(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                               const uint8_t* active, cudaStream_t s);

cudaError_t launch_ok_from_unsat(int F, int K, const uint8_t* unsat, uint8_t* ok, cudaStream_t s);

// Resident pool of the serving loop: the step-form state of up to F frame
// slots of one decoder, kept in HBM across blocks of iterations (jbp_step.cu).
struct PoolState {
    int n, K;
    long long msg_floats;   // K*E*q per frame
    float* msg;             // [F][K][E][q]
    float* y;               // [F][n]
    float* sig;             // [F] noise variance of each frame
    uint8_t* active;        // [F] 1 while the frame iterates
    int32_t* t;             // [F] iterations run
    uint8_t* unsat;         // [F*K]
    uint8_t* ok;            // [F*K]
    uint8_t* hat;           // [F*K*n]
    uint8_t* fin;           // [F] finished during the current block, not yet harvested
};
cudaError_t launch_pool_admit(int m, const int32_t* slot, const float* adm_y, const float* adm_sig,
                              const PoolState& p, cudaStream_t s);
cudaError_t launch_pool_finalize(int F, int T, int early_stop, const PoolState& p, cudaStream_t s);
cudaError_t launch_pool_harvest(int F, const PoolState& p, int32_t* count, int32_t* out_slot, int32_t* out_iters,
                                uint8_t* out_ok, uint8_t* out_hat, cudaStream_t s);

// Fused shared-memory form (jbp_fused.cu).
struct FusedPlan {
    int frames_per_cta;   // frames resident in one CTA
    int threads;          // threads per CTA
    int smem_bytes;       // dynamic shared memory per CTA
    int grid;             // CTAs launched (persistent)
    int variant = 0;      // kernel variant (fused position-major: 1 = lane-pair channel)
};
bool fused_plan(const Graph& g, const DeviceInfo& di, int F, int threads_hint, int fpc_hint,
                FusedPlan* plan);
cudaError_t launch_fused(const Graph& g, const FusedPlan& plan, int F, const float* y, int T,
                         int early_stop, uint8_t* hat, int32_t* iters, uint8_t* ok, float* post,
                         cudaStream_t s);

// A serving pool run by the fused position-major kernel: slot f's message state
// (msg_floats + ch2v_floats floats, in the kernel's shared-memory layout) stays
// in HBM between blocks; a launch runs up to `block` more iterations of every
// active slot (one slot per CTA), loading its state into shared memory and
// storing it back, and stops a slot at its early stop or at T (active = 0,
// fin = 1, its decisions in hat).  t [F]: iterations run, updated.
struct FusedPool {
    float* msg = nullptr;    // [F][msg_floats]
    float* ch2v = nullptr;   // [F][ch2v_floats]
    uint8_t* active = nullptr;
    uint8_t* fin = nullptr;
    int block = 0;
};
// The fused pool's plan (one frame per CTA) and per-slot state sizes; false if
// the position-major kernel does not serve this graph.
bool fused_pool_plan(const Graph& g, const DeviceInfo& di, int cap, int threads_hint, FusedPlan* plan,
                     size_t* msg_floats, size_t* ch2v_floats);
cudaError_t launch_fused_pool(const Graph& g, const FusedPlan& plan, int F, const float* y, int T, int early_stop,
                              uint8_t* hat, int32_t* t, uint8_t* ok, const FusedPool& pool, cudaStream_t s);

// Evidence-interface path (jbp_ura.cu): slot-wise AMP detector and SIC row
// decoder.  Device tables and scalars of one (code, detector) pair.
struct UraDev {
    int n, P, dc, dv, K, Q;      // slots = variables, checks, check and variable degree, rows, field size
    int ns;                      // complex channel uses per slot (rows of the partial DFT)
    int amp_iters, bp_iters, early_stop;
    float log_odds;              // log((1 - rho) / rho)
    float su2;                   // variance of an active coordinate
    float inv_sqrt_ns;           // 1 / sqrt(ns)
    float cancel_log;            // SIC: log-evidence added to a decided symbol
    const int32_t* rows;         // [n*ns] partial-DFT rows of each slot
    const float* tw;             // [2*Q] exp(-2 pi i k / Q), interleaved
    const int32_t* chk_var;      // [P*dc]
    const uint8_t* chk_coef;     // [P*dc]
    const int32_t* var_edge;     // [dv*n] the edges of each variable
    const uint8_t* gf_mul;       // [Q*Q]
    const uint8_t* gf_div;       // [Q*Q]
};
// Warps (frames) per CTA of the SIC kernel, 0 if one frame does not fit.
int sic_warps_per_cta(const UraDev& u, const DeviceInfo& di);
cudaError_t launch_amp(const UraDev& u, const DeviceInfo& di, int F, const float* y, float* S, cudaStream_t s);
cudaError_t launch_match_rows(const DeviceInfo& di, int F, int K, int n, const uint8_t* hat, const uint8_t* truth,
                              int32_t* sym_err, int32_t* cw_err, cudaStream_t s);
cudaError_t launch_sic(const UraDev& u, const DeviceInfo& di, int F, const float* S, uint8_t* hat, int32_t* iters,
                       uint8_t* ok, cudaStream_t s);

// Record the message returned by jbp_last_error() on this thread (jbp_capi.cu).
void set_last_error(const char* msg);

// GF(2^m) tables (jbp_capi.cu), q = 2^m, m = 1..6, field polynomials of jbp.h:
// mul[h*q + x] = h x, div[h*q + x] = h^{-1} x (row 0 of div zero).
void gf_build_tables(int m, uint8_t* mul, uint8_t* div);

// Bytes of message state of one frame in either form: msg [K*E*Q] + ch2v [K*n*Q] floats.
inline int64_t state_bytes(const Graph& g)
{
    return 4ll * g.K * (int64_t)(g.E + g.n) * g.Q;
}

}  // namespace jbp
