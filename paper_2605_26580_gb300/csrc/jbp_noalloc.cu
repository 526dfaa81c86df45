// jbp_noalloc.cu -- jbp_decode_noalloc: a decode that allocates no memory.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or under a strict memory cap, or a process that may
// not call cudaMalloc at all.  jbp_decode_noalloc serves them: it runs the
// step-form decode (channel, check, variable, syndrome kernels) with all of its
// working memory -- the code tables and the per-frame message state -- in one
// file-scope device array of fixed size, kNoallocScratchBytes.  Every GPU that
// loads this library holds that array until the process exits.
//
// The array's name is a host-side stand-in in host code, not a device address,
// so the address is taken with cudaGetSymbolAddress once per device (with that
// device current) and passed to the kernels.  The first call on a device does
// that set-up; make it before any stream capture.  All calls share the array
// and it keeps the last call's contents: each call clears what must start at
// zero.  Calls whose work overlaps on the GPU (different streams, or different
// host threads on one device) race on the array and must be serialised by the
// caller.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "jbp.h"
#include "jbp_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;   // 16 MiB per device
constexpr size_t kTableBytes = size_t(1) << 20;             // host/device table area (first 1 MiB)
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch
    jbp::DeviceInfo di{};
};

std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];
unsigned char g_host_tables[kTableBytes];   // host staging, guarded by g_mu
int nfail(int code, const char* msg)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "jbp_decode_noalloc: %s", msg);
    jbp::set_last_error(buf);
    return code;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// After the last iteration: if a bounded device wait of the staged check
// kernel expired during this call, no frame's outputs can be trusted, so every
// frame gets ok = 0 and iters = -1 (the caller's only sign of it, since the
// call returns before the work runs).
__global__ void k_noalloc_status(const int* err, int F, int K, int32_t* iters, uint8_t* ok)
{
    if (*err == 0) return;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
        iters[f] = -1;
        for (int k = 0; k < K; ++k) ok[(size_t)f * K + k] = 0;
    }
}

}  // namespace

extern "C" int jbp_decode_noalloc(const jbp_code* code, int32_t K, const jbp_channel* chan, int32_t T,
                                  int32_t early_stop, int32_t F, const float* y, uint8_t* hat, int32_t* iters,
                                  uint8_t* ok, void* stream)
{
    if (!code || !chan) return nfail(JBP_EINVAL, "NULL code or channel");
    if (F < 0 || T < 1) return nfail(JBP_EINVAL, "F must be >= 0 and iters >= 1");
    if (F > 0 && (!y || !hat || !iters || !ok)) return nfail(JBP_EINVAL, "NULL buffer");
    const int q = code->q, n = code->n, P = code->P, dc = code->dc, dv = code->dv;
    int m = 0;
    while ((1 << m) < q && m < 8) ++m;
    if (q < 2 || q > 64 || (1 << m) != q) return nfail(JBP_EINVAL, "q must be a power of two in 2..64");
    if (K < 1 || K > jbp::kMaxK) return nfail(JBP_EINVAL, "K must be in 1..16");
    if (n < 1 || P < 1 || dc != 4 || dv < 1 || dv > jbp::kMaxDv || (int64_t)n * dv != (int64_t)P * dc)
        return nfail(JBP_EINVAL, "unsupported code shape (needs regular dv, dc = 4, n*dv = P*dc)");
    if (!code->chk_var || !code->chk_coef) return nfail(JBP_EINVAL, "NULL code arrays");
    if (!(chan->sigma2 > 0.0) || !std::isfinite(chan->sigma2)) return nfail(JBP_EINVAL, "sigma2 must be > 0");
    if (chan->interleave && !chan->perm) return nfail(JBP_EINVAL, "interleave = 1 needs perm");
    const int E = P * dc;

    // table area (first kTableBytes) and per-frame state after it
    const size_t o_var = 0, o_coef = up256(o_var + 4ull * E), o_vedge = up256(o_coef + E),
                 o_use = up256(o_vedge + 4ull * n * dv), o_mul = up256(o_use + 4ull * K * n),
                 o_div = up256(o_mul + (size_t)q * q), o_err = up256(o_div + (size_t)q * q),
                 tables_end = up256(o_err + sizeof(int));
    if (tables_end > kTableBytes) return nfail(JBP_EINVAL, "code too large for the fixed table area (1 MiB)");
    const size_t fs = (size_t)K * E * q * 4, vs = (size_t)K * n * q * 4;
    const size_t o_msg = kTableBytes, o_ch2v = up256(o_msg + fs * F), o_act = up256(o_ch2v + vs * F),
                 o_unsat = up256(o_act + (size_t)F), end = up256(o_unsat + (size_t)F * K);
    if (end > kNoallocScratchBytes) {
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "jbp_decode_noalloc: %d frames need %zu bytes of scratch, more than the fixed %zu "
                      "(at most %zu frames of this shape)",
                      F, end, kNoallocScratchBytes,
                      (size_t)((kNoallocScratchBytes - kTableBytes - 1024) / (fs + vs + 1 + K + 1)));
        jbp::set_last_error(buf);
        return JBP_EINVAL;
    }
    if (F == 0) return JBP_OK;

    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nfail(JBP_ECUDA, "no current CUDA device");
    DeviceSetup& ds = g_dev[dev];
    if (!ds.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return nfail(JBP_ECUDA, cudaGetErrorString(e));
        if (cudaDeviceGetAttribute(&ds.di.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&ds.di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return nfail(JBP_ECUDA, "cudaDeviceGetAttribute failed");
        ds.base = static_cast<unsigned char*>(p);
        ds.ready = true;
    }

    // host-side tables in the static staging buffer
    unsigned char* H = g_host_tables;
    std::memset(H, 0, tables_end);
    int32_t* hvar = reinterpret_cast<int32_t*>(H + o_var);
    uint8_t* hcoef = H + o_coef;
    int32_t* hvedge = reinterpret_cast<int32_t*>(H + o_vedge);
    int32_t* huse = reinterpret_cast<int32_t*>(H + o_use);
    uint8_t* hmul = H + o_mul;
    uint8_t* hdiv = H + o_div;
    // variable degree counters live in huse until use_pos is written
    for (int i = 0; i < n; ++i) huse[i] = 0;
    for (int e = 0; e < E; ++e) {
        const int i = code->chk_var[e];
        if (i < 0 || i >= n) return nfail(JBP_EINVAL, "chk_var out of range");
        if (code->chk_coef[e] < 1 || code->chk_coef[e] >= q) return nfail(JBP_EINVAL, "chk_coef not in 1..q-1");
        if (huse[i] >= dv) return nfail(JBP_EINVAL, "a variable has more than dv edges");
        hvar[e] = i;
        hcoef[e] = code->chk_coef[e];
        hvedge[(size_t)i * dv + huse[i]++] = e;
    }
    for (int i = 0; i < n; ++i)
        if (huse[i] != dv) return nfail(JBP_EINVAL, "a variable has fewer than dv edges");
    for (int i = 0; i < K * n; ++i) huse[i] = -1;
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < n; ++i) {
            const int t = chan->interleave ? chan->perm[(size_t)k * n + i] : i;
            if (t < 0 || t >= n || huse[(size_t)k * n + t] != -1) return nfail(JBP_EINVAL, "perm row is not a permutation");
            huse[(size_t)k * n + t] = i;
        }
    jbp::gf_build_tables(m, hmul, hdiv);
    // the wait-expiry flag at o_err is zero in H (cleared with the tables each call)

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* D = ds.base;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(D, H, tables_end, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = jbp::launch_fill(reinterpret_cast<float*>(D + o_msg), fs / 4 * F, 1.0f, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(D + o_act, 1, (size_t)F, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(D + o_unsat, 0, (size_t)F * K, s)) != cudaSuccess)
        return nfail(JBP_ECUDA, cudaGetErrorString(e));
    jbp::Graph g;
    g.n = n; g.P = P; g.E = E; g.dc = dc; g.dv = dv; g.K = K; g.Q = q;
    g.inv_sigma2 = (float)(1.0 / chan->sigma2);
    g.chk_var = reinterpret_cast<const int32_t*>(D + o_var);
    g.chk_coef = D + o_coef;
    g.var_edge = reinterpret_cast<const int32_t*>(D + o_vedge);
    g.use_pos = reinterpret_cast<const int32_t*>(D + o_use);
    g.gf_mul = D + o_mul;
    g.gf_div = D + o_div;
    g.log_fallbacks = nullptr;
    g.pos_of = nullptr;
    g.slot = nullptr;
    g.tc_error = reinterpret_cast<int*>(D + o_err);
    g.sigma2_f = nullptr;
    g.chk_order = nullptr;
    float* msg = reinterpret_cast<float*>(D + o_msg);
    float* ch2v = reinterpret_cast<float*>(D + o_ch2v);
    uint8_t* active = D + o_act;
    uint8_t* unsat = D + o_unsat;
    jbp::StepCtl c{active, unsat, iters, ok};
    for (int t = 1; t <= T; ++t) {
        if ((e = jbp::launch_channel(g, ds.di, F, y, msg, ch2v, active, s)) != cudaSuccess ||
            (e = jbp::launch_check(g, ds.di, F, msg, active, JBP_PREC_FP32, s)) != cudaSuccess ||
            (e = jbp::launch_var(g, ds.di, F, ch2v, msg, nullptr, hat, active, s)) != cudaSuccess ||
            (e = jbp::launch_syndrome(g, ds.di, F, hat, unsat, active, s)) != cudaSuccess ||
            (e = jbp::launch_finalize(F, K, t, early_stop, c, s)) != cudaSuccess)
            return nfail(JBP_ECUDA, cudaGetErrorString(e));
    }
    k_noalloc_status<<<std::min((F + 255) / 256, 4 * ds.di.sm_count), 256, 0, s>>>(g.tc_error, F, K, iters, ok);
    if ((e = cudaGetLastError()) != cudaSuccess) return nfail(JBP_ECUDA, cudaGetErrorString(e));
    return JBP_OK;
}
