// jbp_capi.cu -- the C ABI (include/jbp.h): contexts, decoder handles, the three
// launch forms, single-step entry points and the continuous-batching serving loop.
#include <algorithm>
#include <array>
#include <memory>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "jbp.h"
#include "jbp_internal.h"

using namespace jbp;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

static int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

static int cuda_fail(cudaError_t e, const char* what)
{
    return fail(JBP_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define JBP_CU(call, what)                                   \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return cuda_fail(_e, (what)); \
    } while (0)

extern "C" const char* jbp_last_error(void) { return g_last_error.c_str(); }

void jbp::set_last_error(const char* msg) { g_last_error = msg; }

static double now_us()
{
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// GF(2^m) tables (host side of the library)
// ---------------------------------------------------------------------------

static int prim_poly(int m)
{
    switch (m) {
        case 1: return 0x3;
        case 2: return 0x7;
        case 3: return 0xB;
        case 4: return 0x13;
        case 5: return 0x25;
        case 6: return 0x43;
        default: return 0;
    }
}

// carry-less product of two polynomials, then reduction modulo the field polynomial
static int gf_mul_host(int a, int b, int m)
{
    int p = 0;
    for (int i = 0; i < m; ++i)
        if ((b >> i) & 1) p ^= a << i;
    const int poly = prim_poly(m);
    for (int i = 2 * m - 2; i >= m; --i)
        if ((p >> i) & 1) p ^= poly << (i - m);
    return p;
}

// q x q tables of GF(2^m): mul[h q + x] = h x and div[h q + x] = h^{-1} x
// (row h = 0 of div is all zero).  The one builder of these tables in the
// library: jbp_create, the evidence decoder, jbp_gf_tables and
// jbp_decode_noalloc all take them from here.
void jbp::gf_build_tables(int m, uint8_t* mul, uint8_t* div)
{
    const int q = 1 << m;
    std::vector<int> inv(q, 0);
    for (int a = 1; a < q; ++a)
        for (int b = 1; b < q; ++b)
            if (gf_mul_host(a, b, m) == 1) inv[a] = b;
    for (int h = 0; h < q; ++h)
        for (int x = 0; x < q; ++x) {
            mul[(size_t)h * q + x] = (uint8_t)gf_mul_host(h, x, m);
            div[(size_t)h * q + x] = (uint8_t)gf_mul_host(inv[h], x, m);
        }
}

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------

namespace {

// A device buffer that only grows; its byte size is recorded so that it can be
// freed without knowing which decoder last used it.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Device buffers of one decode: step-form state and host-path staging.
struct Workspace {
    DevBuf msg, ch2v, active, unsat;             // step form, per frame state
    DevBuf y, hat, iters, ok, post, sig;         // staging for host buffers / serving
    uint64_t gen = 0;                            // bumped on every reallocation
};

struct Request {
    uint64_t ticket;
    jbp_h* h;
    std::vector<float> y;
    float sigma2;   // > 0: this frame's noise variance; otherwise the handle's
    double t_submit;
};

struct Result {
    std::vector<uint8_t> hat;
    std::vector<uint8_t> ok;
    int32_t iters = 0;
};

// Resident pool of the serving loop: step-form state of up to `cap` frame slots
// of one decoder, kept in HBM across blocks of iterations.
struct ServePool {
    jbp_h* h = nullptr;
    int cap = 0;                   // frame slots
    int hi = 0;                    // 1 + highest slot in use
    int n_active = 0;              // slots holding a frame that has not been harvested
    bool running = false;          // a block is in flight
    double last_used = 0;
    int64_t bytes = 0;             // device bytes held
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf msg, ch2v, y, sig, active, t, unsat, ok, hat, fin, adm_slot, adm_y, adm_sig, count;
    // pinned staging of an admission, and the harvest count of the last block
    int32_t* h_adm_slot = nullptr;
    float* h_adm_y = nullptr;
    float* h_adm_sig = nullptr;
    int32_t* h_count = nullptr;
    // harvest area: host-mapped, written by the device (h_*: host view, d_*: device view)
    int32_t* h_slot = nullptr;
    int32_t* h_iters = nullptr;
    uint8_t* h_ok = nullptr;
    uint8_t* h_hat = nullptr;
    int32_t* d_slot = nullptr;
    int32_t* d_iters = nullptr;
    uint8_t* d_ok = nullptr;
    uint8_t* d_hat = nullptr;
    std::vector<Request> req;      // [cap] the request each used slot holds
    std::vector<uint8_t> used;     // [cap]
    std::vector<int> free_list;
    // fused pool: slots keep the fused kernel's position-major state, and a
    // block is one launch of that kernel (launch_fused_pool)
    bool fused = false;
    FusedPlan fplan{};
    size_t fmsg = 0, fch2v = 0;    // floats of a slot's messages and channel messages
};

}  // namespace

struct jbp_ctx {
    jbp_options opt{};
    int device = 0;
    DeviceInfo di{};
    cudaStream_t stream = nullptr;
    cudaStream_t io_in = nullptr, io_out = nullptr;   // host-buffer decodes: copies beside the compute stream
    int64_t budget = 0;
    std::atomic<int64_t> used{0};

    // serving
    std::mutex mu;
    std::condition_variable cv;
    std::condition_variable cv_idle;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> done;
    std::unordered_map<uint64_t, int> pending;   // ticket -> 1 while queued or in flight
    std::vector<double> latencies;
    uint64_t completed = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool server_started = false;
    std::thread server;
    std::vector<std::unique_ptr<ServePool>> serve_pools;   // touched by the server thread only
    int64_t pool_bytes = 0;                                 // device bytes of the pools (server thread)
    std::unordered_map<const jbp_h*, int> pool_of;          // decoders that own a pool (under mu)
    int handles = 0;

    // multi-part decodes: stream pool, fork/join events, graphs keyed by arguments
    std::mutex many_mu;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> pool_ev;
    cudaEvent_t fork_ev = nullptr;
    // jbp_decode_many runs (and captures) on its own stream, ordered after and
    // before the caller's stream by these events: any caller stream works, the
    // legacy default stream included, and a captured graph serves every caller
    cudaStream_t many_stream = nullptr;
    cudaEvent_t many_in = nullptr, many_out = nullptr;
    struct GraphEntry {
        int seen = 0;
        cudaGraphExec_t exec = nullptr;
    };
    std::map<std::vector<uintptr_t>, GraphEntry> graphs;
};

struct jbp_h {
    jbp_ctx* ctx = nullptr;
    int K = 0, Q = 0, m = 0, n = 0, P = 0, dc = 0, dv = 0, E = 0;
    bool var_reg = true;                  // every variable has dv edges
    double sigma2 = 0;
    int32_t* d_chk_var = nullptr;
    uint8_t* d_chk_coef = nullptr;
    int32_t* d_var_edge = nullptr;
    int32_t* d_use_pos = nullptr;
    uint8_t* d_gf_mul = nullptr;
    uint8_t* d_gf_div = nullptr;
    unsigned long long* d_fallbacks = nullptr;
    int32_t* d_pos_of = nullptr;
    int* d_tc_error = nullptr;
    uint16_t* d_slot = nullptr;
    uint16_t* d_chk_order = nullptr;
    unsigned char* d_dft_tab = nullptr;   // tables of the tensor-core channel node (null: trellis)
    size_t dft_bytes = 0;
    int64_t table_bytes = 0;
    Workspace ws;
    std::mutex ws_mu;
    bool fused_ok = false;
    int tune_threads = 0, tune_fpc = 0;   // fused launch shape chosen by the autotuner (0 = default)
    bool tuned = false;
    uint64_t ws_gen = 0;                  // bumped whenever h->ws is reallocated (invalidates graphs)
    bool closing = false;                 // jbp_destroy in progress (under ctx->mu)
    // measured channel-node step times (us) of a serving pool of this decoder at
    // 1 and chan_fb frames, trellis and tensor-core node (serving under AUTO)
    bool chan_cal = false;
    int chan_fb = 1;
    float chan_t1 = 0, chan_tb = 0, chan_d1 = 0, chan_db = 0;

    Graph graph() const
    {
        Graph g;
        g.n = n; g.P = P; g.E = E; g.dc = dc; g.dv = dv; g.K = K; g.Q = Q;
        g.inv_sigma2 = (float)(1.0 / sigma2);
        g.chk_var = d_chk_var; g.chk_coef = d_chk_coef; g.var_edge = d_var_edge;
        g.use_pos = d_use_pos; g.gf_mul = d_gf_mul; g.gf_div = d_gf_div;
        g.log_fallbacks = d_fallbacks;
        g.pos_of = d_pos_of;
        g.slot = d_slot;
        g.tc_error = d_tc_error;
        g.sigma2_f = nullptr;
        g.chk_order = d_chk_order;
        g.dft_tab = d_dft_tab;
        g.var_reg = var_reg ? 1 : 0;
        return g;
    }
};

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------

template <class T>
static int dev_alloc(jbp_ctx* ctx, T** p, size_t count, int64_t* acct)
{
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (ctx->used.load() + (int64_t)bytes > ctx->budget)
        return fail(JBP_ENOMEM, "device memory budget exceeded (%lld + %zu > %lld bytes)",
                    (long long)ctx->used.load(), bytes, (long long)ctx->budget);
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(JBP_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->used += (int64_t)bytes;
    if (acct) *acct += (int64_t)bytes;
    return JBP_OK;
}

static void dev_free(jbp_ctx* ctx, void* p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    ctx->used -= (int64_t)std::max<size_t>(bytes, 16);
}

static int buf_ensure(jbp_ctx* ctx, DevBuf& b, size_t bytes, bool* grew)
{
    bytes = std::max<size_t>(bytes, 16);
    if (bytes <= b.bytes) return JBP_OK;
    dev_free(ctx, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
    int rc = dev_alloc(ctx, reinterpret_cast<unsigned char**>(&b.p), bytes, nullptr);
    if (rc) return rc;
    b.bytes = bytes;
    *grew = true;
    return JBP_OK;
}

static void buf_free(jbp_ctx* ctx, DevBuf& b)
{
    dev_free(ctx, b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
}

static void ws_release(jbp_ctx* ctx, Workspace& w)
{
    for (DevBuf* b : {&w.msg, &w.ch2v, &w.active, &w.unsat, &w.y, &w.hat, &w.iters, &w.ok, &w.post, &w.sig})
        buf_free(ctx, *b);
    w.gen++;
}

static int ws_step(jbp_ctx* ctx, const jbp_h* h, Workspace& w, int F)
{
    const size_t fs = (size_t)h->K * h->E * h->Q, vs = (size_t)h->K * h->n * h->Q;
    bool grew = false;
    int rc;
    if ((rc = buf_ensure(ctx, w.msg, sizeof(float) * fs * F, &grew)) ||
        (rc = buf_ensure(ctx, w.ch2v, sizeof(float) * vs * F, &grew)) ||
        (rc = buf_ensure(ctx, w.active, (size_t)F, &grew)) || (rc = buf_ensure(ctx, w.unsat, (size_t)F * h->K, &grew))) {
        w.gen++;
        return rc;
    }
    if (grew) w.gen++;
    return JBP_OK;
}

static int ws_io(jbp_ctx* ctx, const jbp_h* h, Workspace& w, int F, bool post)
{
    const size_t vs = (size_t)h->K * h->n * h->Q;
    const size_t cap = std::max(F, 1);
    bool grew = false;
    int rc;
    if ((rc = buf_ensure(ctx, w.y, sizeof(float) * cap * h->n, &grew)) ||
        (rc = buf_ensure(ctx, w.hat, cap * h->K * h->n, &grew)) ||
        (rc = buf_ensure(ctx, w.iters, sizeof(int32_t) * cap, &grew)) ||
        (rc = buf_ensure(ctx, w.ok, cap * h->K, &grew)) || (rc = buf_ensure(ctx, w.sig, sizeof(float) * cap, &grew)) ||
        (post && (rc = buf_ensure(ctx, w.post, sizeof(float) * vs * cap, &grew)))) {
        w.gen++;
        return rc;
    }
    if (grew) w.gen++;
    return JBP_OK;
}

template <class T>
static T* P(const DevBuf& b) { return static_cast<T*>(b.p); }

// ---------------------------------------------------------------------------
// decode forms
// ---------------------------------------------------------------------------

static int run_step_iters(jbp_h* h, const Graph& g, Workspace& w, int F, const float* y, uint8_t* hat, int32_t* iters,
                          uint8_t* ok, float* post, cudaStream_t s)
{
    jbp_ctx* ctx = h->ctx;
    const size_t fs = (size_t)h->K * h->E * h->Q;
    float* msg = P<float>(w.msg);
    float* ch2v = P<float>(w.ch2v);
    uint8_t* active = P<uint8_t>(w.active);
    uint8_t* unsat = P<uint8_t>(w.unsat);
    JBP_CU(launch_fill(msg, fs * F, 1.0f, s), "init msg");
    JBP_CU(cudaMemsetAsync(active, 1, (size_t)F, s), "memset active");
    JBP_CU(cudaMemsetAsync(unsat, 0, (size_t)F * h->K, s), "memset unsat");
    StepCtl c{active, unsat, iters, ok};
    for (int t = 1; t <= ctx->opt.iters; ++t) {
        JBP_CU(launch_channel(g, ctx->di, F, y, msg, ch2v, active, s), "channel kernel");
        JBP_CU(launch_check(g, ctx->di, F, msg, active, ctx->opt.precision, s), "check kernel");
        JBP_CU(launch_var(g, ctx->di, F, ch2v, msg, post, hat, active, s), "var kernel");
        JBP_CU(launch_syndrome(g, ctx->di, F, hat, unsat, active, s), "syndrome kernel");
        JBP_CU(launch_finalize(F, h->K, t, ctx->opt.early_stop, c, s), "finalize kernel");
    }
    return JBP_OK;
}

// Decode F frames whose buffers are all on the device, on stream s.
static int decode_device(jbp_h* h, Workspace& w, int form, int F, const float* y, uint8_t* hat, int32_t* iters,
                         uint8_t* ok, float* post, const float* sigma2_f, cudaStream_t s)
{
    if (F == 0) return JBP_OK;
    jbp_ctx* ctx = h->ctx;
    Graph g = h->graph();
    g.sigma2_f = sigma2_f;
    // the fused kernel runs the FP32 butterfly check node; the tensor-core
    // precision variants run in the step form
    if (form == JBP_FORM_AUTO)
        form = (h->fused_ok && ctx->opt.precision == JBP_PREC_FP32 && !h->d_dft_tab) ? JBP_FORM_FUSED : JBP_FORM_STEP;
    if (form == JBP_FORM_FUSED && ctx->opt.precision != JBP_PREC_FP32)
        return fail(JBP_EINVAL, "the fused form runs the FP32 check node; use the step form for precision %d",
                    ctx->opt.precision);
    if (form == JBP_FORM_FUSED && h->d_dft_tab)
        return fail(JBP_EINVAL, "the fused form runs the trellis channel node; use the step form for the DFT node");
    if (form == JBP_FORM_FUSED) {
        if (!h->fused_ok) return fail(JBP_EINVAL, "one frame does not fit the fused form (shared memory)");
        FusedPlan plan;
        if (!fused_plan(g, ctx->di, F, h->tune_threads, h->tune_fpc, &plan)) return fail(JBP_EINVAL, "no fused launch plan");
        JBP_CU(launch_fused(g, plan, F, y, ctx->opt.iters, ctx->opt.early_stop, hat, iters, ok, post, s), "fused kernel");
        return JBP_OK;
    }
    if (form == JBP_FORM_STEP) {
        int rc = ws_step(ctx, h, w, F);
        if (rc) return rc;
        return run_step_iters(h, g, w, F, y, hat, iters, ok, post, s);
    }
    if (form == JBP_FORM_PLAIN) {
        int rc = ws_step(ctx, h, w, 1);
        if (rc) return rc;
        const size_t vs = (size_t)h->K * h->n * h->Q;
        for (int f = 0; f < F; ++f) {
            Graph gf = g;
            if (sigma2_f) gf.sigma2_f = sigma2_f + f;
            rc = run_step_iters(h, gf, w, 1, y + (size_t)f * h->n, hat + (size_t)f * h->K * h->n, iters + f,
                                ok + (size_t)f * h->K, post ? post + vs * f : nullptr, s);
            if (rc) return rc;
        }
        return JBP_OK;
    }
    return fail(JBP_EINVAL, "unknown form %d", form);
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

static void server_main(jbp_ctx* ctx);
static void pool_destroy(jbp_ctx* ctx, ServePool* p);

extern "C" int jbp_context_create(const jbp_options* opt, jbp_ctx** out)
{
    if (!opt || !out) return fail(JBP_EINVAL, "jbp_context_create: NULL argument");
    if (opt->iters < 1) return fail(JBP_EINVAL, "iters must be >= 1 (got %d)", opt->iters);
    if (opt->precision < 0 || opt->precision > 3) return fail(JBP_EINVAL, "bad precision %d", opt->precision);
    if (opt->channel_node < JBP_CHAN_TRELLIS || opt->channel_node > JBP_CHAN_AUTO)
        return fail(JBP_EINVAL, "bad channel_node %d", opt->channel_node);
    if (opt->mem_budget_bytes < 0) return fail(JBP_EINVAL, "negative memory budget");
    int ndev = 0;
    JBP_CU(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (opt->device < 0 || opt->device >= ndev) return fail(JBP_EINVAL, "device %d out of range (%d devices)", opt->device, ndev);
    JBP_CU(cudaSetDevice(opt->device), "cudaSetDevice");
    jbp_ctx* ctx = new (std::nothrow) jbp_ctx();
    if (!ctx) return fail(JBP_ENOMEM, "host allocation failed");
    ctx->opt = *opt;
    if (ctx->opt.block_iters <= 0) ctx->opt.block_iters = 5;
    ctx->device = opt->device;
    cudaError_t e;
    if ((e = cudaDeviceGetAttribute(&ctx->di.sm_count, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&ctx->di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->io_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->io_out, cudaStreamNonBlocking)) != cudaSuccess) {
        for (cudaStream_t st : {ctx->stream, ctx->io_in, ctx->io_out})
            if (st) cudaStreamDestroy(st);
        delete ctx;
        return cuda_fail(e, "context setup");
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    ctx->budget = opt->mem_budget_bytes > 0 ? opt->mem_budget_bytes : (int64_t)(0.9 * (double)free_b);
    *out = ctx;
    return JBP_OK;
}

extern "C" int jbp_context_destroy(jbp_ctx* ctx)
{
    if (!ctx) return fail(JBP_EINVAL, "jbp_context_destroy: NULL context");
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->handles > 0) return fail(JBP_EINVAL, "context still has %d live handles", ctx->handles);
        ctx->stop = true;
    }
    ctx->cv.notify_all();
    if (ctx->server.joinable()) ctx->server.join();
    cudaSetDevice(ctx->device);
    while (!ctx->serve_pools.empty()) {
        pool_destroy(ctx, ctx->serve_pools.back().get());
        ctx->serve_pools.pop_back();
    }
    for (auto& kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (cudaStream_t st : ctx->pool) cudaStreamDestroy(st);
    for (cudaEvent_t ev : ctx->pool_ev) cudaEventDestroy(ev);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->many_stream) cudaStreamDestroy(ctx->many_stream);
    if (ctx->many_in) cudaEventDestroy(ctx->many_in);
    if (ctx->many_out) cudaEventDestroy(ctx->many_out);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->io_in) cudaStreamDestroy(ctx->io_in);
    if (ctx->io_out) cudaStreamDestroy(ctx->io_out);
    delete ctx;
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------

// Order of the K*P check units (k, j) in the fused kernel's check phase.  A
// warp runs 32 consecutive units, and the d-th edge message of unit (k, j) lives
// in shared-memory bank (position mod 32) of that edge, so the d-th loads of a
// warp cost as many wavefronts as the largest number of its units sharing that
// bank.  Greedy fill of each run of 32 with units whose banks are still free,
// then annealed pairwise swaps between runs.  Deterministic (fixed-seed
// xorshift); the order does not change any result.
static std::vector<uint16_t> check_order(int K, int P, int E, const std::vector<uint16_t>& slot)
{
    const int N = K * P, R = (N + 31) / 32;
    std::vector<std::array<uint8_t, kDC>> col(N);
    for (int u = 0; u < N; ++u) {
        const int k = u / P, j = u % P;
        // bank of the edge's message: its position within the row, rotated by
        // 16 for users 2 and 3 (pos_rot of the fused layout)
        for (int d = 0; d < kDC; ++d)
            col[u][d] = (uint8_t)(((slot[(size_t)k * E + kDC * j + d] >> 1) + ((k & 2) << 3)) & 31);
    }
    uint64_t x = 0x9e3779b97f4a7c15ull;
    auto rnd = [&]() {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        return x;
    };
    std::vector<int> rem(N);
    for (int u = 0; u < N; ++u) rem[u] = u;
    for (int i = N - 1; i > 0; --i) std::swap(rem[i], rem[rnd() % (uint64_t)(i + 1)]);
    std::vector<int> order;
    order.reserve(N);
    std::vector<std::array<std::array<int, 32>, kDC>> cnt(R);
    for (int r = 0; r < R; ++r) {
        for (auto& a : cnt[r]) a.fill(0);
        const int want = std::min(32, N - r * 32);
        int got = 0;
        for (int pass = 0; pass < 2 && got < want; ++pass)
            for (size_t i = 0; i < rem.size() && got < want;) {
                const int u = rem[i];
                bool free_all = true;
                for (int d = 0; d < kDC; ++d) free_all = free_all && cnt[r][d][col[u][d]] == 0;
                if (pass == 1 || free_all) {
                    for (int d = 0; d < kDC; ++d) cnt[r][d][col[u][d]]++;
                    order.push_back(u);
                    rem.erase(rem.begin() + i);
                    ++got;
                } else {
                    ++i;
                }
            }
    }
    // Annealed pairwise swaps between runs on the sum of squared bank counts
    // (every collision costs, so the search has a gradient that the largest count
    // alone lacks); the cost of a swap changes only in the two runs' counts.
    if (R > 1) {
        const long iters = 800l * N;
        for (long it = 0; it < iters; ++it) {
            const int i1 = (int)(rnd() % (uint64_t)N), i2 = (int)(rnd() % (uint64_t)N);
            const int r1 = i1 / 32, r2 = i2 / 32;
            if (r1 == r2) continue;
            const int u1 = order[i1], u2 = order[i2];
            int delta = 0;
            for (int d = 0; d < kDC; ++d) {
                const int a = col[u1][d], b = col[u2][d];
                if (a == b) continue;
                // u1 (bank a) leaves r1 for r2, u2 (bank b) leaves r2 for r1
                delta += 2 * (cnt[r1][d][b] - cnt[r1][d][a] + 1) + 2 * (cnt[r2][d][a] - cnt[r2][d][b] + 1);
            }
            // temperature falls linearly from 2 to 0; uniform in [0, 1) from 53 random bits
            const double temp = 2.0 * (1.0 - (double)it / (double)iters);
            const double u01 = (double)(rnd() >> 11) * (1.0 / 9007199254740992.0);
            if (delta <= 0 || (temp > 0.0 && u01 < std::exp(-delta / temp))) {
                std::swap(order[i1], order[i2]);
                for (int d = 0; d < kDC; ++d) {
                    cnt[r1][d][col[u1][d]]--; cnt[r1][d][col[u2][d]]++;
                    cnt[r2][d][col[u2][d]]--; cnt[r2][d][col[u1][d]]++;
                }
            }
        }
    }
    std::vector<uint16_t> out(N);
    for (int i = 0; i < N; ++i) out[i] = (uint16_t)order[i];
    return out;
}

static int chan_calibrate(jbp_ctx* ctx, jbp_h* h);

extern "C" int jbp_create(jbp_ctx* ctx, const jbp_code* code, int32_t K, int32_t q, const jbp_channel* chan,
                          jbp_h** out)
{
    if (!ctx || !code || !chan || !out) return fail(JBP_EINVAL, "jbp_create: NULL argument");
    int m = 0;
    while ((1 << m) < q && m < 8) ++m;
    if (q < 2 || q > 64 || (1 << m) != q) return fail(JBP_EINVAL, "q must be a power of two in 2..64 (got %d)", q);
    if (code->q != q) return fail(JBP_EINVAL, "code->q (%d) != q (%d)", code->q, q);
    if (K < 1 || K > kMaxK) return fail(JBP_EINVAL, "K must be in 1..%d (got %d)", kMaxK, K);
    if (code->n < 1 || code->P < 1) return fail(JBP_EINVAL, "n and P must be >= 1");
    if (code->dc != 3 && code->dc != 4 && code->dc != 6)
        return fail(JBP_EINVAL, "check degree dc must be 3, 4 or 6 (got %d)", code->dc);
    if (code->dv < 1 || code->dv > kMaxDv) return fail(JBP_EINVAL, "dv must be in 1..%d (got %d)", kMaxDv, code->dv);
    if ((int64_t)code->n * code->dv < (int64_t)code->P * code->dc)
        return fail(JBP_EINVAL, "P*dc (%d*%d) edges exceed n*dv (%d*%d)", code->P, code->dc, code->n, code->dv);
    if (ctx->opt.precision != JBP_PREC_FP32 && code->dc != kDC)
        return fail(JBP_EINVAL, "the tensor-core check variants are built for dc = 4 (got %d)", code->dc);
    if (!code->chk_var || !code->chk_coef) return fail(JBP_EINVAL, "NULL code arrays");
    if (!(chan->sigma2 > 0.0) || !std::isfinite(chan->sigma2)) return fail(JBP_EINVAL, "sigma2 must be finite and > 0");
    if (chan->interleave && !chan->perm) return fail(JBP_EINVAL, "interleave = 1 needs perm");
    const int n = code->n, P = code->P, dc = code->dc, dv = code->dv, E = P * dc;

    std::vector<int32_t> var_edge((size_t)n * dv, -1), fill(n, 0);
    for (int e = 0; e < E; ++e) {
        const int i = code->chk_var[e];
        if (i < 0 || i >= n) return fail(JBP_EINVAL, "chk_var[%d] = %d out of range", e, i);
        if (code->chk_coef[e] < 1 || code->chk_coef[e] >= q) return fail(JBP_EINVAL, "chk_coef[%d] = %d not in 1..q-1", e, code->chk_coef[e]);
        if (fill[i] >= dv) return fail(JBP_EINVAL, "variable %d has more than dv = %d edges", i, dv);
        var_edge[(size_t)i * dv + fill[i]++] = e;
    }
    // dv is the largest variable degree: a variable may have fewer edges (an
    // irregular degree profile; its var_edge row ends with -1 entries)
    bool var_reg = true;
    for (int i = 0; i < n; ++i) var_reg = var_reg && fill[i] == dv;
    std::vector<int32_t> use_pos((size_t)K * n, -1);
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < n; ++i) {
            const int t = chan->interleave ? chan->perm[(size_t)k * n + i] : i;
            if (t < 0 || t >= n || use_pos[(size_t)k * n + t] != -1)
                return fail(JBP_EINVAL, "perm row %d is not a permutation of 0..n-1", k);
            use_pos[(size_t)k * n + t] = i;
        }
    // position-major tables of the fused form: pi_k(i) and, per user and edge,
    // pi_k(var)*2 + (rank of the edge among its variable's edges)
    std::vector<int32_t> pos_of((size_t)K * n);
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < n; ++i) pos_of[(size_t)k * n + i] = chan->interleave ? chan->perm[(size_t)k * n + i] : i;
    const bool want_slot = dv == 2 && var_reg && n <= 32767;
    std::vector<uint16_t> slot(want_slot ? (size_t)K * E : 0);
    if (want_slot)
        for (int k = 0; k < K; ++k)
            for (int e = 0; e < E; ++e) {
                const int i = code->chk_var[e];
                const int rank = var_edge[(size_t)i * dv] == e ? 0 : 1;
                slot[(size_t)k * E + e] = (uint16_t)(pos_of[(size_t)k * n + i] * 2 + rank);
            }
    // only where the fused position-major form can run (K <= 4, q <= 16, one
    // frame's state in shared memory)
    const bool want_order = want_slot && dc == kDC && K <= 4 && q <= 16 &&
                            4ll * K * (E + n) * q <= (int64_t)ctx->di.smem_optin;
    std::vector<uint16_t> chk_order;
    if (want_order) chk_order = check_order(K, P, E, slot);
    const DftShape dsh = dft_shape(K, q);
    // AUTO: the transform except where the register-resident trellis (thread shape) applies
    const bool thread_shape = q <= 16 && K <= 4;
    const bool want_dft = (ctx->opt.channel_node == JBP_CHAN_DFT ||
                           (ctx->opt.channel_node == JBP_CHAN_AUTO && !thread_shape)) &&
                          dv == 2 && var_reg && dc == kDC && dsh.ok && dsh.smem <= ctx->di.smem_optin;
    std::vector<unsigned char> dft_tab;   // shape tables, then this handle's message offsets
    if (want_dft) {
        dft_tab.resize(dft_table_bytes(K, q) + dft_offsets_bytes(K, n));
        dft_build_table(K, q, dft_tab.data());
        dft_build_offsets(K, q, n, E, use_pos.data(), var_edge.data(),
                          reinterpret_cast<int32_t*>(dft_tab.data() + dft_table_bytes(K, q)));
    }
    std::vector<uint8_t> gmul((size_t)q * q), gdiv((size_t)q * q);
    gf_build_tables(m, gmul.data(), gdiv.data());
    const int scf = blk_scratch_floats(K, q);
    const int team_lanes = q < 32 ? q : 32;
    if ((size_t)(32 / team_lanes) * scf * sizeof(float) > (size_t)ctx->di.smem_optin)
        return fail(JBP_EINVAL, "K = %d, q = %d: channel trellis does not fit shared memory", K, q);

    JBP_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    jbp_h* h = new (std::nothrow) jbp_h();
    if (!h) return fail(JBP_ENOMEM, "host allocation failed");
    h->ctx = ctx; h->K = K; h->Q = q; h->m = m; h->n = n; h->P = P; h->dc = dc; h->dv = dv; h->E = E;
    h->sigma2 = chan->sigma2;
    h->var_reg = var_reg;
    int rc;
    if ((rc = dev_alloc(ctx, &h->d_chk_var, (size_t)E, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_chk_coef, (size_t)E, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_var_edge, (size_t)n * dv, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_use_pos, (size_t)K * n, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_gf_mul, (size_t)q * q, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_gf_div, (size_t)q * q, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_fallbacks, (size_t)1, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_pos_of, (size_t)K * n, &h->table_bytes)) ||
        (rc = dev_alloc(ctx, &h->d_tc_error, (size_t)1, &h->table_bytes)) ||
        (want_slot && (rc = dev_alloc(ctx, &h->d_slot, (size_t)K * E, &h->table_bytes))) ||
        (want_order && (rc = dev_alloc(ctx, &h->d_chk_order, (size_t)K * P, &h->table_bytes))) ||
        (want_dft && (rc = dev_alloc(ctx, &h->d_dft_tab, dft_tab.size(), &h->table_bytes)))) {
        jbp_destroy(h);
        return rc;
    }
    if (want_dft) h->dft_bytes = dft_tab.size();
    cudaError_t e;
    if ((e = cudaMemcpy(h->d_chk_var, code->chk_var, sizeof(int32_t) * E, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d_chk_coef, code->chk_coef, (size_t)E, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d_var_edge, var_edge.data(), sizeof(int32_t) * var_edge.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d_use_pos, use_pos.data(), sizeof(int32_t) * use_pos.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d_gf_mul, gmul.data(), gmul.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d_gf_div, gdiv.data(), gdiv.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(h->d_fallbacks, 0, sizeof(unsigned long long))) ||
        (e = cudaMemset(h->d_tc_error, 0, sizeof(int))) ||
        (e = cudaMemcpy(h->d_pos_of, pos_of.data(), sizeof(int32_t) * pos_of.size(), cudaMemcpyHostToDevice)) ||
        (want_slot &&
         (e = cudaMemcpy(h->d_slot, slot.data(), sizeof(uint16_t) * slot.size(), cudaMemcpyHostToDevice))) ||
        (want_order && (e = cudaMemcpy(h->d_chk_order, chk_order.data(), sizeof(uint16_t) * chk_order.size(),
                                       cudaMemcpyHostToDevice))) ||
        (want_dft && (e = cudaMemcpy(h->d_dft_tab, dft_tab.data(), dft_tab.size(), cudaMemcpyHostToDevice)))) {
        jbp_destroy(h);
        return cuda_fail(e, "jbp_create: copy tables");
    }
    FusedPlan plan;
    h->fused_ok = fused_plan(h->graph(), ctx->di, 1, 0, 0, &plan);
    cudaGetLastError();
    if (want_dft && ctx->opt.channel_node == JBP_CHAN_AUTO && (rc = chan_calibrate(ctx, h)) != JBP_OK) {
        jbp_destroy(h);
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->handles++;
    }
    *out = h;
    return JBP_OK;
}

// The tensor-core channel node's launches have a latency floor (one CTA per
// tile of 128 channel uses), so a launch over a few frames is faster on the
// trellis.  Under AUTO, jbp_create measures both nodes on a decoder with DFT
// tables at 1 frame and at fb frames (the count whose tiles fill the SMs, at
// most 256 MB of temporary state) on a uniform message state; serving pools then
// take the node that chan_est rates faster for their frame count.
static int chan_calibrate(jbp_ctx* ctx, jbp_h* h)
{
    const DeviceInfo& di = ctx->di;
    const size_t per_frame = (size_t)state_bytes(h->graph()) + sizeof(float) * h->n + 1;
    int fb = std::max(1, (128 * di.sm_count + h->n - 1) / h->n);
    fb = (int)std::max<size_t>(1, std::min<size_t>((size_t)fb, (size_t(256) << 20) / per_frame));
    float *msg = nullptr, *ch2v = nullptr, *y = nullptr;
    uint8_t* act = nullptr;
    int64_t acct = 0;
    int rc;
    if ((rc = dev_alloc(ctx, &msg, (size_t)fb * h->K * h->E * h->Q, &acct)) ||
        (rc = dev_alloc(ctx, &ch2v, (size_t)fb * h->K * h->n * h->Q, &acct)) ||
        (rc = dev_alloc(ctx, &y, (size_t)fb * h->n, &acct)) || (rc = dev_alloc(ctx, &act, (size_t)fb, &acct))) {
        dev_free(ctx, msg, sizeof(float) * (size_t)fb * h->K * h->E * h->Q);
        dev_free(ctx, ch2v, sizeof(float) * (size_t)fb * h->K * h->n * h->Q);
        dev_free(ctx, y, sizeof(float) * (size_t)fb * h->n);
        dev_free(ctx, act, (size_t)fb);
        return rc;
    }
    cudaStream_t s = ctx->stream;
    cudaEvent_t a = nullptr, b = nullptr;
    float t[2][2] = {{0, 0}, {0, 0}};
    cudaError_t e = launch_fill(msg, (size_t)fb * h->K * h->E * h->Q, 1.0f, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, sizeof(float) * (size_t)fb * h->n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(act, 1, (size_t)fb, s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    for (int node = 0; node < 2 && e == cudaSuccess; ++node) {
        Graph g = h->graph();
        if (node == 0) g.dft_tab = nullptr;
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            const int F = i == 0 ? 1 : fb;
            float best = 1e30f;
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                float ms = 0;
                e = cudaEventRecord(a, s);
                if (e == cudaSuccess) e = launch_channel(g, di, F, y, msg, ch2v, act, s);
                if (e == cudaSuccess) e = cudaEventRecord(b, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) best = std::min(best, ms * 1e3f);   // the first launch is a warm-up
            }
            t[node][i] = best;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    dev_free(ctx, msg, sizeof(float) * (size_t)fb * h->K * h->E * h->Q);
    dev_free(ctx, ch2v, sizeof(float) * (size_t)fb * h->K * h->n * h->Q);
    dev_free(ctx, y, sizeof(float) * (size_t)fb * h->n);
    dev_free(ctx, act, (size_t)fb);
    if (e != cudaSuccess || e2 != cudaSuccess) return cuda_fail(e != cudaSuccess ? e : e2, "channel-node calibration");
    h->chan_t1 = t[0][0];
    h->chan_tb = t[0][1];
    h->chan_d1 = t[1][0];
    h->chan_db = t[1][1];
    h->chan_fb = fb;
    h->chan_cal = true;
    return JBP_OK;
}

extern "C" int jbp_destroy(jbp_h* h)
{
    if (!h) return fail(JBP_EINVAL, "jbp_destroy: NULL handle");
    jbp_ctx* ctx = h->ctx;
    bool counted = h->d_gf_div != nullptr;
    {
        std::unique_lock<std::mutex> lk(ctx->mu);
        // cancel queued requests of this handle, wait for its in-flight batches
        for (auto it = ctx->queue.begin(); it != ctx->queue.end();) {
            if (it->h == h) {
                ctx->pending.erase(it->ticket);
                it = ctx->queue.erase(it);
            } else {
                ++it;
            }
        }
        h->closing = true;
        ctx->cv.notify_all();
        // the server finishes the handle's frames in flight, then frees its pool
        ctx->cv_idle.wait(lk, [&] { return ctx->pool_of.count(h) == 0; });
        if (counted) ctx->handles--;
    }
    cudaSetDevice(ctx->device);
    {
        // graphs captured with this handle refer to its tables and workspace
        std::lock_guard<std::mutex> lk(ctx->many_mu);
        for (cudaStream_t st : ctx->pool) cudaStreamSynchronize(st);
        if (ctx->many_stream) cudaStreamSynchronize(ctx->many_stream);
        for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
            bool uses = false;
            for (size_t i = 1; i < it->first.size(); i += 10)
                if (it->first[i] == (uintptr_t)h) uses = true;
            if (uses) {
                if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
                it = ctx->graphs.erase(it);
            } else {
                ++it;
            }
        }
    }
    cudaStreamSynchronize(ctx->stream);
    ws_release(ctx, h->ws);
    dev_free(ctx, h->d_chk_var, sizeof(int32_t) * h->E);
    dev_free(ctx, h->d_chk_coef, (size_t)h->E);
    dev_free(ctx, h->d_var_edge, sizeof(int32_t) * (size_t)h->n * h->dv);
    dev_free(ctx, h->d_use_pos, sizeof(int32_t) * (size_t)h->K * h->n);
    dev_free(ctx, h->d_gf_mul, (size_t)h->Q * h->Q);
    dev_free(ctx, h->d_gf_div, (size_t)h->Q * h->Q);
    dev_free(ctx, h->d_fallbacks, sizeof(unsigned long long));
    dev_free(ctx, h->d_pos_of, sizeof(int32_t) * (size_t)h->K * h->n);
    dev_free(ctx, h->d_dft_tab, h->dft_bytes);
    dev_free(ctx, h->d_tc_error, sizeof(int));
    if (h->d_slot) dev_free(ctx, h->d_slot, sizeof(uint16_t) * (size_t)h->K * h->E);
    if (h->d_chk_order) dev_free(ctx, h->d_chk_order, sizeof(uint16_t) * (size_t)h->K * h->P);
    delete h;
    return JBP_OK;
}

extern "C" int jbp_query(jbp_h* h, int32_t* E, int64_t* state_bytes_per_frame, int32_t* fused)
{
    if (!h) return fail(JBP_EINVAL, "jbp_query: NULL handle");
    if (E) *E = h->E;
    if (state_bytes_per_frame) *state_bytes_per_frame = state_bytes(h->graph());
    if (fused) *fused = h->fused_ok ? 1 : 0;
    return JBP_OK;
}

extern "C" int jbp_query_channel(jbp_h* h, int32_t* node)
{
    if (!h || !node) return fail(JBP_EINVAL, "jbp_query_channel: NULL argument");
    *node = h->d_dft_tab ? JBP_CHAN_DFT : JBP_CHAN_TRELLIS;
    return JBP_OK;
}

extern "C" int jbp_gf_tables(int32_t q, uint8_t* mul, uint8_t* div)
{
    int m = 0;
    while (m < 7 && (1 << m) < q) ++m;
    if (q < 2 || q > 64 || (1 << m) != q) return fail(JBP_EINVAL, "jbp_gf_tables: q = %d (2, 4, ..., 64)", q);
    if (!mul || !div) return fail(JBP_EINVAL, "jbp_gf_tables: NULL argument");
    gf_build_tables(m, mul, div);
    return JBP_OK;
}

extern "C" int jbp_dft_tables(int32_t K, int32_t q, int32_t* shape, void* out, int64_t* bytes)
{
    if (!bytes) return fail(JBP_EINVAL, "jbp_dft_tables: NULL bytes");
    if (q != 16 && q != 32 && q != 64) return fail(JBP_EINVAL, "jbp_dft_tables: q = %d (16, 32 or 64)", q);
    const DftShape S = dft_shape(K, q);
    if (!S.ok) return fail(JBP_EINVAL, "jbp_dft_tables: no DFT form for K = %d, q = %d", K, q);
    *bytes = (int64_t)dft_table_bytes(K, q);
    if (shape) {
        shape[0] = S.L;
        shape[1] = S.W;
        shape[2] = S.KB;
        shape[3] = S.Nc;
        shape[4] = S.chunks;
    }
    if (out) dft_build_table(K, q, static_cast<unsigned char*>(out));
    return JBP_OK;
}

extern "C" int jbp_stats(jbp_h* h, uint64_t* log_fallbacks, int32_t* tc_timeouts)
{
    if (!h) return fail(JBP_EINVAL, "jbp_stats: NULL handle");
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    unsigned long long v = 0;
    int err = 0;
    JBP_CU(cudaDeviceSynchronize(), "jbp_stats");
    JBP_CU(cudaMemcpy(&v, h->d_fallbacks, sizeof v, cudaMemcpyDeviceToHost), "jbp_stats: copy");
    JBP_CU(cudaMemcpy(&err, h->d_tc_error, sizeof err, cudaMemcpyDeviceToHost), "jbp_stats: copy");
    if (log_fallbacks) *log_fallbacks = v;
    if (tc_timeouts) *tc_timeouts = err;
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// decode
// ---------------------------------------------------------------------------

// host-buffer decodes of at least kPipeMinFrames frames run as kPipeChunks parts
// whose copies overlap the other parts' decodes
static constexpr int kPipeChunks = 8;
static constexpr int kPipeMinFrames = 8192;

extern "C" int jbp_decode(jbp_h* h, jbp_batch* b)
{
    if (!h || !b) return fail(JBP_EINVAL, "jbp_decode: NULL argument");
    if (b->F < 0) return fail(JBP_EINVAL, "F must be >= 0");
    if (b->form < JBP_FORM_AUTO || b->form > JBP_FORM_PLAIN) return fail(JBP_EINVAL, "bad form %d", b->form);
    if (b->F == 0) return JBP_OK;
    if (!b->y || !b->hat || !b->iters || !b->ok) return fail(JBP_EINVAL, "jbp_decode: NULL buffer");
    jbp_ctx* ctx = h->ctx;
    JBP_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int F = b->F;
    if (b->on_device) {
        cudaStream_t s = b->stream ? (cudaStream_t)b->stream : ctx->stream;
        std::lock_guard<std::mutex> lk(h->ws_mu);
        return decode_device(h, h->ws, b->form, F, b->y, b->hat, b->iters, b->ok, b->logpost, b->sigma2, s);
    }
    cudaStream_t s = ctx->stream;
    std::lock_guard<std::mutex> lk(h->ws_mu);
    Workspace& w = h->ws;
    int rc = ws_io(ctx, h, w, F, b->logpost != nullptr);
    if (rc) return rc;
    const size_t vs = (size_t)h->K * h->n * h->Q, KN = (size_t)h->K * h->n;
    float* dy = P<float>(w.y);
    float* dsig = P<float>(w.sig);
    float* dpost = P<float>(w.post);
    uint8_t* dhat = P<uint8_t>(w.hat);
    int32_t* dit = P<int32_t>(w.iters);
    uint8_t* dok = P<uint8_t>(w.ok);
    // A large batch goes in kPipeChunks parts: part c's inputs travel on io_in, its
    // decode runs on the compute stream once they are in (parts in order, so the
    // step form's workspace is reused safely), and its results travel back on
    // io_out once it is decoded, so copies overlap the other parts' decodes.
    // Every frame is decoded as it would be in one launch.
    const int parts = F >= kPipeMinFrames ? kPipeChunks : 1;
    cudaEvent_t ev_in[kPipeChunks] = {}, ev_done[kPipeChunks] = {};
    cudaStream_t sin = parts > 1 ? ctx->io_in : s, sout = parts > 1 ? ctx->io_out : s;
    auto cleanup = [&]() {
        for (int c = 0; c < kPipeChunks; ++c) {
            if (ev_in[c]) cudaEventDestroy(ev_in[c]);
            if (ev_done[c]) cudaEventDestroy(ev_done[c]);
        }
    };
    for (int c = 0; c < parts; ++c)
        if (parts > 1 && (cudaEventCreateWithFlags(&ev_in[c], cudaEventDisableTiming) != cudaSuccess ||
                          cudaEventCreateWithFlags(&ev_done[c], cudaEventDisableTiming) != cudaSuccess)) {
            cleanup();
            cudaGetLastError();
            return fail(JBP_ECUDA, "jbp_decode: event creation failed");
        }
    auto part = [&](int c, int& f0, int& nf) {   // the first parts are the larger ones (workspaces only grow)
        const int base = F / parts, rem = F % parts;
        f0 = c * base + std::min(c, rem);
        nf = base + (c < rem ? 1 : 0);
    };
    auto fetch = [&](int c) {   // results of part c back to the caller's buffers
        int f0, nf;
        part(c, f0, nf);
        cudaError_t e;
        if ((parts > 1 && (e = cudaStreamWaitEvent(sout, ev_done[c], 0)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(b->hat + KN * f0, dhat + KN * f0, KN * nf, cudaMemcpyDeviceToHost, sout)) != cudaSuccess ||
            (e = cudaMemcpyAsync(b->iters + f0, dit + f0, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost, sout)) != cudaSuccess ||
            (e = cudaMemcpyAsync(b->ok + (size_t)h->K * f0, dok + (size_t)h->K * f0, (size_t)h->K * nf,
                                 cudaMemcpyDeviceToHost, sout)) != cudaSuccess ||
            (b->logpost && (e = cudaMemcpyAsync(b->logpost + vs * f0, dpost + vs * f0, sizeof(float) * vs * nf,
                                                cudaMemcpyDeviceToHost, sout)) != cudaSuccess))
            return cuda_fail(e, "jbp_decode: copy results");
        return (int)JBP_OK;
    };
    for (int c = 0; c < parts && rc == JBP_OK; ++c) {
        int f0, nf;
        part(c, f0, nf);
        cudaError_t e = cudaMemcpyAsync(dy + (size_t)h->n * f0, b->y + (size_t)h->n * f0, sizeof(float) * h->n * nf,
                                        cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess && b->sigma2)
            e = cudaMemcpyAsync(dsig + f0, b->sigma2 + f0, sizeof(float) * nf, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess && parts > 1 && (e = cudaEventRecord(ev_in[c], sin)) == cudaSuccess)
            e = cudaStreamWaitEvent(s, ev_in[c], 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "jbp_decode: copy inputs");
            break;
        }
        rc = decode_device(h, w, b->form, nf, dy + (size_t)h->n * f0, dhat + KN * f0, dit + f0, dok + (size_t)h->K * f0,
                           b->logpost ? dpost + vs * f0 : nullptr, b->sigma2 ? dsig + f0 : nullptr, s);
        if (rc) break;
        if (parts > 1 && (e = cudaEventRecord(ev_done[c], s)) != cudaSuccess) {
            rc = cuda_fail(e, "jbp_decode: event");
            break;
        }
        // the previous part's results (a copy to pageable memory returns when it is done,
        // by which time this part's decode is queued behind it)
        if (parts > 1 && c > 0) rc = fetch(c - 1);
    }
    if (rc == JBP_OK) rc = fetch(parts - 1);
    const cudaError_t e1 = cudaStreamSynchronize(s), e2 = cudaStreamSynchronize(sin), e3 = cudaStreamSynchronize(sout);
    cleanup();
    if (rc) return rc;
    JBP_CU(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3, "jbp_decode");
    {
        // bounded device waits (tensor-core completions, staged check tiles) record expiry here
        int err = 0;
        JBP_CU(cudaMemcpy(&err, h->d_tc_error, sizeof err, cudaMemcpyDeviceToHost), "jbp_decode: status");
        if (err) return fail(JBP_ETIMEOUT, "a bounded device wait expired");
    }
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// autotuner and multi-part decodes
// ---------------------------------------------------------------------------

// Time candidate fused launch shapes (threads per CTA x frames per CTA) on the
// first min(F, 4 * SMs) frames of a batch, a few iterations each, and keep the
// fastest for this handle.  Every candidate runs the same per-frame arithmetic,
// so the choice changes speed only.  Candidates are the distinct shapes the
// planner resolves (a hint it clamps to an already-seen shape is not re-timed);
// each is scored by the median of kTuneReps timed launches; a candidate whose
// launch or timing fails is skipped.  The handle keeps the resolved shape (never
// a 0 "default" hint), so jbp_tune reports what later fused launches use.
static int autotune(jbp_h* h, int F, const float* y, uint8_t* hat, int32_t* iters, uint8_t* ok,
                    const float* sigma2_f, cudaStream_t s)
{
    constexpr int kTuneReps = 5;
    jbp_ctx* ctx = h->ctx;
    if (!h->fused_ok || F <= 0) return JBP_OK;
    Graph g = h->graph();
    g.sigma2_f = sigma2_f;
    const int Fs = std::min(F, 4 * ctx->di.sm_count);
    const int T = std::min(ctx->opt.iters, 4);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        cudaGetLastError();
        return fail(JBP_ECUDA, "autotune: cudaEventCreate failed");
    }
    float best = 1e30f;
    int bt = 0, bf = 0;
    cudaError_t last = cudaSuccess;
    std::vector<std::pair<int, int>> seen;   // (threads, frames per CTA) of resolved plans
    const int threads_c[] = {128, 192, 256, 384, 512};
    const int fpc_c[] = {1, 2, 4, 8, 16};
    for (int th : threads_c)
        for (int fc : fpc_c) {
            FusedPlan plan;
            if (!fused_plan(g, ctx->di, Fs, th, fc, &plan)) continue;
            const std::pair<int, int> key(plan.threads, plan.frames_per_cta);
            if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
            seen.push_back(key);
            float ms[kTuneReps];
            bool good = true;
            for (int rep = 0; rep < kTuneReps && good; ++rep) {
                cudaError_t e = cudaEventRecord(a, s);
                if (e == cudaSuccess) e = launch_fused(g, plan, Fs, y, T, 0, hat, iters, ok, nullptr, s);
                if (e == cudaSuccess) e = cudaEventRecord(b, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[rep], a, b);
                if (e != cudaSuccess) {
                    last = e;
                    good = false;
                }
            }
            if (!good) {
                cudaGetLastError();   // a rejected launch shape leaves a non-sticky error
                continue;
            }
            std::sort(ms, ms + kTuneReps);
            const float per_frame = ms[kTuneReps / 2] / Fs;
            if (per_frame < best) {
                best = per_frame;
                bt = plan.threads;
                bf = plan.frames_per_cta;
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (bt == 0) {
        const cudaError_t sticky = cudaDeviceSynchronize();
        return fail(JBP_ECUDA, "autotune: no candidate launch shape ran: %s",
                    cudaGetErrorString(sticky != cudaSuccess ? sticky : last));
    }
    h->tune_threads = bt;
    h->tune_fpc = bf;
    h->tuned = true;
    return JBP_OK;
}

extern "C" int jbp_tune(jbp_h* h, const jbp_batch* b, int32_t* threads, int32_t* frames_per_cta)
{
    if (!h) return fail(JBP_EINVAL, "jbp_tune: NULL handle");
    if (!b) {
        // manual shape
        if (!threads || !frames_per_cta || *threads < 0 || *frames_per_cta < 0)
            return fail(JBP_EINVAL, "jbp_tune: a manual shape needs threads and frames_per_cta >= 0");
        h->tune_threads = *threads;
        h->tune_fpc = *frames_per_cta;
        h->tuned = true;
        return JBP_OK;
    }
    if (!b->on_device) return fail(JBP_EINVAL, "jbp_tune: needs a device batch");
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    cudaStream_t s = b->stream ? (cudaStream_t)b->stream : h->ctx->stream;
    int rc = autotune(h, b->F, b->y, b->hat, b->iters, b->ok, b->sigma2, s);
    if (rc) return rc;
    if (threads) *threads = h->tune_threads;
    if (frames_per_cta) *frames_per_cta = h->tune_fpc;
    return JBP_OK;
}

static int many_enqueue(jbp_ctx* ctx, int nparts, jbp_h* const* handles, const jbp_batch* bs, cudaStream_t main)
{
    JBP_CU(cudaEventRecord(ctx->fork_ev, main), "fork");
    // distinct handles go to pool streams round-robin (parts of one handle share
    // its workspace, so they stay in order on one stream)
    std::vector<jbp_h*> order;
    for (int i = 0; i < nparts; ++i)
        if (std::find(order.begin(), order.end(), handles[i]) == order.end()) order.push_back(handles[i]);
    const size_t S = std::min(order.size(), ctx->pool.size());
    for (size_t u = 0; u < S; ++u) JBP_CU(cudaStreamWaitEvent(ctx->pool[u], ctx->fork_ev, 0), "fork wait");
    for (size_t u = 0; u < order.size(); ++u) {
        cudaStream_t st = ctx->pool[u % S];
        for (int i = 0; i < nparts; ++i) {
            if (handles[i] != order[u]) continue;
            const jbp_batch& b = bs[i];
            int rc = decode_device(handles[i], handles[i]->ws, b.form, b.F, b.y, b.hat, b.iters, b.ok, b.logpost,
                                   b.sigma2, st);
            if (rc) return rc;
        }
    }
    for (size_t u = 0; u < S; ++u) {
        JBP_CU(cudaEventRecord(ctx->pool_ev[u], ctx->pool[u]), "join");
        JBP_CU(cudaStreamWaitEvent(main, ctx->pool_ev[u], 0), "join wait");
    }
    return JBP_OK;
}

static int many_run(jbp_ctx* ctx, int32_t nparts, jbp_h* const* handles, const jbp_batch* batches,
                    cudaStream_t main);

extern "C" int jbp_decode_many(jbp_ctx* ctx, int32_t nparts, jbp_h* const* handles, const jbp_batch* batches,
                               void* stream)
{
    if (!ctx || nparts < 0 || (nparts > 0 && (!handles || !batches))) return fail(JBP_EINVAL, "jbp_decode_many: bad argument");
    for (int i = 0; i < nparts; ++i) {
        const jbp_batch& b = batches[i];
        if (!handles[i] || handles[i]->ctx != ctx) return fail(JBP_EINVAL, "part %d: handle of another context", i);
        if (!b.on_device) return fail(JBP_EINVAL, "part %d: jbp_decode_many takes device batches", i);
        if (b.F < 0 || (b.F > 0 && (!b.y || !b.hat || !b.iters || !b.ok))) return fail(JBP_EINVAL, "part %d: bad batch", i);
    }
    JBP_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::lock_guard<std::mutex> lk(ctx->many_mu);
    if (ctx->pool.empty()) {
        ctx->pool.resize(32);
        ctx->pool_ev.resize(32);
        for (int i = 0; i < 32; ++i) {
            JBP_CU(cudaStreamCreateWithFlags(&ctx->pool[i], cudaStreamNonBlocking), "pool stream");
            JBP_CU(cudaEventCreateWithFlags(&ctx->pool_ev[i], cudaEventDisableTiming), "pool event");
        }
        JBP_CU(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "fork event");
        JBP_CU(cudaStreamCreateWithFlags(&ctx->many_stream, cudaStreamNonBlocking), "many stream");
        JBP_CU(cudaEventCreateWithFlags(&ctx->many_in, cudaEventDisableTiming), "many event");
        JBP_CU(cudaEventCreateWithFlags(&ctx->many_out, cudaEventDisableTiming), "many event");
    }
    const cudaStream_t user = stream ? (cudaStream_t)stream : ctx->stream;
    const cudaStream_t main = ctx->many_stream;
    JBP_CU(cudaEventRecord(ctx->many_in, user), "many: order after the caller");
    JBP_CU(cudaStreamWaitEvent(main, ctx->many_in, 0), "many: order after the caller");
    const int rc = many_run(ctx, nparts, handles, batches, main);
    JBP_CU(cudaEventRecord(ctx->many_out, main), "many: order before the caller");
    JBP_CU(cudaStreamWaitEvent(user, ctx->many_out, 0), "many: order before the caller");
    return rc;
}

// jbp_decode_many's work on its own stream: eager on the first call with given
// arguments, captured into a graph on the second, replayed from then on
static int many_run(jbp_ctx* ctx, int32_t nparts, jbp_h* const* handles, const jbp_batch* batches,
                    cudaStream_t main)
{
    std::vector<uintptr_t> key;
    for (int i = 0; i < nparts; ++i) {
        const jbp_batch& b = batches[i];
        for (uintptr_t v : {(uintptr_t)handles[i], (uintptr_t)handles[i]->ws.gen, (uintptr_t)b.F, (uintptr_t)b.y,
                            (uintptr_t)b.hat, (uintptr_t)b.iters, (uintptr_t)b.ok, (uintptr_t)b.logpost,
                            (uintptr_t)b.form, (uintptr_t)b.sigma2})
            key.push_back(v);
    }
    auto& ge = ctx->graphs[key];
    if (ge.exec) {
        JBP_CU(cudaGraphLaunch(ge.exec, main), "graph launch");
        return JBP_OK;
    }
    if (ge.seen == 0) {
        // first call: tune the fused parts, size the workspaces, run eagerly
        for (int i = 0; i < nparts; ++i) {
            jbp_h* h = handles[i];
            const jbp_batch& b = batches[i];
            if (!h->tuned && h->fused_ok && ctx->opt.precision == JBP_PREC_FP32 && !h->d_dft_tab &&
                (b.form == JBP_FORM_AUTO || b.form == JBP_FORM_FUSED)) {
                int rc = autotune(h, b.F, b.y, b.hat, b.iters, b.ok, b.sigma2, main);
                if (rc) return rc;
            }
        }
        ge.seen = 1;
        return many_enqueue(ctx, nparts, handles, batches, main);
    }
    // second call with these arguments: capture the whole decode as one graph
    JBP_CU(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal), "begin capture");
    int rc = many_enqueue(ctx, nparts, handles, batches, main);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(main, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        ge.exec = nullptr;
        return cuda_fail(e, "graph instantiate");
    }
    JBP_CU(cudaGraphLaunch(ge.exec, main), "graph launch");
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// single steps
// ---------------------------------------------------------------------------

static cudaStream_t pick_stream(jbp_h* h, void* s) { return s ? (cudaStream_t)s : h->ctx->stream; }

extern "C" int jbp_step_channel(jbp_h* h, int32_t F, const float* y, float* msg, float* ch2v, void* stream)
{
    if (!h || F < 0 || (F > 0 && (!y || !msg || !ch2v))) return fail(JBP_EINVAL, "jbp_step_channel: bad argument");
    if (reinterpret_cast<uintptr_t>(msg) % 16 || reinterpret_cast<uintptr_t>(ch2v) % 16)
        return fail(JBP_EINVAL, "jbp_step_channel: msg and ch2v must be 16-byte aligned");
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    JBP_CU(launch_channel(h->graph(), h->ctx->di, F, y, msg, ch2v, nullptr, pick_stream(h, stream)), "channel kernel");
    return JBP_OK;
}

extern "C" int jbp_step_check(jbp_h* h, int32_t F, float* msg, int32_t precision, void* stream)
{
    if (!h || F < 0 || (F > 0 && !msg)) return fail(JBP_EINVAL, "jbp_step_check: bad argument");
    if (precision < 0 || precision > 3) return fail(JBP_EINVAL, "bad precision %d", precision);
    // the check kernel moves tiles of msg with bulk copies, which need 16-byte alignment
    if (reinterpret_cast<uintptr_t>(msg) % 16)
        return fail(JBP_EINVAL, "jbp_step_check: msg must be 16-byte aligned");
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    JBP_CU(launch_check(h->graph(), h->ctx->di, F, msg, nullptr, precision, pick_stream(h, stream)), "check kernel");
    return JBP_OK;
}

extern "C" int jbp_step_var(jbp_h* h, int32_t F, const float* ch2v, const float* msg, float* post, uint8_t* hat,
                            void* stream)
{
    if (!h || F < 0 || (F > 0 && (!ch2v || !msg || !hat))) return fail(JBP_EINVAL, "jbp_step_var: bad argument");
    if (reinterpret_cast<uintptr_t>(msg) % 16 || reinterpret_cast<uintptr_t>(ch2v) % 16)
        return fail(JBP_EINVAL, "jbp_step_var: msg and ch2v must be 16-byte aligned");
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    JBP_CU(launch_var(h->graph(), h->ctx->di, F, ch2v, msg, post, hat, nullptr, pick_stream(h, stream)), "var kernel");
    return JBP_OK;
}

extern "C" int jbp_step_syndrome(jbp_h* h, int32_t F, const uint8_t* hat, uint8_t* ok, void* stream)
{
    if (!h || F < 0 || (F > 0 && (!hat || !ok))) return fail(JBP_EINVAL, "jbp_step_syndrome: bad argument");
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    cudaStream_t s = pick_stream(h, stream);
    // ok doubles as the unsatisfied-flag buffer, then is inverted in place
    JBP_CU(cudaMemsetAsync(ok, 0, (size_t)F * h->K, s), "memset ok");
    JBP_CU(launch_syndrome(h->graph(), h->ctx->di, F, hat, ok, nullptr, s), "syndrome kernel");
    JBP_CU(launch_ok_from_unsat(F, h->K, ok, ok, s), "ok kernel");
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// serving: resident pools re-batched every block of iterations
// ---------------------------------------------------------------------------
//
// jbp_submit queues one frame.  A server thread keeps, for every decoder with
// work, a resident pool: the step-form message state of up to `cap` frame slots
// in HBM.  It repeatedly (1) retires each pool whose block finished: the frames
// that finished during it come back through host-mapped memory and are
// published to jbp_poll, and their slots free up; (2) admits queued frames into
// the free slots of their decoder's pool, creating the pool when the memory
// budget allows (idle pools are evicted first); (3) launches the next block
// (ctx->opt.block_iters iterations, each frame stopping at its own early stop
// or at T) of every pool with frames, on the pool's stream, so the pools'
// blocks overlap on the device.  A frame's arithmetic does not depend on the
// other frames of its pool, so each result equals the frame decoded alone in
// the step form.

static constexpr int kPoolMinCap = 32;
static constexpr int kPoolMaxCap = 1024;

// device bytes of one frame slot of a pool (the larger of the step form's state
// and the fused form's, whose rows are padded to 32 positions)
static int64_t pool_frame_bytes(const jbp_h* h)
{
    const int64_t nb32 = (h->n + 31) / 32 * 32;
    const int64_t state = std::max<int64_t>(state_bytes(h->graph()), 12ll * h->K * nb32 * h->Q);
    return state + 8ll * h->n + 24 + 3ll * h->K + (int64_t)h->K * h->n;
}

// A decoder whose frames the fused position-major kernel runs (FP32 check, the
// trellis channel node) keeps its serving pool in that kernel's layout.
static bool pool_wants_fused(const jbp_ctx* ctx, const jbp_h* h)
{
    return h->fused_ok && ctx->opt.precision == JBP_PREC_FP32 && !h->d_dft_tab;
}

static PoolState pool_state(const ServePool& p)
{
    const jbp_h* h = p.h;
    PoolState st;
    st.n = h->n;
    st.K = h->K;
    st.msg_floats = p.fused ? (long long)p.fmsg : (long long)h->K * h->E * h->Q;
    st.msg = P<float>(p.msg);
    st.y = P<float>(p.y);
    st.sig = P<float>(p.sig);
    st.active = P<uint8_t>(p.active);
    st.t = P<int32_t>(p.t);
    st.unsat = P<uint8_t>(p.unsat);
    st.ok = P<uint8_t>(p.ok);
    st.hat = P<uint8_t>(p.hat);
    st.fin = P<uint8_t>(p.fin);
    return st;
}

static void pool_destroy(jbp_ctx* ctx, ServePool* p)
{
    if (p->stream) cudaStreamSynchronize(p->stream);
    for (DevBuf* b : {&p->msg, &p->ch2v, &p->y, &p->sig, &p->active, &p->t, &p->unsat, &p->ok, &p->hat, &p->fin,
                      &p->adm_slot, &p->adm_y, &p->adm_sig, &p->count})
        buf_free(ctx, *b);
    cudaFreeHost(p->h_adm_slot); cudaFreeHost(p->h_adm_y); cudaFreeHost(p->h_adm_sig); cudaFreeHost(p->h_count);
    cudaFreeHost(p->h_slot); cudaFreeHost(p->h_iters); cudaFreeHost(p->h_ok); cudaFreeHost(p->h_hat);
    if (p->done) cudaEventDestroy(p->done);
    if (p->stream) cudaStreamDestroy(p->stream);
    ctx->pool_bytes -= p->bytes;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->pool_of.erase(p->h);
    }
    ctx->cv_idle.notify_all();
}

template <class T>
static int mapped_alloc(T** host, T** dev, size_t count)
{
    JBP_CU(cudaHostAlloc((void**)host, std::max<size_t>(count * sizeof(T), 16), cudaHostAllocMapped), "pinned mapped");
    JBP_CU(cudaHostGetDevicePointer((void**)dev, *host, 0), "mapped device pointer");
    return JBP_OK;
}

static int pool_create(jbp_ctx* ctx, jbp_h* h, int cap, ServePool** out)
{
    std::unique_ptr<ServePool> p(new ServePool());
    p->h = h;
    p->cap = cap;
    const size_t F = (size_t)cap, K = h->K, n = h->n, E = h->E, Q = h->Q;
    if (pool_wants_fused(ctx, h)) {
        p->fused = fused_pool_plan(h->graph(), ctx->di, cap, K == 4 ? 512 : 0, &p->fplan, &p->fmsg, &p->fch2v);
        cudaGetLastError();
    }
    const size_t msg_floats = p->fused ? p->fmsg : K * E * Q, ch2v_floats = p->fused ? p->fch2v : K * n * Q;
    bool g = false;
    const int64_t before = ctx->used.load();
    int rc;
    if ((rc = buf_ensure(ctx, p->msg, sizeof(float) * F * msg_floats, &g)) ||
        (rc = buf_ensure(ctx, p->ch2v, sizeof(float) * F * ch2v_floats, &g)) ||
        (rc = buf_ensure(ctx, p->y, sizeof(float) * F * n, &g)) || (rc = buf_ensure(ctx, p->sig, sizeof(float) * F, &g)) ||
        (rc = buf_ensure(ctx, p->active, F, &g)) || (rc = buf_ensure(ctx, p->t, sizeof(int32_t) * F, &g)) ||
        (rc = buf_ensure(ctx, p->unsat, F * K, &g)) || (rc = buf_ensure(ctx, p->ok, F * K, &g)) ||
        (rc = buf_ensure(ctx, p->hat, F * K * n, &g)) || (rc = buf_ensure(ctx, p->fin, F, &g)) ||
        (rc = buf_ensure(ctx, p->adm_slot, sizeof(int32_t) * F, &g)) ||
        (rc = buf_ensure(ctx, p->adm_y, sizeof(float) * F * n, &g)) ||
        (rc = buf_ensure(ctx, p->adm_sig, sizeof(float) * F, &g)) || (rc = buf_ensure(ctx, p->count, sizeof(int32_t), &g))) {
        p->bytes = ctx->used.load() - before;
        ctx->pool_bytes += p->bytes;
        pool_destroy(ctx, p.get());
        return rc;
    }
    p->bytes = ctx->used.load() - before;
    ctx->pool_bytes += p->bytes;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->pool_of[h] = 1;
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming)) ||
        (e = cudaMallocHost((void**)&p->h_adm_slot, sizeof(int32_t) * F)) ||
        (e = cudaMallocHost((void**)&p->h_adm_y, sizeof(float) * F * n)) ||
        (e = cudaMallocHost((void**)&p->h_adm_sig, sizeof(float) * F)) ||
        (e = cudaMallocHost((void**)&p->h_count, sizeof(int32_t)))) {
        pool_destroy(ctx, p.get());
        return cuda_fail(e, "serving pool setup");
    }
    if ((rc = mapped_alloc(&p->h_slot, &p->d_slot, F)) || (rc = mapped_alloc(&p->h_iters, &p->d_iters, F)) ||
        (rc = mapped_alloc(&p->h_ok, &p->d_ok, F * K)) || (rc = mapped_alloc(&p->h_hat, &p->d_hat, F * K * n))) {
        pool_destroy(ctx, p.get());
        return rc;
    }
    if ((e = cudaMemsetAsync(p->active.p, 0, F, p->stream)) || (e = cudaMemsetAsync(p->fin.p, 0, F, p->stream)) ||
        (e = cudaStreamSynchronize(p->stream))) {
        pool_destroy(ctx, p.get());
        return cuda_fail(e, "serving pool clear");
    }
    p->req.resize(F);
    p->used.assign(F, 0);
    for (int s2 = cap - 1; s2 >= 0; --s2) p->free_list.push_back(s2);
    *out = p.release();
    return JBP_OK;
}

// Publish results; called without the context lock held.
static void publish(jbp_ctx* ctx, std::vector<std::pair<uint64_t, Result>>& out, std::vector<double>& lat)
{
    if (out.empty()) return;
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto& r : out) {
        ctx->done[r.first] = std::move(r.second);
        ctx->pending.erase(r.first);
    }
    ctx->latencies.insert(ctx->latencies.end(), lat.begin(), lat.end());
    ctx->completed += out.size();
    out.clear();
    lat.clear();
}

static void pool_free_slot(ServePool& p, int slot)
{
    p.used[slot] = 0;
    p.req[slot] = Request();
    p.free_list.push_back(slot);
    p.n_active--;
    while (p.hi > 0 && !p.used[p.hi - 1]) p.hi--;
}

// A block of the pool has completed (q = its status): hand out the frames it finished.
static void pool_retire(jbp_ctx* ctx, ServePool& p, cudaError_t q)
{
    const double now = now_us();
    jbp_h* h = p.h;
    std::vector<std::pair<uint64_t, Result>> out;
    std::vector<double> lat;
    if (q != cudaSuccess) {
        cudaGetLastError();
        for (int s2 = 0; s2 < p.cap; ++s2) {
            if (!p.used[s2]) continue;
            Result r;
            r.iters = -1;
            r.hat.assign((size_t)h->K * h->n, 0);
            r.ok.assign((size_t)h->K, 0);
            out.emplace_back(p.req[s2].ticket, std::move(r));
            lat.push_back(now - p.req[s2].t_submit);
            pool_free_slot(p, s2);
        }
        cudaMemsetAsync(p.active.p, 0, (size_t)p.cap, p.stream);
        cudaMemsetAsync(p.fin.p, 0, (size_t)p.cap, p.stream);
        cudaStreamSynchronize(p.stream);
    } else {
        const int cnt = *reinterpret_cast<volatile int32_t*>(p.h_count);
        const size_t KN = (size_t)h->K * h->n;
        for (int i = 0; i < cnt; ++i) {
            const int s2 = p.h_slot[i];
            if (s2 < 0 || s2 >= p.cap || !p.used[s2]) continue;
            Result r;
            r.iters = p.h_iters[i];
            r.ok.assign(p.h_ok + (size_t)i * h->K, p.h_ok + (size_t)(i + 1) * h->K);
            r.hat.assign(p.h_hat + i * KN, p.h_hat + (i + 1) * KN);
            out.emplace_back(p.req[s2].ticket, std::move(r));
            lat.push_back(now - p.req[s2].t_submit);
            pool_free_slot(p, s2);
        }
    }
    publish(ctx, out, lat);
}

// Step time of one channel-node launch over F frames, from two measured points
// (1 and fb frames): linear between them, proportional to F beyond fb.
static float chan_est(float t1, float tb, int fb, int F)
{
    if (F <= 1 || fb <= 1) return F <= 1 ? t1 : tb * (float)F / (float)fb;
    if (F <= fb) return t1 + (tb - t1) * (float)(F - 1) / (float)(fb - 1);
    return tb * (float)F / (float)fb;
}

// Under AUTO a serving pool runs the tensor-core channel node only where it is
// the faster one for the pool's current frame count (chan_calibrate).
static bool pool_use_dft(const jbp_ctx* ctx, const jbp_h* h, int F)
{
    if (!h->d_dft_tab) return false;
    if (ctx->opt.channel_node != JBP_CHAN_AUTO || !h->chan_cal) return true;
    return chan_est(h->chan_d1, h->chan_db, h->chan_fb, F) < chan_est(h->chan_t1, h->chan_tb, h->chan_fb, F);
}

// Stage `take` into free slots and launch the pool's next block.
static int pool_launch(jbp_ctx* ctx, ServePool& p, std::vector<Request>& take)
{
    jbp_h* h = p.h;
    const int m = (int)take.size();
    for (int i = 0; i < m; ++i) {
        const int s2 = p.free_list.back();
        p.free_list.pop_back();
        Request& r = take[i];
        p.h_adm_slot[i] = s2;
        memcpy(p.h_adm_y + (size_t)i * h->n, r.y.data(), sizeof(float) * h->n);
        p.h_adm_sig[i] = r.sigma2 > 0.0f ? r.sigma2 : (float)h->sigma2;
        r.y.clear();
        r.y.shrink_to_fit();
        p.req[s2] = std::move(r);
        p.used[s2] = 1;
        p.n_active++;
        p.hi = std::max(p.hi, s2 + 1);
    }
    take.clear();
    cudaStream_t s = p.stream;
    const PoolState st = pool_state(p);
    if (m > 0) {
        JBP_CU(cudaMemcpyAsync(p.adm_slot.p, p.h_adm_slot, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s), "admit slots");
        JBP_CU(cudaMemcpyAsync(p.adm_y.p, p.h_adm_y, sizeof(float) * (size_t)m * h->n, cudaMemcpyHostToDevice, s), "admit y");
        JBP_CU(cudaMemcpyAsync(p.adm_sig.p, p.h_adm_sig, sizeof(float) * m, cudaMemcpyHostToDevice, s), "admit sigma2");
        JBP_CU(launch_pool_admit(m, P<int32_t>(p.adm_slot), P<float>(p.adm_y), P<float>(p.adm_sig), st, s), "admit");
    }
    Graph g = h->graph();
    g.sigma2_f = P<float>(p.sig);
    const DeviceInfo& di = ctx->di;
    const int F = p.hi;
    if (!pool_use_dft(ctx, h, F)) g.dft_tab = nullptr;
    float* msg = P<float>(p.msg);
    float* ch2v = P<float>(p.ch2v);
    const uint8_t* act = P<uint8_t>(p.active);
    if (p.fused) {
        // one launch runs the block: every active slot up to block_iters more
        // iterations in shared memory, its state back to HBM unless it finished
        FusedPool fp;
        fp.msg = msg;
        fp.ch2v = ch2v;
        fp.active = P<uint8_t>(p.active);
        fp.fin = P<uint8_t>(p.fin);
        fp.block = ctx->opt.block_iters;
        JBP_CU(launch_fused_pool(g, p.fplan, F, P<float>(p.y), ctx->opt.iters, ctx->opt.early_stop,
                                 P<uint8_t>(p.hat), P<int32_t>(p.t), P<uint8_t>(p.ok), fp, s),
               "pool fused block");
    }
    for (int it = 0; it < (p.fused ? 0 : ctx->opt.block_iters); ++it) {
        JBP_CU(launch_channel(g, di, F, P<float>(p.y), msg, ch2v, act, s), "pool channel");
        JBP_CU(launch_check(g, di, F, msg, act, ctx->opt.precision, s), "pool check");
        JBP_CU(launch_var(g, di, F, ch2v, msg, nullptr, P<uint8_t>(p.hat), act, s), "pool var");
        JBP_CU(launch_syndrome(g, di, F, P<uint8_t>(p.hat), P<uint8_t>(p.unsat), act, s), "pool syndrome");
        JBP_CU(launch_pool_finalize(F, ctx->opt.iters, ctx->opt.early_stop, st, s), "pool finalize");
    }
    JBP_CU(cudaMemsetAsync(p.count.p, 0, sizeof(int32_t), s), "harvest clear");
    JBP_CU(launch_pool_harvest(F, st, P<int32_t>(p.count), p.d_slot, p.d_iters, p.d_ok, p.d_hat, s), "harvest");
    JBP_CU(cudaMemcpyAsync(p.h_count, p.count.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "harvest count");
    JBP_CU(cudaEventRecord(p.done, s), "pool event");
    p.running = true;
    p.last_used = now_us();
    return JBP_OK;
}

static ServePool* find_pool(jbp_ctx* ctx, const jbp_h* h)
{
    for (auto& up : ctx->serve_pools)
        if (up->h == h) return up.get();
    return nullptr;
}

// Free device memory for a new pool: destroy idle pools, least recently used first.
static void evict_idle(jbp_ctx* ctx, int64_t need)
{
    while (ctx->pool_bytes + need > ctx->budget / 2) {
        int victim = -1;
        for (int i = 0; i < (int)ctx->serve_pools.size(); ++i) {
            const ServePool& p = *ctx->serve_pools[i];
            if (p.running || p.n_active > 0) continue;
            if (victim < 0 || p.last_used < ctx->serve_pools[victim]->last_used) victim = i;
        }
        if (victim < 0) return;
        pool_destroy(ctx, ctx->serve_pools[victim].get());
        ctx->serve_pools.erase(ctx->serve_pools.begin() + victim);
    }
}

static void fail_requests(jbp_ctx* ctx, std::vector<Request>& reqs)
{
    std::vector<std::pair<uint64_t, Result>> out;
    std::vector<double> lat;
    const double now = now_us();
    for (Request& r : reqs) {
        Result res;
        res.iters = -1;
        res.hat.assign((size_t)r.h->K * r.h->n, 0);
        res.ok.assign((size_t)r.h->K, 0);
        out.emplace_back(r.ticket, std::move(res));
        lat.push_back(now - r.t_submit);
    }
    reqs.clear();
    publish(ctx, out, lat);
}

static void server_main(jbp_ctx* ctx)
{
    cudaSetDevice(ctx->device);
    while (true) {
        bool any_running = false;
        // (1) retire the pools whose block completed
        for (auto& up : ctx->serve_pools) {
            ServePool& p = *up;
            if (!p.running) continue;
            const cudaError_t q = cudaEventQuery(p.done);
            if (q == cudaErrorNotReady) {
                any_running = true;
                continue;
            }
            p.running = false;
            pool_retire(ctx, p, q);
        }
        // (2) decoders with queued frames, in queue order
        std::vector<std::pair<jbp_h*, int>> want;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            for (const Request& r : ctx->queue) {
                auto it = std::find_if(want.begin(), want.end(), [&](const std::pair<jbp_h*, int>& w) { return w.first == r.h; });
                if (it == want.end()) want.emplace_back(r.h, 1);
                else it->second++;
            }
        }
        for (auto& w : want) {
            jbp_h* h = w.first;
            ServePool* p = find_pool(ctx, h);
            if (p && !p->running && p->n_active == 0 && w.second > p->cap && p->cap < kPoolMaxCap) {
                // grow an idle pool that is too small for the queue
                pool_destroy(ctx, p);
                ctx->serve_pools.erase(std::find_if(ctx->serve_pools.begin(), ctx->serve_pools.end(),
                                                    [&](const std::unique_ptr<ServePool>& u) { return u.get() == p; }));
                p = nullptr;
            }
            if (!p) {
                const int64_t per = pool_frame_bytes(h);
                int cap = kPoolMinCap;
                while (cap < kPoolMaxCap && cap < 2 * w.second) cap *= 2;
                evict_idle(ctx, per * cap);
                const int64_t room = ctx->budget / 2 - ctx->pool_bytes;
                cap = (int)std::min<int64_t>(cap, room / per);
                if (cap < 1) {
                    if (ctx->serve_pools.empty()) {
                        // one frame of this decoder does not fit the serving budget
                        std::vector<Request> drop;
                        {
                            std::lock_guard<std::mutex> lk(ctx->mu);
                            for (auto it = ctx->queue.begin(); it != ctx->queue.end();)
                                if (it->h == h) {
                                    drop.push_back(std::move(*it));
                                    it = ctx->queue.erase(it);
                                } else {
                                    ++it;
                                }
                        }
                        fail_requests(ctx, drop);
                    }
                    continue;   // wait for pools to drain
                }
                if (pool_create(ctx, h, cap, &p) != JBP_OK) {
                    p = nullptr;
                    continue;
                }
                ctx->serve_pools.emplace_back(p);
            }
            if (p->running || p->free_list.empty()) continue;
            std::vector<Request> take;
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                for (auto it = ctx->queue.begin(); it != ctx->queue.end() && take.size() < p->free_list.size();)
                    if (it->h == h) {
                        take.push_back(std::move(*it));
                        it = ctx->queue.erase(it);
                    } else {
                        ++it;
                    }
            }
            if (take.empty() && p->n_active == 0) continue;
            if (pool_launch(ctx, *p, take) != JBP_OK) {
                fail_requests(ctx, take);
                cudaGetLastError();
            }
            any_running = any_running || p->running;
        }
        // (3) pools with frames in flight and nothing new: next block
        for (auto& up : ctx->serve_pools) {
            ServePool& p = *up;
            if (p.running || p.n_active == 0) continue;
            std::vector<Request> none;
            if (pool_launch(ctx, p, none) != JBP_OK) cudaGetLastError();
            any_running = any_running || p.running;
        }
        // (4) pools of decoders being destroyed, once drained
        for (size_t i = 0; i < ctx->serve_pools.size();) {
            ServePool& p = *ctx->serve_pools[i];
            bool closing;
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                closing = p.h->closing;
            }
            if (closing && !p.running && p.n_active == 0) {
                pool_destroy(ctx, &p);
                ctx->serve_pools.erase(ctx->serve_pools.begin() + i);
            } else {
                ++i;
            }
        }
        std::unique_lock<std::mutex> lk(ctx->mu);
        if (ctx->stop && !any_running && ctx->queue.empty()) break;
        if (any_running) {
            ctx->cv.wait_for(lk, std::chrono::microseconds(50));
        } else {
            bool closing_pool = false;
            for (auto& up : ctx->serve_pools) closing_pool = closing_pool || up->h->closing;
            if (!closing_pool) ctx->cv.wait(lk, [&] {
                if (ctx->stop || !ctx->queue.empty()) return true;
                for (auto& up : ctx->serve_pools)
                    if (up->h->closing) return true;
                return false;
            });
        }
    }
}

extern "C" int jbp_submit(jbp_h* h, const float* y_frame, double sigma2, uint64_t* ticket)
{
    if (!h || !y_frame || !ticket) return fail(JBP_EINVAL, "jbp_submit: NULL argument");
    if (!std::isfinite(sigma2)) return fail(JBP_EINVAL, "jbp_submit: sigma2 not finite");
    jbp_ctx* ctx = h->ctx;
    Request r;
    r.h = h;
    r.y.assign(y_frame, y_frame + h->n);
    r.sigma2 = (float)sigma2;
    r.t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->stop) return fail(JBP_ECLOSED, "context is shutting down");
        if (!ctx->server_started) {
            ctx->server = std::thread(server_main, ctx);
            ctx->server_started = true;
        }
        r.ticket = ctx->next_ticket++;
        *ticket = r.ticket;
        ctx->pending[r.ticket] = 1;
        ctx->queue.push_back(std::move(r));
    }
    ctx->cv.notify_all();
    return JBP_OK;
}

extern "C" int jbp_poll(jbp_ctx* ctx, uint64_t ticket, uint8_t* hat, int32_t* iters, uint8_t* ok)
{
    if (!ctx) return fail(JBP_EINVAL, "jbp_poll: NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->done.find(ticket);
    if (it == ctx->done.end()) {
        if (ctx->pending.count(ticket)) return JBP_EAGAIN;
        return fail(JBP_ECLOSED, "unknown or already consumed ticket %llu", (unsigned long long)ticket);
    }
    const Result& r = it->second;
    if (r.iters < 0) {
        ctx->done.erase(it);
        return fail(JBP_ECUDA, "request %llu failed on the device", (unsigned long long)ticket);
    }
    if (hat) memcpy(hat, r.hat.data(), r.hat.size());
    if (ok) memcpy(ok, r.ok.data(), r.ok.size());
    if (iters) *iters = r.iters;
    ctx->done.erase(it);
    return JBP_OK;
}

extern "C" int jbp_serving_stats(jbp_ctx* ctx, uint64_t* completed, double* p50, double* p99)
{
    if (!ctx) return fail(JBP_EINVAL, "jbp_serving_stats: NULL context");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        lat = ctx->latencies;
        if (completed) *completed = ctx->completed;
    }
    double a = 0, b = 0;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        a = lat[(size_t)std::floor(0.50 * (lat.size() - 1))];
        b = lat[(size_t)std::floor(0.99 * (lat.size() - 1))];
    }
    if (p50) *p50 = a;
    if (p99) *p99 = b;
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// evidence interface: slot detector and SIC row decoder
// ---------------------------------------------------------------------------

struct jbp_ura {
    jbp_ctx* ctx = nullptr;
    UraDev u{};
    int32_t* d_rows = nullptr;
    float* d_tw = nullptr;
    int32_t* d_chk_var = nullptr;
    uint8_t* d_chk_coef = nullptr;
    int32_t* d_var_edge = nullptr;
    uint8_t* d_gf_mul = nullptr;
    uint8_t* d_gf_div = nullptr;
    int64_t table_bytes = 0;
    std::mutex mu;
    DevBuf S, y, hat, iters, ok;   // workspaces of the host-pointer calls and of jbp_ura_decode
};

extern "C" int jbp_ura_destroy(jbp_ura* u)
{
    if (!u) return fail(JBP_EINVAL, "jbp_ura_destroy: NULL handle");
    jbp_ctx* ctx = u->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, u->d_rows, sizeof(int32_t) * (size_t)u->u.n * u->u.ns);
    dev_free(ctx, u->d_tw, sizeof(float) * 2 * (size_t)u->u.Q);
    dev_free(ctx, u->d_chk_var, sizeof(int32_t) * (size_t)u->u.P * u->u.dc);
    dev_free(ctx, u->d_chk_coef, (size_t)u->u.P * u->u.dc);
    dev_free(ctx, u->d_var_edge, sizeof(int32_t) * (size_t)u->u.dv * u->u.n);
    dev_free(ctx, u->d_gf_mul, (size_t)u->u.Q * u->u.Q);
    dev_free(ctx, u->d_gf_div, (size_t)u->u.Q * u->u.Q);
    for (DevBuf* b : {&u->S, &u->y, &u->hat, &u->iters, &u->ok}) buf_free(ctx, *b);
    if (u->d_gf_div) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->handles--;
    }
    delete u;
    return JBP_OK;
}

extern "C" int jbp_ura_create(jbp_ctx* ctx, const jbp_code* code, const jbp_ura_params* p, jbp_ura** out)
{
    if (!ctx || !code || !p || !out) return fail(JBP_EINVAL, "jbp_ura_create: NULL argument");
    const int q = code->q;
    int m = 0;
    while ((1 << m) < q && m < 8) ++m;
    if ((1 << m) != q || (q != 16 && q != 32 && q != 64))
        return fail(JBP_EINVAL, "q must be 16, 32 or 64 (got %d)", q);
    if (!((code->dv == 2 && (code->dc == 3 || code->dc == 4)) || (code->dv == 3 && code->dc == 6)))
        return fail(JBP_EINVAL, "the row decoder is built for (dv, dc) = (2, 3), (2, 4) or (3, 6) (got (%d, %d))",
                    code->dv, code->dc);
    if (code->n < 1 || code->P < 1 || (int64_t)code->n * code->dv != (int64_t)code->P * code->dc)
        return fail(JBP_EINVAL, "n*dv must equal P*dc with n, P >= 1");
    if (code->n > 32767) return fail(JBP_EINVAL, "n must be <= 32767");
    if (!code->chk_var || !code->chk_coef || !p->rows) return fail(JBP_EINVAL, "NULL code arrays or rows");
    if (p->ns < 1 || p->ns > 32 || p->ns > q) return fail(JBP_EINVAL, "ns must be in 1..min(32, q) (got %d)", p->ns);
    if (p->K < 1 || p->K > 8) return fail(JBP_EINVAL, "K must be in 1..8 (got %d)", p->K);
    if (p->amp_iters < 0 || p->bp_iters < 1) return fail(JBP_EINVAL, "amp_iters >= 0 and bp_iters >= 1 required");
    if (!(p->rho_bg > 0.0 && p->rho_bg < 1.0)) return fail(JBP_EINVAL, "rho_bg must be in (0, 1)");
    if (!(p->sigma_u2 > 0.0) || !std::isfinite(p->sigma_u2)) return fail(JBP_EINVAL, "sigma_u2 must be finite and > 0");
    if (!(p->cancel_log <= 0.0) || !std::isfinite(p->cancel_log)) return fail(JBP_EINVAL, "cancel_log must be finite and <= 0");
    const int n = code->n, P = code->P, dc = code->dc, dv = code->dv, E = P * dc;
    std::vector<int32_t> var_edge((size_t)dv * n), fill(n, 0);
    for (int e = 0; e < E; ++e) {
        const int i = code->chk_var[e];
        if (i < 0 || i >= n) return fail(JBP_EINVAL, "chk_var[%d] = %d out of range", e, i);
        if (code->chk_coef[e] < 1 || code->chk_coef[e] >= q) return fail(JBP_EINVAL, "chk_coef[%d] = %d not in 1..q-1", e, code->chk_coef[e]);
        if (fill[i] >= dv) return fail(JBP_EINVAL, "variable %d has more than dv = %d edges", i, dv);
        var_edge[(size_t)dv * i + fill[i]++] = e;
    }
    for (int i = 0; i < n; ++i)
        if (fill[i] != dv) return fail(JBP_EINVAL, "variable %d has %d edges, expected dv = %d", i, fill[i], dv);
    for (int l = 0; l < n; ++l)
        for (int i = 0; i < p->ns; ++i) {
            const int r = p->rows[(size_t)l * p->ns + i];
            if (r < 0 || r >= q) return fail(JBP_EINVAL, "rows[%d] = %d not in 0..q-1", l * p->ns + i, r);
            for (int i2 = 0; i2 < i; ++i2)
                if (p->rows[(size_t)l * p->ns + i2] == r) return fail(JBP_EINVAL, "slot %d repeats row %d", l, r);
        }
    std::vector<uint8_t> gmul((size_t)q * q), gdiv((size_t)q * q);
    gf_build_tables(m, gmul.data(), gdiv.data());
    // twiddles exp(-2 pi i k / q) from the host's double-precision cos and sin
    std::vector<float> tw((size_t)2 * q);
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < q; ++k) {
        tw[2 * k] = (float)std::cos(two_pi * k / q);
        tw[2 * k + 1] = (float)-std::sin(two_pi * k / q);
    }
    UraDev d{};
    d.n = n; d.P = P; d.dc = dc; d.dv = dv; d.K = p->K; d.Q = q; d.ns = p->ns;
    d.amp_iters = p->amp_iters; d.bp_iters = p->bp_iters; d.early_stop = p->early_stop ? 1 : 0;
    d.log_odds = (float)std::log((1.0 - p->rho_bg) / p->rho_bg);
    d.su2 = (float)p->sigma_u2;
    d.inv_sqrt_ns = (float)(1.0 / std::sqrt((double)p->ns));
    d.cancel_log = (float)p->cancel_log;
    if (sic_warps_per_cta(d, ctx->di) < 1)
        return fail(JBP_EINVAL, "n = %d, q = %d: one frame's row state does not fit shared memory", n, q);

    JBP_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    jbp_ura* u = new (std::nothrow) jbp_ura();
    if (!u) return fail(JBP_ENOMEM, "host allocation failed");
    u->ctx = ctx;
    u->u = d;
    int rc;
    if ((rc = dev_alloc(ctx, &u->d_rows, (size_t)n * p->ns, &u->table_bytes)) ||
        (rc = dev_alloc(ctx, &u->d_tw, (size_t)2 * q, &u->table_bytes)) ||
        (rc = dev_alloc(ctx, &u->d_chk_var, (size_t)E, &u->table_bytes)) ||
        (rc = dev_alloc(ctx, &u->d_chk_coef, (size_t)E, &u->table_bytes)) ||
        (rc = dev_alloc(ctx, &u->d_var_edge, (size_t)dv * n, &u->table_bytes)) ||
        (rc = dev_alloc(ctx, &u->d_gf_mul, (size_t)q * q, &u->table_bytes)) ||
        (rc = dev_alloc(ctx, &u->d_gf_div, (size_t)q * q, &u->table_bytes))) {
        jbp_ura_destroy(u);
        return rc;
    }
    cudaError_t e;
    if ((e = cudaMemcpy(u->d_rows, p->rows, sizeof(int32_t) * (size_t)n * p->ns, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(u->d_tw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(u->d_chk_var, code->chk_var, sizeof(int32_t) * E, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(u->d_chk_coef, code->chk_coef, (size_t)E, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(u->d_var_edge, var_edge.data(), sizeof(int32_t) * var_edge.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(u->d_gf_mul, gmul.data(), gmul.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(u->d_gf_div, gdiv.data(), gdiv.size(), cudaMemcpyHostToDevice))) {
        jbp_ura_destroy(u);
        return cuda_fail(e, "jbp_ura_create: copy tables");
    }
    u->u.rows = u->d_rows; u->u.tw = u->d_tw; u->u.chk_var = u->d_chk_var; u->u.chk_coef = u->d_chk_coef;
    u->u.var_edge = u->d_var_edge; u->u.gf_mul = u->d_gf_mul; u->u.gf_div = u->d_gf_div;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->handles++;
    }
    *out = u;
    return JBP_OK;
}

static int ura_grow(jbp_ura* u, DevBuf& b, size_t bytes)
{
    bool grew = false;
    return buf_ensure(u->ctx, b, bytes, &grew);
}

// One call of the evidence path on device pointers: what = 1 detector, 2 row
// decoder, 3 both (S in the handle's workspace).
static int ura_run(jbp_ura* u, int what, int F, const float* y, float* S, uint8_t* hat, int32_t* iters, uint8_t* ok,
                   cudaStream_t s)
{
    const UraDev& d = u->u;
    if ((what & 1) && d.Q != 32 && d.Q != 64) return fail(JBP_EINVAL, "the slot detector is built for q = 32 and 64");
    if (what == 3) {
        int rc = ura_grow(u, u->S, sizeof(float) * (size_t)F * d.n * d.Q);
        if (rc) return rc;
        S = P<float>(u->S);
    }
    cudaError_t e = cudaSuccess;
    if (what & 1) {
        e = launch_amp(d, u->ctx->di, F, y, S, s);
        if (e != cudaSuccess) return cuda_fail(e, "slot detector launch");
    }
    if (what & 2) {
        e = launch_sic(d, u->ctx->di, F, S, hat, iters, ok, s);
        if (e != cudaSuccess) return cuda_fail(e, "row decoder launch");
    }
    return JBP_OK;
}

static int ura_call(jbp_ura* u, int what, int32_t F, const float* y, float* S_io, const float* S_in, uint8_t* hat,
                    int32_t* iters, uint8_t* ok, int32_t on_device, void* stream)
{
    if (!u) return fail(JBP_EINVAL, "NULL handle");
    if (F < 0) return fail(JBP_EINVAL, "F must be >= 0");
    if (F == 0) return JBP_OK;
    const UraDev& d = u->u;
    if ((what & 1) && !y) return fail(JBP_EINVAL, "NULL y");
    if (what == 1 && !S_io) return fail(JBP_EINVAL, "NULL S");
    if (what == 2 && !S_in) return fail(JBP_EINVAL, "NULL S");
    if ((what & 2) && (!hat || !iters || !ok)) return fail(JBP_EINVAL, "NULL output buffer");
    jbp_ctx* ctx = u->ctx;
    JBP_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::lock_guard<std::mutex> lk(u->mu);
    const size_t ybytes = sizeof(float) * (size_t)F * d.n * d.ns * 2;
    const size_t sbytes = sizeof(float) * (size_t)F * d.n * d.Q;
    const size_t hbytes = (size_t)F * d.K * d.n;
    if (on_device) {
        cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
        return ura_run(u, what, F, y, what == 1 ? S_io : const_cast<float*>(S_in), hat, iters, ok, s);
    }
    cudaStream_t s = ctx->stream;
    int rc;
    if ((what & 1) && (rc = ura_grow(u, u->y, ybytes))) return rc;
    if (what != 3 && (rc = ura_grow(u, u->S, sbytes))) return rc;
    if ((what & 2) && ((rc = ura_grow(u, u->hat, hbytes)) || (rc = ura_grow(u, u->iters, sizeof(int32_t) * F * d.K)) ||
                       (rc = ura_grow(u, u->ok, (size_t)F * d.K))))
        return rc;
    if (what & 1) JBP_CU(cudaMemcpyAsync(P<float>(u->y), y, ybytes, cudaMemcpyHostToDevice, s), "copy y");
    if (what == 2) JBP_CU(cudaMemcpyAsync(P<float>(u->S), S_in, sbytes, cudaMemcpyHostToDevice, s), "copy S");
    rc = ura_run(u, what, F, P<float>(u->y), P<float>(u->S), P<uint8_t>(u->hat), P<int32_t>(u->iters), P<uint8_t>(u->ok), s);
    if (rc) return rc;
    if (what == 1) JBP_CU(cudaMemcpyAsync(S_io, P<float>(u->S), sbytes, cudaMemcpyDeviceToHost, s), "copy S");
    if (what & 2) {
        JBP_CU(cudaMemcpyAsync(hat, P<uint8_t>(u->hat), hbytes, cudaMemcpyDeviceToHost, s), "copy hat");
        JBP_CU(cudaMemcpyAsync(iters, P<int32_t>(u->iters), sizeof(int32_t) * F * d.K, cudaMemcpyDeviceToHost, s), "copy iters");
        JBP_CU(cudaMemcpyAsync(ok, P<uint8_t>(u->ok), (size_t)F * d.K, cudaMemcpyDeviceToHost, s), "copy ok");
    }
    JBP_CU(cudaStreamSynchronize(s), "evidence path");
    return JBP_OK;
}

extern "C" int jbp_amp_evidence(jbp_ura* u, int32_t F, const float* y, float* S, int32_t on_device, void* stream)
{
    return ura_call(u, 1, F, y, S, nullptr, nullptr, nullptr, nullptr, on_device, stream);
}

extern "C" int jbp_sic_decode(jbp_ura* u, int32_t F, const float* S, uint8_t* hat, int32_t* iters, uint8_t* ok,
                              int32_t on_device, void* stream)
{
    return ura_call(u, 2, F, nullptr, nullptr, S, hat, iters, ok, on_device, stream);
}

extern "C" int jbp_ura_decode(jbp_ura* u, int32_t F, const float* y, uint8_t* hat, int32_t* iters, uint8_t* ok,
                              int32_t on_device, void* stream)
{
    return ura_call(u, 3, F, y, nullptr, nullptr, hat, iters, ok, on_device, stream);
}

extern "C" int jbp_match_rows(jbp_ctx* ctx, int32_t F, int32_t K, int32_t n, const uint8_t* hat, const uint8_t* truth,
                              int32_t* sym_err, int32_t* cw_err, int32_t on_device, void* stream)
{
    if (!ctx) return fail(JBP_EINVAL, "jbp_match_rows: NULL context");
    if (F < 0 || K < 1 || K > 8 || n < 1) return fail(JBP_EINVAL, "jbp_match_rows: need F >= 0, K in 1..8, n >= 1");
    if (F == 0) return JBP_OK;
    if (!hat || !truth || !sym_err || !cw_err) return fail(JBP_EINVAL, "jbp_match_rows: NULL buffer");
    JBP_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (on_device) {
        cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
        JBP_CU(launch_match_rows(ctx->di, F, K, n, hat, truth, sym_err, cw_err, s), "row matching");
        return JBP_OK;
    }
    const size_t hb = (size_t)F * K * n;
    DevBuf dh, dx, ds, dc;
    bool g = false;
    int rc;
    if ((rc = buf_ensure(ctx, dh, hb, &g)) || (rc = buf_ensure(ctx, dx, hb, &g)) ||
        (rc = buf_ensure(ctx, ds, sizeof(int32_t) * F, &g)) || (rc = buf_ensure(ctx, dc, sizeof(int32_t) * F, &g))) {
        for (DevBuf* b : {&dh, &dx, &ds, &dc}) buf_free(ctx, *b);
        return rc;
    }
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dh.p, hat, hb, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(dx.p, truth, hb, cudaMemcpyHostToDevice, s)) ||
        (e = launch_match_rows(ctx->di, F, K, n, P<uint8_t>(dh), P<uint8_t>(dx), P<int32_t>(ds), P<int32_t>(dc), s)) ||
        (e = cudaMemcpyAsync(sym_err, ds.p, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(cw_err, dc.p, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
        for (DevBuf* b : {&dh, &dx, &ds, &dc}) buf_free(ctx, *b);
        return cuda_fail(e, "row matching");
    }
    for (DevBuf* b : {&dh, &dx, &ds, &dc}) buf_free(ctx, *b);
    return JBP_OK;
}
