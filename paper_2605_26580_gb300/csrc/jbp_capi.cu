// jbp_capi.cu -- the C ABI (include/jbp.h): contexts, decoder handles, the three
// launch forms, single-step entry points and the continuous-batching serving loop.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/jbp.h"
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

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------

namespace {

// Device buffers of one decode (grown on demand).  Sizes in frames.
struct Workspace {
    int cap_step = 0;      // frames of msg/ch2v/active/unsat
    float* msg = nullptr;
    float* ch2v = nullptr;
    uint8_t* active = nullptr;
    uint8_t* unsat = nullptr;
    int cap_io = 0;        // frames of staging
    bool io_post = false;
    float* y = nullptr;
    uint8_t* hat = nullptr;
    int32_t* iters = nullptr;
    uint8_t* ok = nullptr;
    float* post = nullptr;
    int64_t bytes = 0;
};

struct Request {
    uint64_t ticket;
    jbp_h* h;
    std::vector<float> y;
    double t_submit;
};

struct Result {
    std::vector<uint8_t> hat;
    std::vector<uint8_t> ok;
    int32_t iters = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Workspace ws;
    size_t host_cap = 0;   // bytes of each pinned array below
    float* h_y = nullptr;
    uint8_t* h_hat = nullptr;
    int32_t* h_iters = nullptr;
    uint8_t* h_ok = nullptr;
    bool busy = false;
    jbp_h* h = nullptr;
    std::vector<Request> reqs;
    int64_t state_bytes = 0;
};

}  // namespace

struct jbp_ctx {
    jbp_options opt{};
    int device = 0;
    DeviceInfo di{};
    cudaStream_t stream = nullptr;
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
    std::vector<Slot> slots;
    int64_t inflight_bytes = 0;
    int handles = 0;
};

struct jbp_h {
    jbp_ctx* ctx = nullptr;
    int K = 0, Q = 0, m = 0, n = 0, P = 0, dc = 0, dv = 0, E = 0;
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
    int64_t table_bytes = 0;
    Workspace ws;
    std::mutex ws_mu;
    bool fused_ok = false;

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

static void ws_io_free(jbp_ctx* ctx, const jbp_h* h, Workspace& w);

static void ws_release(jbp_ctx* ctx, const jbp_h* h, Workspace& w)
{
    const size_t fs = (size_t)h->K * h->E * h->Q, vs = (size_t)h->K * h->n * h->Q;
    dev_free(ctx, w.msg, sizeof(float) * fs * w.cap_step);
    dev_free(ctx, w.ch2v, sizeof(float) * vs * w.cap_step);
    dev_free(ctx, w.active, (size_t)w.cap_step);
    dev_free(ctx, w.unsat, (size_t)w.cap_step * h->K);
    ws_io_free(ctx, h, w);
    w = Workspace();
}

static int ws_step(jbp_ctx* ctx, const jbp_h* h, Workspace& w, int F)
{
    if (F <= w.cap_step) return JBP_OK;
    const size_t fs = (size_t)h->K * h->E * h->Q, vs = (size_t)h->K * h->n * h->Q;
    dev_free(ctx, w.msg, sizeof(float) * fs * w.cap_step);
    dev_free(ctx, w.ch2v, sizeof(float) * vs * w.cap_step);
    dev_free(ctx, w.active, (size_t)w.cap_step);
    dev_free(ctx, w.unsat, (size_t)w.cap_step * h->K);
    w.msg = nullptr; w.ch2v = nullptr; w.active = nullptr; w.unsat = nullptr; w.cap_step = 0;
    int rc;
    if ((rc = dev_alloc(ctx, &w.msg, fs * F, nullptr)) || (rc = dev_alloc(ctx, &w.ch2v, vs * F, nullptr)) ||
        (rc = dev_alloc(ctx, &w.active, (size_t)F, nullptr)) || (rc = dev_alloc(ctx, &w.unsat, (size_t)F * h->K, nullptr))) {
        dev_free(ctx, w.msg, sizeof(float) * fs * F);
        dev_free(ctx, w.ch2v, sizeof(float) * vs * F);
        dev_free(ctx, w.active, (size_t)F);
        w.msg = nullptr; w.ch2v = nullptr; w.active = nullptr; w.unsat = nullptr;
        return rc;
    }
    w.cap_step = F;
    return JBP_OK;
}

static void ws_io_free(jbp_ctx* ctx, const jbp_h* h, Workspace& w)
{
    const size_t vs = (size_t)h->K * h->n * h->Q;
    dev_free(ctx, w.y, sizeof(float) * (size_t)w.cap_io * h->n);
    dev_free(ctx, w.hat, (size_t)w.cap_io * h->K * h->n);
    dev_free(ctx, w.iters, sizeof(int32_t) * (size_t)w.cap_io);
    dev_free(ctx, w.ok, (size_t)w.cap_io * h->K);
    if (w.io_post) dev_free(ctx, w.post, sizeof(float) * vs * w.cap_io);
    w.y = nullptr; w.hat = nullptr; w.iters = nullptr; w.ok = nullptr; w.post = nullptr;
    w.cap_io = 0; w.io_post = false;
}

static int ws_io(jbp_ctx* ctx, const jbp_h* h, Workspace& w, int F, bool post)
{
    if (F <= w.cap_io && (!post || w.io_post)) return JBP_OK;
    ws_io_free(ctx, h, w);
    const size_t vs = (size_t)h->K * h->n * h->Q;
    const int cap = std::max(F, 1);
    int rc;
    if ((rc = dev_alloc(ctx, &w.y, (size_t)cap * h->n, nullptr)) || (rc = dev_alloc(ctx, &w.hat, (size_t)cap * h->K * h->n, nullptr)) ||
        (rc = dev_alloc(ctx, &w.iters, (size_t)cap, nullptr)) || (rc = dev_alloc(ctx, &w.ok, (size_t)cap * h->K, nullptr)) ||
        (post && (rc = dev_alloc(ctx, &w.post, vs * cap, nullptr)))) {
        // free what was allocated (null pointers are skipped)
        w.cap_io = cap;
        w.io_post = (w.post != nullptr);
        ws_io_free(ctx, h, w);
        return rc;
    }
    w.cap_io = cap;
    w.io_post = post;
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// decode forms
// ---------------------------------------------------------------------------

static int run_step_iters(jbp_h* h, Workspace& w, int F, const float* y, uint8_t* hat, int32_t* iters,
                          uint8_t* ok, float* post, cudaStream_t s)
{
    jbp_ctx* ctx = h->ctx;
    const Graph g = h->graph();
    const size_t fs = (size_t)h->K * h->E * h->Q;
    JBP_CU(launch_fill(w.msg, fs * F, 1.0f, s), "init msg");
    JBP_CU(cudaMemsetAsync(w.active, 1, (size_t)F, s), "memset active");
    JBP_CU(cudaMemsetAsync(w.unsat, 0, (size_t)F * h->K, s), "memset unsat");
    StepCtl c{w.active, w.unsat, iters, ok};
    for (int t = 1; t <= ctx->opt.iters; ++t) {
        JBP_CU(launch_channel(g, ctx->di, F, y, w.msg, w.ch2v, w.active, s), "channel kernel");
        JBP_CU(launch_check(g, ctx->di, F, w.msg, w.active, ctx->opt.precision, s), "check kernel");
        JBP_CU(launch_var(g, ctx->di, F, w.ch2v, w.msg, post, hat, w.active, s), "var kernel");
        JBP_CU(launch_syndrome(g, ctx->di, F, hat, w.unsat, w.active, s), "syndrome kernel");
        JBP_CU(launch_finalize(F, h->K, t, ctx->opt.early_stop, c, s), "finalize kernel");
    }
    return JBP_OK;
}

// Decode F frames whose buffers are all on the device, on stream s.
static int decode_device(jbp_h* h, Workspace& w, int form, int F, const float* y, uint8_t* hat, int32_t* iters,
                         uint8_t* ok, float* post, cudaStream_t s)
{
    if (F == 0) return JBP_OK;
    jbp_ctx* ctx = h->ctx;
    // the fused kernel runs the FP32 butterfly check node; the tensor-core
    // precision variants run in the step form
    if (form == JBP_FORM_AUTO) form = (h->fused_ok && ctx->opt.precision == JBP_PREC_FP32) ? JBP_FORM_FUSED : JBP_FORM_STEP;
    if (form == JBP_FORM_FUSED && ctx->opt.precision != JBP_PREC_FP32)
        return fail(JBP_EINVAL, "the fused form runs the FP32 check node; use the step form for precision %d",
                    ctx->opt.precision);
    if (form == JBP_FORM_FUSED) {
        if (!h->fused_ok) return fail(JBP_EINVAL, "one frame does not fit the fused form (shared memory)");
        FusedPlan plan;
        if (!fused_plan(h->graph(), ctx->di, F, 0, 0, &plan)) return fail(JBP_EINVAL, "no fused launch plan");
        JBP_CU(launch_fused(h->graph(), plan, F, y, ctx->opt.iters, ctx->opt.early_stop, hat, iters, ok, post, s),
               "fused kernel");
        return JBP_OK;
    }
    if (form == JBP_FORM_STEP) {
        int rc = ws_step(ctx, h, w, F);
        if (rc) return rc;
        return run_step_iters(h, w, F, y, hat, iters, ok, post, s);
    }
    if (form == JBP_FORM_PLAIN) {
        int rc = ws_step(ctx, h, w, 1);
        if (rc) return rc;
        const size_t vs = (size_t)h->K * h->n * h->Q;
        for (int f = 0; f < F; ++f) {
            rc = run_step_iters(h, w, 1, y + (size_t)f * h->n, hat + (size_t)f * h->K * h->n, iters + f,
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

extern "C" int jbp_context_create(const jbp_options* opt, jbp_ctx** out)
{
    if (!opt || !out) return fail(JBP_EINVAL, "jbp_context_create: NULL argument");
    if (opt->iters < 1) return fail(JBP_EINVAL, "iters must be >= 1 (got %d)", opt->iters);
    if (opt->precision < 0 || opt->precision > 3) return fail(JBP_EINVAL, "bad precision %d", opt->precision);
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
        (e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess) {
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
    for (Slot& s : ctx->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        cudaFreeHost(s.h_y); cudaFreeHost(s.h_hat); cudaFreeHost(s.h_iters); cudaFreeHost(s.h_ok);
    }
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------

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
    if (code->dc != 4) return fail(JBP_EINVAL, "only check degree dc = 4 is built (got %d)", code->dc);
    if (code->dv < 1 || code->dv > kMaxDv) return fail(JBP_EINVAL, "dv must be in 1..%d (got %d)", kMaxDv, code->dv);
    if ((int64_t)code->n * code->dv != (int64_t)code->P * code->dc)
        return fail(JBP_EINVAL, "n*dv (%d*%d) != P*dc (%d*%d)", code->n, code->dv, code->P, code->dc);
    if (!code->chk_var || !code->chk_coef) return fail(JBP_EINVAL, "NULL code arrays");
    if (!(chan->sigma2 > 0.0) || !std::isfinite(chan->sigma2)) return fail(JBP_EINVAL, "sigma2 must be finite and > 0");
    if (chan->interleave && !chan->perm) return fail(JBP_EINVAL, "interleave = 1 needs perm");
    const int n = code->n, P = code->P, dc = code->dc, dv = code->dv, E = P * dc;

    std::vector<int32_t> var_edge((size_t)n * dv), fill(n, 0);
    for (int e = 0; e < E; ++e) {
        const int i = code->chk_var[e];
        if (i < 0 || i >= n) return fail(JBP_EINVAL, "chk_var[%d] = %d out of range", e, i);
        if (code->chk_coef[e] < 1 || code->chk_coef[e] >= q) return fail(JBP_EINVAL, "chk_coef[%d] = %d not in 1..q-1", e, code->chk_coef[e]);
        if (fill[i] >= dv) return fail(JBP_EINVAL, "variable %d has more than dv = %d edges", i, dv);
        var_edge[(size_t)i * dv + fill[i]++] = e;
    }
    for (int i = 0; i < n; ++i)
        if (fill[i] != dv) return fail(JBP_EINVAL, "variable %d has %d edges, expected dv = %d", i, fill[i], dv);
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
    const bool want_slot = dv == 2 && n <= 32767;
    std::vector<uint16_t> slot(want_slot ? (size_t)K * E : 0);
    if (want_slot)
        for (int k = 0; k < K; ++k)
            for (int e = 0; e < E; ++e) {
                const int i = code->chk_var[e];
                const int rank = var_edge[(size_t)i * dv] == e ? 0 : 1;
                slot[(size_t)k * E + e] = (uint16_t)(pos_of[(size_t)k * n + i] * 2 + rank);
            }
    std::vector<uint8_t> gmul((size_t)q * q), gdiv((size_t)q * q);
    std::vector<int> inv(q, 0);
    for (int a = 1; a < q; ++a)
        for (int b = 1; b < q; ++b)
            if (gf_mul_host(a, b, m) == 1) inv[a] = b;
    for (int h = 0; h < q; ++h)
        for (int x = 0; x < q; ++x) {
            gmul[(size_t)h * q + x] = (uint8_t)gf_mul_host(h, x, m);
            gdiv[(size_t)h * q + x] = (uint8_t)gf_mul_host(inv[h], x, m);
        }
    const int scf = chan_scratch_floats(K, q);
    const int team_lanes = q < 32 ? q : 32;
    if ((size_t)(32 / team_lanes) * scf * sizeof(float) > (size_t)ctx->di.smem_optin)
        return fail(JBP_EINVAL, "K = %d, q = %d: channel trellis does not fit shared memory", K, q);

    JBP_CU(cudaSetDevice(ctx->device), "cudaSetDevice");
    jbp_h* h = new (std::nothrow) jbp_h();
    if (!h) return fail(JBP_ENOMEM, "host allocation failed");
    h->ctx = ctx; h->K = K; h->Q = q; h->m = m; h->n = n; h->P = P; h->dc = dc; h->dv = dv; h->E = E;
    h->sigma2 = chan->sigma2;
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
        (want_slot && (rc = dev_alloc(ctx, &h->d_slot, (size_t)K * E, &h->table_bytes)))) {
        jbp_destroy(h);
        return rc;
    }
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
         (e = cudaMemcpy(h->d_slot, slot.data(), sizeof(uint16_t) * slot.size(), cudaMemcpyHostToDevice)))) {
        jbp_destroy(h);
        return cuda_fail(e, "jbp_create: copy tables");
    }
    FusedPlan plan;
    h->fused_ok = fused_plan(h->graph(), ctx->di, 1, 0, 0, &plan);
    cudaGetLastError();
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->handles++;
    }
    *out = h;
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
        ctx->cv_idle.wait(lk, [&] {
            for (const Slot& s : ctx->slots)
                if (s.busy && s.h == h) return false;
            return true;
        });
        for (Slot& s : ctx->slots) {
            if (s.h != h) continue;
            ws_release(ctx, h, s.ws);
            s.h = nullptr;
        }
        if (counted) ctx->handles--;
    }
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ws_release(ctx, h, h->ws);
    dev_free(ctx, h->d_chk_var, sizeof(int32_t) * h->E);
    dev_free(ctx, h->d_chk_coef, (size_t)h->E);
    dev_free(ctx, h->d_var_edge, sizeof(int32_t) * (size_t)h->n * h->dv);
    dev_free(ctx, h->d_use_pos, sizeof(int32_t) * (size_t)h->K * h->n);
    dev_free(ctx, h->d_gf_mul, (size_t)h->Q * h->Q);
    dev_free(ctx, h->d_gf_div, (size_t)h->Q * h->Q);
    dev_free(ctx, h->d_fallbacks, sizeof(unsigned long long));
    dev_free(ctx, h->d_pos_of, sizeof(int32_t) * (size_t)h->K * h->n);
    dev_free(ctx, h->d_tc_error, sizeof(int));
    if (h->d_slot) dev_free(ctx, h->d_slot, sizeof(uint16_t) * (size_t)h->K * h->E);
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
        return decode_device(h, h->ws, b->form, F, b->y, b->hat, b->iters, b->ok, b->logpost, s);
    }
    cudaStream_t s = ctx->stream;
    std::lock_guard<std::mutex> lk(h->ws_mu);
    Workspace& w = h->ws;
    int rc = ws_io(ctx, h, w, F, b->logpost != nullptr);
    if (rc) return rc;
    const size_t vs = (size_t)h->K * h->n * h->Q;
    JBP_CU(cudaMemcpyAsync(w.y, b->y, sizeof(float) * (size_t)F * h->n, cudaMemcpyHostToDevice, s), "copy y");
    rc = decode_device(h, w, b->form, F, w.y, w.hat, w.iters, w.ok, b->logpost ? w.post : nullptr, s);
    if (rc) return rc;
    JBP_CU(cudaMemcpyAsync(b->hat, w.hat, (size_t)F * h->K * h->n, cudaMemcpyDeviceToHost, s), "copy hat");
    JBP_CU(cudaMemcpyAsync(b->iters, w.iters, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s), "copy iters");
    JBP_CU(cudaMemcpyAsync(b->ok, w.ok, (size_t)F * h->K, cudaMemcpyDeviceToHost, s), "copy ok");
    if (b->logpost)
        JBP_CU(cudaMemcpyAsync(b->logpost, w.post, sizeof(float) * vs * F, cudaMemcpyDeviceToHost, s), "copy post");
    JBP_CU(cudaStreamSynchronize(s), "jbp_decode");
    if (ctx->opt.precision != JBP_PREC_FP32) {
        int err = 0;
        JBP_CU(cudaMemcpy(&err, h->d_tc_error, sizeof err, cudaMemcpyDeviceToHost), "jbp_decode: status");
        if (err) return fail(JBP_ETIMEOUT, "a tensor-core completion wait expired");
    }
    return JBP_OK;
}

// ---------------------------------------------------------------------------
// single steps
// ---------------------------------------------------------------------------

static cudaStream_t pick_stream(jbp_h* h, void* s) { return s ? (cudaStream_t)s : h->ctx->stream; }

extern "C" int jbp_step_channel(jbp_h* h, int32_t F, const float* y, float* msg, float* ch2v, void* stream)
{
    if (!h || F < 0 || (F > 0 && (!y || !msg || !ch2v))) return fail(JBP_EINVAL, "jbp_step_channel: bad argument");
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    JBP_CU(launch_channel(h->graph(), h->ctx->di, F, y, msg, ch2v, nullptr, pick_stream(h, stream)), "channel kernel");
    return JBP_OK;
}

extern "C" int jbp_step_check(jbp_h* h, int32_t F, float* msg, int32_t precision, void* stream)
{
    if (!h || F < 0 || (F > 0 && !msg)) return fail(JBP_EINVAL, "jbp_step_check: bad argument");
    if (precision < 0 || precision > 3) return fail(JBP_EINVAL, "bad precision %d", precision);
    JBP_CU(cudaSetDevice(h->ctx->device), "cudaSetDevice");
    JBP_CU(launch_check(h->graph(), h->ctx->di, F, msg, nullptr, precision, pick_stream(h, stream)), "check kernel");
    return JBP_OK;
}

extern "C" int jbp_step_var(jbp_h* h, int32_t F, const float* ch2v, const float* msg, float* post, uint8_t* hat,
                            void* stream)
{
    if (!h || F < 0 || (F > 0 && (!ch2v || !msg || !hat))) return fail(JBP_EINVAL, "jbp_step_var: bad argument");
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
// serving: continuous batching across concurrent launches
// ---------------------------------------------------------------------------
//
// jbp_submit queues one frame.  A server thread repeatedly (1) retires finished
// launches, publishing their results, and (2) admits queued frames into a free
// launch slot (its own stream, pinned staging and device workspace) as long as
// the message state of everything in flight stays within the memory budget.
// Frames of one handle that are queued together share a launch; launches of
// different slots overlap on the device.  Each frame's arithmetic does not
// depend on which other frames share its launch.

static constexpr int kSlots = 4;
static constexpr int kMaxServeBatch = 8192;

static int slot_prepare(jbp_ctx* ctx, Slot& s, jbp_h* h, int F)
{
    if (!s.stream) {
        JBP_CU(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "slot stream");
        JBP_CU(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming), "slot event");
    }
    if (s.h != h && (s.ws.cap_step || s.ws.cap_io)) {
        if (s.h) ws_release(ctx, s.h, s.ws);
    }
    s.h = h;
    const size_t need = std::max<size_t>({sizeof(float) * (size_t)F * h->n, (size_t)F * h->K * h->n,
                                          sizeof(int32_t) * (size_t)F, (size_t)F * h->K});
    if (need > s.host_cap) {
        cudaFreeHost(s.h_y); cudaFreeHost(s.h_hat); cudaFreeHost(s.h_iters); cudaFreeHost(s.h_ok);
        s.h_y = nullptr; s.h_hat = nullptr; s.h_iters = nullptr; s.h_ok = nullptr; s.host_cap = 0;
        const size_t cap = std::max(need, (size_t)(1 << 16));
        JBP_CU(cudaMallocHost((void**)&s.h_y, cap), "pinned y");
        JBP_CU(cudaMallocHost((void**)&s.h_hat, cap), "pinned hat");
        JBP_CU(cudaMallocHost((void**)&s.h_iters, cap), "pinned iters");
        JBP_CU(cudaMallocHost((void**)&s.h_ok, cap), "pinned ok");
        s.host_cap = cap;
    }
    return ws_io(ctx, h, s.ws, F, false);
}

static int slot_launch(jbp_ctx* ctx, Slot& s)
{
    jbp_h* h = s.h;
    const int F = (int)s.reqs.size();
    for (int f = 0; f < F; ++f) memcpy(s.h_y + (size_t)f * h->n, s.reqs[f].y.data(), sizeof(float) * h->n);
    JBP_CU(cudaMemcpyAsync(s.ws.y, s.h_y, sizeof(float) * (size_t)F * h->n, cudaMemcpyHostToDevice, s.stream), "serve copy y");
    int rc = decode_device(h, s.ws, JBP_FORM_AUTO, F, s.ws.y, s.ws.hat, s.ws.iters, s.ws.ok, nullptr, s.stream);
    if (rc) return rc;
    JBP_CU(cudaMemcpyAsync(s.h_hat, s.ws.hat, (size_t)F * h->K * h->n, cudaMemcpyDeviceToHost, s.stream), "serve copy hat");
    JBP_CU(cudaMemcpyAsync(s.h_iters, s.ws.iters, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s.stream), "serve copy iters");
    JBP_CU(cudaMemcpyAsync(s.h_ok, s.ws.ok, (size_t)F * h->K, cudaMemcpyDeviceToHost, s.stream), "serve copy ok");
    JBP_CU(cudaEventRecord(s.done, s.stream), "serve event");
    return JBP_OK;
}

static void server_main(jbp_ctx* ctx)
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (true) {
        bool any_busy = false;
        // (1) retire finished launches
        for (Slot& s : ctx->slots) {
            if (!s.busy) continue;
            cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            const double t = now_us();
            jbp_h* h = s.h;
            for (size_t f = 0; f < s.reqs.size(); ++f) {
                Result r;
                r.hat.assign(s.h_hat + f * h->K * h->n, s.h_hat + (f + 1) * h->K * h->n);
                r.ok.assign(s.h_ok + f * h->K, s.h_ok + (f + 1) * h->K);
                r.iters = q == cudaSuccess ? s.h_iters[f] : -1;
                ctx->done[s.reqs[f].ticket] = std::move(r);
                ctx->pending.erase(s.reqs[f].ticket);
                ctx->latencies.push_back(t - s.reqs[f].t_submit);
                ctx->completed++;
            }
            ctx->inflight_bytes -= s.state_bytes;
            s.reqs.clear();
            s.busy = false;
            ctx->cv_idle.notify_all();
        }
        // (2) admit queued frames into free slots
        while (!ctx->queue.empty()) {
            Slot* free_slot = nullptr;
            for (Slot& s : ctx->slots)
                if (!s.busy) { free_slot = &s; break; }
            if (!free_slot) break;
            jbp_h* h = ctx->queue.front().h;
            const int64_t per_frame = state_bytes(h->graph()) + (int64_t)h->n * 4 + (int64_t)h->K * (h->n + 1) + 4;
            std::vector<Request> batch;
            int64_t bytes = 0;
            for (auto it = ctx->queue.begin(); it != ctx->queue.end() && (int)batch.size() < kMaxServeBatch;) {
                if (it->h == h && ctx->inflight_bytes + bytes + per_frame <= ctx->budget / 2) {
                    bytes += per_frame;
                    batch.push_back(std::move(*it));
                    it = ctx->queue.erase(it);
                } else {
                    ++it;
                }
            }
            if (batch.empty()) break;   // over budget: wait for a launch to retire
            Slot& s = *free_slot;
            s.reqs = std::move(batch);
            s.state_bytes = bytes;
            int rc = slot_prepare(ctx, s, h, (int)s.reqs.size());
            if (!rc) rc = slot_launch(ctx, s);
            if (rc) {
                // publish the failure to each ticket
                for (const Request& r : s.reqs) {
                    Result res;
                    res.iters = -1;
                    res.hat.assign((size_t)h->K * h->n, 0);
                    res.ok.assign((size_t)h->K, 0);
                    ctx->done[r.ticket] = std::move(res);
                    ctx->pending.erase(r.ticket);
                }
                s.reqs.clear();
                cudaGetLastError();
                continue;
            }
            s.busy = true;
            any_busy = true;
            ctx->inflight_bytes += bytes;
        }
        if (ctx->stop && !any_busy) break;
        if (any_busy)
            ctx->cv.wait_for(lk, std::chrono::microseconds(20));
        else
            ctx->cv.wait(lk, [&] { return ctx->stop || !ctx->queue.empty(); });
    }
}

extern "C" int jbp_submit(jbp_h* h, const float* y_frame, uint64_t* ticket)
{
    if (!h || !y_frame || !ticket) return fail(JBP_EINVAL, "jbp_submit: NULL argument");
    jbp_ctx* ctx = h->ctx;
    Request r;
    r.h = h;
    r.y.assign(y_frame, y_frame + h->n);
    r.t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->stop) return fail(JBP_ECLOSED, "context is shutting down");
        if (!ctx->server_started) {
            ctx->slots.resize(kSlots);
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
