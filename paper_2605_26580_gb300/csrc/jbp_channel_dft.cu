// jbp_channel_dft.cu -- channel node (kernel (a)) as discrete Fourier transforms
// over the integer symbol-sum alphabet, with the transforms issued as matrix
// products on the 5th-generation tensor cores (tcgen05).
//
// For one channel use with user messages mu_0..mu_{K-1} (length q) and the
// Gaussian score G(u) of the sum value u = 0..K(q-1), the extrinsic message to
// user k is the correlation
//     ch2v_k(a) ~ sum_s E_k(s) G(s + a),   E_k = the integer convolution of mu_j, j != k.
// With a DFT length L >= K(q-1)+1 the circular correlation equals the linear one
// for a = 0..q-1, and with hats for DFTs (e^{-2 pi i f x / L}):
//     X_k(f) = G^(f) conj(prod_{j != k} mu^_j(f)),   ch2v_k(a) ~ sum_f X_k(f) e^{+2 pi i f a / L}.
// Real inputs make the spectra Hermitian, so frequencies 0..L/2 carry everything:
// L real spectral columns, pairs (Re, Im) of f = 1..L/2-1 and the pair (DC, Nyquist).
//
// A CTA of 256 threads takes tiles of 128 channel uses (rows; thread t and
// t + 128 share row t % 128 and split its work).  Per tile:
//   1. each row's mu_j = c2v_e0 * c2v_e1 (its variable's two edges) and a window of
//      W values of G around the most likely sum are staged in shared memory as FP16
//      operands (one term each; lane groups move the message vectors);
//   2. per chunk of Nc spectral columns: one thread issues the forward DFT products
//      (every mu_j, and the G window, against the shared forward matrix) into tensor
//      memory; every thread reads its row's spectra, scales each by its DC term,
//      rotates the window spectrum to its offset, forms the K leave-one-out
//      products X_k by prefix and suffix products (no division) and stages them
//      (hi + lo) as the operand of the inverse DFT, which accumulates over the
//      chunks in tensor memory (K q columns);
//   3. every thread reads the accumulated messages of its users, normalises them
//      to max 1 with the floor, and writes ch2v and the two v2c messages of each
//      variable (the same outputs as the trellis kernels).  A channel use whose
//      peak is too small for the transform to resolve (the other users' beliefs
//      make the observed sum nearly impossible) is left to the FP32 trellis,
//      which a second launch runs on just those channel uses.
// Numerics: products of FP16 terms are exact and accumulate in FP32.  mu and the
// G window are single FP16 terms: a relative rounding of at most 2^-12 per value,
// which perturbs each output by at most (K - 1 + 1) 2^-12 relative.  The DFT
// matrices and the X_k are hi + lo terms (about 2^-22): the inverse transform
// subtracts terms of the size of the whole spectrum, so that part of the error is
// absolute, a fraction of each message's maximum, instead of relative per entry
// as in the FP32 trellis.
// Every mbarrier wait is bounded; on expiry the kernel records an error in
// g.tc_error, frees its tensor memory and returns.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_fp16.h>

#include "jbp_internal.h"
#include "jbp_tc.cuh"

namespace jbp {
namespace {

// two values rounded to FP16 in one packed conversion (first in the low half)
__device__ __forceinline__ uint32_t h2bits(__half2 h) { return *reinterpret_cast<const uint32_t*>(&h); }

// 8 values as one 16-byte core-matrix row of FP16 hi terms and one of lo terms
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2 hh = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
        const float2 back = __half22float2(hh);
        h[i] = h2bits(hh);
        l[i] = h2bits(__floats2half2_rn(v[2 * i] - back.x, v[2 * i + 1] - back.y));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    return make_uint4(h2bits(__floats2half2_rn(v[0], v[1])), h2bits(__floats2half2_rn(v[2], v[3])),
                      h2bits(__floats2half2_rn(v[4], v[5])), h2bits(__floats2half2_rn(v[6], v[7])));
}

struct Cx {
    float r, i;
};
__device__ __forceinline__ Cx cmul(Cx a, Cx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
// a * conj(b)
__device__ __forceinline__ Cx cmulc(Cx a, Cx b) { return {a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i}; }

// X_k = g conj(prod_{j != k} m_j) for every k, by prefix and suffix products
template <int K>
__device__ __forceinline__ void leave_one_out(const Cx (&m)[K], Cx g, Cx (&X)[K])
{
    Cx pre[K];
    pre[0] = {1.0f, 0.0f};
#pragma unroll
    for (int k = 1; k < K; ++k) pre[k] = k == 1 ? m[0] : cmul(pre[k - 1], m[k - 1]);
    Cx suf = {1.0f, 0.0f};
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        const Cx e = k == K - 1 ? pre[k] : k == 0 ? suf : cmul(pre[k], suf);
        X[k] = cmulc(g, e);
        if (k > 0) suf = k == K - 1 ? m[k] : cmul(suf, m[k]);
    }
}

// Smallest peak mass (fraction of the normalised spectra's total) that the
// transform resolves: its absolute error, of order 2^-22 per spectral term,
// stays below about 1e-3 of such a peak.
constexpr float kMinPeak = 1.0f / 4096.0f;

template <int Q, int K>
struct ShapeOf {
    static constexpr DftShape v = dft_shape(K, Q);
};

// Forward products of one chunk (one thread): spectrum of mu_j into columns
// SP + j Nc, of the G window into SP + K Nc.  Terms A*B_hi + A*B_lo.  The
// operand descriptors are the tiles' step-0 descriptors plus constant offsets.
template <int Q, int K, class Sh>
__device__ __forceinline__ void issue_forward(uint32_t tmem, uint64_t dA1, uint64_t dAG, uint64_t dB1)
{
    constexpr DftShape S = Sh::v;
    constexpr int NC = S.Nc, W = S.W, SP = S.KG * Q;
    constexpr uint32_t kA1 = kDftRows * Q * 2, kB1 = NC * S.KB * 2;
    constexpr uint32_t id = tc::idesc_f16(kDftRows, NC, false);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t d = tmem + SP + j * NC;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int ks = 0; ks < Q / 16; ++ks)
                tc::mma_f16(d, dA1 + ((j * kA1 + ks * 256) >> 4), dB1 + ((p * kB1 + ks * 256) >> 4), id, p | ks);
    }
    const uint32_t d = tmem + SP + K * NC;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int ks = 0; ks < W / 16; ++ks)
            tc::mma_f16(d, dAG + ks * 16, dB1 + ((p * kB1 + ks * 256) >> 4), id, p | ks);
}

// Inverse products of chunk c (one thread): X of the pass's user slot k < kn
// against the inverse rows, accumulated into columns k q.
template <int Q, int K, class Sh>
__device__ __forceinline__ void issue_inverse(uint32_t tmem, uint64_t dA3, uint64_t dB3, int c, int kn)
{
    constexpr int NC = Sh::v.Nc;
    constexpr uint32_t kA3 = kDftRows * NC * 2, kB3 = Q * NC * 2;
    constexpr uint32_t id = tc::idesc_f16(kDftRows, Q, false);
#pragma unroll
    for (int k = 0; k < Sh::v.KG; ++k) {
        if (k >= kn) break;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int ks = 0; ks < NC / 16; ++ks)
                tc::mma_f16(tmem + k * Q, dA3 + (((2 * k + (p == 1)) * kA3 + ks * 256) >> 4),
                            dB3 + (((p == 2) * kB3 + ks * 256) >> 4), id, (c > 0) | p | ks);
    }
}

// lanes of one group that moves one (row, user) message vector: a float4 each
template <int Q>
struct Group {
    static constexpr int GL = Q / 4;          // lanes per vector
    static constexpr int PPW = 32 / GL;       // vectors per warp instruction
};

// largest divisor of n that is at most 8
__host__ __device__ constexpr int batch_of(int n)
{
    int b = 8;
    while (n % b) --b;
    return b;
}

template <int GL>
__device__ __forceinline__ float group_max(float x)
{
#pragma unroll
    for (int o = GL / 2; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

__device__ __forceinline__ float max4(float4 v) { return fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)); }
__device__ __forceinline__ float4 mul4(float4 a, float4 b)
{
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 scale4(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }

template <int Q, int K>
__global__ void __launch_bounds__(kDftThreads, 1) k_channel_dft(Graph g, int F, const float* __restrict__ y,
                                                               float* msg, float* ch2v,
                                                               const uint8_t* __restrict__ active)
{
    using Sh = ShapeOf<Q, K>;
    constexpr DftShape S = Sh::v;
    static_assert(S.ok, "no tensor-core channel shape for this (K, q)");
    constexpr int L = S.L, W = S.W, NC = S.Nc, CH = S.chunks, U = S.U, R = kDftRows;
    constexpr int KG = S.KG, NP = S.NP, SP = KG * Q;   // users per pass, passes, first spectrum column
    constexpr int NW = kDftThreads / 32, GL = Group<Q>::GL, PPW = Group<Q>::PPW;
    constexpr int IT = R * K / (NW * PPW);   // (row, user) vectors per lane group and tile
    constexpr int BT = batch_of(IT);         // of which in flight at once
    constexpr uint32_t kA1 = R * Q * 2, kAG = R * W * 2, kB1 = NC * S.KB * 2, kB3 = Q * NC * 2, kA3 = R * NC * 2;
    constexpr uint32_t kChunk = 2 * kB1 + 2 * kB3;
    constexpr int SS = K * Q + 4;   // row stride (floats) of the output stage: rows fall on shifted banks
    static_assert(NP > 1 || R * SS * 4 <= K * kA1 + kAG + 2 * K * kA3,
                  "output stage exceeds the operand tiles it reuses");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* A1 = smem;                 // [K][R x q]           mu_j
    unsigned char* AG = A1 + K * kA1;         // [R x W]              G window
    unsigned char* A3 = AG + kAG;             // [KG][hi, lo][R x Nc] X_k of the pass's users
    unsigned char* BC = A3 + 2 * KG * kA3;    // forward rows (hi, lo), inverse rows (hi, lo) of a chunk
    float2* TW = reinterpret_cast<float2*>(BC + kChunk);         // [L] (cos, sin)(2 pi m / L)
    int* s_off = reinterpret_cast<int*>(TW + L);                 // [R][K][3] offsets of e0, e1 (msg), ch2v
    float* stage = reinterpret_cast<float*>(smem);               // [R][SS] messages (reuses A1, AG, A3)
    __shared__ __align__(8) uint64_t mbar_store;
    __shared__ uint32_t tmem_holder;
    __shared__ int s_rowf[R];          // frame of each row, -1 if the row is not decoded
    __shared__ uint8_t s_weak[2][R];   // per half and row: a user's peak is below kMinPeak

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int m = quarter * 32 + lane;   // this thread's row (= its tensor-memory lane)
    const int gsub = lane / GL, gl = lane % GL;
    const unsigned char* tab = g.dft_tab;
    for (int i = t; i < L; i += blockDim.x) TW[i] = reinterpret_cast<const float2*>(tab + (size_t)CH * kChunk)[i];
    // forward rows of the next forward product (r1) and inverse rows of the next inverse product (r3)
    constexpr int P1 = CH > 1 ? (int)((2 * kB1 / 16 + kDftThreads - 1) / kDftThreads) : 1;
    constexpr int P3 = CH > 1 ? (int)((2 * kB3 / 16 + kDftThreads - 1) / kDftThreads) : 1;
    uint4 r1[P1], r3[P3];
    auto fetch = [&](int c) {   // r1 <- forward rows of chunk c
        const uint4* src = reinterpret_cast<const uint4*>(tab + (size_t)c * kChunk);
#pragma unroll
        for (int i = 0; i < P1; ++i) {
            const int j = t + i * kDftThreads;
            if (j < (int)(2 * kB1 / 16)) r1[i] = src[j];
        }
    };
    auto fetch3 = [&](int c) {   // r3 <- inverse rows of chunk c
        const uint4* src = reinterpret_cast<const uint4*>(tab + (size_t)c * kChunk + 2 * kB1);
#pragma unroll
        for (int i = 0; i < P3; ++i) {
            const int j = t + i * kDftThreads;
            if (j < (int)(2 * kB3 / 16)) r3[i] = src[j];
        }
    };
    auto put1 = [&]() {
        uint4* dst = reinterpret_cast<uint4*>(BC);
#pragma unroll
        for (int i = 0; i < P1; ++i) {
            const int j = t + i * kDftThreads;
            if (j < (int)(2 * kB1 / 16)) dst[j] = r1[i];
        }
    };
    auto put3 = [&]() {
        uint4* dst = reinterpret_cast<uint4*>(BC + 2 * kB1);
#pragma unroll
        for (int i = 0; i < P3; ++i) {
            const int j = t + i * kDftThreads;
            if (j < (int)(2 * kB3 / 16)) dst[j] = r3[i];
        }
    };
    if constexpr (CH == 1) {   // one chunk: the DFT rows stay resident
        const uint4* src = reinterpret_cast<const uint4*>(tab);
        uint4* dst = reinterpret_cast<uint4*>(BC);
        for (int i = t; i < (int)(kChunk / 16); i += blockDim.x) dst[i] = src[i];
    } else {
        fetch(0);
        fetch3(0);
    }
    const uint32_t mbar = tc::smem_addr(&mbar_store);
    if (t == 0) tc::mbar_init(mbar);
    if (warp == 0) tc::tmem_alloc(&tmem_holder, S.tmem_cols);
    tc::proxy_fence();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint64_t dA1 = tc::tile_desc(tc::smem_addr(A1), Q), dAG = tc::tile_desc(tc::smem_addr(AG), W),
                   dB1 = tc::tile_desc(tc::smem_addr(BC), S.KB), dB3 = tc::tile_desc(tc::smem_addr(BC) + 2 * kB1, NC),
                   dA3 = tc::tile_desc(tc::smem_addr(A3), NC);
    uint32_t phase = 0;
    bool ok = true;
    const long total = (long)F * g.n;
    const long tiles = (total + R - 1) / R;
    const size_t us = (size_t)g.E * Q, fs = (size_t)K * us, vs = (size_t)K * g.n * Q;

    const int* __restrict__ tab_off = reinterpret_cast<const int*>(tab + (size_t)CH * kChunk + (size_t)L * 8);

    for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long r = tile * R + m;
        const long f = r < total ? r / g.n : 0;
        const int u = r < total ? (int)(r % g.n) : 0;
        const bool live = r < total && (!active || active[f]);
        GaussTerm gt{};
        int u_lo = 0;
        // 1. the row's message offsets (this half's users, from the handle's table),
        // the G window, then mu by lane groups
        if (half == 0) s_rowf[m] = live ? (int)f : -1;
        if (live) {
            for (int k = half; k < K; k += 2) {
                const int* o = tab_off + ((size_t)u * K + k) * 3;
                int* so = s_off + (m * K + k) * 3;
                so[0] = o[0];
                so[1] = o[1];
                so[2] = o[2];
            }
            gt = gauss_term(y[r], K, Q, frame_inv_s2(g, f));
            u_lo = min(max(gt.ss - W / 2, 0), max(U - W, 0));
        }
        if constexpr (CH > 1) put1();   // forward rows of chunk 0 (the last tile's products are done)
#pragma unroll
        for (int kq = 0; kq < W / 16; ++kq) {   // this half of the G window
            const int kg = half * (W / 16) + kq;
            float e[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int ii = kg * 8 + i, uu = u_lo + ii;
                e[i] = live ? (uu < U ? gt.score(uu) : 0.0f) : (ii == 0 ? 1.0f : 0.0f);
            }
            *reinterpret_cast<uint4*>(AG + tc::tile_off(m, kg, W)) = pack8(e);
        }
        __syncthreads();
        if constexpr (CH > 1) fetch(1);
        // mu_j = c2v_e0 * c2v_e1, max 1: BT vectors per lane group in flight
#pragma unroll 1
        for (int b0 = 0; b0 < IT; b0 += BT) {
            float4 va[BT], vb[BT];
#pragma unroll
            for (int i = 0; i < BT; ++i) {
                const int p = (b0 + i) * NW * PPW + warp * PPW + gsub, mr = p / K, k = p - mr * K;
                const int fr = s_rowf[mr];
                va[i] = vb[i] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
                if (fr >= 0) {
                    const float* mf = msg + (size_t)fr * fs;
                    const int* o = s_off + (mr * K + k) * 3;
                    va[i] = reinterpret_cast<const float4*>(mf + o[0])[gl];
                    vb[i] = reinterpret_cast<const float4*>(mf + o[1])[gl];
                }
            }
#pragma unroll
            for (int i = 0; i < BT; ++i) {
                const int p = (b0 + i) * NW * PPW + warp * PPW + gsub, mr = p / K, k = p - mr * K;
                float4 v = mul4(va[i], vb[i]);
                if (s_rowf[mr] < 0) v = make_float4(gl == 0 ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f);
                const float inv = 1.0f / group_max<GL>(max4(v));
                const float4 w = scale4(v, inv);
                *reinterpret_cast<uint2*>(A1 + k * kA1 + tc::tile_off(mr, gl >> 1, Q) + (gl & 1) * 8) =
                    make_uint2(h2bits(__floats2half2_rn(w.x, w.y)), h2bits(__floats2half2_rn(w.z, w.w)));
            }
        }

        // 2. chunks of the spectrum.  Per chunk c: wait for the forward products of c
        // (and the inverse products of c-1); every thread takes its share of the
        // chunk's spectra into registers; the forward products of c+1 are issued and
        // run while the threads form the X_k of chunk c; then the inverse products of c.
        float inv_dc[K + 1];
        bool weak = false;   // some user's peak below kMinPeak (this thread's users, all passes)
#pragma unroll
        for (int pass = 0; pass < NP; ++pass) {
            const int k0 = pass * KG, kn = min(KG, K - k0);
            if (pass > 0) {
                if constexpr (CH > 1) {   // forward rows of chunk 0 (the previous pass's products are done)
                    put1();
                    fetch(1);
                }
            }
            tc::proxy_fence();
            tc::fence_before();
            __syncthreads();
            if (t == 0) {
                tc::fence_after();
                issue_forward<Q, K, Sh>(tmem, dA1, dAG, dB1);
                tc::mma_commit(mbar);
            }
#pragma unroll 1
            for (int c = 0; c < CH; ++c) {
                // each thread waits on its own; the barrier below settles an expiry for all
                const bool done = tc::spin_wait(mbar, phase);
                phase ^= 1;
                tc::fence_after();
                uint32_t spec[K + 1][NC / 16][8];
#pragma unroll
                for (int j = 0; j <= K; ++j)
#pragma unroll
                    for (int q8 = 0; q8 < NC / 16; ++q8)
                        tc::tmem_ld8_nowait(trow + SP + j * NC + half * (NC / 2) + q8 * 8, spec[j][q8]);
                if (c == 0) {   // DC terms (real, >= 1): every spectrum is scaled to DC 1
                    uint32_t raw[K + 1][8];
#pragma unroll
                    for (int j = 0; j <= K; ++j) tc::tmem_ld8_nowait(trow + SP + j * NC, raw[j]);
                    tc::ld_wait();
#pragma unroll
                    for (int j = 0; j <= K; ++j) inv_dc[j] = 1.0f / __uint_as_float(raw[j][0]);
                }
                tc::ld_wait();
                if constexpr (CH > 1) {
                    put3();                          // inverse rows of chunk c
                    fetch3((c + 1) % CH);
                    if (c + 1 < CH) {
                        put1();                      // forward rows of chunk c + 1
                        fetch((c + 2) % CH);
                    }
                }
                tc::fence_before();
                tc::proxy_fence();
                if (__syncthreads_or(done ? 0 : 1)) {
                    if (t == 0) atomicExch(g.tc_error, 1);
                    ok = false;
                    break;
                }
                if (t == 0 && c + 1 < CH) {
                    tc::fence_after();
                    issue_forward<Q, K, Sh>(tmem, dA1, dAG, dB1);
                }
#pragma unroll
                for (int cq = 0; cq < NC / 16; ++cq) {
                    const int cg = half * (NC / 16) + cq;   // group of 8 columns = 4 frequency pairs
                    float xs[KG][8];
#pragma unroll
                    for (int pp = 0; pp < 4; ++pp) {
                        const int pg = c * (NC / 2) + cg * 4 + pp;
                        Cx mh[K], X[K], gh;
                        if (pg == 0) {   // (DC, Nyquist), both real
#pragma unroll
                            for (int j = 0; j < K; ++j) mh[j] = {__uint_as_float(spec[j][cq][1]) * inv_dc[j], 0.0f};
                            gh = {__uint_as_float(spec[K][cq][1]) * inv_dc[K] * ((u_lo & 1) ? -1.0f : 1.0f), 0.0f};
                            leave_one_out<K>(mh, gh, X);
#pragma unroll
                            for (int k = 0; k < KG; ++k) {
                                xs[k][0] = 1.0f;
                                xs[k][1] = k0 + k < K ? X[k0 + k].r : 0.0f;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < K; ++j)
                                mh[j] = {__uint_as_float(spec[j][cq][2 * pp]) * inv_dc[j],
                                         __uint_as_float(spec[j][cq][2 * pp + 1]) * inv_dc[j]};
                            const Cx gw = {__uint_as_float(spec[K][cq][2 * pp]) * inv_dc[K],
                                           __uint_as_float(spec[K][cq][2 * pp + 1]) * inv_dc[K]};
                            const float2 w = TW[(pg * u_lo) % L];   // window offset: G^ = Gw^ e^{-2 pi i f u_lo / L}
                            gh = {gw.r * w.x + gw.i * w.y, gw.i * w.x - gw.r * w.y};
                            leave_one_out<K>(mh, gh, X);
#pragma unroll
                            for (int k = 0; k < KG; ++k) {
                                xs[k][2 * pp] = k0 + k < K ? X[k0 + k].r : 0.0f;
                                xs[k][2 * pp + 1] = k0 + k < K ? X[k0 + k].i : 0.0f;
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < KG; ++k) {
                        uint4 hi, lo;
                        split8(xs[k], hi, lo);
                        *reinterpret_cast<uint4*>(A3 + (2 * k) * kA3 + tc::tile_off(m, cg, NC)) = hi;
                        *reinterpret_cast<uint4*>(A3 + (2 * k + 1) * kA3 + tc::tile_off(m, cg, NC)) = lo;
                    }
                }
                tc::fence_before();
                tc::proxy_fence();
                __syncthreads();
                if (t == 0) {
                    tc::fence_after();
                    issue_inverse<Q, K, Sh>(tmem, dA3, dB3, c, kn);
                    tc::mma_commit(mbar);
                }
            }
            if (!ok) break;
            if (!tc::wait_bounded(mbar, phase, g.tc_error)) {
                ok = false;
                break;
            }
            phase ^= 1;
            tc::fence_after();
            if constexpr (NP > 1) {
                // this pass's messages straight to ch2v (row threads); the in-place v2c
                // waits until every pass has passed the resolution test
#pragma unroll 1
                for (int k = k0 + half; k < k0 + kn; k += 2) {
                    float mx = -INFINITY;
#pragma unroll
                    for (int c16 = 0; c16 < Q / 16; ++c16) {
                        float o[16];
                        tc::tmem_ld16(trow + (k - k0) * Q + c16 * 16, o);
                        mx = fmaxf(mx, vmax(o));
                    }
                    weak |= !(mx >= kMinPeak * (float)L);
                    const float inv = 1.0f / mx;
                    float* dst = ch2v + f * vs + (live ? s_off[(m * K + k) * 3 + 2] : 0);
#pragma unroll
                    for (int c16 = 0; c16 < Q / 16; ++c16) {
                        float o[16];
                        tc::tmem_ld16(trow + (k - k0) * Q + c16 * 16, o);
                        if (live)
#pragma unroll
                            for (int a = 0; a < 16; a += 4)
                                *reinterpret_cast<float4*>(dst + c16 * 16 + a) =
                                    make_float4(fmaxf(o[a] * inv, kRelFloor), fmaxf(o[a + 1] * inv, kRelFloor),
                                                fmaxf(o[a + 2] * inv, kRelFloor), fmaxf(o[a + 3] * inv, kRelFloor));
                    }
                }
                tc::fence_before();
                __syncthreads();   // accumulators read before the next pass overwrites them
            }
        }   // passes
        if (!ok) break;

        // 3. messages.  With every spectrum scaled to DC 1 the accumulated value is
        // L times the probability mass sum_s E(s) G(s + a) of normalised sequences,
        // computed with an absolute error of order L 2^-22.  A row where some
        // user's peak mass is below kMinPeak is left to the FP32 trellis: nothing
        // is written but a NaN in the first entry of user 0's channel message,
        // which the trellis pass looks for.  Each thread normalises its row's
        // messages into the stage; lane groups then write them out.
        if constexpr (NP == 1) {
#pragma unroll 1
        for (int k = half; k < K; k += 2) {
            float mx = -INFINITY;
#pragma unroll
            for (int c16 = 0; c16 < Q / 16; ++c16) {
                float o[16];
                tc::tmem_ld16(trow + k * Q + c16 * 16, o);
                mx = fmaxf(mx, vmax(o));
            }
            weak |= !(mx >= kMinPeak * (float)L);
            const float inv = 1.0f / mx;
            float* srow = stage + m * SS + k * Q;
#pragma unroll
            for (int c16 = 0; c16 < Q / 16; ++c16) {
                float o[16];
                tc::tmem_ld16(trow + k * Q + c16 * 16, o);
#pragma unroll
                for (int a = 0; a < 16; a += 4)
                    *reinterpret_cast<float4*>(srow + c16 * 16 + a) =
                        make_float4(fmaxf(o[a] * inv, kRelFloor), fmaxf(o[a + 1] * inv, kRelFloor),
                                    fmaxf(o[a + 2] * inv, kRelFloor), fmaxf(o[a + 3] * inv, kRelFloor));
            }
        }
        s_weak[half][m] = weak ? 1 : 0;
        tc::fence_before();
        __syncthreads();
#pragma unroll 1
        for (int b0 = 0; b0 < IT; b0 += BT) {
            float4 c0[BT], c1[BT];
#pragma unroll
            for (int i = 0; i < BT; ++i) {
                const int p = (b0 + i) * NW * PPW + warp * PPW + gsub, mr = p / K, k = p - mr * K;
                const int fr = s_rowf[mr];
                c0[i] = c1[i] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
                if (fr >= 0 && !(s_weak[0][mr] | s_weak[1][mr])) {
                    const float* mf = msg + (size_t)fr * fs;
                    const int* o = s_off + (mr * K + k) * 3;
                    c0[i] = reinterpret_cast<const float4*>(mf + o[0])[gl];
                    c1[i] = reinterpret_cast<const float4*>(mf + o[1])[gl];
                }
            }
#pragma unroll
            for (int i = 0; i < BT; ++i) {
                const int p = (b0 + i) * NW * PPW + warp * PPW + gsub, mr = p / K, k = p - mr * K;
                const int fr = s_rowf[mr];
                const bool emit = fr >= 0 && !(s_weak[0][mr] | s_weak[1][mr]);
                const int* o = s_off + (mr * K + k) * 3;
                float* mf = msg + (size_t)(fr >= 0 ? fr : 0) * fs;
                const float4 ov = reinterpret_cast<const float4*>(stage + mr * SS + k * Q)[gl];
                // v2c of each edge = ch2v * c2v of the other edge, rescaled to max 1
                const float4 v0 = mul4(ov, c1[i]), v1 = mul4(ov, c0[i]);
                const float i0 = 1.0f / group_max<GL>(max4(v0)), i1 = 1.0f / group_max<GL>(max4(v1));
                if (emit) {
                    reinterpret_cast<float4*>(ch2v + (size_t)fr * vs + o[2])[gl] = ov;
                    reinterpret_cast<float4*>(mf + o[0])[gl] = scale4(v0, i0);
                    reinterpret_cast<float4*>(mf + o[1])[gl] = scale4(v1, i1);
                } else if (fr >= 0 && k == 0 && gl == 0) {
                    ch2v[(size_t)fr * vs + o[2]] = __int_as_float(0x7fc00000);
                    if (g.log_fallbacks) atomicAdd(g.log_fallbacks, 1ull);
                }
            }
        }
        } else {
            s_weak[half][m] = weak ? 1 : 0;
            __syncthreads();
#pragma unroll 1
            for (int b0 = 0; b0 < IT; b0 += BT) {
                float4 c0[BT], c1[BT], ov[BT];
#pragma unroll
                for (int i = 0; i < BT; ++i) {
                    const int p = (b0 + i) * NW * PPW + warp * PPW + gsub, mr = p / K, k = p - mr * K;
                    const int fr = s_rowf[mr];
                    c0[i] = c1[i] = ov[i] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
                    if (fr >= 0 && !(s_weak[0][mr] | s_weak[1][mr])) {
                        const float* mf = msg + (size_t)fr * fs;
                        const int* o = s_off + (mr * K + k) * 3;
                        c0[i] = reinterpret_cast<const float4*>(mf + o[0])[gl];
                        c1[i] = reinterpret_cast<const float4*>(mf + o[1])[gl];
                        ov[i] = reinterpret_cast<const float4*>(ch2v + (size_t)fr * vs + o[2])[gl];
                    }
                }
#pragma unroll
                for (int i = 0; i < BT; ++i) {
                    const int p = (b0 + i) * NW * PPW + warp * PPW + gsub, mr = p / K, k = p - mr * K;
                    const int fr = s_rowf[mr];
                    const bool emit = fr >= 0 && !(s_weak[0][mr] | s_weak[1][mr]);
                    const int* o = s_off + (mr * K + k) * 3;
                    float* mf = msg + (size_t)(fr >= 0 ? fr : 0) * fs;
                    const float4 v0 = mul4(ov[i], c1[i]), v1 = mul4(ov[i], c0[i]);
                    const float i0 = 1.0f / group_max<GL>(max4(v0)), i1 = 1.0f / group_max<GL>(max4(v1));
                    if (emit) {
                        reinterpret_cast<float4*>(mf + o[0])[gl] = scale4(v0, i0);
                        reinterpret_cast<float4*>(mf + o[1])[gl] = scale4(v1, i1);
                    } else if (fr >= 0 && k == 0 && gl == 0) {
                        ch2v[(size_t)fr * vs + o[2]] = __int_as_float(0x7fc00000);
                        if (g.log_fallbacks) atomicAdd(g.log_fallbacks, 1ull);
                    }
                }
            }
        }
        __syncthreads();   // the stage and the offsets are read before the next tile overwrites them
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tmem, S.tmem_cols);
    }
}
template <int Q, int K>
cudaError_t channel_dft_qk(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                           const uint8_t* active, cudaStream_t s)
{
    constexpr DftShape S = dft_shape(K, Q);
    if constexpr (!S.ok) {
        return cudaErrorInvalidValue;
    } else {
        if (S.smem > di.smem_optin) return cudaErrorInvalidValue;
        cudaError_t e =
            cudaFuncSetAttribute(k_channel_dft<Q, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, S.smem);
        if (e != cudaSuccess) return e;
        const long tiles = ((long)F * g.n + kDftRows - 1) / kDftRows;
        const int grid = (int)std::max(1L, std::min(tiles, (long)di.sm_count));   // one CTA per SM (tensor memory)
        k_channel_dft<Q, K><<<grid, kDftThreads, S.smem, s>>>(g, F, y, msg, ch2v, active);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return launch_channel_fix(g, di, F, y, msg, ch2v, active, s);
    }
}

template <int Q>
cudaError_t channel_dft_q(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                          const uint8_t* active, cudaStream_t s)
{
    switch (g.K) {
        case 2: return channel_dft_qk<Q, 2>(g, di, F, y, msg, ch2v, active, s);
        case 3: return channel_dft_qk<Q, 3>(g, di, F, y, msg, ch2v, active, s);
        case 4: return channel_dft_qk<Q, 4>(g, di, F, y, msg, ch2v, active, s);
        case 5: return channel_dft_qk<Q, 5>(g, di, F, y, msg, ch2v, active, s);
        case 6: return channel_dft_qk<Q, 6>(g, di, F, y, msg, ch2v, active, s);
        case 7: return channel_dft_qk<Q, 7>(g, di, F, y, msg, ch2v, active, s);
        case 8: return channel_dft_qk<Q, 8>(g, di, F, y, msg, ch2v, active, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_channel_dft(const Graph& g, const DeviceInfo& di, int F, const float* y, float* msg, float* ch2v,
                               const uint8_t* active, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    if (!g.dft_tab || g.dv != 2 || g.dc != kDC || !dft_shape(g.K, g.Q).ok) return cudaErrorInvalidValue;
    switch (g.Q) {
        case 16: return channel_dft_q<16>(g, di, F, y, msg, ch2v, active, s);
        case 32: return channel_dft_q<32>(g, di, F, y, msg, ch2v, active, s);
        case 64: return channel_dft_q<64>(g, di, F, y, msg, ch2v, active, s);
        default: return cudaErrorInvalidValue;
    }
}

size_t dft_table_bytes(int K, int Q)
{
    const DftShape S = dft_shape(K, Q);
    if (!S.ok) return 0;
    return (size_t)S.chunks * (4ull * S.Nc * S.KB + 4ull * Q * S.Nc) + 8ull * S.L;
}

size_t dft_offsets_bytes(int K, int n) { return 12ull * K * n; }

void dft_build_offsets(int K, int Q, int n, int E, const int32_t* use_pos, const int32_t* var_edge, int32_t* out)
{
    for (int u = 0; u < n; ++u)
        for (int k = 0; k < K; ++k) {
            const int var = use_pos[k * n + u];
            const int e0 = var_edge[2 * var], e1 = var_edge[2 * var + 1];
            int32_t* o = out + ((size_t)u * K + k) * 3;
            o[0] = k * E * Q + (e0 >> 2) * 4 * Q + (e0 & 3) * Q;
            o[1] = k * E * Q + (e1 >> 2) * 4 * Q + (e1 & 3) * Q;
            o[2] = (k * n + var) * Q;
        }
}

// Forward row n of the spectrum (pair p = n/2; n even: real part, odd: imaginary
// part of the e^{-2 pi i p x / L} transform; pair 0 = DC and Nyquist), inner index x.
static double forward_entry(int n, int x, int L)
{
    const int p = n / 2;
    if (p == 0) return (n & 1) ? ((x & 1) ? -1.0 : 1.0) : 1.0;
    const double th = 2.0 * M_PI * (double)(((long long)p * x) % L) / L;
    return (n & 1) ? -std::sin(th) : std::cos(th);
}

// Inverse weight of spectral column n for output a: sum over the Hermitian
// spectrum folded onto f = 0..L/2 (factor 2 on the pairs f = 1..L/2-1).
static double inverse_entry(int n, int a, int L)
{
    const int p = n / 2;
    if (p == 0) return (n & 1) ? ((a & 1) ? -1.0 : 1.0) : 1.0;
    const double th = 2.0 * M_PI * (double)(((long long)p * a) % L) / L;
    return (n & 1) ? -2.0 * std::sin(th) : 2.0 * std::cos(th);
}

// FP16 hi and lo terms of x at (row, col) of a (rows x KD) tile; lo tile at +tile_bytes.
// Both are rounded from double directly: through float first, a value just past
// an FP16 midpoint can land on it and round the wrong way.
static void put_split(unsigned char* tile, size_t tile_bytes, int row, int col, int KD, double x)
{
    const __half hi = __double2half(x);
    const __half lo = __double2half(x - (double)__half2float(hi));
    const size_t off = tc::tile_off(row, col / 8, KD) + (col % 8) * 2;
    std::memcpy(tile + off, &hi, 2);
    std::memcpy(tile + tile_bytes + off, &lo, 2);
}

void dft_build_table(int K, int Q, unsigned char* out)
{
    const DftShape S = dft_shape(K, Q);
    if (!S.ok) return;
    const int L = S.L, NC = S.Nc, KB = S.KB;
    const size_t kB1 = (size_t)NC * KB * 2, kB3 = (size_t)Q * NC * 2, kChunk = 2 * kB1 + 2 * kB3;
    std::memset(out, 0, dft_table_bytes(K, Q));
    for (int c = 0; c < S.chunks; ++c) {
        unsigned char* B1 = out + c * kChunk;
        unsigned char* B3 = B1 + 2 * kB1;
        for (int nl = 0; nl < NC; ++nl)
            for (int x = 0; x < KB; ++x) put_split(B1, kB1, nl, x, KB, forward_entry(c * NC + nl, x, L));
        for (int a = 0; a < Q; ++a)
            for (int nl = 0; nl < NC; ++nl) put_split(B3, kB3, a, nl, NC, inverse_entry(c * NC + nl, a, L));
    }
    float* tw = reinterpret_cast<float*>(out + S.chunks * kChunk);
    for (int i = 0; i < L; ++i) {
        const double th = 2.0 * M_PI * i / L;
        tw[2 * i] = (float)std::cos(th);
        tw[2 * i + 1] = (float)std::sin(th);
    }
}

}  // namespace jbp
