// jbp_check_tc.cu -- check node with both Walsh-Hadamard transforms issued as
// dense +-1 matrix products on the 5th-generation tensor cores (tcgen05).
//
// A CTA of 128 threads takes tiles of 128 consecutive edge rows of the step-form
// message array (32 checks x 4 edges; row r = (frame*K + user)*E + e).  Per tile:
//   1. thread t gathers row t's permuted v2c  p~(x) = v2c(h^{-1} x), splits each
//      FP32 value into NSPLIT BF16 terms (hi [, mid] [, lo]) and writes them to
//      shared memory as the A operand (128 x q, K-major, no swizzle);
//   2. one thread issues tcgen05.mma for every split and 16-wide K step against
//      B = the q x q Sylvester matrix (+-1, exact in BF16), accumulating FP32 in
//      tensor memory (TMEM), and commits to an mbarrier;
//   3. every warp reads its 32 TMEM lanes (tcgen05.ld, thread t = row t): the
//      transform P of its row; the leave-one-out product of the three other rows
//      of the check comes from warp shuffles (rows of a check are lanes t^1..t^3);
//   4. the products are split and transformed the same way (second MMA);
//   5. floor, normalise, inverse permutation, store in place.
// Every mbarrier wait is bounded; on expiry the kernel records an error, frees
// its TMEM and returns.
#include <algorithm>

#include <cuda_bf16.h>

#include "jbp_internal.h"
#include "jbp_tc.cuh"

namespace jbp {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTileRows = 128;

using tc::fence_after;
using tc::fence_before;
using tc::proxy_fence;
using tc::smem_addr;

template <int Q>
__device__ __forceinline__ uint32_t tile_off(int m, int kg)
{
    return tc::tile_off(m, kg, Q);
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <int NSPLIT>
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 (&t)[3])
{
    t[0] = __float2bfloat16_rn(x);
    if constexpr (NSPLIT >= 2) {
        float r = x - __bfloat162float(t[0]);
        t[1] = __float2bfloat16_rn(r);
        if constexpr (NSPLIT >= 3) {
            r -= __bfloat162float(t[1]);
            t[2] = __float2bfloat16_rn(r);
        }
    }
}

// write row m's Q values (split into NSPLIT terms) into the A tiles
template <int Q, int NSPLIT>
__device__ __forceinline__ void stage_row(unsigned char* A, int m, const float (&v)[Q])
{
    constexpr uint32_t kTile = kTileRows * Q * 2;
#pragma unroll
    for (int kg = 0; kg < Q / 8; ++kg) {
        __nv_bfloat16 parts[NSPLIT][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            __nv_bfloat16 t[3];
            split_bf16<NSPLIT>(v[kg * 8 + i], t);
#pragma unroll
            for (int s = 0; s < NSPLIT; ++s) parts[s][i] = t[s];
        }
#pragma unroll
        for (int s = 0; s < NSPLIT; ++s)
            *reinterpret_cast<uint4*>(A + s * kTile + tile_off<Q>(m, kg)) =
                make_uint4(pack_bf16(parts[s][0], parts[s][1]), pack_bf16(parts[s][2], parts[s][3]),
                           pack_bf16(parts[s][4], parts[s][5]), pack_bf16(parts[s][6], parts[s][7]));
    }
}

// Issue D = sum_s A_s * B^T over all K steps (one thread), then commit.
template <int Q, int NSPLIT>
__device__ __forceinline__ void issue_transform(uint32_t a_base, uint32_t b_base, uint32_t tmem, uint32_t mbar)
{
    constexpr uint32_t kTile = kTileRows * Q * 2, sbo = (Q / 8) * 128;
    constexpr uint32_t idesc = tc::idesc_f16(kTileRows, Q, true);
    int acc = 0;
#pragma unroll
    for (int s = 0; s < NSPLIT; ++s)
#pragma unroll
        for (int ks = 0; ks < Q / 16; ++ks) {
            const uint64_t ad = tc::smem_desc(a_base + s * kTile + ks * 256, 128, sbo);
            const uint64_t bd = tc::smem_desc(b_base + ks * 256, 128, sbo);
            tc::mma_f16(tmem, ad, bd, idesc, acc);
            acc = 1;
        }
    tc::mma_commit(mbar);
}

template <int Q>
__device__ __forceinline__ void read_row(uint32_t tmem_row, float (&v)[Q])
{
#pragma unroll
    for (int c = 0; c < Q / 16; ++c) {
        float t[16];
        tc::tmem_ld16(tmem_row + c * 16, t);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[c * 16 + i] = t[i];
    }
}

template <int Q, int NSPLIT>
__global__ void __launch_bounds__(kTcThreads) k_check_tc(Graph g, long R, float* msg, const uint8_t* active, int* err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr uint32_t kTile = kTileRows * Q * 2;
    unsigned char* A = smem;                        // NSPLIT tiles
    unsigned char* B = smem + NSPLIT * kTile;       // Q x Q Sylvester matrix
    __shared__ __align__(8) uint64_t mbar_store;
    __shared__ uint32_t tmem_holder;
    __shared__ uint8_t sdiv[Q * Q];
    constexpr int kCols = Q < 32 ? 32 : Q;

    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < Q * Q; i += blockDim.x) sdiv[i] = g.gf_div[i];
    // B[n][k] = (-1)^{popcount(n & k)}
    for (int i = t; i < Q * (Q / 8); i += blockDim.x) {
        const int n = i / (Q / 8), kg = i % (Q / 8);
        __nv_bfloat16 e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) e[j] = __float2bfloat16_rn((__popc(n & (kg * 8 + j)) & 1) ? -1.0f : 1.0f);
        *reinterpret_cast<uint4*>(B + tile_off<Q>(n, kg)) =
            make_uint4(pack_bf16(e[0], e[1]), pack_bf16(e[2], e[3]), pack_bf16(e[4], e[5]), pack_bf16(e[6], e[7]));
    }
    const uint32_t mbar = smem_addr(&mbar_store);
    if (t == 0) tc::mbar_init(mbar);
    if (warp == 0) tc::tmem_alloc(&tmem_holder, kCols);
    proxy_fence();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t a_base = smem_addr(A), b_base = smem_addr(B);
    const long per_frame = (long)g.K * g.E;
    uint32_t phase = 0;

    const long tiles = (R + kTileRows - 1) / kTileRows;
    for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long r = tile * kTileRows + t;
        const bool live = r < R && (!active || active[r / per_frame]);
        float* row = msg + (r < R ? r : 0) * Q;
        int h = 1;
        float v[Q];
        if (live) {
            h = g.chk_coef[r % g.E];
#pragma unroll
            for (int x = 0; x < Q; ++x) v[x] = row[sdiv[h * Q + x]];
        } else {
#pragma unroll
            for (int x = 0; x < Q; ++x) v[x] = 0.0f;
        }
        // forward transform
        stage_row<Q, NSPLIT>(A, t, v);
        proxy_fence();
        __syncthreads();
        if (t == 0) {
            fence_after();
            issue_transform<Q, NSPLIT>(a_base, b_base, tmem, mbar);
        }
        if (!tc::wait_bounded(mbar, phase, err)) break;
        phase ^= 1;
        fence_after();
        read_row<Q>(tmem_row, v);
        // leave-one-out product over the check's four rows (lanes t^1, t^2, t^3)
#pragma unroll
        for (int x = 0; x < Q; ++x) {
            const float a = __shfl_xor_sync(0xffffffffu, v[x], 1);
            const float b = __shfl_xor_sync(0xffffffffu, v[x], 2);
            const float c = __shfl_xor_sync(0xffffffffu, v[x], 3);
            v[x] = a * (b * c);
        }
        // inverse transform (the 1/q factor cancels in the normalisation)
        stage_row<Q, NSPLIT>(A, t, v);
        fence_before();
        proxy_fence();
        __syncthreads();
        if (t == 0) {
            fence_after();
            issue_transform<Q, NSPLIT>(a_base, b_base, tmem, mbar);
        }
        if (!tc::wait_bounded(mbar, phase, err)) break;
        phase ^= 1;
        fence_after();
        read_row<Q>(tmem_row, v);
        if (live) {
            float mx = v[0];
#pragma unroll
            for (int x = 1; x < Q; ++x) mx = fmaxf(mx, v[x]);
            const float fl = kRelFloor * mx, inv = 1.0f / mx;
#pragma unroll
            for (int x = 0; x < Q; ++x) row[sdiv[h * Q + x]] = fmaxf(v[x], fl) * inv;
        }
        fence_before();
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tc::tmem_free(tmem, kCols);
    }
}

template <int Q, int NSPLIT>
cudaError_t check_tc_q(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active, cudaStream_t s)
{
    const size_t smem = (size_t)NSPLIT * kTileRows * Q * 2 + (size_t)Q * Q * 2;
    cudaError_t e = cudaFuncSetAttribute(k_check_tc<Q, NSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_check_tc<Q, NSPLIT>, kTcThreads, smem) != cudaSuccess ||
        occ < 1)
        occ = 1;
    const long R = (long)F * g.K * g.E;
    const long tiles = (R + kTileRows - 1) / kTileRows;
    const int grid = (int)std::max(1L, std::min(tiles, (long)di.sm_count * occ));
    k_check_tc<Q, NSPLIT><<<grid, kTcThreads, smem, s>>>(g, R, msg, active, g.tc_error);
    return cudaGetLastError();
}

template <int Q>
cudaError_t check_tc_split(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active,
                           int precision, cudaStream_t s)
{
    switch (precision) {
        case 1: return check_tc_q<Q, 2>(g, di, F, msg, active, s);   // JBP_PREC_BF16X2
        case 2: return check_tc_q<Q, 1>(g, di, F, msg, active, s);   // JBP_PREC_BF16
        case 3: return check_tc_q<Q, 3>(g, di, F, msg, active, s);   // JBP_PREC_BF16X3
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_check_tc(const Graph& g, const DeviceInfo& di, int F, float* msg, const uint8_t* active,
                            int precision, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    if (g.dc != kDC || !g.tc_error) return cudaErrorInvalidValue;
    switch (g.Q) {
        case 16: return check_tc_split<16>(g, di, F, msg, active, precision, s);
        case 32: return check_tc_split<32>(g, di, F, msg, active, precision, s);
        case 64: return check_tc_split<64>(g, di, F, msg, active, precision, s);
        default: return cudaErrorInvalidValue;   // q < 16: the transform runs as FP32 butterflies
    }
}

}  // namespace jbp
