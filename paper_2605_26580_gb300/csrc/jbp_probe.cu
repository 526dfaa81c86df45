// jbp_probe.cu -- measured FP32 FMA throughput of the device: the denominator
// of the ALU roofline that the channel and fused kernels are reported against.
//
// Every thread runs kChains independent multiply-add chains x <- x*b + c (no
// dependence between chains, so the FMA pipe, not latency, is the limit) for a
// given number of rounds; the grid holds 4 CTAs of 256 threads per SM.  The
// packed form issues the same chains as two-lane FP32 instructions
// (__ffma2_rn), which perform two multiply-adds per lane and instruction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "jbp.h"
#include "jbp_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 4;
constexpr int kUnroll = 16;

template <bool PACKED>
__global__ void __launch_bounds__(kThreads) k_fma_peak(float b, float c, long rounds, float* sink)
{
    const float seed = 1.0f + 1e-7f * (float)(threadIdx.x + blockIdx.x * blockDim.x);
    float acc = 0.0f;
    if constexpr (PACKED) {
        float2 x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = make_float2(seed + 1e-3f * j, seed - 1e-3f * j);
        const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
        for (long r = 0; r < rounds; ++r) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], b2, c2);
        }
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc += x[j].x + x[j].y;
    } else {
        float x[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = seed + 1e-3f * j;
        for (long r = 0; r < rounds; ++r) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], b, c);
        }
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc += x[j];
    }
    // the chains stay near 1 (b < 1, c small): this store never happens, but the
    // compiler cannot know that, so the chains are kept
    if (acc == -1.0f) sink[threadIdx.x] = acc;
}

template <bool PACKED>
cudaError_t run_once(int grid, long rounds, float* sink, cudaEvent_t a, cudaEvent_t b, float* ms)
{
    cudaError_t e = cudaEventRecord(a);
    if (e == cudaSuccess) {
        k_fma_peak<PACKED><<<grid, kThreads>>>(0.9999999f, 1e-7f, rounds, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    return e;
}

}  // namespace

extern "C" int jbp_fp32_peak(int32_t device, double seconds, int32_t packed, double* tflops)
{
    if (!tflops) {
        jbp::set_last_error("jbp_fp32_peak: NULL tflops");
        return JBP_EINVAL;
    }
    if (!(seconds > 0.0) || seconds > 60.0) {
        jbp::set_last_error("jbp_fp32_peak: seconds must be in (0, 60]");
        return JBP_EINVAL;
    }
    *tflops = 0.0;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        jbp::set_last_error("jbp_fp32_peak: no such CUDA device");
        return JBP_ECUDA;
    }
    int sms = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    float* sink = nullptr;
    int rc = JBP_OK;
    do {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0 ||
            cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess ||
            cudaMalloc(&sink, sizeof(float) * kThreads) != cudaSuccess) {
            rc = JBP_ECUDA;
            break;
        }
        const int grid = sms * kCtasPerSm;
        auto once = [&](long rounds, float* ms) {
            return packed ? run_once<true>(grid, rounds, sink, a, b, ms) : run_once<false>(grid, rounds, sink, a, b, ms);
        };
        // calibrate: short launches, then three launches of seconds / 3 each
        long rounds = 2048;
        float ms = 0.0f;
        if (once(rounds, &ms) != cudaSuccess) { rc = JBP_ECUDA; break; }
        while (ms < 20.0f && rounds < (1L << 40)) {
            rounds *= 4;
            if (once(rounds, &ms) != cudaSuccess) { rc = JBP_ECUDA; break; }
        }
        if (rc) break;
        rounds = std::max(1L, (long)(rounds * (seconds * 1e3 / 3.0) / std::max(ms, 1e-3f)));
        double rate[3];
        for (int rep = 0; rep < 3; ++rep) {
            if (once(rounds, &ms) != cudaSuccess) { rc = JBP_ECUDA; break; }
            const double fma_per_lane = (double)rounds * kUnroll * kChains * (packed ? 2 : 1);
            const double flops = 2.0 * fma_per_lane * (double)grid * kThreads;
            rate[rep] = flops / (ms * 1e-3) / 1e12;
        }
        if (rc) break;
        std::sort(rate, rate + 3);
        *tflops = rate[1];   // median of three launches back to back (a sustained rate)
    } while (false);
    if (rc) jbp::set_last_error("jbp_fp32_peak: a CUDA call failed");
    if (sink) cudaFree(sink);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaGetLastError();
    cudaSetDevice(prev);
    return rc;
}
