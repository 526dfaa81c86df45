// jbp_tc.cuh -- building blocks of the kernels that issue 5th-generation tensor
// core matrix products (tcgen05): shared-memory operand descriptors, the
// kind::f16 instruction, completion through an mbarrier, tensor-memory loads.
//
// Operand tiles are K-major without swizzle.  Element (row m, column k) of a
// (rows x KD) 16-bit matrix sits at byte
//     (m/8) * (KD/8) * 128 + (k/8) * 128 + (m%8) * 16 + (k%8) * 2,
// i.e. 8x8 core matrices of 128 contiguous bytes, consecutive along K, then
// along M.  A descriptor for the 16-wide K step ks starts at byte ks * 256 with
// leading-byte offset 128 (next core matrix along K) and stride-byte offset
// (KD/8) * 128 (next core matrix along M or N).
#pragma once

#include <cstdint>

namespace jbp {
namespace tc {

constexpr long long kSpinLimit = 1ll << 24;   // bound of every mbarrier wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of core-matrix row (m, 8*kg .. 8*kg+7) in a (rows x KD) tile
__host__ __device__ __forceinline__ uint32_t tile_off(int m, int kg, int KD)
{
    return (uint32_t)((m >> 3) * (KD / 8) * 128 + kg * 128 + (m & 7) * 16);
}

// shared-memory matrix descriptor: K-major, no swizzle, absolute LBO mode
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version
    return d;
}

// descriptor of the 16-wide K step ks of a (rows x KD) tile at addr
__device__ __forceinline__ uint64_t step_desc(uint32_t addr, int ks, int KD)
{
    return smem_desc(addr + (uint32_t)ks * 256u, 128u, (uint32_t)(KD / 8) * 128u);
}

// descriptor of K step 0 of a (rows x KD) tile at addr.  The start-address
// field holds addr / 16 in 14 bits, which shared-memory offsets never carry out
// of, so the descriptor of byte offset o within the same tile is this plus o / 16
// (step ks: + 16 ks).
__device__ __forceinline__ uint64_t tile_desc(uint32_t addr, int KD)
{
    return smem_desc(addr, 128u, (uint32_t)(KD / 8) * 128u);
}

// instruction descriptor, kind::f16 with FP32 accumulation, A and B K-major.
// bf16 = true: BF16 x BF16; false: FP16 x FP16 (both operands always share a type).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16)
{
    return (1u << 4) | (bf16 ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) [+]= A * B^T, one thread
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// arrive on mbar once every tcgen05 operation issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_init(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make generic-proxy shared-memory writes visible to the tensor cores
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// warp 0 allocates cols tensor-memory columns (a power of two >= 32); the
// address lands in *holder
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, int cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(holder)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, int cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

// 16 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive TMEM columns of this thread's lane (no wait: call ld_wait)
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Bounded wait of this thread on an mbarrier phase; true if the phase completed.
__device__ __forceinline__ bool spin_wait(uint32_t mbar, uint32_t phase)
{
    long long spins = 0;
    bool done = false;
    while (!(done = mbar_try_wait(mbar, phase)) && ++spins < kSpinLimit) {
    }
    return done;
}

// Bounded wait of every thread of the CTA on an mbarrier phase; returns false
// (all threads agree) on expiry, after recording it in *err.
__device__ __forceinline__ bool wait_bounded(uint32_t mbar, uint32_t phase, int* err)
{
    const bool done = spin_wait(mbar, phase);
    const int timed_out = __syncthreads_or(done ? 0 : 1);
    if (timed_out) {
        if (threadIdx.x == 0 && err) atomicExch(err, 1);
        return false;
    }
    return true;
}

}  // namespace tc
}  // namespace jbp
