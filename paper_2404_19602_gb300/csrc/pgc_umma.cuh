// pgc_umma.cuh -- the fifth-generation tensor-core primitives (tcgen05) used by the tensor-core
// reconstruction of the streaming kernel: tensor-memory (TMEM) allocation, the asynchronous
// matrix multiply-accumulate with both operands in shared memory and the accumulator in TMEM,
// its completion through an mbarrier, and TMEM loads into registers.  Inline PTX for sm_103a.
//
// Operand layout (the canonical K-major layout without swizzle): a matrix of R rows x K
// 16-bit elements is cut into core matrices of 8 rows x 16 bytes (8 elements); element (r, k)
// sits at byte
//     (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2
// with LBO the distance between core matrices adjacent along K and SBO the distance between
// core matrices adjacent along the rows.  kUmmaLBO / kUmmaSBO(K) below give the packed form
// used here: the core matrices of one 8-row group are contiguous along K.
#pragma once

#include <cstdint>

namespace pgc {

constexpr uint32_t kUmmaLBO = 128;                                   // one core matrix
__host__ __device__ constexpr uint32_t umma_sbo(int K) { return (uint32_t)(K / 8) * 128u; }
// byte offset of element (r, k) of a K-major operand with K columns (16-bit elements)
__host__ __device__ constexpr uint32_t umma_off(int r, int k, int K)
{
    return (uint32_t)(r / 8) * umma_sbo(K) + (uint32_t)(k / 8) * kUmmaLBO + (uint32_t)(r % 8) * 16u + (uint32_t)(k % 8) * 2u;
}

// Shared-memory matrix descriptor (64 bit): start address >> 4 in bits [0,14), LBO >> 4 in
// [16,30), SBO >> 4 in [32,46), the fixed value 1 in [46,48), base offset 0, relative LBO,
// no swizzle (bits [61,64) = 0).
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16 with FP16 A and B, FP32 accumulator, both operands
// K-major: D format F32 (bits [4,6) = 1), A/B format F16 (0), N >> 3 in [17,23), M >> 4 in [24,29).
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// --- TMEM allocation (one warp, .sync.aligned) ---
__device__ __forceinline__ void tmem_alloc(uint32_t *slot_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot_smem)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// --- ordering of tcgen05 operations around thread synchronisation ---
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// --- D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread ---
__device__ __forceinline__ void umma_f16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}
// arrive once on the mbarrier when every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

// --- mbarrier ---
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
// make the initialised mbarrier visible to the asynchronous proxy (the tensor core's arrive)
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete, giving up after max_tries polls
// (each try_wait itself suspends the thread for a bounded, implementation-defined time).
// Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, uint32_t max_tries)
{
    for (uint32_t t = 0; t < max_tries; ++t)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

// --- TMEM -> registers: lane (32 * (warp % 4) + lane) of the accumulator, 8 / 16 consecutive
// 32-bit columns starting at taddr's column ---
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float v[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// FP16 hi/lo split of a pair: hi = fp16(a), lo = fp16(a - hi), packed two to a 32-bit word
__device__ __forceinline__ void split_f16x2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    uint32_t h;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(b), "f"(a));   // low half = a
    float ha, hb;
    asm("{\n\t.reg .f16 l, u;\n\tmov.b32 {l, u}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, u;\n\t}"
        : "=f"(ha), "=f"(hb)
        : "r"(h));
    uint32_t l;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(b - hb), "f"(a - ha));
    hi = h;
    lo = l;
}

}  // namespace pgc
